// Tensor-core filtered self-join: DSSJ (Sec. 3.5) and kNNSJ (Sec. 3.6) for
// any list of subspaces, with the one dense contraction of the method --
// per-pair squared feature differences times the 0/1 subspace-mask matrix --
// on the 5th-generation tensor cores (tcgen05, kind::f16, FP32 accumulators
// in tensor memory).
//
// For one query i and a tile of 256 candidates j, the A operand holds, per
// candidate, the 15 squared differences (x_j - x_i)^2 rounded to FP16 and a
// constant 1; the B operand holds, per subspace S, its 15 mask bits and minus
// its filter threshold.  So one MMA row gives, for every subspace,
//     D[j][S] ~= sum_{f in S} (x_jf - x_if)^2 - Tf_S,
// and D < 0 marks the candidates that may lie within eps or below the current
// k-th distance.  Tf_S = max(k-th squared distance, eps^2) * (1 + 2^-8) +
// 2^-20, rounded up to FP16: the FP16 rounding of the squared differences is
// <= 2^-11 relative + 2^-25 absolute per term, and the FP32 accumulation adds
// far less, so no true neighbour is lost.  Every candidate that passes is
// recomputed exactly with the library's canonical FP32 fold, and only exact
// results decide counts, sums and kNN lists -- the results are identical to
// the plain FP32 path.
//
// Layout: a CTA (4 warps, one warpgroup) owns a block of 64 subspaces and a
// query block; it handles one query at a time.  Per candidate tile it builds
// A (256 rows, two 128-row MMAs) in shared memory, one thread issues the two
// MMAs into two 64-column TMEM regions and commits to an mbarrier, and each
// warp reads its 32 rows of both regions with tcgen05.ld.  Two subspaces are
// voted on at once by OR-ing the sign bits of four accumulators.  Survivors
// of the exact tests become (d2, subspace, candidate) tuples; the kNN lists
// and the B thresholds are updated once per tile.  Populations whose features
// span more than a unit range are rejected by the host (their squared
// differences could overflow FP16).

#include <cuda_fp16.h>
#include <math_constants.h>

#include <algorithm>

#include "device.cuh"
#include "join.cuh"

namespace snaps {
namespace {

constexpr int kNB = kTcBlockWidth;  // 64 subspaces per block
constexpr int kTcWarps = 4;
constexpr int kTile = 256;
constexpr int kTcStages = 2;
constexpr int kTcInit = 256;         // candidates of tile 0 handled subspace-per-thread first
constexpr int kTcTBuf = 512;         // kNN tuples per warp between flushes (a column pair adds <= 128)
constexpr int kTcFlushAt = kTcTBuf - 128;
constexpr unsigned kLockSpin = 1u << 22;  // bound on waiting for the list lock
constexpr uint32_t kLBO = 128;       // K-direction step between 8x16-byte core matrices
constexpr uint32_t kSBO = 256;       // row-direction step
constexpr uint32_t kTmemCols = 128;  // two 64-column accumulator regions
constexpr int kTcQueries = 4;        // queries per work item

template <int KMAX>
struct TcSmem {
    float4 tile[kTcStages][kTile * 4];           // 32 KB candidate tiles (quad-planar)
    alignas(1024) unsigned char A[2][4096];      // two 128-row A operands, K-major, no swizzle
    alignas(1024) unsigned char B[2048];         // 64-row B operand
    uint2 tbuf[kTcWarps][kTcTBuf];               // event tuples per warp
    float ld[kNB][KMAX + 1];                     // kNN lists by subspace
    int lj[kNB][KMAX + 1];
    unsigned long long esum[kNB];
    unsigned epart[kNB];
    float T[kNB];
    float eps2[kNB];
    float escale[kNB];
    int cnt[kNB];
    uint32_t mask[kNB];
    int slot[kNB];
    int tcount[kTcWarps];
    int changed;
    int lock;                                    // serialises kNN list updates across warps
    uint64_t full[kTcStages];
    uint64_t mma_bar;
    uint32_t tmem_base;
    long long work;
};

__device__ __forceinline__ float eps_up(float e2) {
    return e2 >= 0.f ? __uint_as_float(__float_as_uint(e2) + 1u) : -CUDART_INF_F;
}

// Smem matrix descriptor: K-major, no swizzle, version 1 (sm_100 family).
__device__ __forceinline__ uint64_t smem_desc(const void *p) {
    const uint32_t a = dev::smem_addr(p);
    uint64_t d = (uint64_t)((a >> 4) & 0x3FFFu);
    d |= (uint64_t)((kLBO >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((kSBO >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Byte offset of element (r, k) in a K-major 16-column FP16 operand.
__device__ __forceinline__ uint32_t op_off(int r, int k) {
    return (uint32_t)((r >> 3) * kSBO + (k >> 3) * kLBO + (r & 7) * 16 + (k & 7) * 2);
}

// B row 15 entry for subspace c: minus its conservative FP16 filter threshold.
__device__ __forceinline__ __half neg_filter(float tc) {
    if (!(tc >= 0.f)) return __float2half(1.f);  // inactive subspace: D = +1 > 0 for real rows
    const float t = fminf(tc * (1.f + 0.00390625f) + 9.5367431640625e-07f, 65504.f);
    return __hneg(__float2half_ru(t));
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
        "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
          "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
          "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
}

// Canonical FP32 squared distance of subspace `mask` (highest feature first).
__device__ __forceinline__ float fold_exact(const float (&xq)[16], const float4 *tile, int row,
                                            uint32_t mask)
{
    float xc[16];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const float4 v = tile[q * kTile + row];
        xc[4 * q + 0] = v.x;
        xc[4 * q + 1] = v.y;
        xc[4 * q + 2] = v.z;
        xc[4 * q + 3] = v.w;
    }
    float acc = 0.f;
#pragma unroll
    for (int f = 14; f >= 0; --f) {
        const float d = xc[f] - xq[f];
        acc = fmaf(d * (((mask >> f) & 1u) ? 1.f : 0.f), d, acc);
    }
    return acc;
}

// Append the (d2, column, candidate) tuples of the lanes flagged in `p`.
__device__ __forceinline__ void append(uint2 *buf, int &count, bool p, float d2, int col, int j)
{
    const unsigned b = __ballot_sync(dev::kFull, p);
    if (p) buf[count + __popc(b & ((1u << dev::lane_id()) - 1u))] =
        make_uint2(__float_as_uint(d2), ((unsigned)col << 24) | (unsigned)j);
    count += __popc(b);
}

// Insert one warp's buffered kNN candidates (d2, subspace, candidate) into
// the sorted lists: warp-cooperative, one candidate at a time, by (distance,
// index) -- candidates arrive out of index order across warps.  The caller
// holds the list lock.
template <int KMAX>
__device__ void tc_flush(TcSmem<KMAX> &sm, const uint2 *buf, int count, int k)
{
    const unsigned lane = dev::lane_id();
    for (int b = 0; b < count; b += 32) {
        const int idx = b + (int)lane;
        const bool ok = idx < count;
        const uint2 t = ok ? buf[idx] : make_uint2(0x7f800000u, 0u);
        const int c = (int)(t.y >> 24);
        const int j = (int)(t.y & 0xffffffu);
        const float d2 = __uint_as_float(t.x);
        unsigned kb = __ballot_sync(dev::kFull, ok && d2 <= sm.T[c]);
        while (kb) {
            const int src = __ffs(kb) - 1;
            kb &= kb - 1;
            const int cs = __shfl_sync(dev::kFull, c, src);
            const float ds = __shfl_sync(dev::kFull, d2, src);
            const int js = __shfl_sync(dev::kFull, j, src);
            float T = sm.T[cs];
            if (!(ds < T || (ds == T && js < sm.lj[cs][k - 1]))) continue;
            float my_d = lane < (unsigned)k ? sm.ld[cs][lane] : CUDART_INF_F;
            int my_j = lane < (unsigned)k ? sm.lj[cs][lane] : 0x7fffffff;
            const bool before = lane < (unsigned)k && (my_d < ds || (my_d == ds && my_j < js));
            const int pos = __popc(__ballot_sync(dev::kFull, before));
            const float up_d = __shfl_up_sync(dev::kFull, my_d, 1);
            const int up_j = __shfl_up_sync(dev::kFull, my_j, 1);
            if (lane == (unsigned)pos) {
                my_d = ds;
                my_j = js;
            } else if (lane > (unsigned)pos && lane < (unsigned)k) {
                my_d = up_d;
                my_j = up_j;
            }
            T = __shfl_sync(dev::kFull, my_d, k - 1);
            if (lane < (unsigned)k) {
                sm.ld[cs][lane] = my_d;
                sm.lj[cs][lane] = my_j;
            }
            if (lane == 0) {
                sm.T[cs] = T;
                sm.changed = 1;
            }
            __syncwarp();
        }
    }
}

// Take / release the list lock for a whole warp (bounded wait).
template <int KMAX>
__device__ __forceinline__ bool lock_lists(TcSmem<KMAX> &sm)
{
    int got = 0;
    if (dev::lane_id() == 0) {
        for (unsigned it = 0; it < kLockSpin; ++it) {
            if (atomicCAS(&sm.lock, 0, 1) == 0) {
                got = 1;
                break;
            }
            __nanosleep(64);
        }
        __threadfence_block();
    }
    return __shfl_sync(dev::kFull, got, 0) != 0;
}

template <int KMAX>
__device__ __forceinline__ void unlock_lists(TcSmem<KMAX> &sm)
{
    __syncwarp();
    if (dev::lane_id() == 0) {
        __threadfence_block();
        atomicExch(&sm.lock, 0);
    }
}

template <int KMAX>
__global__ void __launch_bounds__(kTcWarps * 32)
    join_tc_kernel(JoinShape s, const TcBlock *__restrict__ blocks, int n_blocks, JoinOut o,
                   DeviceControl *ctrl)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    TcSmem<KMAX> &sm = *reinterpret_cast<TcSmem<KMAX> *>(smem_raw);
    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const unsigned lane = tid & 31u;
    const int64_t n = s.n;
    const int k = s.k;
    constexpr int kQB = kTcQueries;  // queries per work item
    const long long n_qb = (n + kQB - 1) / kQB;
    const long long total = n_qb * (long long)n_blocks;
    const int n_tiles = (int)(s.n_pad / kTile);
    const float4 *x = s.x;
    const uint32_t idesc = (1u << 4) | ((uint32_t)(kNB >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);

    if (tid == 0) {
        for (int st = 0; st < kTcStages; ++st) dev::mbar_init(&sm.full[st], 1);
        dev::mbar_init(&sm.mma_bar, 1);
        dev::fence_barrier_init();
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         dev::smem_addr(&sm.tmem_base)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = sm.tmem_base;

    uint32_t tiles_used = 0;  // tiles consumed (stage / phase bookkeeping)
    uint32_t mma_used = 0;    // MMA commits waited on
    bool failed = false;
    for (;;) {
        if (tid == 0) sm.work = (long long)atomicAdd(&ctrl->next_work, 1ull);
        __syncthreads();
        const long long w = sm.work;
        __syncthreads();
        if (w >= total || failed) break;
        const TcBlock &blk = blocks[w / n_qb];
        const int64_t q0 = (w % n_qb) * kQB;

        if (tid < kNB) {
            sm.mask[tid] = blk.mask[tid];
            sm.slot[tid] = blk.slot[tid];
            const float e2 = blk.eps2[tid];
            sm.eps2[tid] = e2;
            sm.escale[tid] = dev::eps_scale(e2).scale;
        }
        __syncthreads();

        for (int64_t i = q0; i < q0 + kQB && i < n && !failed; ++i) {
            float xq[16];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float4 v = x[row_quad(i, q)];
                xq[4 * q + 0] = v.x;
                xq[4 * q + 1] = v.y;
                xq[4 * q + 2] = v.z;
                xq[4 * q + 3] = v.w;
            }
            const int orig_i = __float_as_int(xq[15]);  // the query's original index
            // stream the tiles: prologue
            if (tid == 0) {
                for (int t = 0; t < kTcStages && t < n_tiles; ++t) {
                    const uint32_t st = (tiles_used + t) % kTcStages;
                    dev::bulk_load(sm.tile[st], x + (int64_t)t * kTile * 4, kTile * 64, &sm.full[st]);
                }
            }
            if (tid < kTcWarps) sm.tcount[tid] = 0;
            if (tid == 0) {
                sm.lock = 0;
                sm.changed = 0;
            }
            for (int t = 0; t < n_tiles; ++t) {
                const uint32_t st = (tiles_used + t) % kTcStages;
                const bool ok = dev::mbar_wait(&sm.full[st], ((tiles_used + t) / kTcStages) & 1u);
                if (__syncthreads_or(!ok)) {
                    if (tid == 0) {
                        atomicOr(&ctrl->error, kErrTimeout);
                        // let the copies still in flight land before the CTA leaves
                        for (int u = t + 1; u < t + kTcStages && u < n_tiles; ++u)
                            dev::mbar_wait(&sm.full[(tiles_used + u) % kTcStages],
                                           ((tiles_used + u) / kTcStages) & 1u);
                    }
                    failed = true;
                    break;
                }
                const float4 *tile = sm.tile[st];
                const int64_t base = (int64_t)t * kTile;
                if (t == 0) {
                    // ---- set-up: thread c < 64 folds subspace c over the first candidates ----
                    if (tid < kNB) {
                        const int c = tid;
                        const uint32_t mask = sm.mask[c];
                        const bool act = mask != 0u && k > 0;
                        float T = act ? CUDART_INF_F : -CUDART_INF_F;
                        const float e2 = sm.eps2[c];
                        const float sc = sm.escale[c];
                        for (int p = 0; p < KMAX; ++p) {
                            sm.ld[c][p] = CUDART_INF_F;
                            sm.lj[c][p] = 0x7fffffff;
                        }
                        int cnt = 0;
                        unsigned long long qs = 0;
                        const int c_end = (int)std::min<int64_t>(kTcInit, n);
                        for (int r = 0; r < c_end; ++r) {
                            if ((int64_t)r == i || mask == 0u) continue;
                            const float acc = fold_exact(xq, tile, r, mask);
                            if (acc <= e2) {
                                ++cnt;
                                qs += dev::eps_quant(acc, sc);
                            }
                            const int oc = __float_as_int(tile[3 * kTile + r].w);
                            if (act && (acc < T || (acc == T && oc < sm.lj[c][k - 1])))
                                T = dev::private_insert(sm.ld[c], sm.lj[c], k, acc, oc);
                        }
                        sm.T[c] = T;
                        sm.cnt[c] = cnt;
                        sm.esum[c] = qs;
                        sm.epart[c] = 0u;
                        // B operand row c: mask bits, then minus the filter threshold
                        __half row[16];
#pragma unroll
                        for (int f = 0; f < 15; ++f) row[f] = __float2half(((mask >> f) & 1u) ? 1.f : 0.f);
                        row[15] = neg_filter(mask ? fmaxf(T, eps_up(e2)) : -1.f);
#pragma unroll
                        for (int f = 0; f < 16; ++f)
                            *reinterpret_cast<__half *>(sm.B + op_off(c, f)) = row[f];
                    }
                    __syncthreads();  // set-up lists and B complete before tile 0's MMA
                }
                {
                    // ---- A operand: rows tid and tid + 128 of this tile ------------------------
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int r = tid + 128 * h;
                        const int64_t j = base + r;
                        uint32_t wds[8];  // 16 FP16 values, two per word
                        if (j == i || j >= n || j < kTcInit) {
                            // never passes: 65504 per feature, no threshold column
                            const __half2 big = __float2half2_rn(65504.f);
#pragma unroll
                            for (int q = 0; q < 7; ++q) wds[q] = *reinterpret_cast<const uint32_t *>(&big);
                            const __half2 last = __halves2half2(__float2half(65504.f), __float2half(0.f));
                            wds[7] = *reinterpret_cast<const uint32_t *>(&last);
                        } else {
                            float sq[16];
#pragma unroll
                            for (int q = 0; q < 4; ++q) {
                                const float4 v = tile[q * kTile + r];
                                const float d0 = v.x - xq[4 * q], d1 = v.y - xq[4 * q + 1];
                                const float d2 = v.z - xq[4 * q + 2], d3 = v.w - xq[4 * q + 3];
                                sq[4 * q + 0] = d0 * d0;
                                sq[4 * q + 1] = d1 * d1;
                                sq[4 * q + 2] = d2 * d2;
                                sq[4 * q + 3] = d3 * d3;
                            }
                            sq[15] = 1.f;  // threshold column
#pragma unroll
                            for (int q = 0; q < 8; ++q) {
                                const __half2 hv = __floats2half2_rn(sq[2 * q], sq[2 * q + 1]);
                                wds[q] = *reinterpret_cast<const uint32_t *>(&hv);
                            }
                        }
                        unsigned char *Ab = sm.A[h];
                        *reinterpret_cast<uint4 *>(Ab + op_off(tid, 0)) = make_uint4(wds[0], wds[1], wds[2], wds[3]);
                        *reinterpret_cast<uint4 *>(Ab + op_off(tid, 8)) = make_uint4(wds[4], wds[5], wds[6], wds[7]);
                    }
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncthreads();
                {
                    // ---- two MMAs: rows 0..127 -> columns 0..63, rows 128..255 -> 64..127 -----
                    if (tid == 0) {
                        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                        const uint64_t bdesc = smem_desc(sm.B);
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            const uint64_t adesc = smem_desc(sm.A[h]);
                            asm volatile(
                                "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                                "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(
                                    tmem + (uint32_t)(h * kNB)),
                                "l"(adesc), "l"(bdesc), "r"(idesc), "r"(0));
                        }
                        asm volatile(
                            "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                dev::smem_addr(&sm.mma_bar)));
                    }
                    const bool mok = dev::mbar_wait(&sm.mma_bar, mma_used & 1u);
                    ++mma_used;
                    if (__syncthreads_or(!mok)) {
                        if (tid == 0) {
                            atomicOr(&ctrl->error, kErrTimeout);
                            for (int u = t + 1; u < t + kTcStages && u < n_tiles; ++u)
                                dev::mbar_wait(&sm.full[(tiles_used + u) % kTcStages],
                                               ((tiles_used + u) / kTcStages) & 1u);
                        }
                        failed = true;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    // ---- epilogue: warp w owns rows 32w..32w+31 of both regions -----------
                    uint2 *buf = sm.tbuf[warp];
                    int count = sm.tcount[warp];
                    const int ra = 32 * warp + (int)lane, rb = ra + 128;
                    // original indices of this lane's two candidates (float 15 of the rows)
                    const int ja = __float_as_int(tile[3 * kTile + ra].w);
                    const int jb = __float_as_int(tile[3 * kTile + rb].w);
#pragma unroll 1
                    for (int c0 = 0; c0 < kNB; c0 += 32) {
                        uint32_t r0[32], r1[32];
                        const uint32_t lanebase = tmem + ((uint32_t)(32 * warp) << 16);
                        tmem_ld32(lanebase + (uint32_t)c0, r0);
                        tmem_ld32(lanebase + (uint32_t)(kNB + c0), r1);
                        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                        for (int c = 0; c < 32; c += 2) {
                            const uint32_t sgn = (r0[c] | r1[c] | r0[c + 1] | r1[c + 1]) & 0x80000000u;
                            if (__any_sync(dev::kFull, sgn != 0u)) {
#pragma unroll
                                for (int e = 0; e < 2; ++e) {
                                    const int col = c0 + c + e;
                                    const bool pa = (int)r0[c + e] < 0, pb = (int)r1[c + e] < 0;
                                    if (__any_sync(dev::kFull, pa | pb)) {
                                        const uint32_t mask = sm.mask[col];
                                        const float da = pa ? fold_exact(xq, tile, ra, mask) : CUDART_INF_F;
                                        const float db = pb ? fold_exact(xq, tile, rb, mask) : CUDART_INF_F;
                                        // eps: counts and exact sums, aggregated per warp
                                        const float e2 = sm.eps2[col];
                                        const bool ea = da <= e2, eb = db <= e2;
                                        const unsigned ba = __ballot_sync(dev::kFull, ea);
                                        const unsigned bb = __ballot_sync(dev::kFull, eb);
                                        if (ba | bb) {
                                            const float scl = sm.escale[col];
                                            unsigned part = 0;
                                            if (ea) part += dev::eps_quant(da, scl);
                                            if (eb) part += dev::eps_quant(db, scl);
                                            const unsigned sum = __reduce_add_sync(dev::kFull, part);
                                            if (lane == 0) {
                                                atomicAdd(&sm.cnt[col], __popc(ba) + __popc(bb));
                                                atomicAdd(&sm.epart[col], sum);
                                            }
                                        }
                                        // kNN candidates: buffered, inserted under the list lock
                                        const float T = sm.T[col];
                                        append(buf, count, da <= T, da, col, ja);
                                        append(buf, count, db <= T, db, col, jb);
                                    }
                                }
                                if (count > kTcFlushAt) {
                                    if (lock_lists(sm)) {
                                        tc_flush<KMAX>(sm, buf, count, k);
                                        unlock_lists(sm);
                                    } else if (lane == 0) {
                                        atomicOr(&ctrl->error, kErrTimeout);
                                    }
                                    count = 0;
                                }
                            }
                        }
                    }
                    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                    // ---- each warp inserts its own kNN candidates under the list lock -------
                    if (count > 0) {
                        if (lock_lists(sm)) {
                            tc_flush<KMAX>(sm, buf, count, k);
                            unlock_lists(sm);
                        } else if (lane == 0) {
                            atomicOr(&ctrl->error, kErrTimeout);
                        }
                    }
                    __syncthreads();
                    if (warp == 0) {
                        // fold this tile's partial eps sums
                        for (int c = (int)lane; c < kNB; c += 32) {
                            sm.esum[c] += sm.epart[c];
                            sm.epart[c] = 0u;
                        }
                        __syncwarp();
                        if (sm.changed) {
                            for (int c = (int)lane; c < kNB; c += 32) {
                                const uint32_t mask = sm.mask[c];
                                *reinterpret_cast<__half *>(sm.B + op_off(c, 15)) =
                                    neg_filter(mask ? fmaxf(sm.T[c], eps_up(sm.eps2[c])) : -1.f);
                            }
                        }
                        __syncwarp();
                        if (lane == 0) sm.changed = 0;
                        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    }
                }
                __syncthreads();
                if (tid == 0 && t + kTcStages < n_tiles)
                    dev::bulk_load(sm.tile[st], x + (int64_t)(t + kTcStages) * kTile * 4, kTile * 64,
                                   &sm.full[st]);
            }
            if (failed) break;
            tiles_used += n_tiles;

            // ---- this query's results: thread c < 64 reports subspace c ------------------------
            if (tid < kNB && sm.mask[tid] != 0u && (orig_i < 0 || orig_i >= n)) {
                // a row that does not carry its index: report, write nothing
                atomicOr(&ctrl->error, kErrBadRow);
            } else if (tid < kNB && sm.mask[tid] != 0u) {
                const int c = tid;
                const int slot = sm.slot[c];
                float *sc = o.scores + (int64_t)slot * 4 * n;
                const int cnt = sm.cnt[c];
                sc[orig_i] = (float)cnt;
                sc[n + orig_i] = dev::eps_mean(sm.esum[c], cnt, sm.escale[c]);
                if (o.eps_count) o.eps_count[(int64_t)slot * n + orig_i] = cnt;
                if (k > 0) {
                    float msum = 0.f;
                    for (int p = 0; p < k; ++p) {
                        const float dd = sqrtf(sm.ld[c][p]);
                        const int j = sm.lj[c][p];
                        msum += dd;
                        if (j >= 0 && j < n) atomicAdd(&sc[2 * n + j], 1.f);
                        if (o.knn_idx) o.knn_idx[((int64_t)slot * n + orig_i) * k + p] = j;
                        if (o.knn_dist) o.knn_dist[((int64_t)slot * n + orig_i) * k + p] = dd;
                    }
                    sc[3 * n + orig_i] = msum / (float)k;
                }
            }
            __syncthreads();
        }
    }

    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
}

template <int KMAX>
snaps_status launch_tc(const JoinShape &s, const TcBlock *blocks, int n_blocks, const JoinOut &o,
                       DeviceControl *ctrl, cudaStream_t st)
{
    const size_t smem = sizeof(TcSmem<KMAX>) + 1024;  // slack for the 1024-byte alignment
    auto kern = join_tc_kernel<KMAX>;
    SNAPS_CHECK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int dev = 0, sms = 0, per_sm = 0;
    SNAPS_CHECK_CUDA(cudaGetDevice(&dev));
    SNAPS_CHECK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    SNAPS_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kTcWarps * 32, smem));
    if (per_sm < 1) {
        set_error("tensor-core join does not fit on an SM (smem %zu)", smem);
        return SNAPS_ECUDA;
    }
    per_sm = std::min(per_sm, (int)(512 / kTmemCols));  // tensor memory: 512 columns per SM
    const long long n_qb = (s.n + kTcQueries - 1) / kTcQueries;
    const long long total = n_qb * (long long)n_blocks;
    const long long grid = std::min<long long>(total, (long long)sms * per_sm);
    SNAPS_CHECK_CUDA(cudaMemsetAsync(&ctrl->next_work, 0, sizeof(unsigned long long), st));
    kern<<<(unsigned)grid, kTcWarps * 32, smem, st>>>(s, blocks, n_blocks, o, ctrl);
    SNAPS_CHECK_CUDA(cudaGetLastError());
    return SNAPS_OK;
}

}  // namespace

snaps_status launch_join_tc(const JoinShape &s, const TcBlock *blocks, int n_blocks,
                            const JoinOut &o, DeviceControl *ctrl, cudaStream_t st)
{
    if (n_blocks <= 0) return SNAPS_OK;
    if (s.k <= 16) return launch_tc<16>(s, blocks, n_blocks, o, ctrl, st);
    return launch_tc<32>(s, blocks, n_blocks, o, ctrl, st);
}

}  // namespace snaps
