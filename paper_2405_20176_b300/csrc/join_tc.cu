// Tensor-core filtered self-join: DSSJ (Sec. 3.5) and kNNSJ (Sec. 3.6) for
// any list of subspaces, with the one dense contraction of the method --
// per-pair squared feature differences times the 0/1 subspace-mask matrix --
// on the 5th-generation tensor cores (tcgen05, kind::f16 with FP16 or BF16
// operands, FP32 accumulators in tensor memory).
//
// The contraction.  For a query i and 128 candidates j, the B operand holds
// per candidate the 15 squared differences (x_j - x_i)^2 rounded to the
// operand type and a constant 1; the A operand holds per subspace S its 15
// mask bits and minus its filter threshold.  One MMA (M = 128 subspaces,
// N = 128 candidates, K = 16) gives in tensor memory
//     D[S][j] ~= sum_{f in S} (x_jf - x_if)^2 - Tf_S,
// and D < 0 marks the candidates that may lie within eps of the query or
// below the current k-th distance.  Tf_S = max(k-th squared distance, eps^2)
// * (1 + m) + 2^-20, rounded up to the operand type, with m = 2^-8 for FP16
// and 2^-6 for BF16: rounding a squared difference to FP16 is <= 2^-11
// relative (2^-25 absolute below FP16's normal range), to BF16 <= 2^-8
// relative, and the FP32 accumulation of 16 exact products adds far less, so
// no true neighbour is lost.  BF16's wider margin lets more candidates through
// to the exact recompute.  Every candidate that passes is recomputed with the
// library's canonical FP32 fold (FMAs from the highest feature down), and only
// that exact value decides counts, sums and kNN lists: the results are the
// plain FP32 path's, bit for bit.
//
// Mapping.  A CTA owns work items of one query x 256 subspaces (two 128-row A
// operands).  Its 8 consumer warps are the subspace threads: thread s reads
// row s % 128 of the accumulator of half s / 128 -- warp w reaches
// tensor-memory lanes 32 (w % 4) .. 32 (w % 4) + 31 -- and keeps that
// subspace's eps count, exact distance sum and kNN list privately, so events
// need no atomics, locks or buffers.  One producer warp issues the bulk copies
// (TMA) of 256-row candidate tiles into a ring and, per sub-tile of 128
// candidates, the two MMAs into one of two accumulator sets (2 x 128 columns
// each, 512 in all).  The warps meet only at mbarriers: consumers build a
// sub-tile's B rows (half a row each) and arrive on `b_ready`; the producer
// waits for that and for `t_empty` (the accumulator set it will overwrite has
// been read), issues the MMAs and commits them to `mma_done`; consumers wait
// for `mma_done`, filter -- 32 accumulators OR-ed into one sign test --
// recompute and decide the survivors, write tightened thresholds into the A
// copy that batch used (its next reader is issued only after they arrive on
// `t_empty`), and arrive.  Subspaces arrive sorted by dimension, so the
// threads of a warp see similar hit rates.
//
// kNN lists are kept unsorted with their largest entry tracked: a better
// candidate overwrites that entry and the k entries are rescanned (k
// independent loads instead of a dependent shift chain); each list is sorted
// once, when its query's results are written.
//
// Start-up: the 32 rows around the query (in the stored cell order) are
// staged in shared memory and folded exactly first, so the thresholds start
// finite; the stream skips them.  Every wait is bounded and also gives up
// when another warp has raised the CTA's abort flag; the CTA then sets the
// error word, waits for its copies and MMAs in flight, frees its tensor
// memory and leaves.  Populations whose features span more than a unit range
// are rejected by the host (their squared differences could overflow FP16).

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <math_constants.h>

#include <algorithm>

#include "device.cuh"
#include "join.cuh"

namespace snaps {
namespace {

constexpr int kNS = kTcBlockWidth;       // 256 subspaces per block (one query)
constexpr int kM = 128;                  // MMA M: subspaces per A operand
constexpr int kHalves = kNS / kM;        // 2
constexpr int kNC = 128;                 // candidates per sub-tile = MMA N
constexpr int kConsumers = kNS;          // 256: thread s
constexpr int kProducerWarp = kConsumers / 32;
constexpr int kCtaThreads = kConsumers + 32;
constexpr int kTile = 256;               // rows per staged tile (one 16 KB bulk copy)
constexpr int kSubPerTile = kTile / kNC; // 2
constexpr int kStages = 6;               // ring depth in tiles
constexpr int kWarm = 32;                // rows folded exactly before the filter starts
constexpr uint32_t kLBO = 128;           // K-direction step between 8x16-byte core matrices
constexpr uint32_t kSBO = 256;           // row-direction step
constexpr uint32_t kTmemCols = 2 * kHalves * kNC;  // 512: two accumulator sets
static_assert(kHalves == 2 && kTmemCols == 512, "one CTA holds all of an SM's tensor memory");
static_assert(kNC * 2 == kConsumers, "every consumer builds half of one B row");
static_assert(kRowPad % kTile == 0, "padded rows must cover whole tiles");

template <int KMAX>
struct TcSmem {
    float4 ring[kStages][kTile * 4];                   // candidate tiles (quad-planar)
    alignas(1024) unsigned char A[2][kHalves][kM * 32]; // FP16 128 x 16, K-major
    alignas(1024) unsigned char B[2][kNC * 32];         // FP16 128 x 16, K-major
    float ld[KMAX][kConsumers];                         // kNN lists, entry-major: private
    int lj[KMAX][kConsumers];                           // to a thread, distinct banks
    float4 warm[4][kWarm];                              // start-up rows, quad-planar
    float4 xq[4];                                       // the item's query row
    uint64_t full[kStages];                             // tile landed
    uint64_t b_ready[2];                                // B rows written (8 warp arrivals)
    uint64_t t_empty[2];                                // accumulators read (8 warp arrivals)
    uint64_t mma_done[2];                               // MMA batch complete (commit)
    uint64_t cbar;                                      // consumer-only barrier (8 warps)
    uint32_t tmem_base;
    int abort;
};

// Smem matrix descriptor: K-major, no swizzle, version 1 (sm_100 family).
__device__ __forceinline__ uint64_t smem_desc(const void *p)
{
    const uint32_t a = dev::smem_addr(p);
    uint64_t d = (uint64_t)((a >> 4) & 0x3FFFu);
    d |= (uint64_t)((kLBO >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((kSBO >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Byte offset of element (r, k) in a K-major 16-column FP16 operand.
__device__ __forceinline__ uint32_t op_off(int r, int k)
{
    return (uint32_t)((r >> 3) * kSBO + (k >> 3) * kLBO + (r & 7) * 16 + (k & 7) * 2);
}

// Operand element encodings of the two 16-bit forms.
template <bool BF16>
struct Op16 {
    // 1.0, and the "never passes" squared difference of a skipped row
    // (65504 in FP16, 65536 in BF16: finite, and >= 2 of them exceed any
    // threshold of a unit-range population)
    static constexpr uint32_t kOne = BF16 ? 0x3F80u : 0x3C00u;
    static constexpr uint32_t kBig = BF16 ? 0x4780u : 0x7BFFu;
    // relative filter margin: 2^-8 against FP16's 2^-11 rounding of a squared
    // difference, 2^-6 against BF16's 2^-8
    static constexpr float kMargin = BF16 ? 0.015625f : 0.00390625f;
    // instruction descriptor: D = F32, A and B of one type (F16 = 0, BF16 = 1),
    // both K-major; N = 128, M = 128
    static constexpr uint32_t kIdesc = (1u << 4) | ((BF16 ? 1u : 0u) << 7) | ((BF16 ? 1u : 0u) << 10) |
                                       ((uint32_t)(kNC >> 3) << 17) | ((uint32_t)(kM >> 4) << 24);
    static __device__ __forceinline__ uint32_t pack2(float a, float b)
    {
        if constexpr (BF16) {
            const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
            return *reinterpret_cast<const uint32_t *>(&h);
        } else {
            const __half2 h = __floats2half2_rn(a, b);
            return *reinterpret_cast<const uint32_t *>(&h);
        }
    }
    // A row entry 15 for a subspace: minus its conservative filter threshold,
    // rounded up in magnitude
    static __device__ __forceinline__ unsigned short neg_filter(float t)
    {
        if (!(t >= 0.f)) return (unsigned short)kOne;  // nothing to find: D >= +1 - 1 * 0 on real rows
        if constexpr (BF16) {
            const float f = fminf(t * (1.f + kMargin) + 9.5367431640625e-07f, 1e30f);
            return __bfloat16_as_ushort(__hneg(__float2bfloat16_ru(f)));
        } else {
            const float f = fminf(t * (1.f + kMargin) + 9.5367431640625e-07f, 65504.f);
            return __half_as_ushort(__hneg(__float2half_ru(f)));
        }
    }
};

__device__ __forceinline__ float eps_floor(float e2) { return e2 >= 0.f ? e2 : -CUDART_INF_F; }

// Bounded mbarrier wait that also gives up once the CTA's abort flag is set.
__device__ __forceinline__ bool wait_or_abort(uint64_t *bar, unsigned parity, const int *abort)
{
    const uint32_t addr = dev::smem_addr(bar);
    for (unsigned it = 0; it < dev::kSpinLimit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(addr), "r"(parity)
            : "memory");
        if (done) return true;
        if ((it & 63u) == 63u && *(volatile const int *)abort) return false;
    }
    return false;
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32])
{
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

// Canonical FP32 squared distance of subspace `mask` to the candidate at
// `base[p * stride + row]` (quad-planar): FMAs over the squared differences
// from the highest feature down, starting from +0.  Branch-free: a feature
// outside the subspace adds (0 * d) * d = +-0, which leaves the sum unchanged.
__device__ __forceinline__ float fold_exact(const float4 *xq, const float4 *base, int stride, int row,
                                            uint32_t mask, int &orig)
{
    float xc[16], xo[16];
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        const float4 t = base[p * stride + row];
        const float4 u = xq[p];
        xc[4 * p + 0] = t.x;
        xc[4 * p + 1] = t.y;
        xc[4 * p + 2] = t.z;
        xc[4 * p + 3] = t.w;
        xo[4 * p + 0] = u.x;
        xo[4 * p + 1] = u.y;
        xo[4 * p + 2] = u.z;
        xo[4 * p + 3] = u.w;
    }
    orig = __float_as_int(xc[15]);
    float acc = 0.f;
#pragma unroll
    for (int f = 14; f >= 0; --f) {
        const float d = xc[f] - xo[f];
        acc = fmaf(((mask >> f) & 1u) ? d : 0.f, d, acc);
    }
    return acc;
}

// A thread's kNN list: k entries (squared distance, original index) in shared
// memory, unsorted, with its largest entry by (distance, index) tracked in
// registers.  Unused entries are (+inf, INT_MAX).
struct KnnMax {
    float T;   // largest distance: the k-th nearest so far (+inf until k entries)
    int Tj;    // its index
    int Tp;    // its position
};

// One candidate's exact decisions for thread `tid`'s subspace: eps count and
// quantised distance sum, then, when it beats the list's largest entry by
// (distance, index), it takes that entry's place and the new largest is found.
template <int KMAX>
__device__ __forceinline__ void decide(TcSmem<KMAX> &sm, int tid, int k, float d2, int oj, float e2,
                                       float esc, int &cnt, unsigned long long &qs, KnnMax &m)
{
    if (d2 <= e2) {
        ++cnt;
        qs += dev::eps_quant(d2, esc);
    }
    if (d2 < m.T || (d2 == m.T && oj < m.Tj)) {
        sm.ld[m.Tp][tid] = d2;
        sm.lj[m.Tp][tid] = oj;
        float mx = sm.ld[0][tid];
        int mj = sm.lj[0][tid], mp = 0;
        for (int p = 1; p < k; ++p) {
            const float v = sm.ld[p][tid];
            const int j = sm.lj[p][tid];
            const bool gt = v > mx || (v == mx && j > mj);
            mx = gt ? v : mx;
            mj = gt ? j : mj;
            mp = gt ? p : mp;
        }
        m.T = mx;
        m.Tj = mj;
        m.Tp = mp;
    }
}

// Write the A row of subspace r (mask bits, then minus the filter threshold).
template <bool BF16>
__device__ __forceinline__ void write_a_row(unsigned char *A, int r, uint32_t mask, unsigned short thr)
{
    constexpr uint32_t one = Op16<BF16>::kOne;
    uint32_t w[8];
#pragma unroll
    for (int p = 0; p < 8; ++p) {
        const int f0 = 2 * p, f1 = 2 * p + 1;
        const uint32_t lo = ((mask >> f0) & 1u) ? one : 0u;  // 1.0 / 0.0
        const uint32_t hi = f1 == 15 ? (uint32_t)thr : (((mask >> f1) & 1u) ? one : 0u);
        w[p] = lo | (hi << 16);
    }
    *reinterpret_cast<uint4 *>(A + op_off(r, 0)) = make_uint4(w[0], w[1], w[2], w[3]);
    *reinterpret_cast<uint4 *>(A + op_off(r, 8)) = make_uint4(w[4], w[5], w[6], w[7]);
}

template <int KMAX, bool BF16>
__global__ void __launch_bounds__(kCtaThreads, 1)
    join_tc_kernel(JoinShape s, const TcBlock *__restrict__ blocks, int n_blocks, JoinOut o,
                   DeviceControl *ctrl)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *smem_al = smem_raw + ((1024u - (dev::smem_addr(smem_raw) & 1023u)) & 1023u);
    TcSmem<KMAX> &sm = *reinterpret_cast<TcSmem<KMAX> *>(smem_al);
    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const unsigned lane = tid & 31u;

    const int n = (int)s.n;  // <= 2^24
    const int k = s.k;
    const int n_tiles = (int)(s.n_pad / kTile);
    const int n_sub = n_tiles * kSubPerTile;  // even
    const long long total = (long long)n * n_blocks;  // work items: (block, query)
    const float4 *x = s.x;
    // work items of this CTA: blockIdx.x, blockIdx.x + gridDim.x, ...
    const int my_items = total > blockIdx.x ? (int)((total - blockIdx.x + gridDim.x - 1) / gridDim.x) : 0;

    if (tid == 0) {
        for (int st = 0; st < kStages; ++st) dev::mbar_init(&sm.full[st], 1);
        for (int b = 0; b < 2; ++b) {
            dev::mbar_init(&sm.b_ready[b], kConsumers / 32);
            dev::mbar_init(&sm.t_empty[b], kConsumers / 32);
            dev::mbar_init(&sm.mma_done[b], 1);
        }
        dev::mbar_init(&sm.cbar, kConsumers / 32);
        sm.abort = 0;
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

    auto fail = [&]() {
        *(volatile int *)&sm.abort = 1;
        atomicOr(&ctrl->error, kErrTimeout);
    };

    if (warp == kProducerWarp) {
        // ================================ producer ================================================
        if (lane == 0) {
            // The z-th tile of this CTA's stream: tile iv of its work item ii, whose stream
            // starts at the query's own tile and wraps around.
            int ii = 0, iv = 0, it0 = 0;  // next tile to issue: item, tile within item, first tile
            auto item_t0 = [&](int item_iter) {
                const long long item = blockIdx.x + (long long)item_iter * gridDim.x;
                return (int)((item % n) / kTile);
            };
            if (my_items > 0) it0 = item_t0(0);
            long long issued = 0;
            auto issue_next = [&]() {
                if (ii < my_items) {
                    int tt = it0 + iv;
                    if (tt >= n_tiles) tt -= n_tiles;
                    const int st = (int)(issued % kStages);
                    dev::bulk_load(sm.ring[st], x + (int64_t)tt * kTile * 4, kTile * 64, &sm.full[st]);
                    if (++iv == n_tiles) {
                        iv = 0;
                        if (++ii < my_items) it0 = item_t0(ii);
                    }
                }
                ++issued;
            };
            for (int st = 0; st < kStages; ++st) issue_next();
            const long long total_sub = (long long)my_items * n_sub;
            const uint32_t idesc = Op16<BF16>::kIdesc;
            long long g = 0;
            bool ok = true;
            for (; g < total_sub; ++g) {
                const int b = (int)(g & 1);
                const unsigned ph = (unsigned)((g >> 1) & 1);
                ok = wait_or_abort(&sm.b_ready[b], ph, &sm.abort);
                if (ok && g >= 2) ok = wait_or_abort(&sm.t_empty[b], ph ^ 1u, &sm.abort);
                if (!ok) break;
                // sub-tiles <= g - 2 are done with: refill the ring behind them
                if (g >= 2) {
                    const long long tiles_done = (g - 1) / kSubPerTile;
                    while (issued < tiles_done + kStages) issue_next();
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint64_t bdesc = smem_desc(sm.B[b]);
#pragma unroll
                for (int hf = 0; hf < kHalves; ++hf) {
                    const uint64_t adesc = smem_desc(sm.A[b][hf]);
                    const uint32_t dt = tmem + (uint32_t)((b * kHalves + hf) * kNC);
                    asm volatile(
                        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dt),
                        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(0));
                }
                asm volatile(
                    "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                        dev::smem_addr(&sm.mma_done[b])));
            }
            if (!ok) {
                fail();
                // let the copies and MMAs in flight land before the CTA leaves: the last
                // kStages tiles issued (earlier ones were consumed before their slots were refilled)
                const long long real = std::min(issued, (long long)my_items * n_tiles);
                for (long long z = std::max(0ll, real - kStages); z < real; ++z)
                    dev::mbar_wait(&sm.full[z % kStages], (unsigned)((z / kStages) & 1));
                if (g >= 1) dev::mbar_wait(&sm.mma_done[(g - 1) & 1], (unsigned)(((g - 1) >> 1) & 1));
            }
        }
        __syncwarp();
    } else {
        // ================================ consumers ===============================================
        // event role: subspace sidx = half * 128 + arow (TMEM lane arow of half `half`)
        const int half = warp >> 2;
        const int sub = warp & 3;
        const int arow = (sub << 5) | (int)lane;
        const int sidx = half * kM + arow;
        // B-build role: candidate row br of the sub-tile, K half bh
        const int br = tid >> 1;
        const int bh = tid & 1;
        long long gsub = 0;  // global index of this item's first sub-tile
        bool ok = true;
        // every lane of a warp takes the same branch after a wait
        auto wwait = [&](uint64_t *bar, unsigned parity) -> bool {
            return __all_sync(dev::kFull, wait_or_abort(bar, parity, &sm.abort));
        };
        // barrier of the consumer warps (an mbarrier, so that it can give up)
        unsigned cuses = 0;
        auto cbarrier = [&]() -> bool {
            __syncwarp();
            if (lane == 0) dev::mbar_arrive(&sm.cbar);
            return wwait(&sm.cbar, (cuses++) & 1u);
        };

        for (int it = 0; it < my_items && ok; ++it, gsub += n_sub) {
            const long long item = blockIdx.x + (long long)it * gridDim.x;
            const int blk = (int)(item / n);
            const int iq = (int)(item % n);  // the query's stored row
            const TcBlock &bk = blocks[blk];

            // ---- this thread's subspace ------------------------------------------------------------
            const uint32_t mask = bk.mask[sidx];
            const bool act = mask != 0u;
            const float e2 = bk.eps2[sidx];
            const float esc = dev::eps_scale(e2).scale;
            const float4 *xq = sm.xq;
            // ---- B-build role: the query's features of K half bh ----------------------------------
            const float4 bx0 = x[row_quad(iq, 2 * bh)], bx1 = x[row_quad(iq, 2 * bh + 1)];
            // the rows folded exactly first: a window of kWarm rows around the query
            const int wcount = n < kWarm ? n : kWarm;
            const int w0 = std::min(std::max(iq - kWarm / 2, 0), n - wcount);
            if (!cbarrier()) {  // the previous item's shared rows are no longer read
                ok = false;
                break;
            }
            if (tid < 4 * kWarm) {
                const int p = tid / kWarm, r = tid % kWarm;
                sm.warm[p][r] = r < wcount ? x[row_quad(w0 + r, p)] : make_float4(0.f, 0.f, 0.f, 0.f);
            } else if (tid < 4 * kWarm + 4) {
                sm.xq[tid - 4 * kWarm] = x[row_quad(iq, tid - 4 * kWarm)];
            }
#pragma unroll 1
            for (int p = 0; p < KMAX; ++p) {
                sm.ld[p][tid] = CUDART_INF_F;
                sm.lj[p][tid] = 0x7fffffff;
            }
            if (!cbarrier()) {  // start-up rows staged
                ok = false;
                break;
            }

            // ---- start-up: the private list from the window -----------------------------------------
            KnnMax km;
            km.T = (act && k > 0) ? CUDART_INF_F : -CUDART_INF_F;
            km.Tj = 0x7fffffff;
            km.Tp = 0;
            int cnt = 0;
            unsigned long long qs = 0ull;
            if (act) {
#pragma unroll 1
                for (int r = 0; r < wcount; ++r) {
                    if (w0 + r == iq) continue;
                    int oj;
                    const float d2 = fold_exact(xq, &sm.warm[0][0], kWarm, r, mask, oj);
                    decide<KMAX>(sm, tid, k, d2, oj, e2, esc, cnt, qs, km);
                }
            }
            // the threshold last written into each A copy
            float t_w0 = act ? fmaxf(km.T, eps_floor(e2)) : -1.f, t_w1 = t_w0;
            {
                const unsigned short th = Op16<BF16>::neg_filter(t_w0);
                write_a_row<BF16>(sm.A[0][half], arow, mask, th);
                write_a_row<BF16>(sm.A[1][half], arow, mask, th);
            }

            const int t0 = iq / kTile;
            // Build the B rows of sub-tile u (waiting for its tile first when it starts
            // one), then announce them to the producer.
            auto build = [&](int u) -> bool {
                const int v = u / kSubPerTile;
                const long long z = gsub / kSubPerTile + v;
                const int slot = (int)(z % kStages);
                if (u % kSubPerTile == 0 && !wwait(&sm.full[slot], (unsigned)((z / kStages) & 1))) return false;
                int vt = t0 + v;
                if (vt >= n_tiles) vt -= n_tiles;
                const int rr = (u % kSubPerTile) * kNC + br;
                const int j = vt * kTile + rr;
                const bool skip = j >= n || j == iq || (unsigned)(j - w0) < (unsigned)wcount;
                uint4 wd;
                if (skip) {
                    // never passes: every squared difference big, no threshold column
                    constexpr uint32_t big = Op16<BF16>::kBig, big2 = big | (big << 16);
                    wd = make_uint4(big2, big2, big2, bh ? big : big2);
                } else {
                    const float4 c0 = sm.ring[slot][(2 * bh) * kTile + rr];
                    const float4 c1 = sm.ring[slot][(2 * bh + 1) * kTile + rr];
                    const float d0 = c0.x - bx0.x, d1 = c0.y - bx0.y, d2 = c0.z - bx0.z, d3 = c0.w - bx0.w;
                    const float d4 = c1.x - bx1.x, d5 = c1.y - bx1.y, d6 = c1.z - bx1.z, d7 = c1.w - bx1.w;
                    wd.x = Op16<BF16>::pack2(d0 * d0, d1 * d1);
                    wd.y = Op16<BF16>::pack2(d2 * d2, d3 * d3);
                    wd.z = Op16<BF16>::pack2(d4 * d4, d5 * d5);
                    wd.w = Op16<BF16>::pack2(d6 * d6, bh ? 1.f : d7 * d7);
                }
                *reinterpret_cast<uint4 *>(&sm.B[u & 1][op_off(br, 8 * bh)]) = wd;
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncwarp();
                if (lane == 0) dev::mbar_arrive(&sm.b_ready[u & 1]);
                return true;
            };
            ok = build(0);
#pragma unroll 1
            for (int u = 0; u < n_sub && ok; ++u) {
                if (u + 1 < n_sub && !build(u + 1)) {
                    ok = false;
                    break;
                }
                // ---- filter and decide sub-tile u ----------------------------------------------------
                const long long gu = gsub + u;
                const int b = (int)(gu & 1);
                if (!wwait(&sm.mma_done[b], (unsigned)((gu >> 1) & 1))) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const float4 *tl = sm.ring[(gsub / kSubPerTile + u / kSubPerTile) % kStages];
                const int rbase = (u % kSubPerTile) * kNC;
                const uint32_t taddr = tmem + ((uint32_t)(sub * 32) << 16) + (uint32_t)((b * kHalves + half) * kNC);
#pragma unroll 1
                for (int h = 0; h < kNC / 32; ++h) {
                    uint32_t r[32];
                    tmem_ld32(taddr + (uint32_t)(32 * h), r);
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                    uint32_t any = 0u;
#pragma unroll
                    for (int c = 0; c < 32; ++c) any |= r[c];
                    if (act && (int)any < 0) {
                        uint32_t hm = 0u;  // bit c: column c passed the filter
#pragma unroll
                        for (int c = 31; c >= 0; --c) hm = __funnelshift_l(r[c], hm, 1);
                        // two survivors at a time: their folds overlap
                        while (hm) {
                            const int c1 = __ffs(hm) - 1;
                            hm &= hm - 1u;
                            const int c2 = hm ? __ffs(hm) - 1 : c1;
                            const bool two = hm != 0u;
                            hm &= hm - 1u;
                            int o1, o2;
                            const float a1 = fold_exact(xq, tl, kTile, rbase + 32 * h + c1, mask, o1);
                            const float a2 = fold_exact(xq, tl, kTile, rbase + 32 * h + c2, mask, o2);
                            decide<KMAX>(sm, tid, k, a1, o1, e2, esc, cnt, qs, km);
                            if (two) decide<KMAX>(sm, tid, k, a2, o2, e2, esc, cnt, qs, km);
                        }
                    }
                }
                // tightened threshold into the A copy batch gu used: its next reader (batch
                // gu + 2) is issued only after this warp's t_empty arrival
                if (act) {
                    const float tn = fmaxf(km.T, eps_floor(e2));
                    float &tw = b ? t_w1 : t_w0;
                    if (tn != tw) {
                        tw = tn;
                        *reinterpret_cast<unsigned short *>(&sm.A[b][half][op_off(arow, 15)]) =
                            Op16<BF16>::neg_filter(tn);
                    }
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                __syncwarp();
                if (lane == 0) dev::mbar_arrive(&sm.t_empty[b]);
            }
            if (!ok) break;

            // ---- this item's results: thread s reports the query in subspace s --------------------
            const int orig_i = __float_as_int(xq[3].w);
            if (act && (orig_i < 0 || orig_i >= n)) {
                atomicOr(&ctrl->error, kErrBadRow);  // rows that do not carry their index
            } else if (act) {
                const int slot = bk.slot[sidx];
                float *sc = o.scores + (int64_t)slot * 4 * n;
                sc[orig_i] = (float)cnt;
                sc[n + orig_i] = dev::eps_mean(qs, cnt, esc);
                if (o.eps_count) o.eps_count[(int64_t)slot * n + orig_i] = cnt;
                if (k > 0) {
                    // sort the list by (distance, index)
                    for (int p = 1; p < k; ++p) {
                        const float v = sm.ld[p][tid];
                        const int j = sm.lj[p][tid];
                        int q = p;
                        while (q > 0 && (sm.ld[q - 1][tid] > v || (sm.ld[q - 1][tid] == v && sm.lj[q - 1][tid] > j))) {
                            sm.ld[q][tid] = sm.ld[q - 1][tid];
                            sm.lj[q][tid] = sm.lj[q - 1][tid];
                            --q;
                        }
                        sm.ld[q][tid] = v;
                        sm.lj[q][tid] = j;
                    }
                    float msum = 0.f;
                    for (int p = 0; p < k; ++p) {
                        const float dd = sqrtf(sm.ld[p][tid]);
                        const int j = sm.lj[p][tid];
                        msum += dd;
                        if (j >= 0 && j < n) atomicAdd(&sc[2 * n + j], 1.f);
                        if (o.knn_idx) o.knn_idx[((int64_t)slot * n + orig_i) * k + p] = j;
                        if (o.knn_dist) o.knn_dist[((int64_t)slot * n + orig_i) * k + p] = dd;
                    }
                    sc[3 * n + orig_i] = msum / (float)k;
                }
            }
        }
        if (!ok) fail();
    }

    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
}

template <int KMAX, bool BF16>
snaps_status launch_tc(const JoinShape &s, const TcBlock *blocks, int n_blocks, const JoinOut &o,
                       DeviceControl *ctrl, cudaStream_t st)
{
    const size_t smem = sizeof(TcSmem<KMAX>) + 1024;  // slack for the 1024-byte alignment
    auto kern = join_tc_kernel<KMAX, BF16>;
    SNAPS_CHECK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int dev = 0, sms = 0;
    SNAPS_CHECK_CUDA(cudaGetDevice(&dev));
    SNAPS_CHECK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const long long total = s.n * (long long)n_blocks;
    // one CTA per SM: it holds all 512 tensor-memory columns
    const long long grid = std::min<long long>(total, (long long)sms);
    kern<<<(unsigned)grid, kCtaThreads, smem, st>>>(s, blocks, n_blocks, o, ctrl);
    SNAPS_CHECK_CUDA(cudaGetLastError());
    return SNAPS_OK;
}

}  // namespace

snaps_status launch_join_tc(const JoinShape &s, const TcBlock *blocks, int n_blocks, bool bf16,
                            const JoinOut &o, DeviceControl *ctrl, cudaStream_t st)
{
    if (n_blocks <= 0) return SNAPS_OK;
    if (bf16) {
        if (s.k <= 16) return launch_tc<16, true>(s, blocks, n_blocks, o, ctrl, st);
        return launch_tc<32, true>(s, blocks, n_blocks, o, ctrl, st);
    }
    if (s.k <= 16) return launch_tc<16, false>(s, blocks, n_blocks, o, ctrl, st);
    return launch_tc<32, false>(s, blocks, n_blocks, o, ctrl, st);
}

}  // namespace snaps
