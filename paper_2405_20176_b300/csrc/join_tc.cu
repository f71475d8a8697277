// Tensor-core filtered self-join: DSSJ (Sec. 3.5) and kNNSJ (Sec. 3.6) for
// any list of subspaces, with the one dense contraction of the method --
// per-pair squared feature differences times the 0/1 subspace-mask matrix --
// on the 5th-generation tensor cores (tcgen05: kind::f16 with FP16 or BF16
// operands, or kind::tf32 with TF32 operands; FP32 accumulators in tensor
// memory).
//
// The contraction.  For a query i and 128 candidates j, each squared
// difference (x_jf - x_if)^2, scaled by S = 2^11 (exact), is split into a
// high part h = round(s) in the operand type and a low part l = round(s - h).
// Two MMAs (M = 128 subspaces, N = 128 candidates, K = 16), one over the high
// parts and one over the low parts, against the same mask operand (four with
// TF32 parts, whose MMAs take K = 8: two 8-column slices each), leave in
// tensor memory
//     D[S][j] = S * sum_{f in S} (x_jf - x_if)^2 * (1 + e).
// The split leaves 2^-22 relative (FP16, TF32) or 2^-18 (BF16) per term; the FP32
// accumulation of the 30 exact products adds at most 30 roundings of 2^-23
// (the bound for truncating adds; the hardware's own rounding is not
// documented), 3.6e-6.  So |e| <= 3.9e-6 (FP16, TF32) or 7.4e-6 (BF16).  The
// decisions use a margin delta (2^-17 = 7.6e-6 for FP16 and TF32, 2^-15 for BF16)
// that also covers the canonical FP32 fold's own rounding (<= (d + 2) 2^-24),
// plus an absolute slack of 2^-20 (scaled) for FP16 parts below its normal
// range:
//   * D below eps^2 (1 - delta): an eps-neighbour for certain.  It is counted,
//     and its distance sqrt(D / S) enters the exact quantised distance sum;
//   * D within eps^2 (1 +- delta): recomputed with the library's canonical
//     FP32 fold, which decides;
//   * D at or below the k-th distance (1 + delta): recomputed exactly and
//     inserted into the kNN list with the canonical value.
// So eps counts, kNN lists, in-degrees and kNN mean distances are the plain
// FP32 path's, bit for bit; the mean eps distance takes the accumulator's
// distances, within |e| / 2 + 2^-24 (d + 2) of the canonical ones (2.5e-6
// relative for FP16 and TF32, 4.2e-6 for BF16).  Skipped rows (padding, the query itself, the rows folded at start-up)
// carry a large high part in every feature, far above any threshold (every
// threshold is capped at 16 S, above the largest real D of a unit-range
// population, 15 S (1 + delta)).
//
// Mapping.  A CTA owns work items of one query x 256 subspaces (two 128-row A
// operands); the A operands hold only mask bits, so they are written once per
// block of subspaces.  Its 16 consumer warps hold two threads per subspace:
// thread (c, s) reads row s % 128 of the accumulator of half s / 128 --
// warp w reaches tensor-memory lanes 32 (w % 4) .. 32 (w % 4) + 31 -- and
// columns 64 c .. 64 c + 63 of every sub-tile, and keeps its own eps count,
// distance sum and kNN list.  The two lists of a subspace are merged when the
// item ends; meanwhile each thread filters with the smaller of the two k-th
// distances (a candidate at or above the other thread's k-th cannot enter the
// merged list), read from shared memory, where a stale value is only larger.
// A thread first takes the minimum of 32 accumulators and looks at them one by
// one only when it is below the subspace's pass threshold.  One producer warp
// issues the bulk copies (TMA) of 256-row candidate tiles into a ring and, per
// sub-tile of 128 candidates, the four MMAs into one of two accumulator sets
// (2 x 128 columns each, 512 in all).  The warps meet only at mbarriers:
// consumers build a sub-tile's B rows and arrive on `b_ready`; the producer
// waits for that and for `t_empty` (the accumulator set it will overwrite
// has been read), issues the MMAs and commits them to `mma_done`; consumers
// wait for `mma_done`, filter and decide, and arrive on `t_empty`.
//
// kNN lists are max-heaps: a better candidate replaces the largest entry and
// sinks to its place; each list is sorted once, when its query's results are
// written.
//
// Start-up: the 32 rows around the query (in the stored cell order) are
// staged in shared memory and folded exactly first (by the first thread of
// each subspace; the second filters with that thread's k-th distance), so the
// thresholds start finite; the stream skips them.  Every
// wait is bounded and also gives up when another warp has raised the CTA's
// abort flag; the CTA then sets the error word, waits for its copies and MMAs
// in flight, frees its tensor memory and leaves.  Populations whose features
// span more than a unit range are rejected by the host.

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <math_constants.h>

#include <algorithm>

#include "device.cuh"
#include "join.cuh"

namespace snaps {
namespace {

constexpr int kNS = kTcBlockWidth;        // 256 subspaces per block (one query)
constexpr int kM = 128;                   // MMA M: subspaces per A operand
constexpr int kHalves = kNS / kM;         // 2
constexpr int kNC = 128;                  // candidates per sub-tile = MMA N
constexpr int kColParts = 2;              // threads per subspace, 64 columns each
constexpr int kColsPerThread = kNC / kColParts;
constexpr int kConsumers = kNS * kColParts;   // 512
constexpr int kConsumerWarps = kConsumers / 32;
constexpr int kProducerWarp = kConsumerWarps;
constexpr int kCtaThreads = kConsumers + 32;
constexpr int kTile = 256;                // rows per staged tile (one 16 KB bulk copy)
constexpr int kSubPerTile = kTile / kNC;  // 2
constexpr int kWarm = 32;                 // rows folded exactly before the filter starts
constexpr uint32_t kLBO = 128;            // K-direction step between 8x16-byte core matrices
constexpr uint32_t kTmemCols = 2 * kHalves * kNC;  // 512: two accumulator sets
constexpr float kScale = 2048.f;          // S: squared differences are scaled by 2^11
constexpr float kRsqrtScale = 0.02209708691207961f;  // 1 / sqrt(S)
constexpr float kCap = 16.f * kScale;     // every threshold is capped here (> 15 S (1 + delta))
constexpr float kSlack = 9.5367431640625e-07f;  // 2^-20, in scaled units
static_assert(kHalves == 2 && kTmemCols == 512, "one CTA holds all of an SM's tensor memory");
static_assert(kNC * 4 == kConsumers, "every consumer builds four features of one B row");
static_assert(kRowPad % kTile == 0, "padded rows must cover whole tiles");

// Operand forms: FP16 or BF16 parts (kind::f16, K = 16 per MMA, 2-byte
// elements) or TF32 parts (kind::tf32, K = 8 per MMA, 4-byte elements, two
// K-slices per operand).
constexpr int kFormF16 = kTcFormF16, kFormBF16 = kTcFormBF16, kFormTF32 = kTcFormTF32;
template <int FORM>
constexpr int kElemBytes = FORM == kFormTF32 ? 4 : 2;
template <int FORM>
constexpr uint32_t kSBO = 8 * 16 * kElemBytes<FORM>;  // row-direction step: 8 rows of 16 elements
template <int FORM>
constexpr int kSlices = FORM == kFormTF32 ? 2 : 1;       // MMAs per operand over the 16 columns

template <int KMAX, int FORM>
constexpr int kStages = FORM == kFormTF32 ? (KMAX <= 16 ? 6 : 2) : (KMAX <= 16 ? 6 : 4);

template <int KMAX, int FORM>
struct TcSmem {
    static constexpr int kOpBytes = 16 * kElemBytes<FORM>;  // one operand row: 16 columns
    float4 ring[kStages<KMAX, FORM>][kTile * 4];         // candidate tiles (quad-planar)
    alignas(1024) unsigned char A[kHalves][kM * kOpBytes];  // mask bits, 128 x 16, K-major
    alignas(1024) unsigned char Bh[2][kNC * kOpBytes];      // high parts, 128 x 16, K-major
    alignas(1024) unsigned char Bl[2][kNC * kOpBytes];      // low parts
    float ld[KMAX][kConsumers];                         // kNN lists, entry-major: private
    int lj[KMAX][kConsumers];                           // to a thread, distinct banks
    float tk[kConsumers];                               // each thread's current k-th distance
    int pcnt[kNS];                                      // the second thread's eps count and
    unsigned long long pqs[kNS];                        // sum, handed over at the item's end
    float4 warm[4][kWarm];                              // start-up rows, quad-planar
    float4 xq[4];                                       // the item's query row
    uint64_t full[kStages<KMAX, FORM>];                 // tile landed
    uint64_t b_ready[2];                                // B rows written (16 warp arrivals)
    uint64_t t_empty[2];                                // accumulators read (16 warp arrivals)
    uint64_t mma_done[2];                               // MMA batch complete (commit)
    uint64_t cbar;                                      // consumer-only barrier (16 warps)
    uint32_t tmem_base;
    int abort;
};

// Smem matrix descriptor: K-major, no swizzle, version 1 (sm_100 family).
template <int FORM>
__device__ __forceinline__ uint64_t smem_desc(const void *p)
{
    const uint32_t a = dev::smem_addr(p);
    uint64_t d = (uint64_t)((a >> 4) & 0x3FFFu);
    d |= (uint64_t)((kLBO >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((kSBO<FORM> >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Byte offset of element (r, k) in a K-major 16-column operand: 8 x 16-byte
// core matrices, kLBO apart along K and kSBO apart along the rows.
template <int FORM>
__device__ __forceinline__ uint32_t op_off(int r, int k)
{
    constexpr int per = 16 / kElemBytes<FORM>;  // elements in a core matrix row
    return (uint32_t)((r >> 3) * kSBO<FORM> + (k / per) * kLBO + (r & 7) * 16 + (k % per) * kElemBytes<FORM>);
}

// The TF32 value nearest x (ties away from zero in magnitude), as the bits of
// a float whose 13 low mantissa bits are zero: exactly what the tensor core
// reads of a 32-bit operand.
__device__ __forceinline__ uint32_t tf32_bits(float x)
{
    return (__float_as_uint(x) + 0x1000u) & 0xFFFFE000u;
}

// Operand element encodings and error margins of the three forms.
template <int FORM>
struct Op {
    static constexpr bool kBF16 = FORM == kFormBF16, kTF32 = FORM == kFormTF32;
    // 1.0, and the high part of every feature of a skipped row (65504 in FP16,
    // 65536 in BF16 and TF32: two of them exceed every capped threshold)
    static constexpr uint32_t kOne = kTF32 ? 0x3F800000u : kBF16 ? 0x3F80u : 0x3C00u;
    static constexpr uint32_t kBig = kTF32 ? 0x47800000u : kBF16 ? 0x4780u : 0x7BFFu;
    // relative margin of the decisions (see the file comment); TF32 keeps FP16's
    // 10 explicit mantissa bits
    static constexpr float kDelta = kBF16 ? 3.0517578125e-05f : 7.62939453125e-06f;
    // instruction descriptor: D = F32 (bits 4-5), A and B of one type (bits 7-9,
    // 10-12: F16 = 0, BF16 = 1 for kind::f16; TF32 = 2 for kind::tf32), both
    // K-major; N = 128 (bits 17-22, N / 8), M = 128 (bits 24-28, M / 16)
    static constexpr uint32_t kType = kTF32 ? 2u : kBF16 ? 1u : 0u;
    static constexpr uint32_t kIdesc = (1u << 4) | (kType << 7) | (kType << 10) |
                                       ((uint32_t)(kNC >> 3) << 17) | ((uint32_t)(kM >> 4) << 24);
    // high and low parts of a scaled squared difference
    static __device__ __forceinline__ void split(float s, uint32_t &h, uint32_t &l)
    {
        if constexpr (kTF32) {
            h = tf32_bits(s);
            l = tf32_bits(s - __uint_as_float(h));
        } else if constexpr (kBF16) {
            const __nv_bfloat16 a = __float2bfloat16_rn(s);
            const __nv_bfloat16 b = __float2bfloat16_rn(s - __bfloat162float(a));
            h = __bfloat16_as_ushort(a);
            l = __bfloat16_as_ushort(b);
        } else {
            const __half a = __float2half_rn(s);
            const __half b = __float2half_rn(s - __half2float(a));
            h = __half_as_ushort(a);
            l = __half_as_ushort(b);
        }
    }
};

// Bounded mbarrier wait (at most `limit` tries) that also gives up once the
// CTA's abort flag is set.
__device__ __forceinline__ bool wait_or_abort(uint64_t *bar, unsigned parity, const int *abort, unsigned limit)
{
    const uint32_t addr = dev::smem_addr(bar);
    for (unsigned it = 0; it < limit; ++it) {
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
// memory, entry-major, kept as a max-heap (dev::heap_sink_root); its largest
// entry by (distance, index) is mirrored in registers.  Unused entries are
// (+inf, INT_MAX).
struct KnnMax {
    float T;   // largest distance: the k-th nearest so far (+inf until k entries)
    int Tj;    // its index
};

// Insert (d2, oj) into thread `tid`'s list when it beats the largest entry by
// (distance, index).
template <class Smem>
__device__ __forceinline__ void knn_offer(Smem &sm, int tid, int k, float d2, int oj, KnnMax &m)
{
    if (d2 < m.T || (d2 == m.T && oj < m.Tj)) {
        dev::heap_sink_root(&sm.ld[0][tid], &sm.lj[0][tid], kConsumers, k, d2, oj);
        m.T = sm.ld[0][tid];
        m.Tj = sm.lj[0][tid];
    }
}

// The decision thresholds of one thread's subspace, in scaled units.
struct Thresholds {
    float e_lo;    // D below: an eps-neighbour for certain
    float e_hi;    // D at or below (and not below e_lo): decided exactly
    float t_hi;    // D at or below: a kNN candidate, decided exactly
    float pass;    // max(e_hi, t_hi): nothing above it needs a look
};

template <int FORM>
__device__ __forceinline__ Thresholds thresholds(bool act, float e2, float tk)
{
    constexpr float dl = Op<FORM>::kDelta;
    Thresholds t;
    if (!act) {
        t.e_lo = t.e_hi = t.t_hi = t.pass = -CUDART_INF_F;
        return t;
    }
    if (e2 >= 0.f) {
        t.e_lo = fminf(e2 * kScale * (1.f - dl) - kSlack, kCap);
        t.e_hi = fminf(e2 * kScale * (1.f + dl) + kSlack, kCap);
    } else {
        t.e_lo = t.e_hi = -CUDART_INF_F;
    }
    t.t_hi = fminf(tk * kScale * (1.f + dl) + kSlack, kCap);  // +inf (list not full) -> the cap
    t.pass = fmaxf(t.e_hi, t.t_hi);
    return t;
}

// Write the A row of subspace r: its mask bits as 1.0 / 0.0, 0 in column 15.
template <int FORM>
__device__ __forceinline__ void write_a_row(unsigned char *A, int r, uint32_t mask)
{
    constexpr uint32_t one = Op<FORM>::kOne;
    if constexpr (FORM == kFormTF32) {
        // 16 words, four per 16-byte core-matrix row
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            uint32_t w[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int f = 4 * c + e;
                w[e] = (f < 15 && ((mask >> f) & 1u)) ? one : 0u;
            }
            *reinterpret_cast<uint4 *>(A + op_off<FORM>(r, 4 * c)) = make_uint4(w[0], w[1], w[2], w[3]);
        }
    } else {
        uint32_t w[8];
#pragma unroll
        for (int p = 0; p < 8; ++p) {
            const int f0 = 2 * p, f1 = 2 * p + 1;
            const uint32_t lo = ((mask >> f0) & 1u) ? one : 0u;
            const uint32_t hi = (f1 < 15 && ((mask >> f1) & 1u)) ? one : 0u;
            w[p] = lo | (hi << 16);
        }
        *reinterpret_cast<uint4 *>(A + op_off<FORM>(r, 0)) = make_uint4(w[0], w[1], w[2], w[3]);
        *reinterpret_cast<uint4 *>(A + op_off<FORM>(r, 8)) = make_uint4(w[4], w[5], w[6], w[7]);
    }
}

template <int KMAX, int FORM>
__global__ void __launch_bounds__(kCtaThreads, 1)
    join_tc_kernel(JoinShape s, const TcBlock *__restrict__ blocks, int n_blocks, JoinOut o,
                   DeviceControl *ctrl)
{
    constexpr int kSt = kStages<KMAX, FORM>;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *smem_al = smem_raw + ((1024u - (dev::smem_addr(smem_raw) & 1023u)) & 1023u);
    TcSmem<KMAX, FORM> &sm = *reinterpret_cast<TcSmem<KMAX, FORM> *>(smem_al);
    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const unsigned lane = tid & 31u;

    const int n = (int)s.n;  // <= 2^24
    const int k = s.k;
    const int n_tiles = (int)(s.n_pad / kTile);
    const int n_sub = n_tiles * kSubPerTile;  // even
    const long long total = (long long)n * n_blocks;  // work items: (block, query)
    const float4 *x = s.x;
    const unsigned wlimit = s.wait_limit ? s.wait_limit : dev::kSpinLimit;
    // work items of this CTA: blockIdx.x, blockIdx.x + gridDim.x, ...
    const int my_items = total > blockIdx.x ? (int)((total - blockIdx.x + gridDim.x - 1) / gridDim.x) : 0;

    if (tid == 0) {
        for (int st = 0; st < kSt; ++st) dev::mbar_init(&sm.full[st], 1);
        for (int b = 0; b < 2; ++b) {
            dev::mbar_init(&sm.b_ready[b], kConsumerWarps);
            dev::mbar_init(&sm.t_empty[b], kConsumerWarps);
            dev::mbar_init(&sm.mma_done[b], 1);
        }
        dev::mbar_init(&sm.cbar, kConsumerWarps);
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
                    const int st = (int)(issued % kSt);
                    dev::bulk_load(sm.ring[st], x + (int64_t)tt * kTile * 4, kTile * 64, &sm.full[st]);
                    if (++iv == n_tiles) {
                        iv = 0;
                        if (++ii < my_items) it0 = item_t0(ii);
                    }
                }
                ++issued;
            };
            for (int st = 0; st < kSt; ++st) issue_next();
            const long long total_sub = (long long)my_items * n_sub;
            const uint32_t idesc = Op<FORM>::kIdesc;
            long long g = 0;
            bool ok = true;
            for (; g < total_sub; ++g) {
                const int b = (int)(g & 1);
                const unsigned ph = (unsigned)((g >> 1) & 1);
                ok = wait_or_abort(&sm.b_ready[b], ph, &sm.abort, wlimit);
                if (ok && g >= 2) ok = wait_or_abort(&sm.t_empty[b], ph ^ 1u, &sm.abort, wlimit);
                if (!ok) break;
                // sub-tiles <= g - 2 are done with: refill the ring behind them
                if (g >= 2) {
                    const long long tiles_done = (g - 1) / kSubPerTile;
                    while (issued < tiles_done + kSt) issue_next();
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint64_t bh = smem_desc<FORM>(sm.Bh[b]), bl = smem_desc<FORM>(sm.Bl[b]);
#pragma unroll
                for (int hf = 0; hf < kHalves; ++hf) {
                    const uint64_t adesc = smem_desc<FORM>(sm.A[hf]);
                    const uint32_t dt = tmem + (uint32_t)((b * kHalves + hf) * kNC);
                    // per K-slice (the TF32 form has two of eight columns each, 256 bytes
                    // apart, so the descriptors' start addresses step by 256 >> 4 = 16);
                    // the first high-part MMA overwrites the accumulator, the rest add to it
#pragma unroll
                    for (int sl = 0; sl < kSlices<FORM>; ++sl) {
                        const uint64_t step = (uint64_t)(sl * (2 * kLBO >> 4));
                        if constexpr (FORM == kFormTF32) {
                            asm volatile(
                                "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                                "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(dt),
                                "l"(adesc + step), "l"(bh + step), "r"(idesc), "r"(sl));
                            asm volatile(
                                "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                                "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(dt),
                                "l"(adesc + step), "l"(bl + step), "r"(idesc), "r"(1));
                        } else {
                            asm volatile(
                                "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                                "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dt),
                                "l"(adesc + step), "l"(bh + step), "r"(idesc), "r"(sl));
                            asm volatile(
                                "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                                "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dt),
                                "l"(adesc + step), "l"(bl + step), "r"(idesc), "r"(1));
                        }
                    }
                }
                asm volatile(
                    "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                        dev::smem_addr(&sm.mma_done[b])));
            }
            if (!ok) {
                fail();
                // let the copies and MMAs in flight land before the CTA leaves: the last
                // kSt tiles issued (earlier ones were consumed before their slots were refilled)
                const long long real = std::min(issued, (long long)my_items * n_tiles);
                for (long long z = std::max(0ll, real - kSt); z < real; ++z)
                    dev::mbar_wait(&sm.full[z % kSt], (unsigned)((z / kSt) & 1));
                if (g >= 1) dev::mbar_wait(&sm.mma_done[(g - 1) & 1], (unsigned)(((g - 1) >> 1) & 1));
            }
        }
        __syncwarp();
    } else {
        // ================================ consumers ===============================================
        // event role: subspace sidx = half * 128 + arow (tensor-memory lane arow of half `half`),
        // columns 64 cpart .. 64 cpart + 63 of every sub-tile
        const int cpart = warp >> 3;
        const int half = (warp >> 2) & 1;
        const int quarter = warp & 3;
        const int arow = (quarter << 5) | (int)lane;
        const int sidx = half * kM + arow;
        const int partner = tid ^ kNS;
        // B-build role: candidate row br of the sub-tile, features 4 bq .. 4 bq + 3
        const int br = tid >> 2;
        const int bq = tid & 3;
        long long gsub = 0;  // global index of this item's first sub-tile
        int cur_blk = -1;    // the block whose masks the A operands hold
        bool ok = true;
        // every lane of a warp takes the same branch after a wait
        auto wwait = [&](uint64_t *bar, unsigned parity) -> bool {
            return __all_sync(dev::kFull, wait_or_abort(bar, parity, &sm.abort, wlimit));
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
            const float esc_s = esc * kRsqrtScale;  // quantisation of sqrt(D), D = S d^2
            const float4 *xq = sm.xq;
            // ---- B-build role: the query's features 4 bq .. 4 bq + 3 --------------------------------
            const float4 bx = x[row_quad(iq, bq)];
            // the rows folded exactly first: a window of kWarm rows around the query
            const int wcount = n < kWarm ? n : kWarm;
            const int w0 = std::min(std::max(iq - kWarm / 2, 0), n - wcount);
            if (!cbarrier()) {  // the previous item's shared rows and lists are no longer read
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
            sm.tk[tid] = CUDART_INF_F;
            if (blk != cur_blk) {
                // no MMA reads the A operands now: every MMA issued so far was waited for
                if (cpart == 0) write_a_row<FORM>(sm.A[half], arow, mask);
                cur_blk = blk;
            }
            if (!cbarrier()) {  // start-up rows staged, lists cleared, masks written
                ok = false;
                break;
            }

            // ---- start-up: the window, folded exactly by the first thread of each subspace;
            // the second one filters with that thread's k-th distance from the start -----------
            KnnMax km;
            km.T = (act && k > 0) ? CUDART_INF_F : -CUDART_INF_F;
            km.Tj = 0x7fffffff;
            int cnt = 0;
            unsigned long long qs = 0ull;
            if (act && cpart == 0) {
#pragma unroll 1
                for (int r = 0; r < wcount; ++r) {
                    if (w0 + r == iq) continue;
                    int oj;
                    const float d2 = fold_exact(xq, &sm.warm[0][0], kWarm, r, mask, oj);
                    if (d2 <= e2) {
                        ++cnt;
                        qs += dev::eps_quant(d2, esc);
                    }
                    if (k > 0) knn_offer(sm, tid, k, d2, oj, km);
                }
            }
            if (act && k > 0) sm.tk[tid] = km.T;
            Thresholds th = thresholds<FORM>(act, e2, km.T);
            if (!cbarrier()) {  // every thread's start-up k-th distance is published
                ok = false;
                break;
            }

            const int t0 = iq / kTile;
            // Build the B rows of sub-tile u (waiting for its tile first when it starts
            // one), then announce them to the producer.
            auto build = [&](int u) -> bool {
                const int v = u / kSubPerTile;
                const long long z = gsub / kSubPerTile + v;
                const int slot = (int)(z % kSt);
                if (u % kSubPerTile == 0 && !wwait(&sm.full[slot], (unsigned)((z / kSt) & 1))) return false;
                int vt = t0 + v;
                if (vt >= n_tiles) vt -= n_tiles;
                const int rr = (u % kSubPerTile) * kNC + br;
                const int j = vt * kTile + rr;
                const bool skip = j >= n || j == iq || (unsigned)(j - w0) < (unsigned)wcount;
                uint32_t h[4], l[4];
                if (skip) {
                    // never passes: a large high part in every feature
                    constexpr uint32_t big = Op<FORM>::kBig;
                    h[0] = h[1] = h[2] = big;
                    h[3] = bq == 3 ? 0u : big;
                    l[0] = l[1] = l[2] = l[3] = 0u;
                } else {
                    const float4 c = sm.ring[slot][bq * kTile + rr];
                    const float d0 = c.x - bx.x, d1 = c.y - bx.y, d2 = c.z - bx.z, d3 = c.w - bx.w;
                    Op<FORM>::split(d0 * d0 * kScale, h[0], l[0]);
                    Op<FORM>::split(d1 * d1 * kScale, h[1], l[1]);
                    Op<FORM>::split(d2 * d2 * kScale, h[2], l[2]);
                    if (bq == 3) {
                        h[3] = l[3] = 0u;  // float 15 holds the original index, not a feature
                    } else {
                        Op<FORM>::split(d3 * d3 * kScale, h[3], l[3]);
                    }
                }
                const uint32_t off = op_off<FORM>(br, 4 * bq);
                if constexpr (FORM == kFormTF32) {
                    *reinterpret_cast<uint4 *>(&sm.Bh[u & 1][off]) = make_uint4(h[0], h[1], h[2], h[3]);
                    *reinterpret_cast<uint4 *>(&sm.Bl[u & 1][off]) = make_uint4(l[0], l[1], l[2], l[3]);
                } else {
                    *reinterpret_cast<uint2 *>(&sm.Bh[u & 1][off]) =
                        make_uint2(h[0] | (h[1] << 16), h[2] | (h[3] << 16));
                    *reinterpret_cast<uint2 *>(&sm.Bl[u & 1][off]) =
                        make_uint2(l[0] | (l[1] << 16), l[2] | (l[3] << 16));
                }
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
                const float4 *tl = sm.ring[(gsub / kSubPerTile + u / kSubPerTile) % kSt];
                const int rbase = (u % kSubPerTile) * kNC + cpart * kColsPerThread;
                const uint32_t taddr = tmem + ((uint32_t)(quarter * 32) << 16) +
                                       (uint32_t)((b * kHalves + half) * kNC + cpart * kColsPerThread);
                // the smaller of the two threads' k-th distances bounds the merged list
                const float tpart = (act && k > 0) ? sm.tk[partner] : CUDART_INF_F;
                if (act && k > 0) th = thresholds<FORM>(act, e2, fminf(km.T, tpart));
                unsigned qpart = 0u;  // this sub-tile's quantised sums (<= 64 terms of <= 2^20 + 1)
#pragma unroll 1
                for (int h = 0; h < kColsPerThread / 32; ++h) {
                    uint32_t r[32];
                    __syncwarp();  // the load is warp-collective
                    tmem_ld32(taddr + (uint32_t)(32 * h), r);
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                    float mn[16];
#pragma unroll
                    for (int c = 0; c < 16; ++c) mn[c] = fminf(__uint_as_float(r[c]), __uint_as_float(r[c + 16]));
#pragma unroll
                    for (int w = 8; w > 0; w >>= 1)
#pragma unroll
                        for (int c = 0; c < w; ++c) mn[c] = fminf(mn[c], mn[c + w]);
                    if (!(mn[0] < th.pass)) continue;
                    // some accumulator is below the pass threshold: look at each.  Clear
                    // eps-neighbours are counted here, branch-free when the group has any
                    // (every column's quantised distance is formed and the clear ones are
                    // added, so a group costs the same whatever its pattern of hits);
                    // columns in the band around eps and kNN candidates are recomputed
                    // exactly below.
                    uint32_t band = 0u, cand = 0u;
                    if (mn[0] < th.e_lo) {
#pragma unroll
                        for (int c = 0; c < 32; ++c) {
                            const float v = __uint_as_float(r[c]);
                            const bool clear = v < th.e_lo;
                            const unsigned q = dev::eps_quant_fma_pipe(fmaxf(v, 0.f), esc_s);
                            cnt += clear ? 1 : 0;
                            qpart += clear ? q : 0u;
                            band |= (!clear && v <= th.e_hi) ? (1u << c) : 0u;
                            cand |= (v <= th.t_hi) ? (1u << c) : 0u;
                        }
                    } else {
#pragma unroll
                        for (int c = 0; c < 32; ++c) {
                            const float v = __uint_as_float(r[c]);
                            band |= (v <= th.e_hi) ? (1u << c) : 0u;
                            cand |= (v <= th.t_hi) ? (1u << c) : 0u;
                        }
                    }
                    uint32_t need = band | cand;
                    while (need) {
                        const int c = __ffs(need) - 1;
                        const uint32_t bit = 1u << c;
                        need &= need - 1u;
                        int oj;
                        const float d2 = fold_exact(xq, tl, kTile, rbase + 32 * h + c, mask, oj);
                        if ((band & bit) && d2 <= e2) {
                            ++cnt;
                            qs += dev::eps_quant(d2, esc);
                        }
                        if (cand & bit) knn_offer(sm, tid, k, d2, oj, km);
                    }
                    if (cand) th = thresholds<FORM>(act, e2, fminf(km.T, tpart));
                }
                qs += qpart;
                if (act && k > 0) sm.tk[tid] = km.T;
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                __syncwarp();
                if (lane == 0) dev::mbar_arrive(&sm.t_empty[b]);
            }
            if (!ok) break;

            // ---- this item's results: thread (0, s) merges and reports subspace s --------------------
            if (cpart == 1) {
                sm.pcnt[sidx] = cnt;
                sm.pqs[sidx] = qs;
            }
            if (!cbarrier()) {
                ok = false;
                break;
            }
            const int orig_i = __float_as_int(xq[3].w);
            if (cpart == 0 && act && (orig_i < 0 || orig_i >= n)) {
                atomicOr(&ctrl->error, kErrBadRow);  // rows that do not carry their index
            } else if (cpart == 0 && act) {
                cnt += sm.pcnt[sidx];
                qs += sm.pqs[sidx];
                const int slot = bk.slot[sidx];
                float *sc = o.scores + (int64_t)slot * 4 * n;
                sc[orig_i] = (float)cnt;
                sc[n + orig_i] = dev::eps_mean(qs, cnt, esc);
                if (o.eps_count) o.eps_count[(int64_t)slot * n + orig_i] = cnt;
                if (k > 0) {
                    // the partner's entries into this list, then sort it by (distance, index)
                    for (int p = 0; p < k; ++p) knn_offer(sm, tid, k, sm.ld[p][partner], sm.lj[p][partner], km);
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

template <int KMAX, int FORM>
snaps_status launch_tc(const JoinShape &s, const TcBlock *blocks, int n_blocks, const JoinOut &o,
                       DeviceControl *ctrl, cudaStream_t st)
{
    const size_t smem = sizeof(TcSmem<KMAX, FORM>) + 1024;  // slack for the 1024-byte alignment
    static_assert(sizeof(TcSmem<KMAX, FORM>) + 1024 <= 227 * 1024, "the tensor-core join fits one SM");
    auto kern = join_tc_kernel<KMAX, FORM>;
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

snaps_status launch_join_tc(const JoinShape &s, const TcBlock *blocks, int n_blocks, int form,
                            const JoinOut &o, DeviceControl *ctrl, cudaStream_t st)
{
    if (n_blocks <= 0) return SNAPS_OK;
    if (form == kTcFormTF32) {
        if (s.k <= 16) return launch_tc<16, kFormTF32>(s, blocks, n_blocks, o, ctrl, st);
        return launch_tc<32, kFormTF32>(s, blocks, n_blocks, o, ctrl, st);
    }
    if (form == kTcFormBF16) {
        if (s.k <= 16) return launch_tc<16, kFormBF16>(s, blocks, n_blocks, o, ctrl, st);
        return launch_tc<32, kFormBF16>(s, blocks, n_blocks, o, ctrl, st);
    }
    if (s.k <= 16) return launch_tc<16, kFormF16>(s, blocks, n_blocks, o, ctrl, st);
    return launch_tc<32, kFormF16>(s, blocks, n_blocks, o, ctrl, st);
}

}  // namespace snaps
