// Per-subspace finishing steps: every metric mapped onto [0, 1] from its
// population statistics, and the top-n outlier rankings (Sec. 3.4, Table 2).
//
// One CTA per (subspace, metric) row, three passes over the row:
//   1. the population min and max of the metric (for the eps mean distance,
//      over the objects that have eps-neighbours).  Min and max of floats are
//      exact in any precision; the span and its reciprocal are then taken in
//      FP64, once per row.
//   2. every object's normalised value, written out, and a histogram of a
//      2048-bin code that is monotone in the object's place in the ranking
//      (bin 2048 holds the objects without eps-neighbours, which rank first
//      for the eps mean distance).  The scaled value comes from a compensated
//      FP32 evaluation (an exact difference, one correction step of the
//      quotient), within half an ulp of the FP64 quotient plus 2^-20 ulp,
//      instead of an FP64 divide per element, which this part executes at a
//      small fraction of its FP32 rate.
//   3. the bin holding the top_n-th object is found from the histogram; the
//      objects above it (< top_n) and those in it are gathered as (order key,
//      index) pairs and sorted.  When that bin holds more objects than the
//      buffer and they all share one key (ties of an integer metric), the
//      lowest indices are taken by an ordered compaction; otherwise a radix
//      select over the whole row's keys decides (a fallback for rows whose
//      values crowd one bin).
// The row is read from HBM once; passes 2 and 3 find it in L2.  Pass 3
// needs only the ranking code, not the normalised value.

#include <math_constants.h>

#include <algorithm>

#include "device.cuh"
#include "prep.cuh"

namespace snaps {
namespace {

constexpr int kFinThreads = 512;
constexpr int kFinWarps = kFinThreads / 32;
constexpr int kBins = 2048;                         // code bins; bin kBins: no eps-neighbours
constexpr int kBinsPerThread = kBins / kFinThreads; // 4
constexpr int kCap = 4096;                          // (key, index) pairs gathered per row
constexpr int kTopMax = 1024;
static_assert(kBinsPerThread * kFinThreads == kBins, "every thread owns whole bins");

// Order key of a metric value: smaller = more outlying.  Metric values are
// non-negative floats, whose bit patterns order like the values.
__device__ __forceinline__ uint32_t order_key(float v, bool none, int m)
{
    const uint32_t b = __float_as_uint(v);
    switch (m) {
    case SNAPS_SCORE_EPS_COUNT:
    case SNAPS_SCORE_KNN_INDEG:
        return b;  // ascending
    case SNAPS_SCORE_EPS_MEAN:
        return none ? 0u : 0xffffffffu - b;  // no neighbours first, then descending
    default:
        return 0xffffffffu - b;  // descending
    }
}

// Constants of one row's scaling.
struct RowScale {
    float lo, hi;              // population min and max of the metric
    float inv;                 // 1 / span, span = hi - lo in FP64, rounded to FP32
    float span_hi, span_lo;    // span = span_hi + span_lo
    float bscale;              // kBins / span, rounded to FP32
    double span, inv64;        // for spans too small for FP32 reciprocals
    bool up;                   // 1 at the maximum (mean distances), else at the minimum
    bool flat;                 // no spread: every scaled value is 0
    bool wide;                 // the FP32 reciprocal would overflow: scale in FP64
};

__device__ __forceinline__ RowScale row_scale(float lo, float hi, int m)
{
    RowScale c;
    c.lo = lo;
    c.hi = hi;
    c.up = (m == SNAPS_SCORE_EPS_MEAN || m == SNAPS_SCORE_KNN_MEAN);
    c.span = (double)hi - (double)lo;
    c.flat = !(c.span > 0.0);  // also when no object qualifies (lo = +inf, hi = -inf)
    c.inv64 = c.flat ? 0.0 : 1.0 / c.span;
    c.wide = !c.flat && !(c.inv64 < 1.0e30);
    c.inv = (float)c.inv64;
    c.span_hi = (float)c.span;
    c.span_lo = (float)(c.span - (double)c.span_hi);
    c.bscale = c.flat || c.wide ? 0.f : (float)((double)kBins * c.inv64);
    return c;
}

// Normalised value z and ranking code of a qualifying object (value v).
// a - b (a >= b >= 0) is split exactly into s + t (Fast2Sum); q0 = s / span
// to within an ulp; one correction with the exact residual of q0 gives z.
// The code uses s alone: fl(v - lo) is non-decreasing and fl(hi - v)
// non-increasing in v, and so is the truncated product, so a larger code
// never ranks below a smaller one.
__device__ __forceinline__ void scale_one(const RowScale &c, float v, float &z, int &bin)
{
    if (c.flat) {
        z = 0.f;
        bin = 0;
        return;
    }
    const float a = c.up ? v : c.hi;
    const float b = c.up ? c.lo : v;
    if (c.wide) {
        const double q = ((double)a - (double)b) * c.inv64;
        z = fminf(fmaxf((float)q, 0.f), 1.f);
        bin = min(kBins - 1, (int)(((double)a - (double)b) * c.inv64 * (double)kBins));
        return;
    }
    const float s = __fsub_rn(a, b);
    const float t = __fsub_rn(-b, __fsub_rn(s, a));  // a - b = s + t exactly
    const float q0 = __fmul_rn(s, c.inv);
    float r = __fmaf_rn(-q0, c.span_hi, s);
    r = __fmaf_rn(-q0, c.span_lo, r);
    r = __fadd_rn(r, t);
    z = fminf(fmaxf(__fmaf_rn(r, c.inv, q0), 0.f), 1.f);
    bin = min(kBins - 1, __float2int_rz(__fmul_rn(s, c.bscale)));
}

struct FinShared {
    unsigned hist[kBins + 1];
    unsigned long long sel[kCap];
    float red_lo[kFinWarps], red_hi[kFinWarps];
    unsigned warp_sum[kFinWarps];
    int b_star;
    unsigned c_above;      // objects in bins above b_star
    unsigned n_above, n_at;
    unsigned key_min, key_max;  // order keys met in bin b_star
};

// Generic radix select of a row's top_n keys (8 bits a pass, warp-aggregated
// histogram updates), the lowest indices among equal keys by an ordered
// compaction, and a sort of the selected pairs.  Used when a row's values
// crowd the bin that holds its top_n-th object.
__device__ void radix_top_row(const float *s, const float *cnt, int m, int64_t n, int top_n,
                              int32_t *out, FinShared &sh)
{
    unsigned *hist = sh.hist;
    unsigned long long *sel = sh.sel;
    __shared__ uint32_t s_prefix, s_need;
    __shared__ unsigned s_count;
    const unsigned lane = threadIdx.x & 31u;
    const int warp = threadIdx.x >> 5;
    const bool em = m == SNAPS_SCORE_EPS_MEAN;
    auto key_of = [&](int64_t i) { return order_key(s[i], em && cnt[i] == 0.f, m); };

    uint32_t prefix = 0, pmask = 0;
    unsigned need = (unsigned)top_n;
    for (int shift = 24; shift >= 0; shift -= 8) {
        __syncthreads();
        for (int b = threadIdx.x; b < 256; b += blockDim.x) hist[b] = 0;
        __syncthreads();
        const int64_t n_round = (n + 31) / 32 * 32;
        for (int64_t i = threadIdx.x; i < n_round; i += blockDim.x) {
            bool in = false;
            unsigned bin = 0;
            if (i < n) {
                const uint32_t key = key_of(i);
                in = (key & pmask) == prefix;
                bin = (key >> shift) & 255u;
            }
            const unsigned grp = __match_any_sync(dev::kFull, in ? bin : 256u + lane);
            if (in && (__ffs(grp) - 1) == (int)lane) atomicAdd(&hist[bin], __popc(grp));
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned acc = 0;
            int b = 0;
            for (; b < 256; ++b) {
                if (acc + hist[b] >= need) break;
                acc += hist[b];
            }
            s_prefix = prefix | ((uint32_t)b << shift);
            s_need = need - acc;
        }
        __syncthreads();
        prefix = s_prefix;
        need = s_need;
        pmask |= 255u << shift;
    }
    // prefix = the top_n-th smallest key; `need` objects with that key are taken
    if (threadIdx.x == 0) s_count = 0;
    __syncthreads();
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        const uint32_t key = key_of(i);
        if (key < prefix) {
            const unsigned p = atomicAdd(&s_count, 1u);
            sel[p] = ((unsigned long long)key << 32) | (uint32_t)i;
        }
    }
    __syncthreads();
    unsigned base = s_count;
    unsigned left = need;
    for (int64_t c0 = 0; c0 < n && left > 0; c0 += blockDim.x) {
        const int64_t i = c0 + threadIdx.x;
        const bool eq = i < n && key_of(i) == prefix;
        const unsigned bal = __ballot_sync(dev::kFull, eq);
        if (lane == 0) sh.warp_sum[warp] = __popc(bal);
        __syncthreads();
        unsigned before = 0, total = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            if (w < warp) before += sh.warp_sum[w];
            total += sh.warp_sum[w];
        }
        before += __popc(bal & ((1u << lane) - 1u));
        if (eq && before < left) sel[base + before] = ((unsigned long long)prefix << 32) | (uint32_t)i;
        __syncthreads();
        const unsigned took = total < left ? total : left;
        base += took;
        left -= took;
    }
    __syncthreads();
    int size = 1;
    while (size < top_n) size <<= 1;
    for (int i = threadIdx.x + top_n; i < size; i += blockDim.x) sel[i] = ~0ull;
    __syncthreads();
    for (int kk = 2; kk <= size; kk <<= 1)
        for (int jj = kk >> 1; jj > 0; jj >>= 1) {
            for (int i = threadIdx.x; i < size; i += blockDim.x) {
                const int p = i ^ jj;
                if (p > i) {
                    const unsigned long long a = sel[i], b = sel[p];
                    if ((a > b) == ((i & kk) == 0)) {
                        sel[i] = b;
                        sel[p] = a;
                    }
                }
            }
            __syncthreads();
        }
    for (int i = threadIdx.x; i < top_n; i += blockDim.x) out[i] = (int32_t)(uint32_t)(sel[i] & 0xffffffffull);
}

// Ascending bitonic sort of sel[0, count) (count <= kCap) with the block.
__device__ void sort_pairs(unsigned long long *sel, int count)
{
    int size = 1;
    while (size < count) size <<= 1;
    for (int i = threadIdx.x + count; i < size; i += blockDim.x) sel[i] = ~0ull;
    __syncthreads();
    for (int kk = 2; kk <= size; kk <<= 1)
        for (int jj = kk >> 1; jj > 0; jj >>= 1) {
            for (int i = threadIdx.x; i < size; i += blockDim.x) {
                const int p = i ^ jj;
                if (p > i) {
                    const unsigned long long a = sel[i], b = sel[p];
                    if ((a > b) == ((i & kk) == 0)) {
                        sel[i] = b;
                        sel[p] = a;
                    }
                }
            }
            __syncthreads();
        }
}

// Objects with no eps-neighbours take part in the eps mean distance's
// statistics only as "first in the ranking" (z = 1).
__device__ __forceinline__ bool no_neighbours(const float *cnt, int m, int64_t i)
{
    return m == SNAPS_SCORE_EPS_MEAN && cnt[i] == 0.f;
}

// Visit every object of the row: f(i, v, none) gets the object's index, metric
// value and whether it lacks eps-neighbours.  The row's 16-byte aligned body
// is read as float4, two per thread in flight; the few objects before the
// first 16-byte boundary and after the last whole float4 are read singly.  (A
// row starts wherever row * n floats lands; the count row that the eps mean
// distance consults has another alignment and is read singly.)
template <class F>
__device__ __forceinline__ void visit_row(const float *s, const float *cnt, int m, int64_t n, F &&f)
{
    const bool em = m == SNAPS_SCORE_EPS_MEAN;
    const int tid = threadIdx.x;
    const int64_t head = std::min<int64_t>((int64_t)(((16u - ((uintptr_t)s & 15u)) & 15u) >> 2), n);
    const int64_t body = (n - head) >> 2;  // whole float4 units
    const int64_t tail0 = head + 4 * body;
    if (tid < head) f((int64_t)tid, s[tid], em && cnt[tid] == 0.f);
    if (tid < n - tail0) {
        const int64_t i = tail0 + tid;
        f(i, s[i], em && cnt[i] == 0.f);
    }
    const float4 *s4 = reinterpret_cast<const float4 *>(s + head);
    for (int64_t u0 = tid; u0 < body; u0 += 2 * kFinThreads) {
        const int64_t u1 = u0 + kFinThreads;
        const float4 a = s4[u0];
        const float4 b = u1 < body ? s4[u1] : make_float4(0.f, 0.f, 0.f, 0.f);
        float ca[4] = {1.f, 1.f, 1.f, 1.f}, cb[4] = {1.f, 1.f, 1.f, 1.f};
        if (em) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                ca[q] = cnt[head + 4 * u0 + q];
                if (u1 < body) cb[q] = cnt[head + 4 * u1 + q];
            }
        }
        const float va[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) f(head + 4 * u0 + q, va[q], ca[q] == 0.f);
        if (u1 < body) {
            const float vb[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
            for (int q = 0; q < 4; ++q) f(head + 4 * u1 + q, vb[q], cb[q] == 0.f);
        }
    }
}

// The ranking code of a qualifying object alone: the same operations as
// scale_one's, without the normalised value.
__device__ __forceinline__ int code_of(const RowScale &c, float v)
{
    if (c.flat) return 0;
    const float a = c.up ? v : c.hi;
    const float b = c.up ? c.lo : v;
    if (c.wide) return min(kBins - 1, (int)(((double)a - (double)b) * c.inv64 * (double)kBins));
    return min(kBins - 1, __float2int_rz(__fmul_rn(__fsub_rn(a, b), c.bscale)));
}

__global__ void __launch_bounds__(kFinThreads, 3)
    finish_kernel(const float *__restrict__ scores, int64_t n, float *__restrict__ norm, int top_n,
                  int32_t *__restrict__ top)
{
    __shared__ FinShared sh;
    const int64_t row = blockIdx.x;  // slot * 4 + metric
    const int m = (int)(row % 4);
    const float *s = scores + row * n;
    const float *cnt = scores + (row - m) * n;  // metric 0 of the same subspace
    const int tid = threadIdx.x;
    const unsigned lane = tid & 31u;
    const int warp = tid >> 5;

    // ---- pass 1: population min and max ----------------------------------------------
    for (int b = tid; b <= kBins; b += kFinThreads) sh.hist[b] = 0u;
    if (tid == 0) {
        sh.n_above = 0u;
        sh.n_at = 0u;
        sh.key_min = 0xffffffffu;
        sh.key_max = 0u;
    }
    float lo = CUDART_INF_F, hi = -CUDART_INF_F;
    visit_row(s, cnt, m, n, [&](int64_t, float v, bool none) {
        if (!none) {
            lo = fminf(lo, v);
            hi = fmaxf(hi, v);
        }
    });
    for (int o = 16; o > 0; o >>= 1) {
        lo = fminf(lo, __shfl_xor_sync(dev::kFull, lo, o));
        hi = fmaxf(hi, __shfl_xor_sync(dev::kFull, hi, o));
    }
    if (lane == 0) {
        sh.red_lo[warp] = lo;
        sh.red_hi[warp] = hi;
    }
    __syncthreads();
    lo = sh.red_lo[0];
    hi = sh.red_hi[0];
#pragma unroll
    for (int w = 1; w < kFinWarps; ++w) {
        lo = fminf(lo, sh.red_lo[w]);
        hi = fmaxf(hi, sh.red_hi[w]);
    }
    const RowScale c = row_scale(lo, hi, m);

    // ---- pass 2: normalised values and the code histogram ---------------------------
    float *z_out = norm ? norm + row * n : nullptr;
    visit_row(s, cnt, m, n, [&](int64_t i, float v, bool none) {
        float z;
        int bin;
        if (none) {
            z = 1.f;
            bin = kBins;
        } else {
            scale_one(c, v, z, bin);
        }
        if (z_out) z_out[i] = z;
        if (top) atomicAdd(&sh.hist[bin], 1u);
    });
    if (!top) return;
    __syncthreads();

    // ---- the bin of the top_n-th object: bins counted from the most outlying ----------
    {
        unsigned part = 0;
#pragma unroll
        for (int q = 0; q < kBinsPerThread; ++q) part += sh.hist[tid * kBinsPerThread + q];
        // suffix sums over threads (higher threads hold higher bins)
        unsigned incl = part;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_down_sync(dev::kFull, incl, o);
            if (lane + o < 32) incl += y;
        }
        if (lane == 0) sh.warp_sum[warp] = incl;
        __syncthreads();
        unsigned above = sh.hist[kBins];  // objects without eps-neighbours rank first
        for (int w = warp + 1; w < kFinWarps; ++w) above += sh.warp_sum[w];
        above += incl - part;  // bins of the higher lanes of this warp
        const unsigned need = (unsigned)top_n;
        if (tid == 0 && sh.hist[kBins] >= need) {
            sh.b_star = kBins;
            sh.c_above = 0u;
        }
        if (above < need && above + part >= need) {
            for (int q = kBinsPerThread - 1; q >= 0; --q) {
                const unsigned h = sh.hist[tid * kBinsPerThread + q];
                if (above + h >= need) {
                    sh.b_star = tid * kBinsPerThread + q;
                    sh.c_above = above;
                    break;
                }
                above += h;
            }
        }
    }
    __syncthreads();
    const int b_star = sh.b_star;
    const unsigned c_above = sh.c_above;

    // ---- pass 3: gather the objects above that bin and in it ---------------------------
    uint32_t kmin = 0xffffffffu, kmax = 0u;
    visit_row(s, cnt, m, n, [&](int64_t i, float v, bool none) {
        const int bin = none ? kBins : code_of(c, v);
        if (bin < b_star) return;
        const unsigned long long pair = ((unsigned long long)order_key(v, none, m) << 32) | (uint32_t)i;
        if (bin > b_star) {
            sh.sel[atomicAdd(&sh.n_above, 1u)] = pair;
        } else {
            const uint32_t key = (uint32_t)(pair >> 32);
            kmin = min(kmin, key);
            kmax = max(kmax, key);
            const unsigned p = c_above + atomicAdd(&sh.n_at, 1u);
            if (p < kCap) sh.sel[p] = pair;
        }
    });
    kmin = __reduce_min_sync(dev::kFull, kmin);
    kmax = __reduce_max_sync(dev::kFull, kmax);
    if (lane == 0) {
        atomicMin(&sh.key_min, kmin);
        atomicMax(&sh.key_max, kmax);
    }
    __syncthreads();
    int32_t *out = top + row * top_n;
    const unsigned n_at = sh.n_at;
    if (c_above + n_at <= (unsigned)kCap) {
        sort_pairs(sh.sel, (int)(c_above + n_at));
    } else if (sh.key_min == sh.key_max) {
        // one key fills the bin: its lowest indices, in index order
        unsigned base = c_above, left = (unsigned)top_n - c_above;
        for (int64_t c0 = 0; c0 < n && left > 0; c0 += kFinThreads) {
            const int64_t i = c0 + tid;
            bool eq = false;
            if (i < n) eq = (no_neighbours(cnt, m, i) ? kBins : code_of(c, s[i])) == b_star;
            const unsigned bal = __ballot_sync(dev::kFull, eq);
            __syncthreads();
            if (lane == 0) sh.warp_sum[warp] = __popc(bal);
            __syncthreads();
            unsigned before = 0, total = 0;
#pragma unroll
            for (int w = 0; w < kFinWarps; ++w) {
                if (w < warp) before += sh.warp_sum[w];
                total += sh.warp_sum[w];
            }
            before += __popc(bal & ((1u << lane) - 1u));
            if (eq && before < left)
                sh.sel[base + before] = ((unsigned long long)sh.key_min << 32) | (uint32_t)i;
            const unsigned took = total < left ? total : left;
            base += took;
            left -= took;
        }
        __syncthreads();
        sort_pairs(sh.sel, top_n);
    } else {
        radix_top_row(s, cnt, m, n, top_n, out, sh);
        return;
    }
    for (int i = tid; i < top_n; i += kFinThreads) out[i] = (int32_t)(uint32_t)(sh.sel[i] & 0xffffffffull);
}

}  // namespace

snaps_status launch_finish(const float *scores, int64_t n, int n_slots, float *norm, int top_n, int32_t *top,
                           cudaStream_t st)
{
    if (n_slots <= 0 || (!norm && (!top || top_n <= 0))) return SNAPS_OK;
    if (top && (top_n <= 0 || top_n > kTopMax || top_n > n)) {
        set_error("top_n %d out of range (max %d, n %lld)", top_n, kTopMax, (long long)n);
        return SNAPS_EINVAL;
    }
    finish_kernel<<<(unsigned)(n_slots * 4), kFinThreads, 0, st>>>(scores, n, norm, top ? top_n : 0, top);
    SNAPS_CHECK_CUDA(cudaGetLastError());
    return SNAPS_OK;
}

snaps_status launch_norm(const float *scores, int64_t n, int n_slots, float *norm, cudaStream_t st)
{
    return launch_finish(scores, n, n_slots, norm, 0, nullptr, st);
}

snaps_status launch_top(const float *scores, int64_t n, int n_slots, int top_n, int32_t *top, cudaStream_t st)
{
    if (top_n <= 0) return SNAPS_OK;
    return launch_finish(scores, n, n_slots, nullptr, top_n, top, st);
}

}  // namespace snaps
