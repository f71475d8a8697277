// Selection of eps and k by the trade-off between over- and underfitting
// (Sec. 3.5.2, Eq. 2 and 3 for eps; Sec. 3.6.2 for k).
//
// The paper derives the result sets of every grid value from one join at the
// largest value: every eps-neighbour at eps_j < eps_max is one at eps_max, and
// the k_j nearest are the first k_j of the k_max nearest (Sec. 3.5.3, 3.6.2).
// `select_join_kernel` does that for one subspace in one brute-force pass: a
// warp per query, lanes striding over the candidates, the canonical FP32 fold
// (FMAs from the highest feature down, as every join of the library); each
// eps-neighbour at eps_max lands in the histogram bin of the smallest grid
// radius that holds it (count and exact quantised distance, shared-memory
// atomics), and the k_max list is kept warp-cooperatively.  The prefix sums of
// the bins give the count and mean distance at every eps_j.  For k_max <= 32
// the same pass keeps the k_max nearest warp-cooperatively; for larger k_max
// (the paper's k grids reach 4096) `select_knn_kernel` gives each object a CTA
// that keeps its k_max nearest in shared memory.  Either way a neighbour at
// rank t counts toward the in-degree at every k_j > t, and the mean distance
// at k_j is an exact sum of the first k_j distances, each quantised to 2^-30.
// Rankings and top-n lists come from the library's top-n kernel (Sec. 3.4),
// and the host computes Eq. 2 and Eq. 3 from those lists.

#include <math_constants.h>

#include <algorithm>

#include "device.cuh"
#include "select.cuh"

namespace snaps {
namespace {

constexpr int kSelWarps = 8;

__device__ __forceinline__ float fold_mask(const float (&q)[16], const float (&c)[16], uint32_t mask)
{
    float acc = 0.f;
#pragma unroll
    for (int f = 14; f >= 0; --f) {
        const float d = c[f] - q[f];
        acc = fmaf(((mask >> f) & 1u) ? d : 0.f, d, acc);
    }
    return acc;
}

__device__ __forceinline__ void load_row16(const float4 *__restrict__ x, int64_t i, float (&v)[16])
{
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const float4 t = x[row_quad(i, q)];
        v[4 * q + 0] = t.x;
        v[4 * q + 1] = t.y;
        v[4 * q + 2] = t.z;
        v[4 * q + 3] = t.w;
    }
}

// First grid index g with k_g > t: a neighbour at rank t is one of the k_g
// nearest for g and every later grid value.
__device__ __forceinline__ int first_grid_above(const KGrid &kg, int t)
{
    int g = 0;
    while (g < kg.n - 1 && kg.k[g] <= t) ++g;
    return g;
}

__device__ __forceinline__ unsigned long long knn_quant(float d2)
{
    return __float2ull_rn(sqrtf(d2) * (float)(1.0 / kKnnQuantum));
}

__global__ void __launch_bounds__(kSelWarps * 32)
    select_join_kernel(const float4 *__restrict__ x, int n, SelectSpec sp, KGrid kg, float *eps_scores,
                       float *k_scores)
{
    __shared__ unsigned s_cnt[kSelWarps][kSelectMaxGrid];
    __shared__ unsigned long long s_sum[kSelWarps][kSelectMaxGrid];
    const int warp = threadIdx.x >> 5;
    const unsigned lane = dev::lane_id();
    const int p = blockIdx.x * kSelWarps + warp;
    if (p >= n) return;
    for (int b = (int)lane; b < kSelectMaxGrid; b += 32) {
        s_cnt[warp][b] = 0u;
        s_sum[warp][b] = 0ull;
    }
    __syncwarp();
    float q[16];
    load_row16(x, p, q);
    const int qorig = __float_as_int(q[15]);
    const int G = sp.n_eps;
    const float e2max = G > 0 ? sp.e2[G - 1] : -1.f;
    const int k = kg.n > 0 && kg.k[kg.n - 1] <= kSelectWarpK ? kg.k[kg.n - 1] : 0;
    float T = k > 0 ? CUDART_INF_F : -CUDART_INF_F;
    float my_d = CUDART_INF_F;
    int my_j = 0x7fffffff;
    for (int b = 0; b < n; b += 32) {
        const int j = b + (int)lane;
        float d2 = CUDART_INF_F;
        int oj = 0x7fffffff;
        if (j < n && j != p) {
            float c[16];
            load_row16(x, j, c);
            oj = __float_as_int(c[15]);
            d2 = fold_mask(q, c, sp.mask);
        }
        if (d2 <= e2max) {
            int bin = 0;
            while (d2 > sp.e2[bin]) ++bin;  // the smallest radius that holds it
            atomicAdd(&s_cnt[warp][bin], 1u);
            atomicAdd(&s_sum[warp][bin], (unsigned long long)__float2uint_rn(dev::eps_sqrt(d2) * sp.qscale));
        }
        if (k > 0) {
            const int jk = __shfl_sync(dev::kFull, my_j, k - 1);
            const bool want = d2 < T || (d2 == T && oj < jk);
            const unsigned bal = __ballot_sync(dev::kFull, want);
            if (bal) dev::list_insert(bal, d2, oj, my_d, my_j, k, T);
        }
    }
    __syncwarp();
    // counts and mean distances at every grid radius: prefix sums over the bins
    if ((int)lane < G) {
        unsigned c = 0;
        unsigned long long s = 0;
        for (int b = 0; b <= (int)lane; ++b) {
            c += s_cnt[warp][b];
            s += s_sum[warp][b];
        }
        float *row = eps_scores + (int64_t)lane * 4 * n;
        row[qorig] = (float)c;
        row[n + qorig] = c > 0 ? (float)(((double)s / (double)sp.qscale) / (double)c) : 0.f;
    }
    if (k > 0) {
        // lane t holds the neighbour of rank t; prefix sums of the quantised
        // distances give the mean over the k_g nearest at lane k_g - 1
        unsigned long long qs = (int)lane < k ? knn_quant(my_d) : 0ull;
        for (int off = 1; off < 32; off <<= 1) {
            const unsigned long long v = __shfl_up_sync(dev::kFull, qs, off);
            if ((int)lane >= off) qs += v;
        }
        if ((int)lane < k) {
            const int g0 = first_grid_above(kg, (int)lane);
            if (my_j >= 0 && my_j < n) atomicAdd(&k_scores[(int64_t)g0 * 4 * n + 2 * n + my_j], 1.f);
            for (int g = g0; g < kg.n && kg.k[g] <= (int)lane + 1; ++g)
                if (kg.k[g] == (int)lane + 1)
                    k_scores[(int64_t)g * 4 * n + 3 * n + qorig] = (float)((double)qs * kKnnQuantum / (lane + 1));
        }
    }
}

// ---- the k grid for k_max > 32: one CTA per object -----------------------------------------

constexpr int kKnnThreads = 256;

// Ascending bitonic sort of len (a power of two) keys by the whole CTA; ends synchronised.
__device__ void bitonic_sort(unsigned long long *a, int len)
{
    for (int size = 2; size <= len; size <<= 1)
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int t = threadIdx.x; t < (len >> 1); t += blockDim.x) {
                const int lo = ((t & ~(stride - 1)) << 1) | (t & (stride - 1));
                const int hi = lo + stride;
                const bool up = (lo & size) == 0;
                const unsigned long long a0 = a[lo], a1 = a[hi];
                if ((a0 > a1) == up) {
                    a[lo] = a1;
                    a[hi] = a0;
                }
            }
            __syncthreads();
        }
}

// Keys (squared distance bits << 32 | original index) order neighbours by
// (distance, index); every key is distinct.  buf holds cap keys (a power of
// two >= 2 k_max and >= 2 kKnnThreads): candidates below the current k_max-th
// key are appended, and when a round could overflow the buffer it is sorted
// and cut back to its k_max smallest.
__global__ void __launch_bounds__(kKnnThreads)
    select_knn_kernel(const float4 *__restrict__ x, int n, uint32_t mask, KGrid kg, int cap, float *k_scores)
{
    extern __shared__ unsigned long long buf[];
    __shared__ float sq[16];
    __shared__ int s_fill;
    __shared__ unsigned long long s_T;
    __shared__ unsigned long long s_warp[kKnnThreads / 32];
    const int p = blockIdx.x;
    const int tid = threadIdx.x;
    const int kmax = kg.k[kg.n - 1];
    if (tid < 16) {
        const float4 q4 = x[row_quad(p, tid >> 2)];
        sq[tid] = (tid & 3) == 0 ? q4.x : (tid & 3) == 1 ? q4.y : (tid & 3) == 2 ? q4.z : q4.w;
    }
    if (tid == 0) {
        s_fill = 0;
        s_T = ~0ull;
    }
    __syncthreads();
    const int qorig = __float_as_int(sq[15]);
    for (int base = 0; base < n; base += kKnnThreads) {
        const int fill0 = s_fill;  // after the last round's barrier: the same in every thread
        __syncthreads();           // ... and read by all before anyone appends again
        if (fill0 > cap - kKnnThreads) {
            for (int t = fill0 + tid; t < cap; t += kKnnThreads) buf[t] = ~0ull;
            __syncthreads();
            bitonic_sort(buf, cap);
            if (tid == 0) {
                s_fill = kmax;
                s_T = buf[kmax - 1];
            }
            __syncthreads();
        }
        const int j = base + tid;
        if (j < n && j != p) {
            float c[16];
            load_row16(x, j, c);
            float acc = 0.f;
#pragma unroll
            for (int f = 14; f >= 0; --f) {
                const float d = c[f] - sq[f];
                acc = fmaf(((mask >> f) & 1u) ? d : 0.f, d, acc);
            }
            const unsigned long long key =
                ((unsigned long long)__float_as_uint(acc) << 32) | (unsigned)__float_as_int(c[15]);
            if (key < s_T) buf[atomicAdd(&s_fill, 1)] = key;
        }
        __syncthreads();
    }
    const int fill = s_fill;  // >= kmax: every other object was a candidate
    int len = 2 * kKnnThreads;
    while (len < fill) len <<= 1;
    for (int t = fill + tid; t < len; t += kKnnThreads) buf[t] = ~0ull;
    __syncthreads();
    bitonic_sort(buf, len);
    // in-degree contributions and the exact distance sums at every k_g
    const int per = (kmax + kKnnThreads - 1) / kKnnThreads;
    const int t0 = tid * per, t1 = min(kmax, t0 + per);
    unsigned long long local = 0ull;
    for (int t = t0; t < t1; ++t) {
        const unsigned long long key = buf[t];
        const int j = (int)(unsigned)(key & 0xffffffffull);
        local += knn_quant(__uint_as_float((unsigned)(key >> 32)));
        if (j >= 0 && j < n) atomicAdd(&k_scores[(int64_t)first_grid_above(kg, t) * 4 * n + 2 * n + j], 1.f);
    }
    // exclusive prefix of the per-thread sums
    unsigned long long inc = local;
    const unsigned lane = dev::lane_id();
    for (int off = 1; off < 32; off <<= 1) {
        const unsigned long long v = __shfl_up_sync(dev::kFull, inc, off);
        if ((int)lane >= off) inc += v;
    }
    if (lane == 31) s_warp[tid >> 5] = inc;
    __syncthreads();
    unsigned long long before = inc - local;
    for (int w = 0; w < (tid >> 5); ++w) before += s_warp[w];
    // the thread whose range ends a k_g writes its mean
    for (int g = 0; g < kg.n; ++g) {
        const int last = kg.k[g] - 1;
        if (last < t0 || last >= t1) continue;
        unsigned long long s = before;
        for (int t = t0; t <= last; ++t) s += knn_quant(__uint_as_float((unsigned)(buf[t] >> 32)));
        k_scores[(int64_t)g * 4 * n + 3 * n + qorig] = (float)((double)s * kKnnQuantum / kg.k[g]);
    }
}

// In-degree at k_g: row 2 summed over slots 0..g.
__global__ void select_k_finish_kernel(int n, int K, float *k_scores)
{
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        float acc = 0.f;
        for (int g = 0; g < K; ++g) {
            float *r = k_scores + (int64_t)g * 4 * n + 2 * n + j;
            acc += *r;
            *r = acc;
        }
    }
}

int knn_cap(int kmax)
{
    int cap = 2 * kKnnThreads;
    while (cap < 2 * kmax) cap <<= 1;
    return cap;
}

}  // namespace

snaps_status launch_select_join(const float4 *x, int64_t n, const SelectSpec &sp, const KGrid &kg,
                                float *eps_scores, float *k_scores, cudaStream_t st)
{
    const unsigned blocks = (unsigned)((n + kSelWarps - 1) / kSelWarps);
    select_join_kernel<<<blocks, kSelWarps * 32, 0, st>>>(x, (int)n, sp, kg, eps_scores, k_scores);
    SNAPS_CHECK_CUDA(cudaGetLastError());
    return SNAPS_OK;
}

snaps_status launch_select_knn(const float4 *x, int64_t n, uint32_t mask, const KGrid &kg, float *k_scores,
                               cudaStream_t st)
{
    const int kmax = kg.k[kg.n - 1];
    if (kg.n < 1 || kmax > kSelectMaxK || kmax > n - 1) {
        set_error("k_max must be in 1..min(%d, n - 1)", kSelectMaxK);
        return SNAPS_EINVAL;
    }
    const int cap = knn_cap(kmax);
    const size_t smem = sizeof(unsigned long long) * (size_t)cap;
    SNAPS_CHECK_CUDA(cudaFuncSetAttribute(select_knn_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    select_knn_kernel<<<(unsigned)n, kKnnThreads, smem, st>>>(x, (int)n, mask, kg, cap, k_scores);
    SNAPS_CHECK_CUDA(cudaGetLastError());
    return SNAPS_OK;
}

snaps_status launch_select_k_finish(int64_t n, const KGrid &kg, float *k_scores, cudaStream_t st)
{
    const unsigned blocks = (unsigned)std::min<int64_t>((n + 255) / 256, 148 * 8);
    select_k_finish_kernel<<<blocks, 256, 0, st>>>((int)n, kg.n, k_scores);
    SNAPS_CHECK_CUDA(cudaGetLastError());
    return SNAPS_OK;
}

}  // namespace snaps

// ---- eps from selectivity (Sec. 3.5.3) ---------------------------------------------------------
//
// Selectivity is the mean number of eps-neighbours per object, itself
// excluded.  Its estimate at radius r from a sample of m objects is the
// number of sample-to-object distances <= r divided by m.  Pass 0 sums those
// distances (exact quantised u64 sum) for their mean eps_mean, the upper bound
// of the search; pass 1 counts them in n_bins bins of width eps_mean / n_bins
// over [0, eps_mean); the cumulative counts then give, for each target, the
// first bin edge at which the estimate reaches it.

namespace snaps {
namespace {

constexpr int kHistThreads = 256;
constexpr int kHistQueries = 16;  // sampled objects per block, staged in shared memory

// inv[orig] = stored row of every object.
__global__ void inverse_kernel(const float4 *__restrict__ x, int n, int32_t *inv)
{
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x)
        inv[__float_as_int(x[row_quad(p, 3)].w)] = p;
}

__device__ __forceinline__ double hist_eps_mean(const unsigned long long *sum, double count)
{
    return count > 0 ? ((double)*sum * kSelQuantum) / count : 0.0;
}

// Block (g, c): sampled objects kHistQueries g .. +kHistQueries-1 (original
// indices floor(s n / m)) against the c-th slice of all rows.
template <int PASS>
__global__ void __launch_bounds__(kHistThreads)
    selectivity_kernel(const float4 *__restrict__ x, const int32_t *__restrict__ inv, int n, int m,
                       uint32_t mask, int n_bins, double count, unsigned long long *acc)
{
    __shared__ unsigned sh[PASS == 1 ? kSelectHistBins : 1];
    __shared__ float sq[kHistQueries][16];
    __shared__ int srow[kHistQueries];
    __shared__ unsigned long long ssum[kHistThreads / 32];
    if (PASS == 1)
        for (int b = threadIdx.x; b < n_bins; b += blockDim.x) sh[b] = 0u;
    const int s0 = blockIdx.x * kHistQueries;
    const int qs = min(kHistQueries, m - s0);
    for (int t = threadIdx.x; t < kHistQueries * 16; t += blockDim.x) {
        const int s = t >> 4, f = t & 15;
        float v = 0.f;
        if (s < qs) {
            const int row = inv[(int)(((long long)(s0 + s) * n) / m)];
            if (f == 0) srow[s] = row;
            const float4 q4 = x[row_quad(row, f >> 2)];
            v = (f & 3) == 0 ? q4.x : (f & 3) == 1 ? q4.y : (f & 3) == 2 ? q4.z : q4.w;
        } else if (f == 0) {
            srow[s] = -1;
        }
        sq[s][f] = v;
    }
    __syncthreads();
    float inv_bin = 0.f;
    if (PASS == 1) {
        const float em = (float)hist_eps_mean(acc + kSelectHistBins, count);
        inv_bin = em > 0.f ? (float)n_bins / em : 0.f;
    }
    const int per = (n + gridDim.y - 1) / gridDim.y;
    const int j0 = blockIdx.y * per, j1 = min(n, j0 + per);
    unsigned long long qsum = 0ull;
    for (int j = j0 + threadIdx.x; j < j1; j += blockDim.x) {
        float c[16];
        load_row16(x, j, c);
        for (int s = 0; s < qs; ++s) {
            if (j == srow[s]) continue;  // never its own neighbour
            float acc2 = 0.f;
#pragma unroll
            for (int f = 14; f >= 0; --f) {
                const float d = c[f] - sq[s][f];
                acc2 = fmaf(((mask >> f) & 1u) ? d : 0.f, d, acc2);
            }
            const float d = sqrtf(acc2);
            if (PASS == 0) {
                qsum += (unsigned long long)__float2uint_rn(d * (float)(1.0 / kSelQuantum));
            } else {
                const int b = (int)fminf(d * inv_bin, (float)n_bins);  // n_bins: beyond eps_mean
                if (b < n_bins) atomicAdd(&sh[b], 1u);
            }
        }
    }
    if (PASS == 0) {
        for (int o = 16; o > 0; o >>= 1) qsum += __shfl_xor_sync(dev::kFull, qsum, o);
        if (dev::lane_id() == 0) ssum[threadIdx.x >> 5] = qsum;
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned long long t = 0ull;
            for (int w = 0; w < kHistThreads / 32; ++w) t += ssum[w];
            atomicAdd(acc + kSelectHistBins, t);
        }
    } else {
        __syncthreads();
        for (int b = threadIdx.x; b < n_bins; b += blockDim.x)
            if (sh[b]) atomicAdd(&acc[b], (unsigned long long)sh[b]);
    }
}

// One warp: lane t finds, for target t, the first bin b whose cumulative count
// reaches target[t] * m and writes (b + 1) * eps_mean / n_bins (eps_mean when
// no bin does); lane 0 also writes eps_mean.
__global__ void selectivity_pick_kernel(const unsigned long long *__restrict__ acc, int n_bins, double count,
                                        SelectivityTargets tg, float *eps, float *eps_mean)
{
    const int t = threadIdx.x;
    const double em = hist_eps_mean(acc + kSelectHistBins, count);
    if (t == 0 && eps_mean) *eps_mean = (float)em;
    if (t >= tg.n) return;
    const double need = tg.target[t] * (double)tg.m;
    unsigned long long c = 0ull;
    double r = em;
    for (int b = 0; b < n_bins; ++b) {
        c += acc[b];
        if ((double)c >= need) {
            r = (double)(b + 1) * em / (double)n_bins;
            break;
        }
    }
    eps[t] = (float)r;
}

}  // namespace

size_t selectivity_scratch_bytes(int64_t n)
{
    return sizeof(unsigned long long) * (kSelectHistBins + 1) + sizeof(int32_t) * (size_t)n + 256;
}

snaps_status launch_selectivity(const float4 *x, int64_t n, uint32_t mask, int n_bins, const SelectivityTargets &tg,
                                void *scratch, float *eps, float *eps_mean, cudaStream_t st)
{
    if (n_bins < 1 || n_bins > kSelectHistBins) {
        set_error("n_bins must be in 1..%d", kSelectHistBins);
        return SNAPS_EINVAL;
    }
    auto *acc = (unsigned long long *)scratch;
    auto *inv = (int32_t *)(acc + kSelectHistBins + 1);
    inverse_kernel<<<(unsigned)std::min<int64_t>((n + 255) / 256, 148 * 8), 256, 0, st>>>(x, (int)n, inv);
    SNAPS_CHECK_CUDA(cudaGetLastError());
    SNAPS_CHECK_CUDA(cudaMemsetAsync(acc, 0, sizeof(unsigned long long) * (kSelectHistBins + 1), st));
    const double count = (double)tg.m * (double)(n - 1);
    // about 4 blocks per SM over the (sample group, slice) grid
    const int groups = (tg.m + kHistQueries - 1) / kHistQueries;
    const int slices = (int)std::max<int64_t>(
        1, std::min<int64_t>((148 * 4 + groups - 1) / groups, (n + kHistThreads - 1) / kHistThreads));
    const dim3 grid((unsigned)groups, (unsigned)slices);
    selectivity_kernel<0><<<grid, kHistThreads, 0, st>>>(x, inv, (int)n, tg.m, mask, n_bins, count, acc);
    SNAPS_CHECK_CUDA(cudaGetLastError());
    selectivity_kernel<1><<<grid, kHistThreads, 0, st>>>(x, inv, (int)n, tg.m, mask, n_bins, count, acc);
    SNAPS_CHECK_CUDA(cudaGetLastError());
    selectivity_pick_kernel<<<1, 32, 0, st>>>(acc, n_bins, count, tg, eps, eps_mean);
    SNAPS_CHECK_CUDA(cudaGetLastError());
    return SNAPS_OK;
}

}  // namespace snaps
