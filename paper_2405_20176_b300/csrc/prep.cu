// Population preparation: normalisation (Sec. 3.3), missing values (Sec. 2.1),
// the sort-by-cell row order and the per-chunk row copies of the
// subspace-batched join.

#include <math_constants.h>

#include <algorithm>

#include "device.cuh"
#include "prep.cuh"

namespace snaps {
namespace {

// ---- normalisation -------------------------------------------------------------

constexpr int kStatThreads = 1024;

// One block per feature: FP64 min, max, and mean of the non-NaN values, and a
// flag for values the flags do not allow (NaN without NaN->mean, +-inf).
__global__ void __launch_bounds__(kStatThreads)
    col_stats_kernel(const float *__restrict__ in, int64_t n, int f, int nan_ok,
                     ColStats *__restrict__ stats, unsigned *__restrict__ bad)
{
    const int c = blockIdx.x;
    double lo = CUDART_INF, hi = -CUDART_INF, sum = 0.0;
    long long cnt = 0;
    unsigned flag = 0;
    for (int64_t r = threadIdx.x; r < n; r += blockDim.x) {
        const float v = in[r * f + c];
        if (isnan(v)) {
            if (!nan_ok) flag = 1;
            continue;
        }
        if (isinf(v)) {
            flag = 1;
            continue;
        }
        const double d = (double)v;
        lo = fmin(lo, d);
        hi = fmax(hi, d);
        sum += d;
        ++cnt;
    }
    __shared__ double s_lo[32], s_hi[32], s_sum[32];
    __shared__ long long s_cnt[32];
    __shared__ unsigned s_bad[32];
    for (int o = 16; o > 0; o >>= 1) {
        lo = fmin(lo, __shfl_xor_sync(dev::kFull, lo, o));
        hi = fmax(hi, __shfl_xor_sync(dev::kFull, hi, o));
        sum += __shfl_xor_sync(dev::kFull, sum, o);
        cnt += __shfl_xor_sync(dev::kFull, cnt, o);
        flag |= __shfl_xor_sync(dev::kFull, flag, o);
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) {
        s_lo[w] = lo;
        s_hi[w] = hi;
        s_sum[w] = sum;
        s_cnt[w] = cnt;
        s_bad[w] = flag;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const int nw = blockDim.x >> 5;
        for (int i = 1; i < nw; ++i) {
            lo = fmin(lo, s_lo[i]);
            hi = fmax(hi, s_hi[i]);
            sum += s_sum[i];
            cnt += s_cnt[i];
            flag |= s_bad[i];
        }
        stats[c].lo = lo;
        stats[c].hi = hi;
        stats[c].mean = cnt > 0 ? sum / (double)cnt : 0.0;
        stats[c].count = cnt;
        if (flag) atomicOr(bad, 1u);
    }
}

// Write the population rows: (x - lo) / (hi - lo) in FP64 rounded to FP32
// (or the value itself without normalisation), NaN -> the column mean first,
// zeros beyond f, +inf rows for the padding.
__global__ void normalise_rows_kernel(const float *__restrict__ in, int64_t n, int64_t n_pad,
                                      int f, uint32_t flags, const ColStats *__restrict__ stats,
                                      float4 *__restrict__ out)
{
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n_pad;
         r += (int64_t)gridDim.x * blockDim.x) {
        float v[16];
        if (r < n) {
#pragma unroll
            for (int c = 0; c < 16; ++c) {
                float y = 0.f;
                if (c < f) {
                    double d = (double)in[r * f + c];
                    if (isnan(d)) d = stats[c].mean;
                    if (flags & SNAPS_NORM_MINMAX) {
                        const double span = stats[c].hi - stats[c].lo;
                        y = span > 0.0 ? (float)((d - stats[c].lo) / span) : 0.f;
                    } else {
                        y = (float)d;
                    }
                }
                v[c] = y;
            }
            v[15] = __int_as_float((int)r);  // the object's original index (features are 0..14)
        } else {
#pragma unroll
            for (int c = 0; c < 16; ++c) v[c] = CUDART_INF_F;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q)
            out[row_quad(r, q)] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
    }
}

// Rows come out in their original order: float 15 of a stored row holds the
// object's original index.
__global__ void unpack_rows_kernel(const float4 *__restrict__ x, int64_t n, int f,
                                   float *__restrict__ out)
{
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n;
         r += (int64_t)gridDim.x * blockDim.x) {
        const int64_t o = __float_as_int(x[row_quad(r, 3)].w);
        for (int c = 0; c < f; ++c) {
            const float4 v = x[row_quad(r, c / 4)];
            const int e = c % 4;
            out[o * f + c] = e == 0 ? v.x : e == 1 ? v.y : e == 2 ? v.z : v.w;
        }
    }
}

// Cell key of every row for the sort-by-cell index: each of the 15 features
// quantised to 2 bits (4 cells per unit range), bits interleaved from the most
// significant level down, so rows sharing a key prefix are close in every
// feature.
__global__ void cell_key_kernel(const float4 *__restrict__ x, int64_t n, KeyRange kr,
                                uint32_t *__restrict__ keys, int32_t *__restrict__ idx)
{
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n;
         r += (int64_t)gridDim.x * blockDim.x) {
        uint32_t q[15];
#pragma unroll
        for (int qq = 0; qq < 4; ++qq) {
            const float4 v = x[row_quad(r, qq)];
            const float e[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int f = 4 * qq + u;
                if (f < 15) q[f] = (uint32_t)fminf(fmaxf((e[u] - kr.lo[f]) * kr.scale[f] * 4.f, 0.f), 3.f);
            }
        }
        uint32_t key = 0;
#pragma unroll
        for (int b = 1; b >= 0; --b)
#pragma unroll
            for (int f = 0; f < 15; ++f) key = (key << 1) | ((q[f] >> b) & 1u);
        keys[r] = key;
        idx[r] = (int32_t)r;
    }
}

// Chunk keys: Morton order over the chunk's high features (see prep.cuh).
__global__ void chunk_key_kernel(const float4 *__restrict__ x, int64_t n, int f,
                                 const TreeChunk *__restrict__ chunks, int n_chunks, KeyRange kr,
                                 uint64_t *__restrict__ keys, int32_t *__restrict__ vals)
{
    const int64_t total = n * (int64_t)n_chunks;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int g = (int)(e / n);
        const int64_t r = e - (int64_t)g * n;
        const uint32_t high = chunks[g].high;
        float v[16];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float4 t = x[row_quad(r, q)];
            v[4 * q + 0] = t.x;
            v[4 * q + 1] = t.y;
            v[4 * q + 2] = t.z;
            v[4 * q + 3] = t.w;
        }
        // the key's features: H's, or the low ones when H is empty
        const uint32_t fmask = high ? (high << kTreeLowBits) : ((1u << min(f, kTreeLowBits)) - 1u);
        const int nd = __popc(fmask);
        const int bits = min(10, 30 / nd);
        uint32_t q[15];
#pragma unroll
        for (int c = 0; c < 15; ++c) {
            const float u = (v[c] - kr.lo[c]) * kr.scale[c];
            const float top = (float)((1u << bits) - 1u);
            q[c] = (uint32_t)fminf(fmaxf(u * (float)(1u << bits), 0.f), top);
        }
        uint32_t key = 0;
        for (int b = bits - 1; b >= 0; --b)
#pragma unroll
            for (int c = 14; c >= 0; --c)
                if ((fmask >> c) & 1u) key = (key << 1) | ((q[c] >> b) & 1u);
        keys[e] = ((uint64_t)g << 32) | key;
        vals[e] = (int32_t)r;
    }
}

// out[g] <- the rows x[perm[g * n + p]], p = 0..n_pad-1, in the pair-planar
// layout (one thread per row pair a = 64s + l, b = a + 32); padding rows +inf.
__global__ void gather_chunks_kernel(const float4 *__restrict__ x, const int32_t *__restrict__ perm,
                                     const TreeChunk *__restrict__ chunks, int64_t n, int64_t n_pad, int n_chunks,
                                     float4 *__restrict__ out)
{
    const int64_t pairs = n_pad / 2;  // per chunk
    const int64_t total = pairs * (int64_t)n_chunks;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t g = e / pairs;
        const int64_t t = e - g * pairs;  // pair index: step t / 32, lane t % 32
        const int64_t pa = (t >> 5) * 64 + (t & 31), pb = pa + 32;
        float4 ra[4], rb[4];
        const float inf = CUDART_INF_F;
        const int64_t oa = pa < n ? (perm ? perm[g * n + pa] : pa) : -1;
        const int64_t ob = pb < n ? (perm ? perm[g * n + pb] : pb) : -1;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            ra[q] = oa >= 0 ? x[row_quad(oa, q)] : make_float4(inf, inf, inf, inf);
            rb[q] = ob >= 0 ? x[row_quad(ob, q)] : make_float4(inf, inf, inf, inf);
        }
        float va[16] = {ra[0].x, ra[0].y, ra[0].z, ra[0].w, ra[1].x, ra[1].y, ra[1].z, ra[1].w,
                        ra[2].x, ra[2].y, ra[2].z, ra[2].w, ra[3].x, ra[3].y, ra[3].z, ra[3].w};
        float vb[16] = {rb[0].x, rb[0].y, rb[0].z, rb[0].w, rb[1].x, rb[1].y, rb[1].z, rb[1].w,
                        rb[2].x, rb[2].y, rb[2].z, rb[2].w, rb[3].x, rb[3].y, rb[3].z, rb[3].w};
        if (chunks) {
            // compact the chunk's high features into floats 5.. in descending
            // feature order; the floats after them are 0 (padding rows: +inf)
            const uint32_t high = chunks[g].high;
            float ca[10], cb[10];
            int r = 0;
#pragma unroll
            for (int f = 14; f >= 5; --f)
                if ((high >> (f - 5)) & 1u) {
                    ca[r] = va[f];
                    cb[r] = vb[f];
                    ++r;
                }
            for (; r < 10; ++r) {
                ca[r] = oa >= 0 ? 0.f : inf;
                cb[r] = ob >= 0 ? 0.f : inf;
            }
#pragma unroll
            for (int c = 0; c < 10; ++c) {
                va[5 + c] = ca[c];
                vb[5 + c] = cb[c];
            }
        }
        float4 *dst = out + g * n_pad * 4;
#pragma unroll
        for (int q = 0; q < 8; ++q)
            dst[pair_plane(pa, q)] = make_float4(va[2 * q], vb[2 * q], va[2 * q + 1], vb[2 * q + 1]);
    }
}

// One warp per (copy, step): lane l holds rows 64s + l and 64s + 32 + l.
__global__ void chunk_boxes_kernel(const float4 *__restrict__ copies, int64_t n_pad, int n_chunks,
                                   float2 *__restrict__ boxes)
{
    const int64_t n_steps = n_pad / 64;
    const int64_t total = n_steps * n_chunks;
    const unsigned lane = threadIdx.x & 31u;
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t e = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; e < total; e += warps) {
        const int64_t g = e / n_steps, st = e - g * n_steps;
        const float4 *src = copies + g * n_pad * 4;
#pragma unroll
        for (int b = 0; b < 10; ++b) {
            const int f = 5 + b;
            const float4 v = src[pair_plane(st * 64 + lane, f >> 1)];
            float lo = (f & 1) ? fminf(v.z, v.w) : fminf(v.x, v.y);
            float hi = (f & 1) ? fmaxf(v.z, v.w) : fmaxf(v.x, v.y);
            for (int o = 16; o > 0; o >>= 1) {
                lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
                hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
            }
            if (lane == 0) boxes[(g * 10 + b) * n_steps + st] = make_float2(lo, hi);
        }
    }
}

// Sorted row p <- original row perm[p]; padding rows are +inf.
__global__ void gather_rows_kernel(const float4 *__restrict__ src, const int32_t *__restrict__ perm,
                                   int64_t n, int64_t n_pad, float4 *__restrict__ dst)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n_pad;
         p += (int64_t)gridDim.x * blockDim.x) {
        if (p < n) {
            const int64_t o = perm[p];
#pragma unroll
            for (int q = 0; q < 4; ++q) dst[row_quad(p, q)] = src[row_quad(o, q)];
        } else {
            const float inf = CUDART_INF_F;
#pragma unroll
            for (int q = 0; q < 4; ++q) dst[row_quad(p, q)] = make_float4(inf, inf, inf, inf);
        }
    }
}

}  // namespace

snaps_status launch_normalise(const float *in_dev, int64_t n, int64_t n_pad, int f,
                              uint32_t flags, ColStats *stats, unsigned *bad, float4 *out,
                              cudaStream_t st)
{
    SNAPS_CHECK_CUDA(cudaMemsetAsync(bad, 0, sizeof(unsigned), st));
    col_stats_kernel<<<f, kStatThreads, 0, st>>>(in_dev, n, f, (flags & SNAPS_NAN_TO_MEAN) ? 1 : 0,
                                                 stats, bad);
    SNAPS_CHECK_CUDA(cudaGetLastError());
    const int64_t blocks = std::min<int64_t>((n_pad + 255) / 256, 148 * 16);
    normalise_rows_kernel<<<(unsigned)blocks, 256, 0, st>>>(in_dev, n, n_pad, f, flags, stats, out);
    SNAPS_CHECK_CUDA(cudaGetLastError());
    return SNAPS_OK;
}

snaps_status launch_cell_keys(const float4 *x, int64_t n, const KeyRange &kr, uint32_t *keys,
                              int32_t *idx, cudaStream_t st)
{
    const int64_t blocks = std::min<int64_t>((n + 255) / 256, 148 * 16);
    cell_key_kernel<<<(unsigned)blocks, 256, 0, st>>>(x, n, kr, keys, idx);
    SNAPS_CHECK_CUDA(cudaGetLastError());
    return SNAPS_OK;
}

snaps_status launch_chunk_keys(const float4 *x, int64_t n, int f, const TreeChunk *chunks, int n_chunks,
                               const KeyRange &kr, uint64_t *keys, int32_t *vals, cudaStream_t st)
{
    const int64_t total = n * (int64_t)n_chunks;
    const int64_t blocks = std::min<int64_t>((total + 255) / 256, 148 * 16);
    chunk_key_kernel<<<(unsigned)blocks, 256, 0, st>>>(x, n, f, chunks, n_chunks, kr, keys, vals);
    SNAPS_CHECK_CUDA(cudaGetLastError());
    return SNAPS_OK;
}

snaps_status launch_chunk_boxes(const float4 *copies, int64_t n_pad, int n_chunks, float2 *boxes,
                                cudaStream_t st)
{
    const int64_t warps = (n_pad / 64) * n_chunks;
    const unsigned blocks = (unsigned)std::min<int64_t>((warps * 32 + 255) / 256, 148 * 16);
    chunk_boxes_kernel<<<blocks, 256, 0, st>>>(copies, n_pad, n_chunks, boxes);
    SNAPS_CHECK_CUDA(cudaGetLastError());
    return SNAPS_OK;
}

snaps_status launch_gather_chunks(const float4 *x, const int32_t *perm, const TreeChunk *chunks, int64_t n,
                                  int64_t n_pad, int n_chunks, float4 *out, cudaStream_t st)
{
    const int64_t total = n_pad / 2 * (int64_t)n_chunks;
    const int64_t blocks = std::min<int64_t>((total + 255) / 256, 148 * 16);
    gather_chunks_kernel<<<(unsigned)blocks, 256, 0, st>>>(x, perm, chunks, n, n_pad, n_chunks, out);
    SNAPS_CHECK_CUDA(cudaGetLastError());
    return SNAPS_OK;
}

snaps_status launch_gather_rows(const float4 *src, const int32_t *perm, int64_t n, int64_t n_pad,
                                float4 *dst, cudaStream_t st)
{
    const int64_t blocks = std::min<int64_t>((n_pad + 255) / 256, 148 * 16);
    gather_rows_kernel<<<(unsigned)blocks, 256, 0, st>>>(src, perm, n, n_pad, dst);
    SNAPS_CHECK_CUDA(cudaGetLastError());
    return SNAPS_OK;
}

snaps_status launch_unpack(const float4 *x, int64_t n, int f, float *out, cudaStream_t st)
{
    const int64_t blocks = std::min<int64_t>((n + 255) / 256, 148 * 16);
    unpack_rows_kernel<<<(unsigned)blocks, 256, 0, st>>>(x, n, f, out);
    SNAPS_CHECK_CUDA(cudaGetLastError());
    return SNAPS_OK;
}

}  // namespace snaps
