// Grid-indexed self-join for low-dimensional subspaces: DSSJ (Sec. 3.5) and
// kNNSJ (Sec. 3.6) through a sort-by-cell index (the paper indexes up to
// c <= 6 of a subspace's dimensions, Sec. 3.8.1; here up to three of the <= 4
// features of a subspace, the highest ones).
//
// Index.  For a subspace S with d <= 4 features, every object gets the cell
// (floor((x_f - lo_f) / w)) over the D = min(d, 3) highest features f of S on
// a grid of cell width w >= eps (widened where needed so that the grid has at
// most 2^22 cells), and the objects are sorted by
// cell id (row-major, the lowest feature fastest).  cell_start[c] is the first
// sorted position of cell c, so the objects of a run of cells along the
// fastest dimension are one contiguous range.  The sorted objects are stored
// as one float4 each (the subspace's features from the highest index down,
// zero padded) plus their original indices.
//
// Join.  A warp owns one query.  Every eps-neighbour lies in the 3^D block of
// cells around the query's own (w >= eps, and w carries a 2^-10 margin so
// that rounding in the cell computation cannot separate two points by more
// than one cell), so the warp scans those ranges -- lanes striding over the
// candidates -- counts eps-neighbours with ballot/popc, sums their quantised
// distances exactly and keeps the kNN list warp-cooperatively.  When the k-th
// distance still exceeds the cell width afterwards (sparse regions, outliers),
// rings of cells at Chebyshev distance r = 2, 3, ... are scanned for the kNN
// list until (r - 1) w exceeds it: no object outside the scanned cells can be
// nearer (a subspace distance is at least the distance over the index
// features).  Distances are the library's canonical FP32 fold (FMAs from the
// highest feature down), so results equal every other path's bit for bit.

#include <cub/cub.cuh>
#include <math_constants.h>

#include <algorithm>

#include "device.cuh"
#include "grid.cuh"

namespace snaps {
namespace {

constexpr int kGridWarps = 8;

__device__ __forceinline__ int cell_of(float v, float lo, float inv_w, int nc)
{
    const int c = (int)floorf((v - lo) * inv_w);
    return c < 0 ? 0 : (c >= nc ? nc - 1 : c);
}

// Cell coordinates of a gathered point (components in descending feature
// order: the index dimensions are the first D of x, y, z).
__device__ __forceinline__ void point_cell(const GridSpec &g, float4 p, int (&c)[3])
{
    const float v[3] = {p.x, p.y, p.z};
#pragma unroll
    for (int t = 0; t < 3; ++t) c[t] = t < g.D ? cell_of(v[t], g.lo[t], g.inv_w, g.nc[t]) : 0;
}

__device__ __forceinline__ int cell_lin(const GridSpec &g, const int (&c)[3])
{
    int id = 0;
#pragma unroll
    for (int t = 0; t < 3; ++t)
        if (t < g.D) id = id * g.nc[t] + c[t];
    return id;
}

// The subspace's features of stored row i, highest feature first, zero padded.
__device__ __forceinline__ float4 gather_point(const float4 *__restrict__ x, int64_t i, const GridSpec &g)
{
    float f[16];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const float4 t = x[row_quad(i, q)];
        f[4 * q + 0] = t.x;
        f[4 * q + 1] = t.y;
        f[4 * q + 2] = t.z;
        f[4 * q + 3] = t.w;
    }
    float v[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        const int ft = g.feat[t];
        float a = 0.f;
#pragma unroll
        for (int q = 0; q < 15; ++q) a = (q == ft) ? f[q] : a;
        v[t] = t < g.d ? a : 0.f;
    }
    return make_float4(v[0], v[1], v[2], v[3]);
}

__global__ void grid_keys_kernel(const float4 *__restrict__ x, int64_t n, GridSpec g, uint32_t *keys,
                                 int32_t *vals)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int c[3];
        point_cell(g, gather_point(x, i, g), c);
        keys[i] = (uint32_t)cell_lin(g, c);
        vals[i] = (int32_t)i;
    }
}

// cell_start[c] = first sorted position whose key is >= c, for c = 0..ncells.
__global__ void grid_starts_kernel(const uint32_t *__restrict__ keys, int64_t n, int ncells, int32_t *start)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p <= n; p += (int64_t)gridDim.x * blockDim.x) {
        const int hi = p < n ? (int)keys[p] : ncells;
        const int lo = p > 0 ? (int)keys[p - 1] + 1 : 0;
        for (int c = lo; c <= hi; ++c) start[c] = (int32_t)p;
    }
}

__global__ void grid_gather_kernel(const float4 *__restrict__ x, const int32_t *__restrict__ perm, int64_t n,
                                   GridSpec g, float4 *pts, int32_t *orig)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = perm[p];
        const float4 v = gather_point(x, i, g);
        if (g.d <= 2)
            reinterpret_cast<float2 *>(pts)[p] = make_float2(v.x, v.y);  // 8-byte points
        else
            pts[p] = v;
        orig[p] = __float_as_int(x[row_quad(i, 3)].w);
    }
}

__device__ __forceinline__ float fold4(float4 a, float4 q)
{
    // canonical order: highest feature first (component x), padding adds exact zeros
    float acc = 0.f;
    float d = a.x - q.x;
    acc = fmaf(d, d, acc);
    d = a.y - q.y;
    acc = fmaf(d, d, acc);
    d = a.z - q.z;
    acc = fmaf(d, d, acc);
    d = a.w - q.w;
    acc = fmaf(d, d, acc);
    return acc;
}

// Subspaces of <= 2 features keep 8-byte points; the fold is the float4 fold
// without the two padding FMAs, which add exact zeros.
__device__ __forceinline__ float fold4(float2 a, float2 q)
{
    float acc = 0.f;
    float d = a.x - q.x;
    acc = fmaf(d, d, acc);
    d = a.y - q.y;
    acc = fmaf(d, d, acc);
    return acc;
}

__device__ __forceinline__ void point_cell(const GridSpec &g, float2 p, int (&c)[3])
{
    point_cell(g, make_float4(p.x, p.y, 0.f, 0.f), c);
}

// Per-warp state of one query's join.
constexpr int kScanUnroll = 4;  // candidate batches of 32 loaded ahead in a scan

template <typename V>
struct QueryState {
    V q;
    int qrow;                // the query's position in cell order
    int qorig;
    float e2;
    float esc;
    int k;
    float T;                 // current k-th squared distance (warp-uniform)
    float my_d;              // lane t < k holds list entry t
    int my_j;
    unsigned cnt;            // eps-neighbours (warp-uniform)
    unsigned long long qs;   // this lane's quantised distance sum
};

// Scan sorted positions [beg, end) for the eps join (when do_eps) and the kNN list.
template <typename V>
__device__ __forceinline__ void scan_range(const V *__restrict__ pts, const int32_t *__restrict__ orig,
                                           int beg, int end, QueryState<V> &st, bool do_eps)
{
    const unsigned lane = dev::lane_id();
    for (int b0 = beg; b0 < end; b0 += 32 * kScanUnroll) {
        // the rows of kScanUnroll batches are in flight before any is used
        V pv[kScanUnroll];
#pragma unroll
        for (int u = 0; u < kScanUnroll; ++u) {
            const int j = b0 + 32 * u + (int)lane;
            pv[u] = j < end ? pts[j] : V{};
        }
#pragma unroll
        for (int u = 0; u < kScanUnroll; ++u) {
        const int j = b0 + 32 * u + (int)lane;
        const bool valid = j < end && j != st.qrow;  // never its own neighbour
        const float d2 = valid ? fold4(pv[u], st.q) : CUDART_INF_F;
        if (do_eps) {
            const bool e = d2 <= st.e2;
            st.cnt += __popc(__ballot_sync(dev::kFull, e));
            if (e) st.qs += dev::eps_quant(d2, st.esc);
        }
        if (st.k > 0) {
            // candidates at or below the k-th distance are rare once the list
            // is full: their original indices and the exact rule (a tie goes
            // to the smaller original index) are taken only then
            const bool cand = valid && d2 <= st.T;
            if (__ballot_sync(dev::kFull, cand)) {
                const int oj = cand ? orig[j] : 0x7fffffff;
                const int jk = __shfl_sync(dev::kFull, st.my_j, st.k - 1);
                const bool want = cand && (d2 < st.T || oj < jk);
                const unsigned bal = __ballot_sync(dev::kFull, want);
                if (bal) dev::list_insert(bal, d2, oj, st.my_d, st.my_j, st.k, st.T);
            }
        }
        }
    }
}

// Scan the cells of index-space row (c0, c1) [the leading D - 1 coordinates]
// from last-dimension cell a to b (inclusive, clipped).
template <typename V>
__device__ __forceinline__ void scan_cells(const GridSpec &g, const V *pts, const int32_t *orig,
                                           const int32_t *start, int i0, int i1, int a, int b,
                                           QueryState<V> &st, bool do_eps)
{
    const int nl = g.D == 2 ? g.nc[1] : g.nc[2];
    a = max(a, 0);
    b = min(b, nl - 1);
    if (a > b) return;
    const int la = g.D == 2 ? i0 * g.nc[1] + a : (i0 * g.nc[1] + i1) * g.nc[2] + a;
    scan_range(pts, orig, start[la], start[la + (b - a) + 1], st, do_eps);
}

template <typename V>
__global__ void __launch_bounds__(kGridWarps * 32, 2)
    grid_join_kernel(const V *__restrict__ pts, const int32_t *__restrict__ orig,
                     const int32_t *__restrict__ start, int n, GridSpec g, int k, JoinOut o)
{
    const int warp = threadIdx.x >> 5;
    const unsigned lane = dev::lane_id();
    const int p = blockIdx.x * kGridWarps + warp;
    if (p >= n) return;
    QueryState<V> st;
    st.q = pts[p];
    st.qrow = p;
    st.qorig = orig[p];
    st.e2 = g.eps2;
    st.esc = dev::eps_scale(g.eps2).scale;
    st.k = k;
    st.T = k > 0 ? CUDART_INF_F : -CUDART_INF_F;
    st.my_d = CUDART_INF_F;
    st.my_j = 0x7fffffff;
    st.cnt = 0;
    st.qs = 0ull;
    int c[3];
    point_cell(g, st.q, c);
    const bool do_eps = g.eps2 >= 0.f;
    const int D = g.D;
    // the (2R + 1)^D block: every eps-neighbour is inside it.  The query's own
    // cell goes first, so that the kNN threshold is tight before the rest is scanned.
    const int R = g.R;
    const int cl = D == 2 ? c[1] : c[2];
    scan_cells(g, pts, orig, start, c[0], c[1], cl, cl, st, do_eps);
    if (D == 2) {
        for (int i0 = max(c[0] - R, 0); i0 <= min(c[0] + R, g.nc[0] - 1); ++i0) {
            if (i0 == c[0]) {
                scan_cells(g, pts, orig, start, i0, 0, cl - R, cl - 1, st, do_eps);
                scan_cells(g, pts, orig, start, i0, 0, cl + 1, cl + R, st, do_eps);
            } else {
                scan_cells(g, pts, orig, start, i0, 0, cl - R, cl + R, st, do_eps);
            }
        }
    } else {
        for (int i0 = max(c[0] - R, 0); i0 <= min(c[0] + R, g.nc[0] - 1); ++i0)
            for (int i1 = max(c[1] - R, 0); i1 <= min(c[1] + R, g.nc[1] - 1); ++i1) {
                if (i0 == c[0] && i1 == c[1]) {
                    scan_cells(g, pts, orig, start, i0, i1, cl - R, cl - 1, st, do_eps);
                    scan_cells(g, pts, orig, start, i0, i1, cl + 1, cl + R, st, do_eps);
                } else {
                    scan_cells(g, pts, orig, start, i0, i1, cl - R, cl + R, st, do_eps);
                }
            }
    }
    // kNN rings: objects in ring r are at least (r - 1) w away
    if (k > 0) {
        const int span = max(g.nc[0], max(D > 1 ? g.nc[1] : 0, D > 2 ? g.nc[2] : 0));
        for (int r = R + 1; r <= span; ++r) {
            const float reach = (float)(r - 1) * g.w * (1.f - 1.f / 1024.f);
            if (reach * reach > st.T) break;
            if (D == 2) {
                for (int i0 = c[0] - r; i0 <= c[0] + r; ++i0) {
                    if (i0 < 0 || i0 >= g.nc[0]) continue;
                    if (abs(i0 - c[0]) == r) {
                        scan_cells(g, pts, orig, start, i0, 0, c[1] - r, c[1] + r, st, false);
                    } else {
                        scan_cells(g, pts, orig, start, i0, 0, c[1] - r, c[1] - r, st, false);
                        scan_cells(g, pts, orig, start, i0, 0, c[1] + r, c[1] + r, st, false);
                    }
                }
            } else {
                for (int i0 = c[0] - r; i0 <= c[0] + r; ++i0) {
                    if (i0 < 0 || i0 >= g.nc[0]) continue;
                    for (int i1 = c[1] - r; i1 <= c[1] + r; ++i1) {
                        if (i1 < 0 || i1 >= g.nc[1]) continue;
                        if (max(abs(i0 - c[0]), abs(i1 - c[1])) == r) {
                            scan_cells(g, pts, orig, start, i0, i1, c[2] - r, c[2] + r, st, false);
                        } else {
                            scan_cells(g, pts, orig, start, i0, i1, c[2] - r, c[2] - r, st, false);
                            scan_cells(g, pts, orig, start, i0, i1, c[2] + r, c[2] + r, st, false);
                        }
                    }
                }
            }
        }
    }
    // ---- results --------------------------------------------------------------------------------
    unsigned long long qs = st.qs;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) qs += __shfl_xor_sync(dev::kFull, qs, off);
    const int oi = st.qorig;
    float *sc = o.scores + (int64_t)g.slot * 4 * n;
    if (lane == 0) {
        sc[oi] = do_eps ? (float)st.cnt : 0.f;
        sc[n + oi] = do_eps ? dev::eps_mean(qs, (int)st.cnt, st.esc) : 0.f;
        if (o.eps_count) o.eps_count[(int64_t)g.slot * n + oi] = do_eps ? (int)st.cnt : 0;
    }
    if (k > 0) {
        const float dd = lane < (unsigned)k ? sqrtf(st.my_d) : 0.f;
        // the mean over the k entries in list order, summed as every other path sums it
        float seq = 0.f;
        for (int t = 0; t < k; ++t) seq += __shfl_sync(dev::kFull, dd, t);
        if (lane < (unsigned)k) {
            const int j = st.my_j;
            if (j >= 0 && j < n) atomicAdd(&sc[2 * n + j], 1.f);
            if (o.knn_idx) o.knn_idx[((int64_t)g.slot * n + oi) * k + lane] = j;
            if (o.knn_dist) o.knn_dist[((int64_t)g.slot * n + oi) * k + lane] = dd;
        }
        if (lane == 0) sc[3 * n + oi] = seq / (float)k;
    }
}

}  // namespace

namespace {
size_t al256(size_t b) { return (b + 255) & ~size_t(255); }
size_t sort_temp_bytes(int64_t n)
{
    size_t cub_bytes = 0;
    cub::DeviceRadixSort::SortPairs(nullptr, cub_bytes, (const uint32_t *)nullptr, (uint32_t *)nullptr,
                                    (const int32_t *)nullptr, (int32_t *)nullptr, (int)n, 0, 32);
    return cub_bytes;
}
}  // namespace

size_t grid_scratch_bytes(int64_t n, int max_cells)
{
    return 4 * al256(n * 4) + al256(n * 16) + al256(n * 4) + al256((size_t)(max_cells + 1) * 4) +
           al256(sort_temp_bytes(n));
}

GridBufs grid_carve(void *base, int64_t n, int max_cells)
{
    char *p = (char *)base;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        void *r = p + off;
        off += al256(bytes);
        return r;
    };
    GridBufs b;
    b.k_in = (uint32_t *)take(n * 4);
    b.k_out = (uint32_t *)take(n * 4);
    b.v_in = (int32_t *)take(n * 4);
    b.v_out = (int32_t *)take(n * 4);
    b.pts = (float4 *)take(n * 16);
    b.orig = (int32_t *)take(n * 4);
    b.start = (int32_t *)take((size_t)(max_cells + 1) * 4);
    b.tmp_bytes = sort_temp_bytes(n);
    b.tmp = take(b.tmp_bytes);
    return b;
}

int grid_key_bits(const GridSpec &g)
{
    int bits = 1;
    while ((1ll << bits) < (long long)g.ncells) ++bits;
    return bits;
}

snaps_status run_grid_subspace(const JoinShape &s, const GridSpec &g, const JoinOut &o, const GridBufs &b,
                               cudaStream_t st)
{
    const int64_t n = s.n;
    const int threads = 256;
    const int blocks = (int)std::min<int64_t>((n + threads - 1) / threads, 148 * 16);
    grid_keys_kernel<<<blocks, threads, 0, st>>>(s.x, n, g, b.k_in, b.v_in);
    SNAPS_CHECK_CUDA(cudaGetLastError());
    size_t tb = b.tmp_bytes;
    SNAPS_CHECK_CUDA(cub::DeviceRadixSort::SortPairs(b.tmp, tb, b.k_in, b.k_out, b.v_in, b.v_out, (int)n, 0,
                                                     grid_key_bits(g), st));
    grid_starts_kernel<<<(int)std::min<int64_t>(n / threads + 1, 148 * 16), threads, 0, st>>>(b.k_out, n, g.ncells,
                                                                                            b.start);
    SNAPS_CHECK_CUDA(cudaGetLastError());
    grid_gather_kernel<<<blocks, threads, 0, st>>>(s.x, b.v_out, n, g, b.pts, b.orig);
    SNAPS_CHECK_CUDA(cudaGetLastError());
    const unsigned jb = (unsigned)((n + kGridWarps - 1) / kGridWarps);
    if (g.d <= 2)
        grid_join_kernel<float2><<<jb, kGridWarps * 32, 0, st>>>(reinterpret_cast<const float2 *>(b.pts), b.orig,
                                                                  b.start, (int)n, g, s.k, o);
    else
        grid_join_kernel<float4><<<jb, kGridWarps * 32, 0, st>>>(b.pts, b.orig, b.start, (int)n, g, s.k, o);
    SNAPS_CHECK_CUDA(cudaGetLastError());
    return SNAPS_OK;
}

}  // namespace snaps
