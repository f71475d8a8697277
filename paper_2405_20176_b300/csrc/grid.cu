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
// zero padded; a float2 for subspaces of two features) plus their original
// indices.
//
// Join.  Every eps-neighbour of a query lies in the (2R + 1)^D block of
// cells around its own (R w >= eps, and w carries a 2^-10 margin so that
// rounding in the cell computation cannot separate two points by more than R
// cells).  grid_tile_kernel gives a CTA 256 consecutive queries in cell order
// and, per row segment of them, stages the union of their blocks in shared
// memory once; every thread tests all of it against its query, counts
// eps-neighbours, sums their quantised distances exactly and keeps a private
// kNN list.  When a query's k-th distance is not below R w afterwards
// (sparse regions, outliers), grid_ring_kernel joins it again, a warp per
// query, scanning rings of cells at Chebyshev distance r = R + 1, R + 2, ...
// until (r - 1) w exceeds the k-th distance: no object outside the scanned
// cells can be nearer (a subspace distance is at least the distance over the
// index features).  Distances are the library's canonical FP32 fold (FMAs
// from the highest feature down), so results equal every other path's bit for
// bit.

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

// One warp joins the query at sorted position p: the block, then rings.
template <typename V>
__device__ __forceinline__ void warp_query(const V *__restrict__ pts, const int32_t *__restrict__ orig,
                                           const int32_t *__restrict__ start, int n, const GridSpec &g, int k,
                                           const JoinOut &o, int p)
{
    const unsigned lane = dev::lane_id();
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

// Queries whose kNN list the cell-tile join could not certify (listed in
// `ring`, *ring_n of them): a warp per query, grid-stride.
template <typename V>
__global__ void __launch_bounds__(kGridWarps * 32, 2)
    grid_ring_kernel(const V *__restrict__ pts, const int32_t *__restrict__ orig,
                     const int32_t *__restrict__ start, int n, GridSpec g, int k, JoinOut o,
                     const int32_t *__restrict__ ring, const int32_t *__restrict__ ring_n)
{
    const int warp = threadIdx.x >> 5;
    const int m = *ring_n;
    for (int i = blockIdx.x * kGridWarps + warp; i < m; i += gridDim.x * kGridWarps) {
        const int p = ring[i];
        if (p >= 0 && p < n) warp_query(pts, orig, start, n, g, k, o, p);
    }
}

// ---- cell-tile join ------------------------------------------------------------------------------
//
// A CTA owns kTileQ consecutive sorted positions, one query per thread.  It
// splits them into segments that share the leading cell coordinates (one
// row of cells along the fastest dimension); the queries of a segment lie in
// cells cl_lo..cl_hi of that row, so the union of their (2R + 1)^D blocks is
// the (2R + 1)^(D - 1) neighbouring rows, each restricted to cells
// cl_lo - R .. cl_hi + R: one contiguous range of sorted positions per row.
// Those candidates are staged in shared memory kTileC at a time and every
// thread tests all of them against its query, so a candidate is read from
// global memory once per segment instead of once per query.  Candidates
// outside a query's own block are tested too; they only make its kNN list
// tighter sooner, and every decision is the exact canonical distance.
//
// Each thread keeps its eps count, exact quantised sum and a kNN list kept as
// a max-heap (dev::heap_sink_root) privately.  A query whose k-th distance is not
// below R w afterwards (the reach beyond which the rings begin) may have
// nearer objects outside the scanned block; it is appended to the ring list
// and joined afresh by grid_ring_kernel, and this kernel writes nothing for it.
constexpr int kTileQ = 256;   // queries per CTA
constexpr int kTileC = 1024;  // candidates staged per round

template <typename V, int KMAX>
struct TileSmem {
    static constexpr int NF = sizeof(V) / sizeof(float);  // 2 or 4 stored features
    float cand[NF][kTileC + 4];  // feature-planar, so that a float4 read holds four candidates
    int corig[kTileC];           // their original indices
    float ld[KMAX][kTileQ];      // kNN lists, entry-major: thread t owns column t
    int lj[KMAX][kTileQ];
};

__device__ __forceinline__ float comp(const float2 &v, int f) { return f == 0 ? v.x : v.y; }
__device__ __forceinline__ float comp(const float4 &v, int f)
{
    return f == 0 ? v.x : (f == 1 ? v.y : (f == 2 ? v.z : v.w));
}

__device__ __forceinline__ int fastest_cell(const GridSpec &g, const int (&c)[3]) { return g.D == 2 ? c[1] : c[2]; }

template <typename V, int KMAX>
__global__ void __launch_bounds__(kTileQ, 4)
    grid_tile_kernel(const V *__restrict__ pts, const int32_t *__restrict__ orig,
                     const int32_t *__restrict__ start, int n, GridSpec g, int k, JoinOut o,
                     int32_t *__restrict__ ring, int32_t *__restrict__ ring_n)
{
    extern __shared__ __align__(16) unsigned char tile_smem[];
    TileSmem<V, KMAX> &sm = *reinterpret_cast<TileSmem<V, KMAX> *>(tile_smem);
    constexpr int NF = TileSmem<V, KMAX>::NF;
    const int t = threadIdx.x;
    const int p0 = blockIdx.x * kTileQ;
    const int p1 = min(p0 + kTileQ, n);
    const int D = g.D, R = g.R;
    const int nl = D == 2 ? g.nc[1] : g.nc[2];  // cells along the fastest dimension
    const bool do_eps = g.eps2 >= 0.f;
    const float e2 = g.eps2;
    const float esc = dev::eps_scale(g.eps2).scale;
    const unsigned q_eps = dev::eps_quant_fma_pipe(e2, esc);  // a candidate beyond eps adds this
    // objects outside a query's (2R + 1)^D block are at least this far away
    const float reach = (float)R * g.w * (1.f - 1.f / 1024.f);
    const float reach2 = reach * reach;
    float *sc = o.scores + (int64_t)g.slot * 4 * n;

    int pos = p0;
    while (pos < p1) {  // every thread computes the same segments
        int c[3];
        point_cell(g, pts[pos], c);
        const int row0 = D == 2 ? c[0] * g.nc[1] : (c[0] * g.nc[1] + c[1]) * g.nc[2];
        const int se = min(p1, (int)start[row0 + nl]);  // > pos: pos lies in this row
        int ce[3];
        point_cell(g, pts[se - 1], ce);
        const int a = max(fastest_cell(g, c) - R, 0);
        const int b = min(fastest_cell(g, ce) + R, nl - 1);

        const int q = pos + t;
        const bool act = q < se;
        const V qv = act ? pts[q] : V{};
        float2 nq[NF];
#pragma unroll
        for (int f = 0; f < NF; ++f) nq[f] = make_float2(-comp(qv, f), -comp(qv, f));
#pragma unroll 1
        for (int e = 0; e < KMAX; ++e) {
            sm.ld[e][t] = CUDART_INF_F;
            sm.lj[e][t] = 0x7fffffff;
        }
        float T = (act && k > 0) ? CUDART_INF_F : -CUDART_INF_F;  // largest list entry
        int Tj = 0x7fffffff;
        unsigned cnt = 0;
        unsigned long long qs = 0ull;

        // stage and test the candidates at sorted positions [beg, end)
        auto scan = [&](int beg, int end) {
#pragma unroll 1
                for (int c0 = beg; c0 < end; c0 += kTileC) {
                    const int cn = min(kTileC, end - c0);
                    __syncthreads();  // the previous round's candidates are no longer read
                    for (int u = t; u < cn; u += kTileQ) {
                        const V pv = pts[c0 + u];
#pragma unroll
                        for (int f = 0; f < NF; ++f) sm.cand[f][u] = comp(pv, f);
                        sm.corig[u] = orig[c0 + u];
                    }
                    // partners of the last candidates up to a multiple of four: never an
                    // eps-neighbour, and no kNN entry (cp < cend)
                    if (t < 4 * NF) sm.cand[t >> 2][cn + (t & 3)] = 1e18f;
                    __syncthreads();
                    if (!act) continue;
                    const int cend = c0 + cn;
                    unsigned qb = 0u;  // this round's biased sum over all its candidates (wraps)
                    const unsigned cnt0 = cnt;
#pragma unroll 2
                    for (int u = 0; u < cn; u += 4) {
                        // the canonical fold of four candidates, two per f32x2 instruction,
                        // highest feature first
                        float2 acc[2];
#pragma unroll
                        for (int f = 0; f < NF; ++f) {
                            const float4 v = *reinterpret_cast<const float4 *>(&sm.cand[f][u]);
                            const float2 d0 = __fadd2_rn(make_float2(v.x, v.y), nq[f]);
                            const float2 d1 = __fadd2_rn(make_float2(v.z, v.w), nq[f]);
                            acc[0] = f == 0 ? __fmul2_rn(d0, d0) : __ffma2_rn(d0, d0, acc[0]);
                            acc[1] = f == 0 ? __fmul2_rn(d1, d1) : __ffma2_rn(d1, d1, acc[1]);
                        }
                        // eps: branch-free (the query itself, at d2 = 0, is counted here and
                        // taken off at the end)
#pragma unroll
                        for (int h = 0; h < 4; ++h) {
                            const float d2 = (h & 1) ? acc[h >> 1].y : acc[h >> 1].x;
                            cnt += d2 <= e2 ? 1u : 0u;
                            qb += dev::eps_quant_biased(fminf(d2, e2), esc);
                        }
                        // kNN: one test for the four, then each
                        if (fminf(fminf(acc[0].x, acc[0].y), fminf(acc[1].x, acc[1].y)) <= T) {
#pragma unroll
                        for (int h = 0; h < 4; ++h) {
                            const float d2 = (h & 1) ? acc[h >> 1].y : acc[h >> 1].x;
                            if (d2 <= T) {
                                const int cp = c0 + u + h;
                                if (cp != q && cp < cend) {
                                    const int oj = sm.corig[u + h];
                                    if (d2 < T || oj < Tj) {
                                        dev::heap_sink_root(&sm.ld[0][t], &sm.lj[0][t], kTileQ, k, d2, oj);
                                        T = sm.ld[0][t];
                                        Tj = sm.lj[0][t];
                                    }
                                }
                            }
                        }
                        }
                    }
                    // the neighbours' exact sum: <= kTileC terms of <= 2^20 + 1
                    qs += dev::eps_round_sum(qb, (unsigned)((cn + 3) & ~3), cnt - cnt0, q_eps);
                }
        };
        // the segment's own cells first and then the rows outwards, so that the
        // kNN thresholds are tight early and few candidates reach the insertion
        const int cl_lo = fastest_cell(g, c), cl_hi = fastest_cell(g, ce);
        {
            const int base = (D == 2 ? c[0] : c[0] * g.nc[1] + c[1]) * nl;
            const int m0 = start[base + cl_lo], m1 = start[base + cl_hi + 1];
            scan(m0, m1);
            scan(start[base + a], m0);
            scan(m1, start[base + b + 1]);
        }
        const int r1max = D == 3 ? 2 * R : 0;
#pragma unroll 1
        for (int r0 = 0; r0 <= 2 * R; ++r0) {
            const int i0 = c[0] + ((r0 & 1) ? -((r0 + 1) >> 1) : (r0 >> 1));  // c0, c0 - 1, c0 + 1, ...
            if (i0 < 0 || i0 >= g.nc[0]) continue;
#pragma unroll 1
            for (int r1 = 0; r1 <= r1max; ++r1) {
                const int i1 = c[1] + ((r1 & 1) ? -((r1 + 1) >> 1) : (r1 >> 1));
                if (D == 3 && (i1 < 0 || i1 >= g.nc[1])) continue;
                if (r0 == 0 && r1 == 0) continue;  // the own row, done above
                const int lead = D == 2 ? i0 : i0 * g.nc[1] + i1;
                scan(start[lead * nl + a], start[lead * nl + b + 1]);
            }
        }
        if (act && do_eps) --cnt;  // the query, at distance 0, is in its own block

        if (act) {
            if (k > 0 && !(reach2 > T)) {
                // nearer objects may lie beyond the block: the ring search decides
                ring[atomicAdd(ring_n, 1)] = q;
            } else {
                const int oi = orig[q];
                sc[oi] = do_eps ? (float)cnt : 0.f;
                sc[n + oi] = do_eps ? dev::eps_mean(qs, (int)cnt, esc) : 0.f;
                if (o.eps_count) o.eps_count[(int64_t)g.slot * n + oi] = do_eps ? (int)cnt : 0;
                if (k > 0) {
                    // sort the list by (distance, index), then the mean in that order
                    for (int e = 1; e < k; ++e) {
                        const float v = sm.ld[e][t];
                        const int j = sm.lj[e][t];
                        int r = e;
                        while (r > 0 && (sm.ld[r - 1][t] > v || (sm.ld[r - 1][t] == v && sm.lj[r - 1][t] > j))) {
                            sm.ld[r][t] = sm.ld[r - 1][t];
                            sm.lj[r][t] = sm.lj[r - 1][t];
                            --r;
                        }
                        sm.ld[r][t] = v;
                        sm.lj[r][t] = j;
                    }
                    float msum = 0.f;
                    for (int e = 0; e < k; ++e) {
                        const float dd = sqrtf(sm.ld[e][t]);
                        const int j = sm.lj[e][t];
                        msum += dd;
                        if (j >= 0 && j < n) atomicAdd(&sc[2 * n + j], 1.f);
                        if (o.knn_idx) o.knn_idx[((int64_t)g.slot * n + oi) * k + e] = j;
                        if (o.knn_dist) o.knn_dist[((int64_t)g.slot * n + oi) * k + e] = dd;
                    }
                    sc[3 * n + oi] = msum / (float)k;
                }
            }
        }
        pos = se;
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
           al256(sort_temp_bytes(n)) + al256(n * 4) + al256(4);
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
    b.ring = (int32_t *)take(n * 4);
    b.ring_n = (int32_t *)take(4);
    return b;
}

namespace {
// The cell-tile join over all queries, then the ring search for the queries
// it could not certify.
template <typename V, int KMAX>
snaps_status launch_tile(const V *pts, const GridBufs &b, int n, const GridSpec &g, int k, const JoinOut &o,
                         cudaStream_t st)
{
    const size_t smem = sizeof(TileSmem<V, KMAX>);
    auto tk = grid_tile_kernel<V, KMAX>;
    SNAPS_CHECK_CUDA(cudaFuncSetAttribute(tk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const unsigned tb = (unsigned)((n + kTileQ - 1) / kTileQ);
    tk<<<tb, kTileQ, smem, st>>>(pts, b.orig, b.start, n, g, k, o, b.ring, b.ring_n);
    SNAPS_CHECK_CUDA(cudaGetLastError());
    if (k > 0) {
        // a warp per listed query; the list length is only known on the device
        const unsigned rb = (unsigned)std::min<int64_t>(((int64_t)n + kGridWarps - 1) / kGridWarps, 148 * 8);
        grid_ring_kernel<V><<<rb, kGridWarps * 32, 0, st>>>(pts, b.orig, b.start, n, g, k, o, b.ring, b.ring_n);
        SNAPS_CHECK_CUDA(cudaGetLastError());
    }
    return SNAPS_OK;
}
}  // namespace

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
    SNAPS_CHECK_CUDA(cudaMemsetAsync(b.ring_n, 0, sizeof(int32_t), st));
    if (g.d <= 2) {
        const float2 *p2 = reinterpret_cast<const float2 *>(b.pts);
        if (s.k <= 16) return launch_tile<float2, 16>(p2, b, (int)n, g, s.k, o, st);
        return launch_tile<float2, 32>(p2, b, (int)n, g, s.k, o, st);
    }
    if (s.k <= 16) return launch_tile<float4, 16>(b.pts, b, (int)n, g, s.k, o, st);
    return launch_tile<float4, 32>(b.pts, b, (int)n, g, s.k, o, st);
}

}  // namespace snaps
