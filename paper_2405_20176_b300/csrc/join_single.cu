// Subspace-at-a-time self-join: DSSJ (Sec. 3.5) and kNNSJ (Sec. 3.6) of
// subspaces that do not share a 32-subspace chunk with another requested one
// (random subspace sets, single subspaces such as the full 15-feature space).
//
// Mapping.  Launch row y is entry y % 32 of group y / 32 (a MaskGroup; an
// unused entry has mask 0 and its CTAs return at once).  A CTA owns 256
// consecutive stored rows as queries, one per thread, and streams every row
// of the population through shared memory, 256 at a time.  A staged
// candidate keeps only the subspace's d features, highest first and
// feature-planar, so that one 128-bit read gives four candidates and the
// canonical fold (FMAs from the highest feature down) runs two candidates per
// f32x2 instruction, fully unrolled for the subspace's dimension.  The stream
// starts at the CTA's own rows, which are neighbours in the stored cell
// order, so the kNN thresholds are tight early; it then wraps around.
//
// Each thread keeps its eps count, the exact quantised distance sum and a
// kNN list kept as a max-heap (dev::heap_sink_root).  The query meets itself
// once in the stream (distance 0); that eps hit is taken off at the end and
// the kNN test skips it by position.  Results equal every other path's bit
// for bit.

#include <math_constants.h>

#include <algorithm>

#include "device.cuh"
#include "join.cuh"

namespace snaps {
namespace {

constexpr int kSQ = 256;   // queries per CTA, one per thread
constexpr int kSC = 256;   // candidates staged per round
constexpr int kMaxF = 15;  // features of the largest subspace

template <int KMAX>
struct SingleSmem {
    float cand[kMaxF][kSC + 4];  // compact subspace features, feature-planar
    int corig[kSC];              // original indices of the staged candidates
    float qf[kMaxF][kSQ];        // the CTA's queries, compact: thread t owns column t
    float ld[KMAX][kSQ];         // kNN lists, entry-major: thread t owns column t
    int lj[KMAX][kSQ];
};

// The 16 floats of stored row r (15 features, then the original index's bits).
__device__ __forceinline__ void load_row(const float4 *__restrict__ x, int64_t r, float (&v)[16])
{
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const float4 t = x[row_quad(r, q)];
        v[4 * q + 0] = t.x;
        v[4 * q + 1] = t.y;
        v[4 * q + 2] = t.z;
        v[4 * q + 3] = t.w;
    }
}

template <int D, int KMAX>
__device__ __forceinline__ void join_one(SingleSmem<KMAX> &sm, const float4 *__restrict__ x, int n, uint32_t mask,
                                         float e2, int slot, int k, const JoinOut &o, int p0)
{
    const int t = threadIdx.x;
    const int q = p0 + t;
    const bool act = q < n;
    const bool do_eps = e2 >= 0.f;
    const float esc = dev::eps_scale(e2).scale;
    const unsigned q_eps = dev::eps_quant_fma_pipe(e2, esc);  // a candidate beyond eps adds this

    // this thread's query, compact
    int qorig = 0;
    if (act) {
        float v[16];
        load_row(x, q, v);
#pragma unroll
        for (int f = kMaxF - 1; f >= 0; --f)
            if ((mask >> f) & 1u) sm.qf[__popc(mask >> (f + 1))][t] = v[f];
        qorig = __float_as_int(v[15]);
    }
    float2 nq[D];
#pragma unroll
    for (int p = 0; p < D; ++p) {
        const float a = act ? -sm.qf[p][t] : 0.f;
        nq[p] = make_float2(a, a);
    }
#pragma unroll 1
    for (int e = 0; e < KMAX; ++e) {
        sm.ld[e][t] = CUDART_INF_F;
        sm.lj[e][t] = 0x7fffffff;
    }
    float T = (act && k > 0) ? CUDART_INF_F : -CUDART_INF_F;  // largest list entry
    int Tj = 0x7fffffff;
    unsigned cnt = 0;
    unsigned long long qs = 0ull;

    auto scan = [&](int beg, int end) {
#pragma unroll 1
        for (int c0 = beg; c0 < end; c0 += kSC) {
            const int cn = min(kSC, end - c0);
            __syncthreads();  // the previous round's candidates are no longer read
            for (int u = t; u < cn; u += kSQ) {
                float v[16];
                load_row(x, c0 + u, v);
#pragma unroll
                for (int f = kMaxF - 1; f >= 0; --f)
                    if ((mask >> f) & 1u) sm.cand[__popc(mask >> (f + 1))][u] = v[f];
                sm.corig[u] = __float_as_int(v[15]);
            }
            // partners of the last candidates up to a multiple of four: never an
            // eps-neighbour, and no kNN entry (cp < cend)
            if (t < 4 * D) sm.cand[t >> 2][cn + (t & 3)] = 1e18f;
            __syncthreads();
            if (!act) continue;
            const int cend = c0 + cn;
            unsigned qb = 0u;  // this round's biased sum over all its candidates (wraps)
            const unsigned cnt0 = cnt;
#pragma unroll 2
            for (int u = 0; u < cn; u += 4) {
                float2 acc[2];
#pragma unroll
                for (int p = 0; p < D; ++p) {
                    const float4 v = *reinterpret_cast<const float4 *>(&sm.cand[p][u]);
                    const float2 d0 = __fadd2_rn(make_float2(v.x, v.y), nq[p]);
                    const float2 d1 = __fadd2_rn(make_float2(v.z, v.w), nq[p]);
                    acc[0] = p == 0 ? __fmul2_rn(d0, d0) : __ffma2_rn(d0, d0, acc[0]);
                    acc[1] = p == 0 ? __fmul2_rn(d1, d1) : __ffma2_rn(d1, d1, acc[1]);
                }
                // eps: branch-free; the query itself (d2 = 0) is counted and taken off at the end
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
                                    dev::heap_sink_root(&sm.ld[0][t], &sm.lj[0][t], kSQ, k, d2, oj);
                                    T = sm.ld[0][t];
                                    Tj = sm.lj[0][t];
                                }
                            }
                        }
                    }
                }
            }
            // the neighbours' exact sum: <= kSC terms of <= 2^20 + 1
            qs += dev::eps_round_sum(qb, (unsigned)((cn + 3) & ~3), cnt - cnt0, q_eps);
        }
    };
    scan(p0, n);  // the CTA's own rows first, then the rest
    scan(0, p0);
    if (!act) return;
    if (do_eps) --cnt;  // the query, at distance 0

    float *sc = o.scores + (int64_t)slot * 4 * n;
    const int oi = qorig;
    if (oi < 0 || oi >= n) return;  // rows always carry their index; nothing to write otherwise
    sc[oi] = do_eps ? (float)cnt : 0.f;
    sc[n + oi] = do_eps ? dev::eps_mean(qs, (int)cnt, esc) : 0.f;
    if (o.eps_count) o.eps_count[(int64_t)slot * n + oi] = do_eps ? (int)cnt : 0;
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
            if (o.knn_idx) o.knn_idx[((int64_t)slot * n + oi) * k + e] = j;
            if (o.knn_dist) o.knn_dist[((int64_t)slot * n + oi) * k + e] = dd;
        }
        sc[3 * n + oi] = msum / (float)k;
    }
}

template <int KMAX>
__global__ void __launch_bounds__(kSQ, 2)
    join_single_kernel(JoinShape s, const MaskGroup *__restrict__ groups, JoinOut o)
{
    extern __shared__ __align__(16) unsigned char single_smem[];
    SingleSmem<KMAX> &sm = *reinterpret_cast<SingleSmem<KMAX> *>(single_smem);
    const MaskGroup &g = groups[blockIdx.y >> 5];
    const int entry = (int)(blockIdx.y & 31u);
    const uint32_t mask = g.mask[entry];
    if (mask == 0u) return;  // an unused entry: the whole CTA leaves before any barrier
    const int n = (int)s.n;
    const int p0 = (int)blockIdx.x * kSQ;
    const float e2 = g.eps2[entry];
    const int slot = g.slot[entry];
    switch (__popc(mask)) {
    case 2: join_one<2, KMAX>(sm, s.x, n, mask, e2, slot, s.k, o, p0); break;
    case 3: join_one<3, KMAX>(sm, s.x, n, mask, e2, slot, s.k, o, p0); break;
    case 4: join_one<4, KMAX>(sm, s.x, n, mask, e2, slot, s.k, o, p0); break;
    case 5: join_one<5, KMAX>(sm, s.x, n, mask, e2, slot, s.k, o, p0); break;
    case 6: join_one<6, KMAX>(sm, s.x, n, mask, e2, slot, s.k, o, p0); break;
    case 7: join_one<7, KMAX>(sm, s.x, n, mask, e2, slot, s.k, o, p0); break;
    case 8: join_one<8, KMAX>(sm, s.x, n, mask, e2, slot, s.k, o, p0); break;
    case 9: join_one<9, KMAX>(sm, s.x, n, mask, e2, slot, s.k, o, p0); break;
    case 10: join_one<10, KMAX>(sm, s.x, n, mask, e2, slot, s.k, o, p0); break;
    case 11: join_one<11, KMAX>(sm, s.x, n, mask, e2, slot, s.k, o, p0); break;
    case 12: join_one<12, KMAX>(sm, s.x, n, mask, e2, slot, s.k, o, p0); break;
    case 13: join_one<13, KMAX>(sm, s.x, n, mask, e2, slot, s.k, o, p0); break;
    case 14: join_one<14, KMAX>(sm, s.x, n, mask, e2, slot, s.k, o, p0); break;
    case 15: join_one<15, KMAX>(sm, s.x, n, mask, e2, slot, s.k, o, p0); break;
    default: break;  // the host rejects masks of fewer than 2 features
    }
}

// The work-list form: CTA b finds its item by a binary search over the
// items' first CTAs, then joins that item's 256 queries from row
// 256 (b - first_cta) exactly as join_single_kernel does.
template <int KMAX>
__global__ void __launch_bounds__(kSQ, 2)
    join_worklist_kernel(const WorkItem *__restrict__ items, int n_items)
{
    extern __shared__ __align__(16) unsigned char single_smem[];
    SingleSmem<KMAX> &sm = *reinterpret_cast<SingleSmem<KMAX> *>(single_smem);
    const int b = (int)blockIdx.x;
    int lo = 0, hi = n_items - 1;  // the last item whose first CTA is <= b
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (items[mid].first_cta <= b) lo = mid;
        else hi = mid - 1;
    }
    const WorkItem it = items[lo];
    const int p0 = (b - it.first_cta) * kSQ;
    if (it.mask == 0u || p0 >= it.n) return;  // the whole CTA leaves before any barrier
    JoinOut o{it.scores, nullptr, nullptr, nullptr};
    switch (__popc(it.mask)) {
    case 2: join_one<2, KMAX>(sm, it.x, it.n, it.mask, it.eps2, 0, it.k, o, p0); break;
    case 3: join_one<3, KMAX>(sm, it.x, it.n, it.mask, it.eps2, 0, it.k, o, p0); break;
    case 4: join_one<4, KMAX>(sm, it.x, it.n, it.mask, it.eps2, 0, it.k, o, p0); break;
    case 5: join_one<5, KMAX>(sm, it.x, it.n, it.mask, it.eps2, 0, it.k, o, p0); break;
    case 6: join_one<6, KMAX>(sm, it.x, it.n, it.mask, it.eps2, 0, it.k, o, p0); break;
    case 7: join_one<7, KMAX>(sm, it.x, it.n, it.mask, it.eps2, 0, it.k, o, p0); break;
    case 8: join_one<8, KMAX>(sm, it.x, it.n, it.mask, it.eps2, 0, it.k, o, p0); break;
    case 9: join_one<9, KMAX>(sm, it.x, it.n, it.mask, it.eps2, 0, it.k, o, p0); break;
    case 10: join_one<10, KMAX>(sm, it.x, it.n, it.mask, it.eps2, 0, it.k, o, p0); break;
    case 11: join_one<11, KMAX>(sm, it.x, it.n, it.mask, it.eps2, 0, it.k, o, p0); break;
    case 12: join_one<12, KMAX>(sm, it.x, it.n, it.mask, it.eps2, 0, it.k, o, p0); break;
    case 13: join_one<13, KMAX>(sm, it.x, it.n, it.mask, it.eps2, 0, it.k, o, p0); break;
    case 14: join_one<14, KMAX>(sm, it.x, it.n, it.mask, it.eps2, 0, it.k, o, p0); break;
    case 15: join_one<15, KMAX>(sm, it.x, it.n, it.mask, it.eps2, 0, it.k, o, p0); break;
    default: break;  // the host rejects masks of fewer than 2 features
    }
}

template <int KMAX>
snaps_status launch_worklist(const WorkItem *items, int n_items, int n_ctas, cudaStream_t st)
{
    const size_t smem = sizeof(SingleSmem<KMAX>);
    auto kern = join_worklist_kernel<KMAX>;
    SNAPS_CHECK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<(unsigned)n_ctas, kSQ, smem, st>>>(items, n_items);
    SNAPS_CHECK_CUDA(cudaGetLastError());
    return SNAPS_OK;
}

template <int KMAX>
snaps_status launch_single(const JoinShape &s, const MaskGroup *groups, int n_groups, const JoinOut &o,
                           cudaStream_t st)
{
    const size_t smem = sizeof(SingleSmem<KMAX>);
    auto kern = join_single_kernel<KMAX>;
    SNAPS_CHECK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const dim3 grid((unsigned)((s.n + kSQ - 1) / kSQ), (unsigned)(n_groups * 32));
    kern<<<grid, kSQ, smem, st>>>(s, groups, o);
    SNAPS_CHECK_CUDA(cudaGetLastError());
    return SNAPS_OK;
}

}  // namespace

snaps_status launch_join_worklist(const WorkItem *items, int n_items, int n_ctas, int kmax, cudaStream_t st)
{
    if (n_items <= 0 || n_ctas <= 0) return SNAPS_OK;
    if (kmax <= 16) return launch_worklist<16>(items, n_items, n_ctas, st);
    return launch_worklist<32>(items, n_items, n_ctas, st);
}

snaps_status launch_join_single(const JoinShape &s, const MaskGroup *groups, int n_groups, const JoinOut &o,
                                cudaStream_t st)
{
    if (n_groups <= 0 || s.n <= 0) return SNAPS_OK;
    if (n_groups * 32 > 65535) return SNAPS_EINVAL;  // more subspaces than there are (32,752)
    if (s.k <= 16) return launch_single<16>(s, groups, n_groups, o, st);
    return launch_single<32>(s, groups, n_groups, o, st);
}

}  // namespace snaps
