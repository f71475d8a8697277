// Lane-per-subspace self-join: DSSJ (Sec. 3.5) and kNNSJ (Sec. 3.6) for any
// list of subspaces.
//
// A warp owns one query object and up to 32 subspaces, one per lane.  Every
// candidate object is broadcast to the whole warp from a shared-memory tile;
// each lane folds the squared feature differences of its own subspace (from
// the highest feature index down, one FMA per feature, so every path of the
// library produces the same FP32 bits), tests the eps radius and keeps its
// own sorted kNN list.  The CTA's warps (different queries, same subspaces)
// share each tile, which is staged by 1-D bulk copies (TMA) through an
// mbarrier pipeline.  Work items (subspace group x query block) are handed
// out by an atomic counter so the persistent CTAs balance themselves.
//
// This form suits arbitrary, sparse subspace sets; dense sets of subspaces go
// to the subspace-batched tree kernel, which shares arithmetic across
// subspaces.

#include <math_constants.h>

#include <algorithm>

#include "device.cuh"
#include "join.cuh"

namespace snaps {
namespace {

constexpr int kLmWarps = 8;
constexpr int kTile = 256;  // rows per staged tile (16 KB)
constexpr int kStages = 3;
static_assert(kRowPad % kTile == 0, "padded rows must cover whole tiles");

template <int KMAX>
struct LmSmem {
    float4 tile[kStages][kTile * 4];
    float ld[kLmWarps][KMAX][32];  // kNN lists, entry-major so lanes hit distinct banks
    int lj[kLmWarps][KMAX][32];
    uint64_t bar[kStages];
    long long work;
};

template <int KMAX>
__global__ void __launch_bounds__(kLmWarps * 32)
    join_lanemask_kernel(JoinShape s, const MaskGroup *__restrict__ groups, int n_groups,
                         JoinOut o, DeviceControl *ctrl)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    LmSmem<KMAX> &sm = *reinterpret_cast<LmSmem<KMAX> *>(smem_raw);
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int64_t n = s.n;
    const int k = s.k;
    const long long n_qb = (n + kLmWarps - 1) / kLmWarps;
    const long long total = n_qb * (long long)n_groups;
    const int n_tiles = (int)(s.n_pad / kTile);
    const float4 *x = s.x;

    if (threadIdx.x == 0) {
        for (int st = 0; st < kStages; ++st) dev::mbar_init(&sm.bar[st], 1);
        dev::fence_barrier_init();
    }
    __syncthreads();

    uint32_t used = 0;  // tiles this CTA has consumed so far (same in every thread)
    for (;;) {
        if (threadIdx.x == 0) sm.work = (long long)atomicAdd(&ctrl->next_work, 1ull);
        __syncthreads();
        const long long w = sm.work;
        __syncthreads();
        if (w >= total) break;
        const int g = (int)(w / n_qb);
        const int64_t i = (w % n_qb) * kLmWarps + warp;
        const bool valid = i < n;

        const MaskGroup &grp = groups[g];
        const uint32_t mask = grp.mask[lane];
        const bool active = mask != 0u && valid;
        const float e2 = active ? grp.eps2[lane] : -1.f;
        float wgt[15];
#pragma unroll
        for (int f = 0; f < 15; ++f) wgt[f] = ((mask >> f) & 1u) ? 1.f : 0.f;
        float xq[16];
        int orig_i = 0;  // the query's original index (float 15 of its stored row)
        if (valid) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float4 v = x[row_quad(i, q)];
                xq[4 * q + 0] = v.x;
                xq[4 * q + 1] = v.y;
                xq[4 * q + 2] = v.z;
                xq[4 * q + 3] = v.w;
            }
            orig_i = __float_as_int(xq[15]);
        }
        float T = (active && k > 0) ? CUDART_INF_F : -CUDART_INF_F;
        for (int p = 0; p < KMAX; ++p) {
            sm.ld[warp][p][lane] = CUDART_INF_F;
            sm.lj[warp][p][lane] = 0x7fffffff;
        }
        int cnt = 0;
        unsigned long long qsum = 0;
        const float escale = dev::eps_scale(e2).scale;

        if (threadIdx.x == 0) {
            for (int t = 0; t < kStages && t < n_tiles; ++t) {
                const uint32_t st = (used + t) % kStages;
                dev::bulk_load(sm.tile[st], x + (int64_t)t * kTile * 4, kTile * 64, &sm.bar[st]);
            }
        }
        for (int t = 0; t < n_tiles; ++t) {
            const uint32_t st = (used + t) % kStages;
            const uint32_t parity = ((used + t) / kStages) & 1u;
            const bool ok = dev::mbar_wait(&sm.bar[st], parity);
            if (__syncthreads_or(!ok)) {
                if (threadIdx.x == 0) atomicOr(&ctrl->error, kErrTimeout);
                // let the copies still in flight land before the CTA leaves
                for (int u = t + 1; u < t + kStages && u < n_tiles; ++u)
                    dev::mbar_wait(&sm.bar[(used + u) % kStages], ((used + u) / kStages) & 1u);
                return;
            }
            if (valid) {
                const float4 *tile = sm.tile[st];
                const int64_t base = (int64_t)t * kTile;
                const int c_end = (int)std::min<int64_t>(kTile, n - base);
                for (int c = 0; c < c_end; ++c) {
                    const int64_t j = base + c;
                    if (j == i) continue;
                    float xc[16];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const float4 v = tile[q * kTile + c];
                        xc[4 * q + 0] = v.x;
                        xc[4 * q + 1] = v.y;
                        xc[4 * q + 2] = v.z;
                        xc[4 * q + 3] = v.w;
                    }
                    float acc = 0.f;
#pragma unroll
                    for (int f = 14; f >= 0; --f) {
                        const float d = xc[f] - xq[f];
                        acc = fmaf(d * wgt[f], d, acc);
                    }
                    if (acc <= e2) {
                        ++cnt;
                        qsum += dev::eps_quant(acc, escale);
                    }
                    const int oc = __float_as_int(xc[15]);  // candidate's original index
                    if (acc < T || (acc == T && k > 0 && oc < sm.lj[warp][k - 1][lane])) {
                        // sorted insertion into this lane's list (entries strided by 32),
                        // by (distance, original index)
                        float *ld = &sm.ld[warp][0][lane];
                        int *lj = &sm.lj[warp][0][lane];
                        int p = k - 1;
                        while (p > 0) {
                            const float pd = ld[(p - 1) * 32];
                            const int pj = lj[(p - 1) * 32];
                            if (!(acc < pd || (acc == pd && oc < pj))) break;
                            ld[p * 32] = pd;
                            lj[p * 32] = pj;
                            --p;
                        }
                        ld[p * 32] = acc;
                        lj[p * 32] = oc;
                        T = ld[(k - 1) * 32];
                    }
                }
            }
            __syncthreads();
            if (threadIdx.x == 0 && t + kStages < n_tiles)
                dev::bulk_load(sm.tile[st], x + (int64_t)(t + kStages) * kTile * 4, kTile * 64,
                               &sm.bar[st]);
        }
        used += n_tiles;

        if (active && (orig_i < 0 || orig_i >= n)) {
            // a row that does not carry its index: report, write nothing
            atomicOr(&ctrl->error, kErrBadRow);
        } else if (active) {
            const int slot = grp.slot[lane];
            float *sc = o.scores + (int64_t)slot * 4 * n;
            sc[orig_i] = (float)cnt;
            sc[n + orig_i] = dev::eps_mean(qsum, cnt, escale);
            if (o.eps_count) o.eps_count[(int64_t)slot * n + orig_i] = cnt;
            if (k > 0) {
                float msum = 0.f;
                for (int p = 0; p < k; ++p) {
                    const float d = sqrtf(sm.ld[warp][p][lane]);
                    const int j = sm.lj[warp][p][lane];
                    msum += d;
                    if (j >= 0 && j < n) atomicAdd(&sc[2 * n + j], 1.f);
                    if (o.knn_idx) o.knn_idx[((int64_t)slot * n + orig_i) * k + p] = j;
                    if (o.knn_dist) o.knn_dist[((int64_t)slot * n + orig_i) * k + p] = d;
                }
                sc[3 * n + orig_i] = msum / (float)k;
            }
        }
    }
}

template <int KMAX>
snaps_status launch_lm(const JoinShape &s, const MaskGroup *groups, int n_groups,
                       const JoinOut &o, DeviceControl *ctrl, cudaStream_t st)
{
    const size_t smem = sizeof(LmSmem<KMAX>);
    auto kern = join_lanemask_kernel<KMAX>;
    SNAPS_CHECK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int dev = 0, sms = 0, per_sm = 0;
    SNAPS_CHECK_CUDA(cudaGetDevice(&dev));
    SNAPS_CHECK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    SNAPS_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kLmWarps * 32, smem));
    if (per_sm < 1) {
        set_error("lane-per-subspace join does not fit on an SM (smem %zu)", smem);
        return SNAPS_ECUDA;
    }
    const long long n_qb = (s.n + kLmWarps - 1) / kLmWarps;
    const long long total = n_qb * (long long)n_groups;
    const long long grid = std::min<long long>(total, (long long)sms * per_sm);
    SNAPS_CHECK_CUDA(cudaMemsetAsync(&ctrl->next_work, 0, sizeof(unsigned long long), st));
    kern<<<(unsigned)grid, kLmWarps * 32, smem, st>>>(s, groups, n_groups, o, ctrl);
    SNAPS_CHECK_CUDA(cudaGetLastError());
    return SNAPS_OK;
}

}  // namespace

snaps_status launch_join_lanemask(const JoinShape &s, const MaskGroup *groups, int n_groups,
                                  const JoinOut &o, DeviceControl *ctrl, cudaStream_t st)
{
    if (n_groups <= 0) return SNAPS_OK;
    if (s.k <= 16) return launch_lm<16>(s, groups, n_groups, o, ctrl, st);
    return launch_lm<32>(s, groups, n_groups, o, ctrl, st);
}

}  // namespace snaps
