// Device-side building blocks shared by the join kernels.
#pragma once

#include <cuda_runtime.h>
#include <math_constants.h>
#include <stdint.h>

namespace snaps {
namespace dev {

constexpr unsigned kFull = 0xffffffffu;
// Spin limit of every mbarrier wait: far longer than any healthy tile copy,
// short enough that a lost copy ends the kernel instead of hanging the GPU.
constexpr unsigned kSpinLimit = 1u << 26;

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// ---- mbarrier + 1-D bulk copy (TMA) ------------------------------------------

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void fence_barrier_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Plain arrival (count 1) on the barrier.
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// Arm the barrier for `bytes` of incoming transactions and issue one bulk copy
// of `bytes` (multiple of 16, both addresses 16-byte aligned).
__device__ __forceinline__ void bulk_load(void *dst_smem, const void *src, unsigned bytes,
                                          uint64_t *bar) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_addr(dst_smem)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// Wait for phase `parity` of the barrier; false if the spin limit ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity) {
    uint32_t addr = smem_addr(bar);
    for (unsigned it = 0; it < kSpinLimit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(addr), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// ---- eps distance sums ----------------------------------------------------------
//
// The mean eps-neighbour distance needs sum(dist) over the neighbours.  Each
// distance (<= eps) is quantised to an integer multiple of eps / 2^20 and the
// integers are summed exactly (64-bit totals), so the sum does not depend on
// the order in which kernels visit neighbours: every path of the library
// returns the same bits.  The quantisation error is <= 2^-21 eps per term.
// One quantised term is <= 2^20 (+ rounding), so a warp's 64 terms of one
// step fit a 32-bit warp reduction.

constexpr float kEpsQuantUnits = 1048576.f;  // 2^20 steps per eps

struct EpsScale {
    float scale;  // 2^20 / eps, or 0 when eps == 0 (all such distances are 0)
    float eps;
};

__device__ __forceinline__ EpsScale eps_scale(float eps2) {
    EpsScale e;
    e.eps = eps2 > 0.f ? sqrtf(eps2) : 0.f;
    e.scale = e.eps > 0.f ? kEpsQuantUnits / e.eps : 0.f;
    return e;
}

// Square root of a squared eps-neighbour distance for the distance sum: the
// hardware approximation (sqrt.approx.f32), identical in every kernel; its
// relative error is far below the 2^-20 eps quantisation step.
__device__ __forceinline__ float eps_sqrt(float d2) {
    float r;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(d2));
    return r;
}

__device__ __forceinline__ unsigned eps_quant(float d2, float scale) {
    return __float2uint_rn(eps_sqrt(d2) * scale);
}

// eps_quant's value, for the eps-neighbours of a subspace (scale maps eps to
// 2^20), without the conversion unit: the product p < 2^22 is rounded as
// eps_quant rounds it, and adding 1.5 * 2^23 (an even integer, in a binade
// where floats are the integers) rounds p to the nearest integer, ties to
// even, exactly as __float2uint_rn does.  The _rn intrinsics are never fused
// into one FMA, which would round once instead of twice.
__device__ __forceinline__ unsigned eps_quant_fma_pipe(float d2, float scale) {
    const float p = __fmul_rn(eps_sqrt(d2), scale);
    return __float_as_uint(__fadd_rn(p, 12582912.f)) - 0x4B400000u;
}

// eps_quant_fma_pipe's value plus 0x4B400000 (the bits of the rounded float).
// A branch-free kernel adds this for every candidate, with d2 capped at eps^2:
// a candidate beyond eps then adds eps_quant_fma_pipe(eps^2) + 0x4B400000, a
// known constant, and one correction per round of candidates
// (eps_round_sum) leaves the exact sum of the neighbours' quantised
// distances, with no per-candidate select.  The 32-bit sum wraps; the result
// is exact while the neighbours' true sum fits 32 bits.
__device__ __forceinline__ unsigned eps_quant_biased(float d2, float scale) {
    const float p = __fmul_rn(eps_sqrt(d2), scale);
    return __float_as_uint(__fadd_rn(p, 12582912.f));
}

// The exact quantised sum of a round's eps-neighbours from the biased sum of
// all `slots` candidates of the round (`hits` of them within eps) and the
// quantised value of eps^2 itself.
__device__ __forceinline__ unsigned eps_round_sum(unsigned biased, unsigned slots, unsigned hits, unsigned q_eps) {
    return biased - slots * 0x4B400000u - (slots - hits) * q_eps;
}

// Mean distance from the exact quantised sum.
__device__ __forceinline__ float eps_mean(unsigned long long qsum, int cnt, float scale) {
    if (cnt <= 0 || scale == 0.f) return 0.f;
    return ((float)qsum / scale) / (float)cnt;
}

// ---- warp-cooperative kNN list ------------------------------------------------
//
// A list of up to k (squared distance, index) entries sorted ascending by
// (distance, index) lives in shared memory; lane t < k holds entry t while the
// warp works on it.  Unused entries are (+inf, INT_MAX).

// Insert every lane flagged in `ballot` (candidates (d2, j), lanes in
// ascending j order) into the list held in (my_d, my_j).  T is the list's
// current k-th squared distance (warp-uniform) and is updated.
__device__ __forceinline__ void list_insert(unsigned ballot, float d2, int j, float &my_d,
                                            int &my_j, int k, float &T) {
    const unsigned lane = lane_id();
    while (ballot) {
        const int src = __ffs(ballot) - 1;
        ballot &= ballot - 1;
        const float cd = __shfl_sync(kFull, d2, src);
        const int cj = __shfl_sync(kFull, j, src);
        if (!(cd < T || (cd == T && cj < __shfl_sync(kFull, my_j, k - 1)))) continue;
        const bool before = lane < (unsigned)k && (my_d < cd || (my_d == cd && my_j < cj));
        const int pos = __popc(__ballot_sync(kFull, before));
        const float up_d = __shfl_up_sync(kFull, my_d, 1);
        const int up_j = __shfl_up_sync(kFull, my_j, 1);
        if (lane == (unsigned)pos) {
            my_d = cd;
            my_j = cj;
        } else if (lane > (unsigned)pos && lane < (unsigned)k) {
            my_d = up_d;
            my_j = up_j;
        }
        T = __shfl_sync(kFull, my_d, k - 1);
    }
}

// A kNN list as a max-heap of k (squared distance, original index) entries,
// entry p at ld[p * stride], lj[p * stride]; entry 0 is the largest by
// (distance, index), the current k-th nearest.  Replace it with (d2, j),
// which must be smaller, and sink the new entry to its place: at most
// log2(k) levels, where an unsorted list needs a rescan of all k entries.
// The list is sorted once, when its query's results are written.
__device__ __forceinline__ bool knn_key_gt(float a, int ja, float b, int jb)
{
    return a > b || (a == b && ja > jb);
}

__device__ __forceinline__ void heap_sink_root(float *ld, int *lj, int stride, int k, float d2, int j)
{
    int p = 0;
    for (;;) {
        int c = 2 * p + 1;
        if (c >= k) break;
        float cd = ld[c * stride];
        int cj = lj[c * stride];
        if (c + 1 < k) {
            const float rd = ld[(c + 1) * stride];
            const int rj = lj[(c + 1) * stride];
            if (knn_key_gt(rd, rj, cd, cj)) {
                c = c + 1;
                cd = rd;
                cj = rj;
            }
        }
        if (!knn_key_gt(cd, cj, d2, j)) break;
        ld[p * stride] = cd;
        lj[p * stride] = cj;
        p = c;
    }
    ld[p * stride] = d2;
    lj[p * stride] = j;
}

}  // namespace dev
}  // namespace snaps
