// Parameter selection by the over-/underfitting trade-off (Sec. 3.5.2, Eq. 2
// and 3; Sec. 3.6.2): one join per subspace at the largest eps and k of the
// grids, from which the results at every grid value are derived.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace snaps {

constexpr int kSelectMaxGrid = 64;  // grid values per parameter
constexpr int kSelectHistBins = 4096;  // bins of the selectivity histogram

constexpr int kSelectMaxK = 4096;       // largest k of a k grid
constexpr int kSelectWarpK = 32;        // k_max up to this: warp-held lists
constexpr double kKnnQuantum = 1.0 / 1073741824.0;  // 2^-30: quantum of the exact kNN distance sums

// One subspace's eps grid, as the select join kernel takes it.
struct SelectSpec {
    uint32_t mask;
    int n_eps;                    // 0: no eps grid
    float e2[kSelectMaxGrid];     // ascending squared radii eps_j^2
    float qscale;                 // 2^24 / eps_max: quantisation of the distance sums
};

struct KGrid {
    int n;                        // 0: no k grid
    int k[kSelectMaxGrid];        // strictly ascending; k[n - 1] = k_max
};

// One pass over all candidates of every object for the eps grid and, when
// k_max <= kSelectWarpK, the k grid.  eps_scores: n_eps slots x 4 rows x n
// (rows 0 and 1: eps-neighbour count and mean distance at eps_j, by original
// index).  k_scores: kg.n slots x 4 rows x n; row 2 of slot g receives, per
// object, the number of lists that hold it at a rank in [k_{g-1}, k_g) (must
// start at zero; launch_select_k_finish turns them into in-degrees); row 3 is
// the mean distance to the k_g nearest.
snaps_status launch_select_join(const float4 *x, int64_t n, const SelectSpec &sp, const KGrid &kg,
                                float *eps_scores, float *k_scores, cudaStream_t st);

// The k grid when k_max > kSelectWarpK: one CTA per object keeps its k_max
// nearest in shared memory; writes rows 2 and 3 of k_scores as above.
snaps_status launch_select_knn(const float4 *x, int64_t n, uint32_t mask, const KGrid &kg, float *k_scores,
                               cudaStream_t st);

// Row 2 of every k slot: prefix sums over the slots, giving the in-degree at k_g.
snaps_status launch_select_k_finish(int64_t n, const KGrid &kg, float *k_scores, cudaStream_t st);

// Radii for target selectivities of one subspace (Sec. 3.5.3): m sampled
// objects (original indices floor(s n / m)) against all others; eps_mean is
// the mean of those distances, the histogram has n_bins bins over
// [0, eps_mean), and eps[t] is the first bin edge at which the sampled mean
// neighbour count reaches target[t] (eps_mean if none does).  scratch holds
// selectivity_scratch_bytes(n); eps (n targets floats) and eps_mean (1 float,
// may be NULL) are device memory.
constexpr int kSelectMaxTargets = 32;
constexpr double kSelQuantum = 1.0 / 1048576.0;  // distance quantum of the exact mean

struct SelectivityTargets {
    int n;  // targets
    int m;  // sampled objects, 1..n
    double target[kSelectMaxTargets];  // mean neighbours per object, > 0
};

size_t selectivity_scratch_bytes(int64_t n);
snaps_status launch_selectivity(const float4 *x, int64_t n, uint32_t mask, int n_bins, const SelectivityTargets &tg,
                                void *scratch, float *eps, float *eps_mean, cudaStream_t st);

}  // namespace snaps
