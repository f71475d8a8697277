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

// One subspace's eps grid and k_max, as the select join kernel takes them.
struct SelectSpec {
    uint32_t mask;
    int n_eps;                    // 0: no eps grid
    float e2[kSelectMaxGrid];     // ascending squared radii eps_j^2
    float qscale;                 // 2^24 / eps_max: quantisation of the distance sums
    int kmax;                     // 0: no kNN lists
};

struct KGrid {
    int n;
    int k[kSelectMaxGrid];        // ascending, <= kmax
};

// eps_scores: n_eps slots x 4 rows x n (rows 0 and 1 written: eps-neighbour
// count and mean distance at eps_j, by original index); knn_idx / knn_d2:
// n x kmax, the k_max nearest (original indices, squared distances) of every
// object, nearest first.
snaps_status launch_select_join(const float4 *x, int64_t n, const SelectSpec &sp, float *eps_scores,
                                int32_t *knn_idx, float *knn_d2, cudaStream_t st);

// k_scores: kg.n slots x 4 rows x n; rows 2 (in-degree, added to: must start
// at zero) and 3 (mean kNN distance) at every k_j.
snaps_status launch_select_k(const int32_t *knn_idx, const float *knn_d2, int64_t n, int kmax, const KGrid &kg,
                             float *k_scores, cudaStream_t st);

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
