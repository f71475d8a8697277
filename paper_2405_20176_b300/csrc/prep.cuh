// Launchers for population preparation and per-subspace finishing kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace snaps {

struct ColStats {
    double lo, hi, mean;
    long long count;  // non-NaN values
};

// in_dev: n x f row-major floats on the device.  stats: f entries.  bad: one
// word set non-zero when a value is NaN (without SNAPS_NAN_TO_MEAN) or +-inf.
// out: the padded quad-planar population (n_pad rows).
snaps_status launch_normalise(const float *in_dev, int64_t n, int64_t n_pad, int f,
                              uint32_t flags, ColStats *stats, unsigned *bad, float4 *out,
                              cudaStream_t st);

// Copy the first f features of the n population rows out as n x f row-major.
snaps_status launch_unpack(const float4 *x, int64_t n, int f, float *out, cudaStream_t st);

// norm[slot][m][i] from scores[slot][m][i] (n_slots x 4 x n each).
snaps_status launch_norm(const float *scores, int64_t n, int n_slots, float *norm, cudaStream_t st);

// top[slot][m][0..top_n) from scores (n_slots x 4 x n).
snaps_status launch_top(const float *scores, int64_t n, int n_slots, int top_n, int32_t *top,
                        cudaStream_t st);

}  // namespace snaps
