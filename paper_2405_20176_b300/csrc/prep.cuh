// Launchers for population preparation and per-subspace finishing kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"
#include "join.cuh"

namespace snaps {

struct ColStats {
    double lo, hi, mean;
    long long count;  // non-NaN values
};

// in_dev: n x f row-major floats on the device.  stats: f entries.  bad: one
// word set non-zero when a value is NaN (without SNAPS_NAN_TO_MEAN) or +-inf.
// out: the padded quad-planar population (n_pad rows) in the input's order;
// float 15 of every real row holds its original index.
snaps_status launch_normalise(const float *in_dev, int64_t n, int64_t n_pad, int f,
                              uint32_t flags, ColStats *stats, unsigned *bad, float4 *out,
                              cudaStream_t st);

// Maps each stored feature onto [0, 1] for cell keys: (v - lo) * scale.
struct KeyRange {
    float lo[16];
    float scale[16];
};

// Sort-by-cell index: 30-bit cell keys (2 bits per feature, interleaved) and
// the identity permutation, then the rows gathered into sorted order.
snaps_status launch_cell_keys(const float4 *x, int64_t n, const KeyRange &kr, uint32_t *keys,
                              int32_t *idx, cudaStream_t st);
snaps_status launch_gather_rows(const float4 *src, const int32_t *perm, int64_t n, int64_t n_pad,
                                float4 *dst, cudaStream_t st);

// Per-chunk orders for the subspace-batched join.  For chunk g of `chunks`
// (high part H), keys[g * n + r] = g << 32 | the Morton key of row r over the
// features in H (feature 5 + b for bit b of H; features 0..4 when H = 0), each
// quantised to min(10, 30 / |features|) bits; vals[g * n + r] = r.
snaps_status launch_chunk_keys(const float4 *x, int64_t n, int f, const TreeChunk *chunks, int n_chunks,
                               const KeyRange &kr, uint64_t *keys, int32_t *vals, cudaStream_t st);

// out[g] (n_pad rows each, pair-planar layout) <- the rows of x in chunk g's
// sorted order perm[g * n ..] (perm NULL: x's own order); padding rows are +inf.
// chunks non-NULL: each copy holds its chunk's high features compacted, the
// highest first, in floats 5.., and 0 after them (+inf in padding rows).
snaps_status launch_gather_chunks(const float4 *x, const int32_t *perm, const TreeChunk *chunks, int64_t n,
                                  int64_t n_pad, int n_chunks, float4 *out, cudaStream_t st);

// Step boxes of chunk row copies: boxes[(g * 10 + b) * (n_pad / 64) + s] =
// (min, max) of float 5 + b over the 64 rows of step s of copy g (padding
// rows count as +inf).
snaps_status launch_chunk_boxes(const float4 *copies, int64_t n_pad, int n_chunks, float2 *boxes,
                                cudaStream_t st);

// Copy the first f features of the n population rows out as n x f row-major,
// in the objects' original order.
snaps_status launch_unpack(const float4 *x, int64_t n, int f, float *out, cudaStream_t st);

// The finishing kernel (finish.cu), one launch for both outputs:
// norm[slot][m][i] from scores[slot][m][i] (n_slots x 4 x n each; NULL skips
// it) and top[slot][m][0..top_n) (NULL or top_n == 0 skips it).
snaps_status launch_finish(const float *scores, int64_t n, int n_slots, float *norm, int top_n, int32_t *top,
                           cudaStream_t st);
snaps_status launch_norm(const float *scores, int64_t n, int n_slots, float *norm, cudaStream_t st);
snaps_status launch_top(const float *scores, int64_t n, int n_slots, int top_n, int32_t *top,
                        cudaStream_t st);

}  // namespace snaps
