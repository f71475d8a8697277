// Shared definitions of libsnaps: status plumbing, the device-side layout of
// a population and the warp-level building blocks of the joins.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "snaps.h"

namespace snaps {

// ---- host-side error plumbing ---------------------------------------------

// Record a message for snaps_last_error() on the calling thread.
void set_error(const char *fmt, ...);
void clear_error();

#define SNAPS_CHECK_CUDA(expr)                                                        \
    do {                                                                              \
        cudaError_t _e = (expr);                                                      \
        if (_e != cudaSuccess) {                                                      \
            ::snaps::set_error("%s failed: %s (%s:%d)", #expr, cudaGetErrorString(_e), \
                               __FILE__, __LINE__);                                   \
            return SNAPS_ECUDA;                                                       \
        }                                                                             \
    } while (0)

#define SNAPS_TRY(expr)                      \
    do {                                     \
        snaps_status _s = (expr);            \
        if (_s != SNAPS_OK) return _s;       \
    } while (0)

// ---- population layout -------------------------------------------------------

// Every object is a row of 16 floats: features 0..f-1, then zeros.  Rows are
// grouped in tiles of kRowPad rows, and a tile is stored quad-planar: the
// first float4 (features 0-3) of all its rows, then the second float4 of all
// rows, and so on -- 16 KB per tile, contiguous, so one 1-D bulk copy stages a
// tile and lanes reading consecutive rows hit distinct shared-memory banks.
// The row count is padded to whole tiles with rows whose 16 floats are +inf,
// so any squared distance to a padding row is +inf and fails every radius and
// kNN test without a bounds check.
constexpr int kRowFloats = 16;
constexpr int kRowPad = 256;

// float4 index of quad q (features 4q..4q+3) of row i.
__host__ __device__ inline int64_t row_quad(int64_t i, int q) {
    return ((i / kRowPad) * 4 + q) * kRowPad + (i % kRowPad);
}

// Pair-planar layout of the subspace-batched join's per-chunk row copies.  The
// 64 rows of step s = p / 64 form 8 planes of 32 float4; lane l's float4 in
// plane q holds features 2q and 2q + 1 of rows a = 64s + l and b = 64s + 32 + l
// as (a[2q], b[2q], a[2q + 1], b[2q + 1]), so that one 16-byte load gives two
// (a, b) operand pairs for the f32x2 instructions.
// float4 index of plane q of row p's pair:
__host__ __device__ inline int64_t pair_plane(int64_t p, int q) {
    return ((p >> 6) * 8 + q) * 32 + (p & 31);
}
// float index of feature f of row p:
__host__ __device__ inline int64_t pair_float(int64_t p, int f) {
    return pair_plane(p, f >> 1) * 4 + (f & 1) * 2 + ((p >> 5) & 1);
}

inline int64_t padded_rows(int64_t n) { return (n + kRowPad - 1) / kRowPad * kRowPad; }

// Default squared radius for a d-feature subspace: eps = 0.05 sqrt(d), so
// eps^2 = 0.0025 d, evaluated in FP64 and rounded once to FP32.
inline float default_eps2(int d) { return (float)(0.0025 * (double)d); }

// Control block in device memory shared by a launch: a work counter for the
// persistent kernels and an error word a bounded wait sets when it gives up.
struct DeviceControl {
    unsigned long long next_work;
    unsigned int error;   // 0 = fine; otherwise a kErr* code
    unsigned int pad;
    // subspace-batched join: 64-row steps of the candidate streams that were
    // loaded (not skipped by their box bound), and all steps, summed over the
    // launches since they were last cleared
    unsigned long long steps_loaded;
    unsigned long long steps_total;
};
constexpr unsigned kErrTimeout = 1u;
constexpr unsigned kErrBadRow = 2u;  // a row's stored original index is out of range

}  // namespace snaps
