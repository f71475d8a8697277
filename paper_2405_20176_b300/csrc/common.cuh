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
};
constexpr unsigned kErrTimeout = 1u;

}  // namespace snaps
