// Sort-by-cell grid index and grid-indexed self-join for low-dimensional
// subspaces (DSSJ, Sec. 3.5; kNNSJ, Sec. 3.6; index design after Sec. 3.8.1).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"
#include "join.cuh"

namespace snaps {

// Subspaces of at most this many features can take the grid path; the grid
// indexes at most kGridIndexDims of them (the highest), and every candidate
// found through it is refined with all of the subspace's features.
constexpr int kGridMaxDim = 4;
constexpr int kGridIndexDims = 3;
// Largest number of cells of one subspace's grid.
constexpr int kGridMaxCells = 1 << 22;

// One subspace's grid, as planned on the host.
struct GridSpec {
    int d;            // features in the subspace (2..kGridMaxDim)
    int D;            // index dimensions: min(d, kGridIndexDims)
    int feat[4];      // the subspace's features, highest first; -1 past d
    float lo[3];      // grid origin per index dimension (stored feature units)
    float w, inv_w;   // cell width and its inverse: R w >= eps, with a 2^-10 margin
    int R;            // block radius in cells: every eps-neighbour is within R cells per dimension
    int nc[3];        // cells per index dimension
    int ncells;       // product of nc
    float eps2;       // squared radius; < 0: no eps join
    int slot;         // output slot (index into the request's mask list)
};

// Device buffers of one subspace's index, carved out of one scratch block.
struct GridBufs {
    uint32_t *k_in, *k_out;  // cell keys before / after the sort
    int32_t *v_in, *v_out;   // row numbers before / after the sort
    float4 *pts;             // gathered subspace features in cell order
    int32_t *orig;           // their original indices
    int32_t *start;          // cell starts (ncells + 1)
    void *tmp;               // radix-sort temporary storage
    size_t tmp_bytes;
    int32_t *ring;           // queries left to the ring search (sorted positions)
    int32_t *ring_n;         // their number
};

// Device bytes the index of n objects with up to max_cells cells needs, and
// the buffers inside a block of that size (base NULL: sizes only).
size_t grid_scratch_bytes(int64_t n, int max_cells);
GridBufs grid_carve(void *base, int64_t n, int max_cells);

// Key bits of subspace g's cell ids (the radix sort's end bit).
int grid_key_bits(const GridSpec &g);

// Build subspace g's index over the population s.x (keys, radix sort by cell,
// cell starts, gathered points) in `b`, then run the grid join, writing slot
// g.slot of `o` (row 2, the in-degree, must be zero beforehand).
snaps_status run_grid_subspace(const JoinShape &s, const GridSpec &g, const JoinOut &o, const GridBufs &b,
                               cudaStream_t st);

}  // namespace snaps
