// Host-visible description of one join launch, shared by the join kernels and
// the C-ABI layer.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace snaps {

// Up to 32 subspaces handled together by the lane-per-subspace kernel.  An
// unused entry has mask 0.
struct MaskGroup {
    uint32_t mask[32];
    float eps2[32];   // squared radius; < 0 disables the eps join for that subspace
    int32_t slot[32]; // output slot (index into the request's mask list)
};

// The 2^kTreeLowBits subspaces (H << kTreeLowBits) | L, L = 0..2^kTreeLowBits-1,
// of one high part H, as scheduled for the subspace-batched tree kernel.
constexpr int kTreeLowBits = 5;
constexpr int kTreeWidth = 1 << kTreeLowBits;
// A chunk goes to the subspace-batched kernel when at least this many of its
// subspaces are requested.  Its shared walk costs about 45 FP32-pipe
// operations per candidate pair whatever the number requested (plus about 3
// per requested subspace for events); a subspace joined on its own costs about
// 1.25 d + 8 (18 at d = 8).  Below four, the lone joins cost less.
constexpr int kTreeMinActive = 4;
struct TreeChunk {
    uint32_t high;                 // H
    uint32_t active;               // bit L set when subspace (H << 5) | L is requested
    float eps2[kTreeWidth];        // per L, as in MaskGroup
    int32_t slot[kTreeWidth];
};

// Up to 256 subspaces of any kind, as scheduled for the tensor-core join (two
// MMAs of M = 128 share each B operand).  An unused entry has mask 0.
constexpr int kTcBlockWidth = 256;
struct TcBlock {
    uint32_t mask[kTcBlockWidth];
    float eps2[kTcBlockWidth];
    int32_t slot[kTcBlockWidth];
};

// Outputs of a join.  `scores` is always present: n_slots x 4 x n floats; the
// join writes rows 0 (eps count), 1 (eps mean distance) and 3 (kNN mean
// distance) and adds 1 to row 2 (in-degree) of every kNN list member, so row 2
// must be zero before the launch.
struct JoinOut {
    float *scores;
    int32_t *knn_idx;   // n_slots x n x k, or null
    float *knn_dist;    // n_slots x n x k, or null
    int32_t *eps_count; // n_slots x n, or null
};

struct JoinShape {
    const float4 *x;    // n_pad rows of 16 floats (4 float4)
    int64_t n;
    int64_t n_pad;
    int k;              // 0 disables the kNN join
    // subspace-batched join only: float4 offset between the row copies of
    // consecutive chunks (each chunk's rows in its own order); 0 = one shared copy
    int64_t chunk_stride = 0;
    // subspace-batched join only, optional: per chunk, the (min, max) of each
    // high feature 5 + b over the 64 rows of every step of its row copy, at
    // box[chunk * box_stride + b * (n_pad / 64) + step]
    const float2 *box = nullptr;
    int64_t box_stride = 0;
    // subspace-batched join only: every chunk's copy holds its high features
    // compacted, the highest first, in floats 5.. (0 after them); the boxes
    // then follow the same order
    bool compact = false;
    // tensor-core join only: spins after which a pipeline wait gives up and the
    // launch reports kErrTimeout (0 = dev::kSpinLimit).  Waits for copies and
    // MMAs already in flight, on the way out, always use dev::kSpinLimit.
    unsigned wait_limit = 0;
};

// Launch the lane-per-subspace join over `n_groups` groups (device array).
snaps_status launch_join_lanemask(const JoinShape &s, const MaskGroup *groups, int n_groups,
                                  const JoinOut &o, DeviceControl *ctrl, cudaStream_t st);

// Launch the subspace-at-a-time join over every used entry of `n_groups`
// groups (device array): one launch row per entry, a CTA per 256 queries.
snaps_status launch_join_single(const JoinShape &s, const MaskGroup *groups, int n_groups,
                                const JoinOut &o, cudaStream_t st);

// One subspace of one population in a work list that spans several calls
// (the serving loop fuses the subspaces joined on their own of every small
// request it admits together into one launch).  The CTA's output goes to
// scores[4][n] of that subspace: eps count, mean eps distance, in-degree (added
// to, so it must start at zero) and mean kNN distance.
struct WorkItem {
    const float4 *x;   // the population's stored rows (n_pad rows)
    float *scores;     // this subspace's 4 x n block
    int n;
    int k;             // 1..32
    uint32_t mask;
    float eps2;        // < 0 disables the eps join
    int first_cta;     // the item's first CTA in the launch (items in order)
    int pad;
};

// Launch the subspace-at-a-time join over a work list of `n_items` items
// (device array) whose CTAs number `n_ctas` in all (item i owns CTAs
// first_cta[i] .. first_cta[i + 1] - 1, one per 256 queries); every item's k
// must be <= kmax (16 or 32).
snaps_status launch_join_worklist(const WorkItem *items, int n_items, int n_ctas, int kmax, cudaStream_t st);

// Operand forms of the tensor-core join.
constexpr int kTcFormF16 = 0, kTcFormBF16 = 1, kTcFormTF32 = 2;

// Launch the tensor-core filtered join over `n_blocks` blocks (device array)
// with FP16, BF16 or TF32 high/low parts (`form`).  Requires every feature of
// the population to span at most 1.
snaps_status launch_join_tc(const JoinShape &s, const TcBlock *blocks, int n_blocks, int form,
                            const JoinOut &o, DeviceControl *ctrl, cudaStream_t st);

// Launch the subspace-batched tree join over `n_chunks` chunks (device array).
// `s.x` holds the rows in the pair-planar layout (common.cuh): one copy per
// chunk, s.chunk_stride float4 apart, or one shared copy (chunk_stride 0).
snaps_status launch_join_tree(const JoinShape &s, const TreeChunk *chunks, int n_chunks,
                              const JoinOut &o, DeviceControl *ctrl, cudaStream_t st);

}  // namespace snaps
