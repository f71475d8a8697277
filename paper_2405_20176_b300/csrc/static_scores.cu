// snaps_scores_static: scoring without any device allocation.
//
// Some callers cannot let a library allocate device memory: a process that
// shares one GPU under a fixed, pre-planned memory budget, or code that must
// not call cudaMalloc / cudaFree because those calls can synchronise the
// device and stall other work in flight.  This entry point serves them.  The
// caller passes its features and outputs in device memory; everything else the
// joins need (the normalised, padded population, the column statistics, the
// kernels' control block and the subspace plan) lives in one file-scope
// static device array of fixed size, kStaticScratchBytes, that every GPU which
// loads the library keeps until the process exits.  The call allocates
// nothing, on the device or on the host.
//
// Sharing: every call on a device uses the same array, and the array keeps the
// last call's contents.  The call clears what must start at zero (the control
// block and the in-degree rows of the outputs).  Calls whose GPU work overlaps
// -- on two streams, or from two host threads -- race on the array; issue them
// one after the other.

#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "common.cuh"
#include "join.cuh"
#include "prep.cuh"
#include "pointers.h"

namespace snaps {
namespace {

constexpr int64_t kStaticMaxN = 32768;            // objects
constexpr int kStaticMaxMasks = 32768;            // subspaces per call
constexpr int kStaticMaxChunks = 1024;            // 2^(15 - 5) high parts
constexpr int kStaticMaxGroups = kStaticMaxMasks / 32;

constexpr size_t align256(size_t v) { return (v + 255) & ~size_t(255); }
constexpr size_t kOffPop = 0;
constexpr size_t kPopBytes = align256((size_t)kStaticMaxN * kRowFloats * sizeof(float));
constexpr size_t kOffPair = kOffPop + kPopBytes;  // the rows again, pair-planar (tree join)
constexpr size_t kOffStats = kOffPair + kPopBytes;
constexpr size_t kOffBad = kOffStats + align256(sizeof(ColStats) * 16);
constexpr size_t kOffCtrl = kOffBad + 256;
constexpr size_t kOffChunks = kOffCtrl + align256(sizeof(DeviceControl));
constexpr size_t kOffGroups = kOffChunks + align256(sizeof(TreeChunk) * kStaticMaxChunks);
constexpr size_t kStaticScratchBytes = kOffGroups + align256(sizeof(MaskGroup) * kStaticMaxGroups);

// The scratch array.  In host code its name is only a stand-in; the device
// address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_static_mu;

// Host staging of the subspace plan: fixed arrays, no heap.
TreeChunk g_plan_chunks[kStaticMaxChunks];
MaskGroup g_plan_groups[kStaticMaxGroups];
int16_t g_slot_of[kStaticMaxChunks * kTreeWidth];
int16_t g_count_of[kStaticMaxChunks];
uint16_t g_lone[kStaticMaxMasks];

float default_or_given_eps2(const uint16_t *masks, const float *eps, int m)
{
    return eps ? eps[m] * eps[m] : default_eps2(__builtin_popcount(masks[m]));
}

// Device (or managed) memory that the kernels on `device` may use; memory of
// another GPU does not qualify.
bool device_memory(const void *p, int device) { return ptr_kind(p, device) == PtrKind::Device; }

}  // namespace
}  // namespace snaps

using namespace snaps;

#define STATIC_FAIL(code, ...)          \
    do {                                \
        snaps::set_error(__VA_ARGS__);  \
        return code;                    \
    } while (0)

extern "C" snaps_status snaps_scores_static(int device, const float *feat, int64_t n, int f,
                                            uint32_t flags, const uint16_t *masks, int n_masks,
                                            int k, const float *eps, float *scores, int32_t *top,
                                            int top_n, void *stream)
{
    clear_error();
    if (device < 0 || device >= kMaxDevices) STATIC_FAIL(SNAPS_EINVAL, "device %d out of range", device);
    if (!feat || !masks || !scores) STATIC_FAIL(SNAPS_EINVAL, "feat, masks and scores must be non-NULL");
    if (n < 2 || n > kStaticMaxN)
        STATIC_FAIL(SNAPS_EINVAL, "n must be in 2..%lld for the allocation-free call (got %lld)",
                    (long long)kStaticMaxN, (long long)n);
    if (f < 1 || f > SNAPS_MAX_FEATURES) STATIC_FAIL(SNAPS_EINVAL, "f must be in 1..15 (got %d)", f);
    if (flags & ~(SNAPS_NORM_MINMAX | SNAPS_NAN_TO_MEAN)) STATIC_FAIL(SNAPS_EINVAL, "unknown flags 0x%x", flags);
    if (n_masks < 1 || n_masks > kStaticMaxMasks)
        STATIC_FAIL(SNAPS_EINVAL, "n_masks must be in 1..%d for the allocation-free call (got %d)",
                    kStaticMaxMasks, n_masks);
    if (k < 1 || k > SNAPS_MAX_K || k > n - 1)
        STATIC_FAIL(SNAPS_EINVAL, "k must be in 1..min(%d, n-1) (got %d)", SNAPS_MAX_K, k);
    if (top && (top_n < 1 || top_n > 1024 || top_n > n))
        STATIC_FAIL(SNAPS_EINVAL, "top_n must be in 1..min(1024, n) (got %d)", top_n);
    for (int m = 0; m < n_masks; ++m) {
        const uint32_t v = masks[m];
        if (__builtin_popcount(v) < 2 || (v >> f) != 0)
            STATIC_FAIL(SNAPS_EINVAL, "mask %d (0x%x) must have 2..%d bits, all below feature %d", m, v, f, f);
        if (eps && !(eps[m] >= 0.f && eps[m] < 3.0e18f))
            STATIC_FAIL(SNAPS_EINVAL, "eps[%d] must be a finite value >= 0", m);
    }
    // the caller's current device is restored on every return path
    DeviceScope device_scope(device);
    if (device_scope.error() != cudaSuccess)
        STATIC_FAIL(SNAPS_ECUDA, "cudaSetDevice(%d) failed: %s", device, cudaGetErrorString(device_scope.error()));
    if (!device_memory(feat, device) || !device_memory(scores, device) || (top && !device_memory(top, device)))
        STATIC_FAIL(SNAPS_EINVAL, "feat, scores and top must be memory of device %d for the allocation-free call",
                    device);

    std::lock_guard<std::mutex> guard(g_static_mu);
    // The array's device address, with this device current.  Looked up on
    // every call: after a context reset the module is loaded again and the
    // address can change.  The first call on a device may make the CUDA driver
    // load the library's device code, and with it create the array.
    void *addr = nullptr;
    {
        const cudaError_t e = cudaGetSymbolAddress(&addr, g_static_scratch);
        if (e != cudaSuccess || !addr)
            STATIC_FAIL(SNAPS_ECUDA, "cudaGetSymbolAddress of the static scratch failed: %s",
                        cudaGetErrorString(e));
    }
    char *base = (char *)addr;
    float4 *pop = (float4 *)(base + kOffPop);
    float4 *pair = (float4 *)(base + kOffPair);
    ColStats *stats = (ColStats *)(base + kOffStats);
    unsigned *bad = (unsigned *)(base + kOffBad);
    DeviceControl *ctrl = (DeviceControl *)(base + kOffCtrl);
    TreeChunk *d_chunks = (TreeChunk *)(base + kOffChunks);
    MaskGroup *d_groups = (MaskGroup *)(base + kOffGroups);
    cudaStream_t st = (cudaStream_t)stream;

    // Plan: chunks with >= 2 requested subspaces go to the tree kernel, the
    // rest (and repeats) to the lane-per-subspace kernel.
    const int n_chunk = f > kTreeLowBits ? 1 << (f - kTreeLowBits) : 1;
    for (int i = 0; i < n_chunk * kTreeWidth; ++i) g_slot_of[i] = -1;
    std::memset(g_count_of, 0, sizeof(int16_t) * n_chunk);
    int n_lone = 0;
    for (int m = 0; m < n_masks; ++m) {
        const uint32_t v = masks[m];
        int16_t &slot = g_slot_of[(v >> kTreeLowBits) * kTreeWidth + (v & (kTreeWidth - 1))];
        if (slot >= 0) {
            g_lone[n_lone++] = (uint16_t)m;
            continue;
        }
        slot = (int16_t)m;
        ++g_count_of[v >> kTreeLowBits];
    }
    int n_chunks = 0;
    for (int c = 0; c < n_chunk; ++c) {
        if (g_count_of[c] == 0) continue;
        if (g_count_of[c] == 1) {
            for (int L = 0; L < kTreeWidth; ++L)
                if (g_slot_of[c * kTreeWidth + L] >= 0) g_lone[n_lone++] = (uint16_t)g_slot_of[c * kTreeWidth + L];
            continue;
        }
        TreeChunk &ch = g_plan_chunks[n_chunks++];
        ch.high = (uint32_t)c;
        ch.active = 0;
        for (int L = 0; L < kTreeWidth; ++L) {
            const int m = g_slot_of[c * kTreeWidth + L];
            ch.slot[L] = m;
            ch.eps2[L] = m >= 0 ? default_or_given_eps2(masks, eps, m) : -1.f;
            if (m >= 0) ch.active |= 1u << L;
        }
    }
    int n_groups = 0;
    for (int b = 0; b < n_lone; b += 32) {
        MaskGroup &g = g_plan_groups[n_groups++];
        for (int l = 0; l < 32; ++l) {
            if (b + l < n_lone) {
                const int m = g_lone[b + l];
                g.mask[l] = masks[m];
                g.eps2[l] = default_or_given_eps2(masks, eps, m);
                g.slot[l] = m;
            } else {
                g.mask[l] = 0;
                g.eps2[l] = -1.f;
                g.slot[l] = -1;
            }
        }
    }

    const int64_t n_pad = padded_rows(n);
    if (n_chunks > 0)
        SNAPS_CHECK_CUDA(cudaMemcpyAsync(d_chunks, g_plan_chunks, sizeof(TreeChunk) * n_chunks,
                                         cudaMemcpyHostToDevice, st));
    if (n_groups > 0)
        SNAPS_CHECK_CUDA(cudaMemcpyAsync(d_groups, g_plan_groups, sizeof(MaskGroup) * n_groups,
                                         cudaMemcpyHostToDevice, st));
    SNAPS_CHECK_CUDA(cudaMemsetAsync(ctrl, 0, sizeof(DeviceControl), st));
    SNAPS_CHECK_CUDA(cudaMemsetAsync(scores, 0, (size_t)n_masks * 4 * n * sizeof(float), st));
    SNAPS_TRY(launch_normalise(feat, n, n_pad, f, flags, stats, bad, pop, st));
    unsigned h_bad = 0, h_err = 0;
    SNAPS_CHECK_CUDA(cudaMemcpyAsync(&h_bad, bad, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    SNAPS_CHECK_CUDA(cudaStreamSynchronize(st));
    if (h_bad) STATIC_FAIL(SNAPS_EINVAL, "features must be finite (NaN is allowed only with SNAPS_NAN_TO_MEAN)");
    JoinShape shape{pop, n, n_pad, k};
    JoinOut out{scores, nullptr, nullptr, nullptr};
    if (n_chunks > 0) {
        // the tree join reads the rows in the pair-planar layout (one copy, input order)
        SNAPS_TRY(launch_gather_chunks(pop, nullptr, nullptr, n, n_pad, 1, pair, st));
        JoinShape ts = shape;
        ts.x = pair;
        SNAPS_TRY(launch_join_tree(ts, d_chunks, n_chunks, out, ctrl, st));
    }
    SNAPS_TRY(launch_join_lanemask(shape, d_groups, n_groups, out, ctrl, st));
    if (top) SNAPS_TRY(launch_top(scores, n, n_masks, top_n, top, st));
    SNAPS_CHECK_CUDA(cudaMemcpyAsync(&h_err, &ctrl->error, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    SNAPS_CHECK_CUDA(cudaStreamSynchronize(st));
    if (h_err & kErrBadRow) STATIC_FAIL(SNAPS_ECUDA, "a join kernel met rows without a valid original index (error word 0x%x)", h_err);
    if (h_err) STATIC_FAIL(SNAPS_ETIMEOUT, "a device-side wait gave up (error word 0x%x)", h_err);
    return SNAPS_OK;
}
