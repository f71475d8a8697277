// C ABI of libsnaps (include/snaps.h): contexts, resident populations, the
// synchronous join / scoring calls and the continuous-batching request loop.

#include <cuda_runtime.h>

#include <cub/device/device_radix_sort.cuh>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <tuple>
#include <vector>

#include "common.cuh"
#include "join.cuh"
#include "prep.cuh"
#include "grid.cuh"
#include "select.cuh"
#include "pointers.h"

// ---- error plumbing -----------------------------------------------------------------

namespace snaps {
namespace {
thread_local char g_err[512] = "";
}
const char *last_error_message() { return g_err; }
void set_error(const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}
void clear_error() { g_err[0] = '\0'; }
}  // namespace snaps

using namespace snaps;

#define FAIL(code, ...)                 \
    do {                                \
        snaps::set_error(__VA_ARGS__);  \
        return code;                    \
    } while (0)

// Make `dev` current for the rest of the entry point; the caller's current
// device is restored when the entry point returns.
#define ON_DEVICE(dev)                                                                    \
    DeviceScope device_scope_(dev);                                                      \
    if (device_scope_.error() != cudaSuccess)                                            \
    FAIL(SNAPS_ECUDA, "cudaSetDevice(%d) failed: %s", (int)(dev),                        \
         cudaGetErrorString(device_scope_.error()))

// ---- objects -------------------------------------------------------------------------

namespace {

using Clock = std::chrono::steady_clock;

// Grow-only device buffer charged to a context's budget.
struct Scratch {
    void *ptr = nullptr;
    size_t cap = 0;
};

struct Request;

struct Slot {
    cudaStream_t stream = nullptr;
    Scratch scratch;
    DeviceControl *ctrl = nullptr;
    std::thread worker;
};

}  // namespace

struct snaps_ctx {
    int device = 0;
    size_t budget = 0;
    size_t held = 0;  // bytes allocated through this context
    std::mutex mem_mu;

    // synchronous calls share one scratch area and control block
    std::mutex sync_mu;
    Scratch scratch;
    DeviceControl *ctrl = nullptr;

    // serving
    std::mutex q_mu;
    std::condition_variable q_cv;    // workers wait for work / memory
    std::condition_variable done_cv; // pollers wait for completion
    std::deque<Request *> queue;
    std::unordered_map<uint64_t, Request *> tickets;
    uint64_t next_ticket = 1;
    size_t reserved = 0;  // bytes reserved by admitted requests
    int n_slots = 4;
    std::vector<Slot *> slots;
    bool stopping = false;
    std::atomic<long long> fused_launches{0};  // launches that joined two or more requests
    std::atomic<long long> fused_requests{0};  // requests served by those launches
    std::atomic<int> n_pops{0};

    // kernels one radix sort launches, by n (counted from a stream capture
    // that records the sort without running it; only while tracing)
    std::mutex cap_mu;
    cudaStream_t cap_stream = nullptr;
    std::unordered_map<int64_t, int> sort_kernels;

    // spins after which a tensor-core pipeline wait gives up (0 = the default)
    std::atomic<unsigned> wait_limit{0};

    // index route per (population size class, subspace dimension, k class),
    // recorded by snaps_autotune
    std::mutex tune_mu;
    std::unordered_map<uint32_t, snaps_tune_entry> tune;
    // fewest subspaces a tensor-core block carries, per (size class, k class),
    // recorded by snaps_autotune_tc; a value set by snaps_set_tc_min_fill
    // (> 0) overrides it for every size
    std::unordered_map<uint32_t, int> tc_fill;
    std::atomic<int> tc_fill_override{0};

    // tracing
    std::mutex tr_mu;
    bool tracing = false;
    struct Mark { int phase; int kernels; cudaEvent_t a, b; };
    std::vector<Mark> marks;
    std::vector<cudaEvent_t> spare;
};

struct snaps_pop {
    snaps_ctx *ctx = nullptr;
    int64_t n = 0, n_pad = 0;
    int f = 0;
    bool unit_range = false;  // every stored feature spans <= 1 (tensor-core filter allowed)
    float4 *x = nullptr;
    size_t bytes = 0;
    KeyRange kr{};           // maps stored features onto [0, 1] for cell keys
    std::atomic<int> inflight{0};
};

namespace {

struct Request {
    uint64_t ticket = 0;
    snaps_request req{};
    std::vector<uint16_t> masks;
    std::vector<float> eps;
    size_t footprint = 0;
    // every subspace joined on its own (plain form, no chunk of kTreeMinActive
    // or more, no grid index) and little work: may share a launch with others
    bool fusable = false;
    Clock::time_point t_submit, t_admit, t_done;
    bool done = false;
    bool running = false;
    snaps_status status = SNAPS_OK;
};

snaps_status ctx_alloc(snaps_ctx *ctx, size_t bytes, void **p)
{
    {
        std::lock_guard<std::mutex> g(ctx->mem_mu);
        if (ctx->held + bytes > ctx->budget)
            FAIL(SNAPS_ENOMEM, "allocation of %zu bytes exceeds the HBM budget (%zu of %zu held)",
                 bytes, ctx->held, ctx->budget);
        ctx->held += bytes;
    }
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        std::lock_guard<std::mutex> g(ctx->mem_mu);
        ctx->held -= bytes;
        cudaGetLastError();
        FAIL(SNAPS_ENOMEM, "cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
    }
    return SNAPS_OK;
}

void ctx_free(snaps_ctx *ctx, void *p, size_t bytes)
{
    if (!p) return;
    cudaFree(p);
    std::lock_guard<std::mutex> g(ctx->mem_mu);
    ctx->held -= bytes;
}

snaps_status scratch_reserve(snaps_ctx *ctx, Scratch &s, size_t bytes)
{
    if (bytes <= s.cap) return SNAPS_OK;
    ctx_free(ctx, s.ptr, s.cap);
    s.ptr = nullptr;
    s.cap = 0;
    bytes = (bytes + (1u << 20) - 1) & ~size_t((1u << 20) - 1);
    SNAPS_TRY(ctx_alloc(ctx, bytes, &s.ptr));
    s.cap = bytes;
    return SNAPS_OK;
}

bool is_device_ptr(const void *p)
{
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// EINVAL for a caller buffer in another GPU's memory: the kernels on the
// context's device would fault on it.
snaps_status check_not_foreign(const void *p, int device, const char *name)
{
    if (p && ptr_kind(p, device) == PtrKind::Foreign)
        FAIL(SNAPS_EINVAL, "%s is device memory of another GPU (the context runs on device %d)", name, device);
    return SNAPS_OK;
}

inline int popc16(uint32_t m) { return __builtin_popcount(m); }

// Carve aligned sub-buffers out of one scratch block.
struct Carver {
    size_t off = 0;
    char *base = nullptr;
    template <class T>
    T *take(size_t count)
    {
        off = (off + 255) & ~size_t(255);
        T *p = base ? reinterpret_cast<T *>(base + off) : nullptr;
        off += count * sizeof(T);
        return p;
    }
};

// Everything one scoring / join call needs, independent of who calls it.
struct JobSpec {
    snaps_pop *pop = nullptr;
    const uint16_t *masks = nullptr;
    int n_masks = 0;
    int k = 0;                 // 0: no kNN join
    const float *eps = nullptr;
    bool want_eps = true;
    uint32_t precision = SNAPS_FP32;
    float *scores = nullptr;   // n_masks x 4 x n
    float *norm = nullptr;
    int32_t *top = nullptr;
    int top_n = 0;
    int32_t *knn_idx = nullptr;
    float *knn_dist = nullptr;
    int32_t *eps_count = nullptr;
    float *eps_mean = nullptr;
};

snaps_status validate(const JobSpec &j)
{
    if (!j.pop) FAIL(SNAPS_EINVAL, "population is NULL");
    const snaps_pop *p = j.pop;
    if (j.n_masks < 1) FAIL(SNAPS_EINVAL, "n_masks must be >= 1 (got %d)", j.n_masks);
    if (!j.masks) FAIL(SNAPS_EINVAL, "masks is NULL");
    if (is_device_ptr(j.masks)) FAIL(SNAPS_EINVAL, "masks must be a host array");
    if (j.eps && is_device_ptr(j.eps)) FAIL(SNAPS_EINVAL, "eps must be a host array");
    {
        const int dev = p->ctx->device;
        SNAPS_TRY(check_not_foreign(j.scores, dev, "scores"));
        SNAPS_TRY(check_not_foreign(j.norm, dev, "norm"));
        SNAPS_TRY(check_not_foreign(j.top, dev, "top"));
        SNAPS_TRY(check_not_foreign(j.knn_idx, dev, "idx"));
        SNAPS_TRY(check_not_foreign(j.knn_dist, dev, "dist"));
        SNAPS_TRY(check_not_foreign(j.eps_count, dev, "count"));
        SNAPS_TRY(check_not_foreign(j.eps_mean, dev, "mean_dist"));
    }
    for (int m = 0; m < j.n_masks; ++m) {
        const uint32_t v = j.masks[m];
        if (popc16(v) < 2 || (v >> p->f) != 0)
            FAIL(SNAPS_EINVAL, "mask %d (0x%x) must have 2..%d bits, all below feature %d", m, v,
                 p->f, p->f);
        if (j.eps && !(j.eps[m] >= 0.f && j.eps[m] < 3.0e18f))
            FAIL(SNAPS_EINVAL, "eps[%d] must be a finite value >= 0", m);
    }
    if (j.k < 0 || j.k > SNAPS_MAX_K || (j.k > 0 && j.k > p->n - 1))
        FAIL(SNAPS_EINVAL, "k must be in 1..min(%d, n-1) (got %d, n %lld)", SNAPS_MAX_K, j.k,
             (long long)p->n);
    if (j.top && (j.top_n < 1 || j.top_n > 1024 || j.top_n > p->n))
        FAIL(SNAPS_EINVAL, "top_n must be in 1..min(1024, n) (got %d)", j.top_n);
    const uint32_t form = j.precision & 0xFFu, index = j.precision & ~0xFFu;
    if (form != SNAPS_FP32 && form != SNAPS_TC_F16 && form != SNAPS_TC_BF16 && form != SNAPS_TC_TF32)
        FAIL(SNAPS_EINVAL, "unknown precision %u", j.precision);
    if (index != 0u && index != SNAPS_INDEX_GRID && index != SNAPS_INDEX_NONE)
        FAIL(SNAPS_EINVAL, "unknown index choice in precision 0x%x", j.precision);
    if (form != SNAPS_FP32 && !p->unit_range)
        FAIL(SNAPS_EINVAL, "the tensor-core forms need every feature to span at most 1 "
                           "(index the population with SNAPS_NORM_MINMAX)");
    return SNAPS_OK;
}

// Split the requested subspaces between the tree kernel (chunks with >= kTreeMinActive
// requested subspaces) and the subspace-at-a-time kernel (everything else,
// listed in groups of 32).
struct Plan {
    std::vector<TreeChunk> chunks;
    std::vector<MaskGroup> groups;
    std::vector<TcBlock> blocks;
    std::vector<GridSpec> grids;  // low-dimensional subspaces on the grid index
    int grid_max_cells = 0;
    int order_batch = 0;  // chunks whose row orders are built at a time
};

// Device bytes for the per-chunk row orders of one batch of chunks: the row
// copies, sort keys and values (double-buffered) and the sort's temporary
// storage.
constexpr size_t kOrderBytes = size_t(4) << 30;

size_t order_chunk_bytes(const snaps_pop *p)
{
    return (size_t)p->n_pad * kRowFloats * sizeof(float) + (size_t)p->n * 2 * (sizeof(uint64_t) + sizeof(int32_t)) +
           (size_t)(p->n_pad / 64) * 10 * sizeof(float2);
}

int order_end_bit(int batch)
{
    int hb = 0;
    while ((1 << hb) < batch) ++hb;
    return 32 + hb;
}

size_t order_sort_temp(int64_t items, int end_bit)
{
    size_t bytes = 0;
    cub::DeviceRadixSort::SortPairs(nullptr, bytes, (const uint64_t *)nullptr, (uint64_t *)nullptr,
                                    (const int32_t *)nullptr, (int32_t *)nullptr, (int)items, 0, end_bit);
    return bytes;
}

// The grid of one low-dimensional subspace: cell width eps (the default radius
// when there is no eps join or eps is 0) with a 2^-10 margin, widened where
// needed so that the grid has at most kGridMaxCells cells.
// Key of the autotuner's table: floor(log2 n), the dimension, and whether the
// kNN lists take the k <= 16 or the k <= 32 form of the joins.
uint32_t tune_key(int64_t n, int d, int k)
{
    int nb = 0;
    while ((int64_t(1) << (nb + 1)) <= n) ++nb;
    return ((uint32_t)nb << 16) | ((uint32_t)d << 8) | (k > 16 ? 1u : 0u);
}

bool tune_lookup(snaps_ctx *ctx, int64_t n, int d, int k, snaps_tune_entry *e)
{
    std::lock_guard<std::mutex> g(ctx->tune_mu);
    auto it = ctx->tune.find(tune_key(n, d, k));
    if (it == ctx->tune.end()) return false;
    *e = it->second;
    return true;
}

// Fewest subspaces for which the tensor-core forms fill a block: the
// context's override, else snaps_autotune_tc's choice for this size and k
// class, else the built-in SNAPS_TC_MIN_FILL.
int tc_min_fill(snaps_ctx *ctx, int64_t n, int k)
{
    const int o = ctx->tc_fill_override.load();
    if (o > 0) return o;
    std::lock_guard<std::mutex> g(ctx->tune_mu);
    auto it = ctx->tc_fill.find(tune_key(n, 0, k));
    return it == ctx->tc_fill.end() ? SNAPS_TC_MIN_FILL : it->second;
}

GridSpec make_grid(const JobSpec &j, int m, float eps2, float cell_mult)
{
    const snaps_pop *p = j.pop;
    const uint32_t mask = j.masks[m];
    GridSpec g{};
    g.d = popc16(mask);
    g.D = std::min(g.d, kGridIndexDims);
    int t = 0;
    for (int f = 14; f >= 0; --f)
        if ((mask >> f) & 1u) g.feat[t++] = f;
    for (; t < 4; ++t) g.feat[t] = -1;
    const double eps = eps2 > 0.f ? std::sqrt((double)eps2) : std::sqrt(0.0025 * g.d);
    // cells eps (1 + 2^-10) * cell_mult wide: for cell_mult = 1 / R, R cells
    // per eps and a (2R + 1)^D block; for cell_mult >= 1, one cell and a 3^D block
    const double e1 = eps * (1.0 + 1.0 / 1024.0);
    const int r_req = cell_mult < 1.f ? std::max(1, (int)std::lround(1.0 / (double)cell_mult)) : 1;
    double w = cell_mult < 1.f ? e1 / r_req : e1 * std::max(1.0, (double)cell_mult);
    const int cap = (int)std::floor(std::pow((double)kGridMaxCells, 1.0 / g.D));
    double span[3];
    for (int q = 0; q < g.D; ++q) {
        const int f = g.feat[q];
        span[q] = p->kr.scale[f] > 0.f ? 1.0 / (double)p->kr.scale[f] : 0.0;
        g.lo[q] = p->kr.lo[f];
        w = std::max(w, span[q] / (cap - 1));
    }
    g.w = (float)w;
    g.inv_w = (float)(1.0 / w);
    // cells widened to respect the cell cap need fewer of them per eps
    g.R = std::max(1, std::min(r_req, (int)std::ceil(e1 / w - 1e-9)));
    g.ncells = 1;
    for (int q = 0; q < g.D; ++q) {
        g.nc[q] = std::min(cap, (int)std::floor(span[q] / w) + 1);
        g.ncells *= g.nc[q];
    }
    for (int q = g.D; q < 3; ++q) g.nc[q] = 1;
    g.eps2 = eps2;
    g.slot = m;
    return g;
}

Plan make_plan(const JobSpec &j)
{
    Plan pl;
    auto eps2_of = [&](int m) -> float {
        if (!j.want_eps) return -1.f;
        if (j.eps) return j.eps[m] * j.eps[m];
        return default_eps2(popc16(j.masks[m]));
    };
    // subspaces of <= kGridMaxDim features on the grid index (sort-by-cell, Sec. 3.8.1)
    const uint32_t index = j.precision & ~0xFFu;
    // requested subspaces per 32-subspace chunk: a subspace that shares its
    // chunk rides the tree kernel's shared walk; a lone one (and every one in
    // the tensor-core form) is joined on its own
    const bool tc_form = (j.precision & 0xFFu) != SNAPS_FP32;
    std::unordered_map<uint32_t, int> per_chunk;
    for (int m = 0; m < j.n_masks; ++m) ++per_chunk[(uint32_t)j.masks[m] >> kTreeLowBits];
    std::vector<int> rest;
    for (int m = 0; m < j.n_masks; ++m) {
        const int d = popc16(j.masks[m]);
        bool grid = false;
        // built-in cell width: a third of eps for a two-feature index (the 7 x 7
        // block covers 5.4 eps^2 around the eps-disk instead of 9 eps^2), eps
        // for a three-feature one
        float mult = d <= 2 ? 1.f / 3.f : 1.f;
        if (d <= kGridMaxDim && index != SNAPS_INDEX_NONE) {
            // the built-in rule: the index pays from SNAPS_GRID_AUTO_N objects on.
            // snaps_autotune's choice (grid against a subspace joined on its own)
            // decides for the subspaces that would be joined on their own.
            snaps_tune_entry te;
            const bool tuned = tune_lookup(j.pop->ctx, j.pop->n, d, j.k, &te);
            const bool alone = tc_form || per_chunk[(uint32_t)j.masks[m] >> kTreeLowBits] < kTreeMinActive;
            if (tuned) mult = te.cell_mult;
            grid = index == SNAPS_INDEX_GRID ||
                   (tuned && alone ? te.grid != 0 : j.pop->n >= SNAPS_GRID_AUTO_N);
        }
        if (grid) {
            pl.grids.push_back(make_grid(j, m, eps2_of(m), mult));
            pl.grid_max_cells = std::max(pl.grid_max_cells, pl.grids.back().ncells);
        } else {
            rest.push_back(m);
        }
    }
    if (tc_form) {
        // The tensor-core join takes any subspaces, a block of kTcBlockWidth
        // at a time, sorted by dimension so that the threads of a warp see
        // similar hit rates.  A block costs about the same however few
        // subspaces it carries, so a block is formed only with at least
        // min_fill of them; the subspaces left over (all of them in a small
        // request) take the plain FP32 routes below, which return the same
        // counts, lists and in-degrees.
        std::vector<int> order = rest;
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
            const int da = popc16(j.masks[a]), db = popc16(j.masks[b]);
            return da != db ? da < db : j.masks[a] < j.masks[b];
        });
        const int fill = std::max(1, tc_min_fill(j.pop->ctx, j.pop->n, j.k));
        int nr = (int)order.size();
        const int tail = nr % kTcBlockWidth;
        if (fill > kTcBlockWidth) nr = 0;
        else if (tail > 0 && tail < fill) nr -= tail;
        rest.assign(order.begin() + nr, order.end());
        for (int b = 0; b < nr; b += kTcBlockWidth) {
            TcBlock blk{};
            for (int c = 0; c < kTcBlockWidth; ++c) {
                const int m = b + c < nr ? order[b + c] : j.n_masks;
                if (m < j.n_masks) {
                    blk.mask[c] = j.masks[m];
                    blk.eps2[c] = !j.want_eps ? -1.f
                                  : j.eps ? j.eps[m] * j.eps[m]
                                          : default_eps2(popc16(j.masks[m]));
                    blk.slot[c] = m;
                } else {
                    blk.mask[c] = 0;
                    blk.eps2[c] = -1.f;
                    blk.slot[c] = -1;
                }
            }
            pl.blocks.push_back(blk);
        }
    }
    const int f = j.pop->f;
    const int n_chunk = f > kTreeLowBits ? 1 << (f - kTreeLowBits) : 1;
    std::vector<int> first(size_t(n_chunk) * kTreeWidth, -1);
    std::vector<int> count(n_chunk, 0);
    std::vector<int> extra;  // duplicates of an already-placed subspace
    for (int m : rest) {
        const uint32_t v = j.masks[m];
        const uint32_t c = v >> kTreeLowBits, L = v & (kTreeWidth - 1);
        int &slot = first[size_t(c) * kTreeWidth + L];
        if (slot >= 0) {
            extra.push_back(m);
            continue;
        }
        slot = m;
        ++count[c];
    }
    std::vector<int> lone = extra;
    for (int c = 0; c < n_chunk; ++c) {
        if (count[c] == 0) continue;
        if (count[c] < kTreeMinActive) {
            for (int L = 0; L < kTreeWidth; ++L)
                if (first[size_t(c) * kTreeWidth + L] >= 0) lone.push_back(first[size_t(c) * kTreeWidth + L]);
            continue;
        }
        TreeChunk ch{};
        ch.high = (uint32_t)c;
        ch.active = 0;
        for (int L = 0; L < kTreeWidth; ++L) {
            const int m = first[size_t(c) * kTreeWidth + L];
            ch.slot[L] = m;
            ch.eps2[L] = m >= 0 ? eps2_of(m) : -1.f;
            if (m >= 0) ch.active |= 1u << L;
        }
        pl.chunks.push_back(ch);
    }
    std::sort(lone.begin(), lone.end());
    for (size_t b = 0; b < lone.size(); b += 32) {
        MaskGroup g{};
        for (int l = 0; l < 32; ++l) {
            const size_t q = b + l;
            if (q < lone.size()) {
                const int m = lone[q];
                g.mask[l] = j.masks[m];
                g.eps2[l] = eps2_of(m);
                g.slot[l] = m;
            } else {
                g.mask[l] = 0;
                g.eps2[l] = -1.f;
                g.slot[l] = -1;
            }
        }
        pl.groups.push_back(g);
    }
    if (!pl.chunks.empty()) {
        const size_t per = order_chunk_bytes(j.pop);
        pl.order_batch = (int)std::max<size_t>(1, std::min<size_t>(pl.chunks.size(), kOrderBytes / per));
    }
    return pl;
}

// Device bytes a job needs beyond the population, and the layout inside them.
struct Layout {
    float *scores = nullptr;
    float *norm = nullptr;
    int32_t *top = nullptr;
    int32_t *knn_idx = nullptr;
    float *knn_dist = nullptr;
    int32_t *eps_count = nullptr;
    TreeChunk *chunks = nullptr;
    MaskGroup *groups = nullptr;
    TcBlock *blocks = nullptr;
    char *grid = nullptr;  // one subspace's grid index at a time
    // per-chunk row orders (one batch)
    float4 *ocopy = nullptr;
    float2 *obox = nullptr;  // step boxes of the copies
    uint64_t *okeys = nullptr, *okeys2 = nullptr;
    int32_t *ovals = nullptr, *ovals2 = nullptr;
    void *otmp = nullptr;
    size_t otmp_bytes = 0;
    size_t bytes = 0;
};

Layout layout_job(const JobSpec &j, const Plan &pl, char *base, bool dev_scores, bool dev_norm,
                  bool dev_top, bool dev_idx, bool dev_dist, bool dev_cnt)
{
    Carver cv;
    cv.base = base;
    Layout L;
    const size_t n = (size_t)j.pop->n, nm = (size_t)j.n_masks;
    L.scores = dev_scores ? j.scores : cv.take<float>(nm * 4 * n);
    if (j.norm) L.norm = dev_norm ? j.norm : cv.take<float>(nm * 4 * n);
    if (j.top) L.top = dev_top ? j.top : cv.take<int32_t>(nm * 4 * (size_t)j.top_n);
    if (j.knn_idx) L.knn_idx = dev_idx ? j.knn_idx : cv.take<int32_t>(nm * n * (size_t)j.k);
    if (j.knn_dist) L.knn_dist = dev_dist ? j.knn_dist : cv.take<float>(nm * n * (size_t)j.k);
    if (j.eps_count) L.eps_count = dev_cnt ? j.eps_count : cv.take<int32_t>(nm * n);
    L.chunks = cv.take<TreeChunk>(pl.chunks.size());
    L.groups = cv.take<MaskGroup>(pl.groups.size());
    L.blocks = cv.take<TcBlock>(pl.blocks.size());
    if (!pl.grids.empty()) L.grid = cv.take<char>(grid_scratch_bytes(j.pop->n, pl.grid_max_cells));
    if (pl.order_batch > 0) {
        const size_t g = (size_t)pl.order_batch;
        const int64_t items = (int64_t)g * j.pop->n;
        L.ocopy = cv.take<float4>(g * (size_t)j.pop->n_pad * 4);
        L.obox = cv.take<float2>(g * (size_t)(j.pop->n_pad / 64) * 10);
        L.okeys = cv.take<uint64_t>((size_t)items);
        L.okeys2 = cv.take<uint64_t>((size_t)items);
        L.ovals = cv.take<int32_t>((size_t)items);
        L.ovals2 = cv.take<int32_t>((size_t)items);
        L.otmp_bytes = order_sort_temp(items, order_end_bit(pl.order_batch));
        L.otmp = cv.take<char>(L.otmp_bytes);
    }
    L.bytes = cv.off + 256;
    return L;
}

size_t job_footprint(const JobSpec &j)
{
    Plan pl = make_plan(j);
    Layout L = layout_job(j, pl, nullptr, is_device_ptr(j.scores), is_device_ptr(j.norm),
                          is_device_ptr(j.top), is_device_ptr(j.knn_idx), is_device_ptr(j.knn_dist),
                          is_device_ptr(j.eps_count));
    return L.bytes;
}

// Record a CUDA event pair around a launch when the context is tracing.
struct TraceScope {
    snaps_ctx *ctx;
    int phase;
    cudaStream_t st;
    int kernels;
    cudaEvent_t a = nullptr, b = nullptr;
    TraceScope(snaps_ctx *c, int ph, cudaStream_t s, int nk = 1) : ctx(c), phase(ph), st(s), kernels(nk)
    {
        std::lock_guard<std::mutex> g(ctx->tr_mu);
        if (!ctx->tracing) return;
        a = take();
        b = take();
        if (a && b) cudaEventRecord(a, st);
    }
    cudaEvent_t take()
    {
        if (!ctx->spare.empty()) {
            cudaEvent_t e = ctx->spare.back();
            ctx->spare.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        return e;
    }
    ~TraceScope()
    {
        if (!a || !b) return;
        cudaEventRecord(b, st);
        std::lock_guard<std::mutex> g(ctx->tr_mu);
        ctx->marks.push_back({phase, kernels, a, b});
    }
};

// How many kernels cub::DeviceRadixSort::SortPairs launches for `items`
// (key, value) pairs over key bits [0, end_bit): the sort is recorded by a
// stream capture on a private stream (recording runs nothing) and its kernel
// nodes are counted; cached per shape.  Used only to report launch counts
// while tracing.
template <class K>
snaps_status sort_kernel_count(snaps_ctx *ctx, int64_t items, int end_bit, void *tmp, size_t tmp_bytes,
                               const K *k_in, K *k_out, const int32_t *i_in, int32_t *i_out, int *count)
{
    std::lock_guard<std::mutex> g(ctx->cap_mu);
    const int64_t key = (items << 8) | ((int64_t)sizeof(K) << 6) | end_bit;
    auto it = ctx->sort_kernels.find(key);
    if (it != ctx->sort_kernels.end()) {
        *count = it->second;
        return SNAPS_OK;
    }
    if (!ctx->cap_stream)
        SNAPS_CHECK_CUDA(cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
    SNAPS_CHECK_CUDA(cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal));
    const cudaError_t ce = cub::DeviceRadixSort::SortPairs(tmp, tmp_bytes, k_in, k_out, i_in, i_out, (int)items,
                                                           0, end_bit, ctx->cap_stream);
    cudaGraph_t graph = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(ctx->cap_stream, &graph);
    if (ce != cudaSuccess || ee != cudaSuccess || !graph) {
        if (graph) cudaGraphDestroy(graph);
        set_error("recording a radix sort failed: %s", cudaGetErrorString(ce != cudaSuccess ? ce : ee));
        return SNAPS_ECUDA;
    }
    size_t nn = 0;
    cudaError_t ge = cudaGraphGetNodes(graph, nullptr, &nn);
    std::vector<cudaGraphNode_t> nodes(nn);
    if (ge == cudaSuccess && nn) ge = cudaGraphGetNodes(graph, nodes.data(), &nn);
    int kernels = 0;
    for (size_t q = 0; ge == cudaSuccess && q < nn; ++q) {
        cudaGraphNodeType t;
        ge = cudaGraphNodeGetType(nodes[q], &t);
        if (ge == cudaSuccess && t == cudaGraphNodeTypeKernel) ++kernels;
    }
    cudaGraphDestroy(graph);
    if (ge != cudaSuccess) {
        set_error("reading a recorded radix sort failed: %s", cudaGetErrorString(ge));
        return SNAPS_ECUDA;
    }
    ctx->sort_kernels[key] = kernels;
    *count = kernels;
    return SNAPS_OK;
}

bool tracing_on(snaps_ctx *ctx)
{
    std::lock_guard<std::mutex> g(ctx->tr_mu);
    return ctx->tracing;
}

// Run one job on `st` with `scratch`.  Returns after host outputs are written
// (it synchronises the stream when any output is host memory, or when
// `sync` is set).
snaps_status run_job(snaps_ctx *ctx, const JobSpec &j, cudaStream_t st, Scratch &scratch,
                     DeviceControl *ctrl, bool sync)
{
    SNAPS_TRY(validate(j));
    snaps_pop *p = j.pop;
    const int64_t n = p->n;
    const size_t nm = (size_t)j.n_masks;
    const bool dev_scores = is_device_ptr(j.scores), dev_norm = is_device_ptr(j.norm),
               dev_top = is_device_ptr(j.top), dev_idx = is_device_ptr(j.knn_idx),
               dev_dist = is_device_ptr(j.knn_dist), dev_cnt = is_device_ptr(j.eps_count);
    Plan pl = make_plan(j);
    Layout L0 = layout_job(j, pl, nullptr, dev_scores, dev_norm, dev_top, dev_idx, dev_dist, dev_cnt);
    SNAPS_TRY(scratch_reserve(ctx, scratch, L0.bytes));
    Layout L = layout_job(j, pl, (char *)scratch.ptr, dev_scores, dev_norm, dev_top, dev_idx,
                          dev_dist, dev_cnt);

    if (!pl.chunks.empty())
        SNAPS_CHECK_CUDA(cudaMemcpyAsync(L.chunks, pl.chunks.data(),
                                         pl.chunks.size() * sizeof(TreeChunk),
                                         cudaMemcpyHostToDevice, st));
    if (!pl.groups.empty())
        SNAPS_CHECK_CUDA(cudaMemcpyAsync(L.groups, pl.groups.data(),
                                         pl.groups.size() * sizeof(MaskGroup),
                                         cudaMemcpyHostToDevice, st));
    if (!pl.blocks.empty())
        SNAPS_CHECK_CUDA(cudaMemcpyAsync(L.blocks, pl.blocks.data(),
                                         pl.blocks.size() * sizeof(TcBlock),
                                         cudaMemcpyHostToDevice, st));
    SNAPS_CHECK_CUDA(cudaMemsetAsync(L.scores, 0, nm * 4 * (size_t)n * sizeof(float), st));
    SNAPS_CHECK_CUDA(cudaMemsetAsync(&ctrl->error, 0, sizeof(unsigned), st));

    JoinShape shape{p->x, n, p->n_pad, j.k};
    shape.wait_limit = ctx->wait_limit.load();
    JoinOut out{L.scores, L.knn_idx, L.knn_dist, L.eps_count};
    const int n_chunks = (int)pl.chunks.size();
    for (int b0 = 0; b0 < n_chunks; b0 += pl.order_batch) {
        // every chunk gets its rows in its own order (Morton over its high
        // features), so that a query's stream starts among its neighbours in
        // the features all 32 of the chunk's subspaces share
        const int g = std::min(pl.order_batch, n_chunks - b0);
        const int64_t items = (int64_t)g * n;
        const int end_bit = order_end_bit(g);
        int sort_kernels = 0;
        if (tracing_on(ctx))
            SNAPS_TRY(sort_kernel_count<uint64_t>(ctx, items, end_bit, L.otmp, L.otmp_bytes, L.okeys, L.okeys2,
                                                  L.ovals, L.ovals2, &sort_kernels));
        {
            TraceScope ts(ctx, SNAPS_PHASE_ORDER, st, 3 + sort_kernels);
            SNAPS_TRY(launch_chunk_keys(p->x, n, p->f, L.chunks + b0, g, p->kr, L.okeys, L.ovals, st));
            size_t tb = L.otmp_bytes;
            SNAPS_CHECK_CUDA(cub::DeviceRadixSort::SortPairs(L.otmp, tb, L.okeys, L.okeys2, L.ovals, L.ovals2,
                                                             (int)items, 0, end_bit, st));
            SNAPS_TRY(launch_gather_chunks(p->x, L.ovals2, L.chunks + b0, n, p->n_pad, g, L.ocopy, st));
            SNAPS_TRY(launch_chunk_boxes(L.ocopy, p->n_pad, g, L.obox, st));
        }
        JoinShape cs = shape;
        cs.x = L.ocopy;
        cs.chunk_stride = p->n_pad * 4;
        cs.box = L.obox;
        cs.compact = true;
        cs.box_stride = (p->n_pad / 64) * 10;
        TraceScope ts(ctx, SNAPS_PHASE_JOIN_TREE, st);
        SNAPS_TRY(launch_join_tree(cs, L.chunks + b0, g, out, ctrl, st));
    }
    if (!pl.groups.empty()) {
        TraceScope ts(ctx, SNAPS_PHASE_JOIN_LANE, st);
        SNAPS_TRY(launch_join_single(shape, L.groups, (int)pl.groups.size(), out, st));
    }
    if (!pl.blocks.empty()) {
        TraceScope ts(ctx, SNAPS_PHASE_JOIN_TC, st);
        const uint32_t form = j.precision & 0xFFu;
        SNAPS_TRY(launch_join_tc(shape, L.blocks, (int)pl.blocks.size(),
                                 form == SNAPS_TC_TF32 ? kTcFormTF32 : form == SNAPS_TC_BF16 ? kTcFormBF16
                                                                                              : kTcFormF16,
                                 out, ctrl, st));
    }
    if (!pl.grids.empty()) {
        const GridBufs gb = grid_carve(L.grid, n, pl.grid_max_cells);
        for (const GridSpec &g : pl.grids) {
            int sort_kernels = 0;
            if (tracing_on(ctx))
                SNAPS_TRY(sort_kernel_count<uint32_t>(ctx, n, grid_key_bits(g), gb.tmp, gb.tmp_bytes, gb.k_in,
                                                      gb.k_out, gb.v_in, gb.v_out, &sort_kernels));
            TraceScope ts(ctx, SNAPS_PHASE_GRID, st, 4 + sort_kernels);
            SNAPS_TRY(run_grid_subspace(shape, g, out, gb, st));
        }
    }
    if (j.norm || j.top) {
        // one finishing kernel for the normalised metrics and the rankings
        TraceScope ts(ctx, j.norm ? SNAPS_PHASE_NORM : SNAPS_PHASE_TOP, st);
        SNAPS_TRY(launch_finish(L.scores, n, j.n_masks, L.norm, j.top ? j.top_n : 0, L.top, st));
    }

    bool host_out = false;
    auto d2h = [&](void *dst, const void *src, size_t bytes) -> snaps_status {
        SNAPS_CHECK_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, st));
        host_out = true;
        return SNAPS_OK;
    };
    if (j.scores && !dev_scores) SNAPS_TRY(d2h(j.scores, L.scores, nm * 4 * n * sizeof(float)));
    if (j.norm && !dev_norm) SNAPS_TRY(d2h(j.norm, L.norm, nm * 4 * n * sizeof(float)));
    if (j.top && !dev_top) SNAPS_TRY(d2h(j.top, L.top, nm * 4 * (size_t)j.top_n * sizeof(int32_t)));
    if (j.knn_idx && !dev_idx)
        SNAPS_TRY(d2h(j.knn_idx, L.knn_idx, nm * n * (size_t)j.k * sizeof(int32_t)));
    if (j.knn_dist && !dev_dist)
        SNAPS_TRY(d2h(j.knn_dist, L.knn_dist, nm * n * (size_t)j.k * sizeof(float)));
    if (j.eps_count && !dev_cnt)
        SNAPS_TRY(d2h(j.eps_count, L.eps_count, nm * n * sizeof(int32_t)));
    if (j.eps_mean) {
        // row 1 of every subspace's 4 x n block
        const cudaMemcpyKind kind =
            is_device_ptr(j.eps_mean) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
        SNAPS_CHECK_CUDA(cudaMemcpy2DAsync(j.eps_mean, n * sizeof(float), L.scores + n,
                                           4 * n * sizeof(float), n * sizeof(float), nm, kind, st));
        if (kind == cudaMemcpyDeviceToHost) host_out = true;
    }
    if (host_out || sync) {
        unsigned err = 0;
        SNAPS_CHECK_CUDA(cudaMemcpyAsync(&err, &ctrl->error, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
        SNAPS_CHECK_CUDA(cudaStreamSynchronize(st));
        if (err & kErrBadRow) FAIL(SNAPS_ECUDA, "a join kernel met rows without a valid original index (error word 0x%x)", err);
        if (err) FAIL(SNAPS_ETIMEOUT, "a device-side wait gave up (error word 0x%x)", err);
    }
    return SNAPS_OK;
}

// ---- serving ---------------------------------------------------------------------------

JobSpec spec_of(Request *r)
{
    JobSpec j;
    j.pop = r->req.pop;
    j.masks = r->masks.data();
    j.n_masks = (int)r->masks.size();
    j.k = r->req.k;
    j.eps = r->eps.empty() ? nullptr : r->eps.data();
    j.precision = r->req.precision;
    j.scores = r->req.scores;
    j.norm = r->req.norm;
    j.top = r->req.top;
    j.top_n = r->req.top ? r->req.top_n : 0;
    return j;
}

// Serving: requests that share one launch.  At most kFuseMaxBatch requests,
// each of at most kFuseMaxWork candidate-pair evaluations (n (n - 1) x
// subspaces), so that one batch stays short next to the requests that arrive
// while it runs.
constexpr int kFuseMaxBatch = 32;
constexpr double kFuseMaxWork = 4.0e10;

bool fusable_plan(const JobSpec &j, const Plan &pl)
{
    const double work = (double)j.pop->n * (double)(j.pop->n - 1) * (double)j.n_masks;
    return pl.chunks.empty() && pl.grids.empty() && pl.blocks.empty() && !j.knn_idx && !j.knn_dist &&
           !j.eps_count && !j.eps_mean && work <= kFuseMaxWork;
}

// Run fusable requests together: each gets its own outputs and scratch, and
// the subspaces of all of them are joined by one work-list launch per kNN-list
// size (k <= 16, k <= 32) -- a small request then no longer fills the GPU on
// its own.  The finishing kernel and the copies follow per request.  Returns
// the batch's status (every request in it gets the same).
snaps_status run_batch(snaps_ctx *ctx, const std::vector<JobSpec> &jobs, cudaStream_t st, Scratch &scratch,
                       DeviceControl *ctrl)
{
    struct Part {
        Plan pl;
        Layout L;
        size_t off = 0;
        bool dev_scores, dev_norm, dev_top;
    };
    std::vector<Part> parts(jobs.size());
    size_t total = 0;
    std::vector<WorkItem> items[2];
    int ctas[2] = {0, 0};
    for (size_t q = 0; q < jobs.size(); ++q) {
        const JobSpec &j = jobs[q];
        Part &pt = parts[q];
        pt.pl = make_plan(j);
        pt.dev_scores = is_device_ptr(j.scores);
        pt.dev_norm = is_device_ptr(j.norm);
        pt.dev_top = is_device_ptr(j.top);
        pt.L = layout_job(j, pt.pl, nullptr, pt.dev_scores, pt.dev_norm, pt.dev_top, false, false, false);
        pt.off = total;
        total += (pt.L.bytes + 255) & ~size_t(255);
        for (const MaskGroup &g : pt.pl.groups)
            for (int l = 0; l < 32; ++l) {
                if (g.mask[l] == 0u) continue;
                WorkItem w{};
                w.x = j.pop->x;
                w.n = (int)j.pop->n;
                w.k = j.k;
                w.mask = g.mask[l];
                w.eps2 = g.eps2[l];
                const int c = j.k <= 16 ? 0 : 1;
                w.first_cta = ctas[c];
                ctas[c] += (int)((j.pop->n + 255) / 256);
                w.scores = nullptr;                 // known once the layout is
                w.pad = (int)q << 16 | g.slot[l];   // request and output slot until then
                items[c].push_back(w);
            }
    }
    const size_t item_off = total;
    total += sizeof(WorkItem) * (items[0].size() + items[1].size()) + 256;
    SNAPS_TRY(scratch_reserve(ctx, scratch, total));
    char *base = (char *)scratch.ptr;
    for (size_t q = 0; q < jobs.size(); ++q) {
        Part &pt = parts[q];
        pt.L = layout_job(jobs[q], pt.pl, base + pt.off, pt.dev_scores, pt.dev_norm, pt.dev_top, false, false, false);
        SNAPS_CHECK_CUDA(cudaMemsetAsync(pt.L.scores, 0, (size_t)jobs[q].n_masks * 4 * jobs[q].pop->n * sizeof(float), st));
    }
    for (int c = 0; c < 2; ++c)
        for (WorkItem &w : items[c]) {
            const int q = w.pad >> 16, slot = w.pad & 0xffff;
            w.scores = parts[q].L.scores + (size_t)slot * 4 * jobs[q].pop->n;
            w.pad = 0;
        }
    SNAPS_CHECK_CUDA(cudaMemsetAsync(&ctrl->error, 0, sizeof(unsigned), st));
    WorkItem *dev_items = (WorkItem *)(base + ((item_off + 255) & ~size_t(255)));
    {
        TraceScope ts(ctx, SNAPS_PHASE_JOIN_LANE, st, (items[0].empty() ? 0 : 1) + (items[1].empty() ? 0 : 1));
        WorkItem *d = dev_items;
        for (int c = 0; c < 2; ++c) {
            if (items[c].empty()) continue;
            SNAPS_CHECK_CUDA(cudaMemcpyAsync(d, items[c].data(), sizeof(WorkItem) * items[c].size(),
                                             cudaMemcpyHostToDevice, st));
            SNAPS_TRY(launch_join_worklist(d, (int)items[c].size(), ctas[c], c == 0 ? 16 : 32, st));
            d += items[c].size();
        }
    }
    for (size_t q = 0; q < jobs.size(); ++q) {
        const JobSpec &j = jobs[q];
        const Part &pt = parts[q];
        const int64_t n = j.pop->n;
        const size_t nm = (size_t)j.n_masks;
        if (j.norm || j.top) {
            TraceScope ts(ctx, j.norm ? SNAPS_PHASE_NORM : SNAPS_PHASE_TOP, st);
            SNAPS_TRY(launch_finish(pt.L.scores, n, j.n_masks, pt.L.norm, j.top ? j.top_n : 0, pt.L.top, st));
        }
        if (j.scores && !pt.dev_scores)
            SNAPS_CHECK_CUDA(cudaMemcpyAsync(j.scores, pt.L.scores, nm * 4 * n * sizeof(float), cudaMemcpyDeviceToHost, st));
        if (j.norm && !pt.dev_norm)
            SNAPS_CHECK_CUDA(cudaMemcpyAsync(j.norm, pt.L.norm, nm * 4 * n * sizeof(float), cudaMemcpyDeviceToHost, st));
        if (j.top && !pt.dev_top)
            SNAPS_CHECK_CUDA(cudaMemcpyAsync(j.top, pt.L.top, nm * 4 * (size_t)j.top_n * sizeof(int32_t),
                                             cudaMemcpyDeviceToHost, st));
    }
    unsigned err = 0;
    SNAPS_CHECK_CUDA(cudaMemcpyAsync(&err, &ctrl->error, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    SNAPS_CHECK_CUDA(cudaStreamSynchronize(st));
    if (err) FAIL(SNAPS_ECUDA, "a fused join met an error (error word 0x%x)", err);
    return SNAPS_OK;
}

// A request of more than kUnitWork candidate-pair evaluations runs in parts
// of its subspace list, each about that much work, and between parts the slot
// serves the small requests queued meanwhile: a large request then delays them
// by one part, not by all of its work.  A part holds whole launch units: a
// multiple of 32 subspaces (one subset-tree chunk, when the list runs chunk by
// chunk) in the FP32 form, a multiple of a tensor-core block in the
// tensor-core forms, whose launch costs a full block however few subspaces it
// carries.
constexpr double kUnitWork = 2.0e11;

int part_size(const JobSpec &j, double pairs)
{
    const int unit = (j.precision & 0xFFu) == SNAPS_FP32 ? (1 << kTreeLowBits) : kTcBlockWidth;
    const int per = std::max(1, (int)(kUnitWork / pairs));
    if (per < unit && (j.precision & 0xFFu) == SNAPS_FP32) return per;
    return std::max(unit, per / unit * unit);
}

// Complete finished requests and wake their pollers.
void complete(snaps_ctx *ctx, const std::vector<Request *> &done, snaps_status s, size_t grow)
{
    {
        std::lock_guard<std::mutex> lk(ctx->q_mu);
        ctx->reserved -= grow;
        for (Request *r : done) {
            r->status = s;
            r->done = true;
            r->running = false;
            r->t_done = Clock::now();
            r->req.pop->inflight.fetch_sub(1);
        }
    }
    ctx->done_cv.notify_all();
    ctx->q_cv.notify_all();
}

snaps_status run_fused(snaps_ctx *ctx, const std::vector<Request *> &batch, Slot *slot)
{
    if (batch.size() == 1) return run_job(ctx, spec_of(batch[0]), slot->stream, slot->scratch, slot->ctrl, true);
    std::vector<JobSpec> jobs;
    for (Request *b : batch) jobs.push_back(spec_of(b));
    const snaps_status s = run_batch(ctx, jobs, slot->stream, slot->scratch, slot->ctrl);
    ctx->fused_launches.fetch_add(1);
    ctx->fused_requests.fetch_add((long long)batch.size());
    return s;
}

// Between the parts of a large request: the fusable requests at the head of
// the queue whose scratch fits the slot's as it is (no allocation), run
// together.
void serve_waiting(snaps_ctx *ctx, Slot *slot)
{
    std::vector<Request *> batch;
    {
        std::lock_guard<std::mutex> lk(ctx->q_mu);
        size_t need = 0;
        while (!ctx->queue.empty() && (int)batch.size() < kFuseMaxBatch) {
            Request *h = ctx->queue.front();
            if (!h->fusable || need + h->footprint + 4096 > slot->scratch.cap) break;
            ctx->queue.pop_front();
            need += h->footprint + 4096;
            h->running = true;
            h->t_admit = Clock::now();
            batch.push_back(h);
        }
    }
    if (batch.empty()) return;
    complete(ctx, batch, run_fused(ctx, batch, slot), 0);
}

// Run one request, in parts when it is large.
snaps_status run_request(snaps_ctx *ctx, Request *r, Slot *slot)
{
    const JobSpec full = spec_of(r);
    const double pairs = (double)full.pop->n * (double)(full.pop->n - 1);
    if (pairs * full.n_masks <= kUnitWork) return run_job(ctx, full, slot->stream, slot->scratch, slot->ctrl, true);
    const int per = part_size(full, pairs);
    if (per >= full.n_masks) return run_job(ctx, full, slot->stream, slot->scratch, slot->ctrl, true);
    const size_t n = (size_t)full.pop->n;
    snaps_status s = SNAPS_OK;
    for (int m0 = 0; m0 < full.n_masks && s == SNAPS_OK; m0 += per) {
        JobSpec part = full;
        const int m = std::min(per, full.n_masks - m0);
        part.masks = full.masks + m0;
        part.n_masks = m;
        if (full.eps) part.eps = full.eps + m0;
        if (full.scores) part.scores = full.scores + (size_t)m0 * 4 * n;
        if (full.norm) part.norm = full.norm + (size_t)m0 * 4 * n;
        if (full.top) part.top = full.top + (size_t)m0 * 4 * (size_t)full.top_n;
        s = run_job(ctx, part, slot->stream, slot->scratch, slot->ctrl, true);
        if (s == SNAPS_OK && m0 + per < full.n_masks) serve_waiting(ctx, slot);
    }
    return s;
}

void worker_loop(snaps_ctx *ctx, Slot *slot)
{
    cudaSetDevice(ctx->device);
    for (;;) {
        std::vector<Request *> batch;
        size_t grow = 0;
        {
            std::unique_lock<std::mutex> lk(ctx->q_mu);
            for (;;) {
                if (ctx->stopping && ctx->queue.empty()) return;
                if (!ctx->queue.empty()) {
                    Request *h = ctx->queue.front();
                    // admission by HBM footprint, in arrival order
                    size_t held;
                    {
                        std::lock_guard<std::mutex> g(ctx->mem_mu);
                        held = ctx->held;
                    }
                    const size_t g0 = h->footprint > slot->scratch.cap ? h->footprint : 0;
                    if (held + ctx->reserved + g0 <= ctx->budget || ctx->reserved == 0) {
                        ctx->queue.pop_front();
                        batch.push_back(h);
                        // continuous batching: the fusable requests queued right behind a
                        // fusable one join its launch, while the budget allows
                        size_t need = h->footprint;
                        while (h->fusable && !ctx->queue.empty() && (int)batch.size() < kFuseMaxBatch) {
                            Request *nx = ctx->queue.front();
                            if (!nx->fusable) break;
                            const size_t need2 = need + nx->footprint + 4096;
                            const size_t g2 = need2 > slot->scratch.cap ? need2 : 0;
                            if (held + ctx->reserved + g2 > ctx->budget) break;
                            ctx->queue.pop_front();
                            batch.push_back(nx);
                            need = need2;
                        }
                        grow = need > slot->scratch.cap ? need : 0;
                        ctx->reserved += grow;
                        for (Request *b : batch) {
                            b->running = true;
                            b->t_admit = Clock::now();
                        }
                        break;
                    }
                }
                ctx->q_cv.wait(lk);
            }
        }
        const snaps_status s = batch.size() == 1 ? run_request(ctx, batch[0], slot) : run_fused(ctx, batch, slot);
        complete(ctx, batch, s, grow);
    }
}

snaps_status start_slots(snaps_ctx *ctx)
{
    while ((int)ctx->slots.size() < ctx->n_slots) {
        Slot *s = new Slot();
        SNAPS_CHECK_CUDA(cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking));
        void *c = nullptr;
        SNAPS_TRY(ctx_alloc(ctx, sizeof(DeviceControl), &c));
        s->ctrl = (DeviceControl *)c;
        s->worker = std::thread(worker_loop, ctx, s);
        ctx->slots.push_back(s);
    }
    return SNAPS_OK;
}

}  // namespace

// ---- C ABI --------------------------------------------------------------------------------

extern "C" {

const char *snaps_version(void) { return "0.1.0"; }

const char *snaps_last_error(void) { return snaps::last_error_message(); }

snaps_status snaps_create(int device, size_t hbm_budget_bytes, snaps_ctx **out)
{
    clear_error();
    if (!out) FAIL(SNAPS_EINVAL, "out is NULL");
    *out = nullptr;
    int count = 0;
    SNAPS_CHECK_CUDA(cudaGetDeviceCount(&count));
    if (device < 0 || device >= count) FAIL(SNAPS_EINVAL, "device %d out of range (%d devices)", device, count);
    ON_DEVICE(device);
    size_t free_b = 0, total_b = 0;
    SNAPS_CHECK_CUDA(cudaMemGetInfo(&free_b, &total_b));
    snaps_ctx *ctx = new snaps_ctx();
    ctx->device = device;
    ctx->budget = hbm_budget_bytes ? hbm_budget_bytes : (size_t)(0.9 * (double)free_b);
    void *c = nullptr;
    snaps_status s = ctx_alloc(ctx, sizeof(DeviceControl), &c);
    if (s != SNAPS_OK) {
        delete ctx;
        return s;
    }
    ctx->ctrl = (DeviceControl *)c;
    SNAPS_CHECK_CUDA(cudaMemset(ctx->ctrl, 0, sizeof(DeviceControl)));
    *out = ctx;
    return SNAPS_OK;
}

snaps_status snaps_destroy(snaps_ctx *ctx)
{
    clear_error();
    if (!ctx) return SNAPS_OK;
    DeviceScope device_scope(ctx->device);
    {
        std::lock_guard<std::mutex> lk(ctx->q_mu);
        ctx->stopping = true;
    }
    ctx->q_cv.notify_all();
    for (Slot *s : ctx->slots) {
        if (s->worker.joinable()) s->worker.join();
        ctx_free(ctx, s->scratch.ptr, s->scratch.cap);
        ctx_free(ctx, s->ctrl, sizeof(DeviceControl));
        cudaStreamDestroy(s->stream);
        delete s;
    }
    for (auto &kv : ctx->tickets) delete kv.second;
    for (auto &m : ctx->marks) {
        cudaEventDestroy(m.a);
        cudaEventDestroy(m.b);
    }
    for (cudaEvent_t e : ctx->spare) cudaEventDestroy(e);
    if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
    ctx_free(ctx, ctx->scratch.ptr, ctx->scratch.cap);
    ctx_free(ctx, ctx->ctrl, sizeof(DeviceControl));
    delete ctx;
    return SNAPS_OK;
}

snaps_status snaps_mem_info(const snaps_ctx *ctx, size_t *held, size_t *budget)
{
    clear_error();
    if (!ctx) FAIL(SNAPS_EINVAL, "ctx is NULL");
    auto *c = const_cast<snaps_ctx *>(ctx);
    std::lock_guard<std::mutex> g(c->mem_mu);
    if (held) *held = c->held;
    if (budget) *budget = c->budget;
    return SNAPS_OK;
}


snaps_status snaps_index(snaps_ctx *ctx, const float *feat, int64_t n, int f, uint32_t flags,
                         void *stream, snaps_pop **out)
{
    clear_error();
    if (!ctx || !feat || !out) FAIL(SNAPS_EINVAL, "ctx, feat and out must be non-NULL");
    *out = nullptr;
    if (n < 2 || n > (int64_t(1) << 24)) FAIL(SNAPS_EINVAL, "n must be in 2..2^24 (got %lld)", (long long)n);
    if (f < 1 || f > SNAPS_MAX_FEATURES) FAIL(SNAPS_EINVAL, "f must be in 1..15 (got %d)", f);
    if (flags & ~(SNAPS_NORM_MINMAX | SNAPS_NAN_TO_MEAN)) FAIL(SNAPS_EINVAL, "unknown flags 0x%x", flags);
    ON_DEVICE(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    snaps_pop *p = new snaps_pop();
    p->ctx = ctx;
    p->n = n;
    p->f = f;
    p->n_pad = padded_rows(n);
    p->bytes = (size_t)p->n_pad * kRowFloats * sizeof(float);
    void *xp = nullptr;
    snaps_status s = ctx_alloc(ctx, p->bytes, &xp);
    if (s != SNAPS_OK) {
        delete p;
        return s;
    }
    p->x = (float4 *)xp;
    // staging: input copy (when on the host) + column statistics + flag
    const size_t in_bytes = (size_t)n * f * sizeof(float);
    SNAPS_TRY(check_not_foreign(feat, ctx->device, "feat"));
    const bool dev_in = is_device_ptr(feat);
    const size_t aux = 256 + sizeof(ColStats) * 16 + 256;
    void *stage = nullptr;
    s = ctx_alloc(ctx, (dev_in ? 0 : in_bytes) + aux, &stage);
    if (s != SNAPS_OK) {
        ctx_free(ctx, p->x, p->bytes);
        delete p;
        return s;
    }
    char *sb = (char *)stage;
    unsigned *bad = (unsigned *)sb;
    ColStats *stats = (ColStats *)(sb + 256);
    const float *in = dev_in ? feat : (const float *)(sb + aux);
    auto fail = [&](snaps_status code) {
        cudaStreamSynchronize(st);
        ctx_free(ctx, stage, (dev_in ? 0 : in_bytes) + aux);
        ctx_free(ctx, p->x, p->bytes);
        delete p;
        return code;
    };
    if (!dev_in && cudaMemcpyAsync((void *)in, feat, in_bytes, cudaMemcpyHostToDevice, st) != cudaSuccess) {
        set_error("copying the features to the device failed");
        return fail(SNAPS_ECUDA);
    }
    {
        TraceScope ts(ctx, SNAPS_PHASE_INDEX, st, 2);
        s = launch_normalise(in, n, p->n_pad, f, flags, stats, bad, p->x, st);
    }
    if (s != SNAPS_OK) return fail(s);
    unsigned hbad = 0;
    ColStats hstats[SNAPS_MAX_FEATURES];
    if (cudaMemcpyAsync(&hbad, bad, sizeof(unsigned), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(hstats, stats, sizeof(ColStats) * f, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        set_error("normalisation failed: %s", cudaGetErrorString(cudaGetLastError()));
        return fail(SNAPS_ECUDA);
    }
    if (hbad) {
        set_error("features must be finite (NaN is allowed only with SNAPS_NAN_TO_MEAN)");
        return fail(SNAPS_EINVAL);
    }
    ctx_free(ctx, stage, (dev_in ? 0 : in_bytes) + aux);
    for (int c = 0; c < 16; ++c) {
        p->kr.lo[c] = 0.f;
        p->kr.scale[c] = c < f ? 1.f : 0.f;
    }
    if (!(flags & SNAPS_NORM_MINMAX))
        for (int c = 0; c < f; ++c) {
            const double span = hstats[c].hi - hstats[c].lo;
            p->kr.lo[c] = (float)hstats[c].lo;
            p->kr.scale[c] = span > 0.0 ? (float)(1.0 / span) : 0.f;
        }
    // ---- sort-by-cell index: rows reordered by their 15-feature cell key, so
    // a tile of consecutive rows is a spatial neighbourhood.  Stored rows keep
    // their original index in float 15.
    {
        size_t cub_bytes = 0;
        cub::DeviceRadixSort::SortPairs(nullptr, cub_bytes, (const uint32_t *)nullptr, (uint32_t *)nullptr,
                                        (const int32_t *)nullptr, (int32_t *)nullptr, (int)n, 0, 30, st);
        const size_t rows_bytes = p->bytes;
        const size_t arr = ((size_t)n * 4 + 255) & ~size_t(255);
        const size_t sort_bytes = rows_bytes + 4 * arr + cub_bytes + 256;
        void *sb2 = nullptr;
        s = ctx_alloc(ctx, sort_bytes, &sb2);
        if (s != SNAPS_OK) {
            ctx_free(ctx, p->x, p->bytes);
            delete p;
            return s;
        }
        char *b2 = (char *)sb2;
        float4 *rows = (float4 *)b2;
        uint32_t *k_in = (uint32_t *)(b2 + rows_bytes);
        uint32_t *k_out = (uint32_t *)(b2 + rows_bytes + arr);
        int32_t *i_in = (int32_t *)(b2 + rows_bytes + 2 * arr);
        int32_t *i_out = (int32_t *)(b2 + rows_bytes + 3 * arr);
        void *tmp = b2 + rows_bytes + 4 * arr;
        int sort_kernels = 0;
        snaps_status ss = SNAPS_OK;
        if (tracing_on(ctx))
            ss = sort_kernel_count<uint32_t>(ctx, n, 30, tmp, cub_bytes, k_in, k_out, i_in, i_out, &sort_kernels);
        cudaError_t ce = cudaSuccess;
        if (ss == SNAPS_OK) {
            TraceScope ts(ctx, SNAPS_PHASE_INDEX, st, 2 + sort_kernels);
            ce = cudaMemcpyAsync(rows, p->x, rows_bytes, cudaMemcpyDeviceToDevice, st);
            if (ce == cudaSuccess) ss = launch_cell_keys(rows, n, p->kr, k_in, i_in, st);
            if (ss == SNAPS_OK && ce == cudaSuccess)
                ce = cub::DeviceRadixSort::SortPairs(tmp, cub_bytes, k_in, k_out, i_in, i_out, (int)n, 0, 30, st);
            if (ss == SNAPS_OK && ce == cudaSuccess) ss = launch_gather_rows(rows, i_out, n, p->n_pad, p->x, st);
        }
        if (ss == SNAPS_OK && ce == cudaSuccess) ce = cudaStreamSynchronize(st);
        ctx_free(ctx, sb2, sort_bytes);
        if (ss != SNAPS_OK || ce != cudaSuccess) {
            if (ce != cudaSuccess) set_error("sort-by-cell index failed: %s", cudaGetErrorString(ce));
            ctx_free(ctx, p->x, p->bytes);
            delete p;
            return ss != SNAPS_OK ? ss : SNAPS_ECUDA;
        }
    }
    p->unit_range = true;
    if (!(flags & SNAPS_NORM_MINMAX))
        for (int c = 0; c < f; ++c)
            if (!(hstats[c].hi - hstats[c].lo <= 1.0)) p->unit_range = false;
    ctx->n_pops.fetch_add(1);
    *out = p;
    return SNAPS_OK;
}

snaps_status snaps_release(snaps_pop *pop)
{
    clear_error();
    if (!pop) return SNAPS_OK;
    if (pop->inflight.load() > 0) FAIL(SNAPS_EBUSY, "population has %d requests in flight", pop->inflight.load());
    snaps_ctx *ctx = pop->ctx;
    DeviceScope device_scope(ctx->device);
    cudaDeviceSynchronize();
    ctx_free(ctx, pop->x, pop->bytes);
    ctx->n_pops.fetch_sub(1);
    delete pop;
    return SNAPS_OK;
}

snaps_status snaps_pop_shape(const snaps_pop *pop, int64_t *n, int *f)
{
    clear_error();
    if (!pop) FAIL(SNAPS_EINVAL, "pop is NULL");
    if (n) *n = pop->n;
    if (f) *f = pop->f;
    return SNAPS_OK;
}

snaps_status snaps_pop_features(const snaps_pop *pop, float *out, void *stream)
{
    clear_error();
    if (!pop || !out) FAIL(SNAPS_EINVAL, "pop and out must be non-NULL");
    snaps_ctx *ctx = pop->ctx;
    ON_DEVICE(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const size_t bytes = (size_t)pop->n * pop->f * sizeof(float);
    SNAPS_TRY(check_not_foreign(out, ctx->device, "out"));
    if (is_device_ptr(out)) return launch_unpack(pop->x, pop->n, pop->f, out, st);
    void *tmp = nullptr;
    SNAPS_TRY(ctx_alloc(ctx, bytes, &tmp));
    snaps_status s = launch_unpack(pop->x, pop->n, pop->f, (float *)tmp, st);
    if (s == SNAPS_OK) {
        if (cudaMemcpyAsync(out, tmp, bytes, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) {
            set_error("copying the features out failed");
            s = SNAPS_ECUDA;
        }
    }
    ctx_free(ctx, tmp, bytes);
    return s;
}

snaps_status snaps_knn_selfjoin(snaps_pop *pop, const uint16_t *masks, int n_masks, int k,
                                int32_t *idx, float *dist, void *stream)
{
    clear_error();
    if (!pop) FAIL(SNAPS_EINVAL, "pop is NULL");
    if (!idx) FAIL(SNAPS_EINVAL, "idx is NULL");
    if (k < 1) FAIL(SNAPS_EINVAL, "k must be >= 1 (got %d)", k);
    ON_DEVICE(pop->ctx->device);
    JobSpec j;
    j.pop = pop;
    j.masks = masks;
    j.n_masks = n_masks;
    j.k = k;
    j.want_eps = false;
    j.knn_idx = idx;
    j.knn_dist = dist;
    std::lock_guard<std::mutex> g(pop->ctx->sync_mu);
    return run_job(pop->ctx, j, (cudaStream_t)stream, pop->ctx->scratch, pop->ctx->ctrl, false);
}

snaps_status snaps_eps_selfjoin(snaps_pop *pop, const uint16_t *masks, int n_masks,
                                const float *eps, int32_t *count, float *mean_dist, void *stream)
{
    clear_error();
    if (!pop) FAIL(SNAPS_EINVAL, "pop is NULL");
    ON_DEVICE(pop->ctx->device);
    JobSpec j;
    j.pop = pop;
    j.masks = masks;
    j.n_masks = n_masks;
    j.k = 0;
    j.eps = eps;
    j.want_eps = true;
    j.eps_count = count;
    j.eps_mean = mean_dist;
    std::lock_guard<std::mutex> g(pop->ctx->sync_mu);
    return run_job(pop->ctx, j, (cudaStream_t)stream, pop->ctx->scratch, pop->ctx->ctrl, false);
}

namespace {

// Eq. 2's intersection count of two top-n lists (sorted copies, two-pointer merge).
int top_overlap(const int32_t *a, const int32_t *b, int n)
{
    std::vector<int32_t> x(a, a + n), y(b, b + n);
    std::sort(x.begin(), x.end());
    std::sort(y.begin(), y.end());
    int c = 0;
    for (size_t p = 0, q = 0; p < x.size() && q < y.size();) {
        if (x[p] == y[q]) {
            ++c;
            ++p;
            ++q;
        } else if (x[p] < y[q]) {
            ++p;
        } else {
            ++q;
        }
    }
    return c;
}

// U^min, U^max (Eq. 2) of one metric over a grid of G top-n lists (list g at
// tops + g * stride), and the selected index (Eq. 3; the first on ties).
int select_grid(const int32_t *tops, size_t stride, int G, int top_n, float *u_min, float *u_max)
{
    int best = 0, best_gap = INT32_MAX;
    for (int g = 0; g < G; ++g) {
        const int cmin = top_overlap(tops, tops + g * stride, top_n);
        const int cmax = top_overlap(tops + (G - 1) * stride, tops + g * stride, top_n);
        u_min[g] = (float)cmin / (float)top_n;
        u_max[g] = (float)cmax / (float)top_n;
        const int gap = std::abs(cmin - cmax);
        if (gap < best_gap) {
            best_gap = gap;
            best = g;
        }
    }
    return best;
}

}  // namespace

snaps_status snaps_select(snaps_pop *pop, const uint16_t *masks, int n_masks, const float *eps_min,
                          const float *eps_max, int n_eps, const int32_t *k_grid, int n_k, int top_n,
                          float *u_eps, int32_t *eps_select, float *u_k, int32_t *k_select, void *stream)
{
    clear_error();
    if (!pop) FAIL(SNAPS_EINVAL, "pop is NULL");
    ON_DEVICE(pop->ctx->device);
    snaps_ctx *ctx = pop->ctx;
    const int64_t n = pop->n;
    if (n_masks < 1 || !masks || is_device_ptr(masks)) FAIL(SNAPS_EINVAL, "masks: a host array of >= 1 masks");
    for (int m = 0; m < n_masks; ++m)
        if (popc16(masks[m]) < 2 || (masks[m] >> pop->f) != 0)
            FAIL(SNAPS_EINVAL, "mask %d (0x%x) must have 2..%d bits, all below feature %d", m, masks[m], pop->f,
                 pop->f);
    SNAPS_TRY(check_not_foreign(u_eps, ctx->device, "u_eps"));
    SNAPS_TRY(check_not_foreign(eps_select, ctx->device, "eps_select"));
    SNAPS_TRY(check_not_foreign(u_k, ctx->device, "u_k"));
    SNAPS_TRY(check_not_foreign(k_select, ctx->device, "k_select"));
    const bool want_eps = u_eps || eps_select, want_k = u_k || k_select;
    if (!want_eps && !want_k) FAIL(SNAPS_EINVAL, "no output requested");
    if (want_eps) {
        if (n_eps < 2 || n_eps > kSelectMaxGrid) FAIL(SNAPS_EINVAL, "n_eps must be in 2..%d", kSelectMaxGrid);
        if (!eps_min || !eps_max || is_device_ptr(eps_min) || is_device_ptr(eps_max))
            FAIL(SNAPS_EINVAL, "eps_min / eps_max: host arrays of n_masks values");
        for (int m = 0; m < n_masks; ++m)
            if (!(eps_min[m] >= 0.f && eps_max[m] > eps_min[m] && eps_max[m] < 1e18f))
                FAIL(SNAPS_EINVAL, "subspace %d: need 0 <= eps_min < eps_max (finite)", m);
    }
    if (want_k) {
        if (n_k < 2 || n_k > kSelectMaxGrid) FAIL(SNAPS_EINVAL, "n_k must be in 2..%d", kSelectMaxGrid);
        if (!k_grid || is_device_ptr(k_grid)) FAIL(SNAPS_EINVAL, "k_grid: a host array");
        for (int g = 0; g < n_k; ++g)
            if (k_grid[g] < 1 || (g > 0 && k_grid[g] <= k_grid[g - 1]))
                FAIL(SNAPS_EINVAL, "k_grid must be strictly ascending from >= 1");
        if (k_grid[n_k - 1] > SNAPS_SELECT_MAX_K || k_grid[n_k - 1] > n - 1)
            FAIL(SNAPS_EINVAL, "k_grid values must be <= min(%d, n - 1)", SNAPS_SELECT_MAX_K);
    }
    if (top_n < 1 || top_n > 1024 || top_n > n) FAIL(SNAPS_EINVAL, "top_n must be in 1..min(1024, n)");
    const int G = want_eps ? n_eps : 0, K = want_k ? n_k : 0;
    const int kmax = want_k ? k_grid[n_k - 1] : 0;
    const int slots = std::max(G, K);
    cudaStream_t st = (cudaStream_t)stream;

    std::lock_guard<std::mutex> lock(ctx->sync_mu);
    Carver cv;
    auto layout = [&](char *base) {
        cv = Carver();
        cv.base = base;
        float *es = cv.take<float>((size_t)std::max(G, 1) * 4 * n);
        float *ks = cv.take<float>((size_t)std::max(K, 1) * 4 * n);
        int32_t *tp = cv.take<int32_t>((size_t)slots * 4 * top_n);
        return std::make_tuple(es, ks, tp);
    };
    layout(nullptr);
    SNAPS_TRY(scratch_reserve(ctx, ctx->scratch, cv.off + 256));
    auto [eps_scores, k_scores, tops_dev] = layout((char *)ctx->scratch.ptr);
    std::vector<int32_t> tops((size_t)slots * 4 * top_n);
    std::vector<float> ue((size_t)n_masks * 4 * std::max(G, 1)), uk((size_t)n_masks * 4 * std::max(K, 1));
    std::vector<int32_t> es((size_t)n_masks * 2), kse((size_t)n_masks * 2);

    for (int m = 0; m < n_masks; ++m) {
        SelectSpec sp{};
        sp.mask = masks[m];
        sp.n_eps = G;
        if (G > 0) {
            for (int g = 0; g < G; ++g) {
                const float e = (float)((double)eps_min[m] + g * ((double)eps_max[m] - (double)eps_min[m]) / (G - 1));
                sp.e2[g] = e * e;
            }
            sp.qscale = (float)(16777216.0 / (double)eps_max[m]);
        }
        KGrid kg{};
        kg.n = K;
        for (int g = 0; g < K; ++g) kg.k[g] = k_grid[g];
        const bool wide_k = K > 0 && kmax > kSelectWarpK;
        SNAPS_CHECK_CUDA(cudaMemsetAsync(eps_scores, 0, (size_t)std::max(G, 1) * 4 * n * sizeof(float), st));
        SNAPS_CHECK_CUDA(cudaMemsetAsync(k_scores, 0, (size_t)std::max(K, 1) * 4 * n * sizeof(float), st));
        {
            TraceScope ts(ctx, SNAPS_PHASE_SELECT, st, (G > 0 || !wide_k ? 1 : 0) + (K > 0 ? 1 : 0) + wide_k);
            if (G > 0 || !wide_k) {
                KGrid none{};
                SNAPS_TRY(launch_select_join(pop->x, n, sp, wide_k ? none : kg, eps_scores, k_scores, st));
            }
            if (wide_k) SNAPS_TRY(launch_select_knn(pop->x, n, masks[m], kg, k_scores, st));
            if (K > 0) SNAPS_TRY(launch_select_k_finish(n, kg, k_scores, st));
        }
        for (int half = 0; half < 2; ++half) {
            const int S = half == 0 ? G : K;
            if (S == 0) continue;
            {
                TraceScope ts(ctx, SNAPS_PHASE_TOP, st);
                SNAPS_TRY(launch_top(half == 0 ? eps_scores : k_scores, n, S, top_n, tops_dev, st));
            }
            SNAPS_CHECK_CUDA(cudaMemcpyAsync(tops.data(), tops_dev, (size_t)S * 4 * top_n * sizeof(int32_t),
                                             cudaMemcpyDeviceToHost, st));
            SNAPS_CHECK_CUDA(cudaStreamSynchronize(st));
            for (int r = 0; r < 2; ++r) {
                const int row = half == 0 ? r : 2 + r;  // eps: count, mean; k: in-degree, mean
                float *u = (half == 0 ? ue.data() : uk.data()) + ((size_t)m * 2 + r) * 2 * S;
                const int sel = select_grid(tops.data() + (size_t)row * top_n, (size_t)4 * top_n, S, top_n, u,
                                            u + S);
                (half == 0 ? es : kse)[(size_t)m * 2 + r] = sel;
            }
        }
    }
    auto put = [&](void *dst, const void *src, size_t bytes) -> snaps_status {
        if (!dst) return SNAPS_OK;
        const cudaMemcpyKind kind = is_device_ptr(dst) ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost;
        SNAPS_CHECK_CUDA(cudaMemcpyAsync(dst, src, bytes, kind, st));
        return SNAPS_OK;
    };
    if (G > 0) {
        SNAPS_TRY(put(u_eps, ue.data(), (size_t)n_masks * 4 * G * sizeof(float)));
        SNAPS_TRY(put(eps_select, es.data(), (size_t)n_masks * 2 * sizeof(int32_t)));
    }
    if (K > 0) {
        SNAPS_TRY(put(u_k, uk.data(), (size_t)n_masks * 4 * K * sizeof(float)));
        SNAPS_TRY(put(k_select, kse.data(), (size_t)n_masks * 2 * sizeof(int32_t)));
    }
    SNAPS_CHECK_CUDA(cudaStreamSynchronize(st));
    return SNAPS_OK;
}

snaps_status snaps_autotune(snaps_pop *pop, int k, snaps_tune_entry *out, void *stream)
{
    clear_error();
    if (!pop) FAIL(SNAPS_EINVAL, "pop is NULL");
    ON_DEVICE(pop->ctx->device);
    snaps_ctx *ctx = pop->ctx;
    const int64_t n = pop->n;
    const int f = pop->f;
    if (k < 1 || k > SNAPS_MAX_K || k > n - 1) FAIL(SNAPS_EINVAL, "k must be in 1..min(%d, n - 1)", SNAPS_MAX_K);
    if (f < 2) FAIL(SNAPS_EINVAL, "the population needs >= 2 features");
    cudaStream_t st = (cudaStream_t)stream;
    static const float kMults[SNAPS_TUNE_CELLS] = {1.f, 0.5f, 1.f / 3.f};

    // the population it times: this one, or an evenly strided sample of it
    snaps_pop *tp = pop;
    float *feat = nullptr, *sample = nullptr;
    auto cleanup = [&]() {
        if (tp != pop) snaps_release(tp);
        if (feat) cudaFree(feat);
        if (sample) cudaFree(sample);
    };
    const int64_t m = std::min<int64_t>(n, SNAPS_TUNE_MAX_N);
    if (m < n) {
        const int64_t stride = n / m;
        if (cudaMalloc(&feat, sizeof(float) * (size_t)n * f) != cudaSuccess ||
            cudaMalloc(&sample, sizeof(float) * (size_t)m * f) != cudaSuccess) {
            cleanup();
            FAIL(SNAPS_ENOMEM, "no device memory for the tuning sample");
        }
        snaps_status r = snaps_pop_features(pop, feat, stream);
        if (r == SNAPS_OK &&
            cudaMemcpy2DAsync(sample, sizeof(float) * f, feat, sizeof(float) * f * stride, sizeof(float) * f,
                              (size_t)m, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
            r = SNAPS_ECUDA;
        if (r == SNAPS_OK) r = snaps_index(ctx, sample, m, f, 0u, stream, &tp);
        if (r != SNAPS_OK) {
            tp = pop;
            cleanup();
            FAIL(r == SNAPS_ECUDA ? SNAPS_ECUDA : r, "building the tuning sample failed");
        }
    }
    const int kk = (int)std::min<int64_t>(k, m - 1);
    float *scores = nullptr;
    if (cudaMalloc(&scores, sizeof(float) * 2 * 4 * (size_t)m) != cudaSuccess) {
        cleanup();
        FAIL(SNAPS_ENOMEM, "no device memory for the tuning scores");
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    snaps_tune_entry res[3] = {};
    snaps_status r = SNAPS_OK;
    // ms of one call over `masks` with `precision`, after one untimed call
    auto timed = [&](const uint16_t *masks, uint32_t precision, double *ms) -> snaps_status {
        for (int rep = 0; rep < 2; ++rep) {
            if (rep == 1 && cudaEventRecord(e0, st) != cudaSuccess) return SNAPS_ECUDA;
            const snaps_status q = snaps_scores(tp, masks, 2, kk, nullptr, precision, scores, nullptr, nullptr, 0,
                                                stream);
            if (q != SNAPS_OK) return q;
        }
        float t = 0.f;
        if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&t, e0, e1) != cudaSuccess)
            return SNAPS_ECUDA;
        *ms = t / 2.0;  // per subspace
        return SNAPS_OK;
    };
    for (int d = 2; d <= kGridMaxDim && d <= f && r == SNAPS_OK; ++d) {
        // two subspaces of d features: the lowest and the highest features
        const uint16_t masks[2] = {(uint16_t)((1u << d) - 1u), (uint16_t)(((1u << d) - 1u) << (f - d))};
        snaps_tune_entry &e = res[d - 2];
        e.d = d;
        r = timed(masks, SNAPS_FP32 | SNAPS_INDEX_NONE, &e.ms_brute);
        for (int c = 0; c < SNAPS_TUNE_CELLS && r == SNAPS_OK; ++c) {
            // the grid at this cell width, through the table the planner reads
            snaps_tune_entry probe = e;
            probe.grid = 1;
            probe.cell_mult = kMults[c];
            {
                std::lock_guard<std::mutex> g(ctx->tune_mu);
                ctx->tune[tune_key(tp->n, d, kk)] = probe;
            }
            r = timed(masks, SNAPS_FP32 | SNAPS_INDEX_GRID, &e.ms_grid[c]);
        }
        if (r != SNAPS_OK) break;
        int best = 0;
        for (int c = 1; c < SNAPS_TUNE_CELLS; ++c)
            if (e.ms_grid[c] < e.ms_grid[best]) best = c;
        e.grid = e.ms_grid[best] < e.ms_brute ? 1 : 0;
        e.cell_mult = kMults[best];
    }
    {
        // the choices hold for populations of this one's size class; a sample's
        // probe entries are dropped
        std::lock_guard<std::mutex> g(ctx->tune_mu);
        for (int d = 2; d <= kGridMaxDim; ++d) {
            if (tp != pop) ctx->tune.erase(tune_key(tp->n, d, kk));
            if (r == SNAPS_OK && res[d - 2].d == d) ctx->tune[tune_key(n, d, k)] = res[d - 2];
            else ctx->tune.erase(tune_key(n, d, k));
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(scores);
    cleanup();
    if (r != SNAPS_OK) return r;
    if (out) std::memcpy(out, res, sizeof(res));
    return SNAPS_OK;
}

snaps_status snaps_autotune_tc(snaps_pop *pop, int k, uint32_t precision, snaps_tc_tune *out, void *stream)
{
    clear_error();
    if (!pop) FAIL(SNAPS_EINVAL, "pop is NULL");
    if (precision != SNAPS_TC_F16 && precision != SNAPS_TC_BF16 && precision != SNAPS_TC_TF32)
        FAIL(SNAPS_EINVAL, "precision must be SNAPS_TC_F16, SNAPS_TC_BF16 or SNAPS_TC_TF32 (got %u)", precision);
    if (!pop->unit_range) FAIL(SNAPS_EINVAL, "the tensor-core forms need every feature to span at most 1");
    ON_DEVICE(pop->ctx->device);
    snaps_ctx *ctx = pop->ctx;
    const int64_t n = pop->n;
    const int f = pop->f;
    if (k < 1 || k > SNAPS_MAX_K || k > n - 1) FAIL(SNAPS_EINVAL, "k must be in 1..min(%d, n - 1)", SNAPS_MAX_K);
    if (f < 3) FAIL(SNAPS_EINVAL, "the population needs >= 3 features");
    cudaStream_t st = (cudaStream_t)stream;

    // The subspaces timed: every subspace of 3..12 of the f features, in a
    // fixed pseudo-random order (a multiplicative hash of the mask), the first
    // kTcBlockWidth of them -- a block of mixed dimensions, as a request of
    // random subspaces fills one.
    std::vector<uint16_t> all;
    for (uint32_t v = 1; v < (1u << f); ++v) {
        const int d = popc16(v);
        if (d >= 3 && d <= 12) all.push_back((uint16_t)v);
    }
    std::stable_sort(all.begin(), all.end(), [](uint16_t a, uint16_t b) {
        return (uint32_t)(a * 2654435761u) < (uint32_t)(b * 2654435761u);
    });
    const int nb = (int)std::min<size_t>(all.size(), kTcBlockWidth);
    const int nl = std::min(nb, 32);

    // the population it times: this one, or an evenly strided sample of it
    snaps_pop *tp = pop;
    float *feat = nullptr, *sample = nullptr, *scores = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    const int saved = ctx->tc_fill_override.exchange(1);  // every block on the tensor cores while timing
    auto cleanup = [&]() {
        ctx->tc_fill_override.store(saved);
        if (tp != pop) snaps_release(tp);
        if (feat) cudaFree(feat);
        if (sample) cudaFree(sample);
        if (scores) cudaFree(scores);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    };
    const int64_t m = std::min<int64_t>(n, SNAPS_TUNE_MAX_N);
    if (m < n) {
        const int64_t stride = n / m;
        if (cudaMalloc(&feat, sizeof(float) * (size_t)n * f) != cudaSuccess ||
            cudaMalloc(&sample, sizeof(float) * (size_t)m * f) != cudaSuccess) {
            cleanup();
            FAIL(SNAPS_ENOMEM, "no device memory for the tuning sample");
        }
        snaps_status r = snaps_pop_features(pop, feat, stream);
        if (r == SNAPS_OK &&
            cudaMemcpy2DAsync(sample, sizeof(float) * f, feat, sizeof(float) * f * stride, sizeof(float) * f,
                              (size_t)m, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
            r = SNAPS_ECUDA;
        if (r == SNAPS_OK) r = snaps_index(ctx, sample, m, f, 0u, stream, &tp);
        if (r != SNAPS_OK) {
            tp = pop;
            cleanup();
            FAIL(r == SNAPS_ECUDA ? SNAPS_ECUDA : r, "building the tuning sample failed");
        }
    }
    const int kk = (int)std::min<int64_t>(k, m - 1);
    if (cudaMalloc(&scores, sizeof(float) * (size_t)nb * 4 * (size_t)m) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cleanup();
        FAIL(SNAPS_ENOMEM, "no device memory for the tuning scores");
    }
    // ms of one call over the first `count` subspaces, after one untimed call
    auto timed = [&](int count, uint32_t prec, double *ms) -> snaps_status {
        for (int rep = 0; rep < 2; ++rep) {
            if (rep == 1 && cudaEventRecord(e0, st) != cudaSuccess) return SNAPS_ECUDA;
            const snaps_status q = snaps_scores(tp, all.data(), count, kk, nullptr, prec | SNAPS_INDEX_NONE, scores,
                                                nullptr, nullptr, 0, stream);
            if (q != SNAPS_OK) return q;
        }
        float t = 0.f;
        if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&t, e0, e1) != cudaSuccess)
            return SNAPS_ECUDA;
        *ms = t;
        return SNAPS_OK;
    };
    snaps_tc_tune res{};
    snaps_status r = timed(nb, precision, &res.ms_block);
    double ms_group = 0.0;
    if (r == SNAPS_OK) r = timed(nl, SNAPS_FP32, &ms_group);
    cleanup();
    if (r != SNAPS_OK) return r;
    res.ms_lone = ms_group / nl;
    // the block pays once it carries more subspaces than its time buys on their own
    const double need = res.ms_lone > 0.0 ? std::ceil(res.ms_block / res.ms_lone) : (double)SNAPS_TC_NEVER;
    res.min_fill = (int)std::min<double>(SNAPS_TC_NEVER, std::max(1.0, need));
    {
        std::lock_guard<std::mutex> g(ctx->tune_mu);
        ctx->tc_fill[tune_key(n, 0, k)] = res.min_fill;
    }
    if (out) *out = res;
    return SNAPS_OK;
}

snaps_status snaps_set_tc_min_fill(snaps_ctx *ctx, int fill)
{
    clear_error();
    if (!ctx) FAIL(SNAPS_EINVAL, "ctx is NULL");
    if (fill < 0 || fill > SNAPS_TC_NEVER) FAIL(SNAPS_EINVAL, "fill must be in 0..%d (got %d)", SNAPS_TC_NEVER, fill);
    ctx->tc_fill_override.store(fill);
    return SNAPS_OK;
}

snaps_status snaps_autotune_set(snaps_ctx *ctx, int64_t n, int k, const snaps_tune_entry *e)
{
    clear_error();
    if (!ctx || !e) FAIL(SNAPS_EINVAL, "ctx and e must not be NULL");
    if (n < 2 || k < 0 || k > SNAPS_MAX_K) FAIL(SNAPS_EINVAL, "need n >= 2 and 0 <= k <= %d", SNAPS_MAX_K);
    if (e->d < 2 || e->d > kGridMaxDim) FAIL(SNAPS_EINVAL, "d must be in 2..%d", kGridMaxDim);
    if (!(e->cell_mult > 0.f && e->cell_mult <= 64.f)) FAIL(SNAPS_EINVAL, "cell_mult must be in (0, 64]");
    std::lock_guard<std::mutex> g(ctx->tune_mu);
    ctx->tune[tune_key(n, e->d, k)] = *e;
    return SNAPS_OK;
}

snaps_status snaps_autotune_clear(snaps_ctx *ctx)
{
    clear_error();
    if (!ctx) FAIL(SNAPS_EINVAL, "ctx is NULL");
    std::lock_guard<std::mutex> g(ctx->tune_mu);
    ctx->tune.clear();
    ctx->tc_fill.clear();
    return SNAPS_OK;
}

static_assert(SNAPS_SELECTIVITY_MAX_BINS == kSelectHistBins, "histogram bins of the C ABI and the kernel");

snaps_status snaps_eps_selectivity(snaps_pop *pop, const uint16_t *masks, int n_masks, const double *targets,
                                   int n_targets, int n_sample, int n_bins, float *eps, float *eps_mean,
                                   void *stream)
{
    clear_error();
    if (!pop) FAIL(SNAPS_EINVAL, "pop is NULL");
    ON_DEVICE(pop->ctx->device);
    snaps_ctx *ctx = pop->ctx;
    const int64_t n = pop->n;
    if (n < 2) FAIL(SNAPS_EINVAL, "need at least 2 objects");
    if (n_masks < 1 || !masks || is_device_ptr(masks)) FAIL(SNAPS_EINVAL, "masks: a host array of >= 1 masks");
    for (int m = 0; m < n_masks; ++m)
        if (popc16(masks[m]) < 2 || (masks[m] >> pop->f) != 0)
            FAIL(SNAPS_EINVAL, "mask %d (0x%x) must have 2..%d bits, all below feature %d", m, masks[m], pop->f,
                 pop->f);
    if (n_targets < 1 || n_targets > kSelectMaxTargets)
        FAIL(SNAPS_EINVAL, "n_targets must be in 1..%d", kSelectMaxTargets);
    if (!targets || is_device_ptr(targets)) FAIL(SNAPS_EINVAL, "targets: a host array");
    for (int t = 0; t < n_targets; ++t)
        if (!(targets[t] > 0.0 && targets[t] <= (double)(n - 1)))
            FAIL(SNAPS_EINVAL, "target %d must be in (0, n - 1]", t);
    if (n_sample < 1 || n_sample > SNAPS_SELECTIVITY_MAX_SAMPLE)
        FAIL(SNAPS_EINVAL, "n_sample must be in 1..%d", SNAPS_SELECTIVITY_MAX_SAMPLE);
    if (n_bins < 1 || n_bins > SNAPS_SELECTIVITY_MAX_BINS)
        FAIL(SNAPS_EINVAL, "n_bins must be in 1..%d", SNAPS_SELECTIVITY_MAX_BINS);
    if (!eps) FAIL(SNAPS_EINVAL, "eps is NULL");
    SNAPS_TRY(check_not_foreign(eps, ctx->device, "eps"));
    SNAPS_TRY(check_not_foreign(eps_mean, ctx->device, "eps_mean"));
    SelectivityTargets tg{};
    tg.n = n_targets;
    tg.m = (int)std::min<int64_t>(n_sample, n);
    if ((double)tg.m * (double)(n - 1) > 2199023255552.0)  // 2^41 distances keep the u64 sum exact
        FAIL(SNAPS_EINVAL, "n_sample * (n - 1) must stay below 2^41");
    for (int t = 0; t < n_targets; ++t) tg.target[t] = targets[t];
    cudaStream_t st = (cudaStream_t)stream;

    std::lock_guard<std::mutex> lock(ctx->sync_mu);
    const size_t work = (selectivity_scratch_bytes(n) + 255) & ~(size_t)255;
    const size_t outs = sizeof(float) * (size_t)n_masks * (n_targets + 1);
    SNAPS_TRY(scratch_reserve(ctx, ctx->scratch, work + outs + 256));
    char *base = (char *)ctx->scratch.ptr;
    float *eps_dev = (float *)(base + work);
    float *mean_dev = eps_dev + (size_t)n_masks * n_targets;
    {
        TraceScope ts(ctx, SNAPS_PHASE_SELECT, st, 4 * n_masks);
        for (int m = 0; m < n_masks; ++m)
            SNAPS_TRY(launch_selectivity(pop->x, n, masks[m], n_bins, tg, base, eps_dev + (size_t)m * n_targets,
                                         mean_dev + m, st));
    }
    auto put = [&](void *dst, const void *src, size_t bytes) -> snaps_status {
        if (!dst) return SNAPS_OK;
        const cudaMemcpyKind kind = is_device_ptr(dst) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
        SNAPS_CHECK_CUDA(cudaMemcpyAsync(dst, src, bytes, kind, st));
        return SNAPS_OK;
    };
    SNAPS_TRY(put(eps, eps_dev, sizeof(float) * (size_t)n_masks * n_targets));
    SNAPS_TRY(put(eps_mean, mean_dev, sizeof(float) * (size_t)n_masks));
    SNAPS_CHECK_CUDA(cudaStreamSynchronize(st));
    return SNAPS_OK;
}

snaps_status snaps_scores(snaps_pop *pop, const uint16_t *masks, int n_masks, int k,
                          const float *eps, uint32_t precision, float *scores, float *norm,
                          int32_t *top, int top_n, void *stream)
{
    clear_error();
    if (!pop) FAIL(SNAPS_EINVAL, "pop is NULL");
    if (k < 1) FAIL(SNAPS_EINVAL, "k must be >= 1 (got %d)", k);
    ON_DEVICE(pop->ctx->device);
    JobSpec j;
    j.pop = pop;
    j.masks = masks;
    j.n_masks = n_masks;
    j.k = k;
    j.eps = eps;
    j.want_eps = true;
    j.precision = precision;
    j.scores = scores;
    j.norm = norm;
    j.top = (top && top_n > 0) ? top : nullptr;
    j.top_n = j.top ? top_n : 0;
    std::lock_guard<std::mutex> g(pop->ctx->sync_mu);
    return run_job(pop->ctx, j, (cudaStream_t)stream, pop->ctx->scratch, pop->ctx->ctrl, false);
}

snaps_status snaps_set_slots(snaps_ctx *ctx, int slots)
{
    clear_error();
    if (!ctx) FAIL(SNAPS_EINVAL, "ctx is NULL");
    if (slots < 1 || slots > 64) FAIL(SNAPS_EINVAL, "slots must be in 1..64 (got %d)", slots);
    std::lock_guard<std::mutex> lk(ctx->q_mu);
    if (!ctx->slots.empty() && slots < (int)ctx->slots.size())
        FAIL(SNAPS_EBUSY, "slots can only grow once serving has started");
    ctx->n_slots = slots;
    return SNAPS_OK;
}

snaps_status snaps_submit(snaps_ctx *ctx, const snaps_request *req, uint64_t *ticket)
{
    clear_error();
    if (!ctx || !req || !ticket) FAIL(SNAPS_EINVAL, "ctx, req and ticket must be non-NULL");
    if (!req->pop || req->pop->ctx != ctx) FAIL(SNAPS_EINVAL, "request population does not belong to this context");
    if (req->k < 1) FAIL(SNAPS_EINVAL, "k must be >= 1 (got %d)", req->k);
    ON_DEVICE(ctx->device);
    Request *r = new Request();
    r->req = *req;
    if (req->n_masks < 1 || !req->masks) {
        delete r;
        FAIL(SNAPS_EINVAL, "a request needs at least one mask");
    }
    r->masks.assign(req->masks, req->masks + req->n_masks);
    if (req->eps) r->eps.assign(req->eps, req->eps + req->n_masks);
    r->req.masks = nullptr;
    r->req.eps = nullptr;
    JobSpec j = spec_of(r);
    snaps_status s = validate(j);
    if (s != SNAPS_OK) {
        delete r;
        return s;
    }
    r->footprint = job_footprint(j);
    r->fusable = fusable_plan(j, make_plan(j));
    if (r->footprint > ctx->budget) {
        const size_t need = r->footprint;
        delete r;
        FAIL(SNAPS_ENOMEM, "request needs %zu bytes, over the budget of %zu", need, ctx->budget);
    }
    {
        std::lock_guard<std::mutex> lk(ctx->q_mu);
        s = start_slots(ctx);
        if (s != SNAPS_OK) {
            delete r;
            return s;
        }
        r->ticket = ctx->next_ticket++;
        r->t_submit = Clock::now();
        r->req.pop->inflight.fetch_add(1);
        ctx->tickets[r->ticket] = r;
        ctx->queue.push_back(r);
        *ticket = r->ticket;
    }
    ctx->q_cv.notify_all();
    return SNAPS_OK;
}

snaps_status snaps_poll(snaps_ctx *ctx, uint64_t ticket, int64_t timeout_us, snaps_result *out)
{
    clear_error();
    if (!ctx) FAIL(SNAPS_EINVAL, "ctx is NULL");
    std::unique_lock<std::mutex> lk(ctx->q_mu);
    auto it = ctx->tickets.find(ticket);
    if (it == ctx->tickets.end()) FAIL(SNAPS_EINVAL, "unknown ticket %llu", (unsigned long long)ticket);
    Request *r = it->second;
    if (!r->done) {
        if (timeout_us == 0) return SNAPS_EAGAIN;
        if (timeout_us < 0)
            ctx->done_cv.wait(lk, [&] { return r->done; });
        else if (!ctx->done_cv.wait_for(lk, std::chrono::microseconds(timeout_us), [&] { return r->done; }))
            return SNAPS_EAGAIN;
    }
    if (out) {
        out->status = r->status;
        const auto us = [](Clock::duration d) { return std::chrono::duration<double, std::micro>(d).count(); };
        out->queue_us = r->status == SNAPS_ECANCELED ? us(r->t_done - r->t_submit) : us(r->t_admit - r->t_submit);
        out->latency_us = us(r->t_done - r->t_submit);
        out->objects_x_subspaces = r->req.pop ? r->req.pop->n * (int64_t)r->masks.size() : 0;
    }
    ctx->tickets.erase(it);
    delete r;
    return SNAPS_OK;
}

snaps_status snaps_cancel(snaps_ctx *ctx, uint64_t ticket)
{
    clear_error();
    if (!ctx) FAIL(SNAPS_EINVAL, "ctx is NULL");
    std::lock_guard<std::mutex> lk(ctx->q_mu);
    auto it = ctx->tickets.find(ticket);
    if (it == ctx->tickets.end()) FAIL(SNAPS_EINVAL, "unknown ticket %llu", (unsigned long long)ticket);
    Request *r = it->second;
    if (r->done || r->running) FAIL(SNAPS_EBUSY, "request %llu is already running or finished", (unsigned long long)ticket);
    for (auto q = ctx->queue.begin(); q != ctx->queue.end(); ++q) {
        if (*q == r) {
            ctx->queue.erase(q);
            break;
        }
    }
    r->status = SNAPS_ECANCELED;
    r->done = true;
    r->t_done = Clock::now();
    r->req.pop->inflight.fetch_sub(1);
    ctx->done_cv.notify_all();
    return SNAPS_OK;
}

snaps_status snaps_serving_stats(snaps_ctx *ctx, int64_t *fused_launches, int64_t *fused_requests)
{
    clear_error();
    if (!ctx) FAIL(SNAPS_EINVAL, "ctx is NULL");
    if (fused_launches) *fused_launches = ctx->fused_launches.load();
    if (fused_requests) *fused_requests = ctx->fused_requests.load();
    return SNAPS_OK;
}

snaps_status snaps_set_wait_limit(snaps_ctx *ctx, unsigned spins)
{
    clear_error();
    if (!ctx) FAIL(SNAPS_EINVAL, "ctx is NULL");
    ctx->wait_limit.store(spins);
    return SNAPS_OK;
}

snaps_status snaps_trace(snaps_ctx *ctx, int enable)
{
    clear_error();
    if (!ctx) FAIL(SNAPS_EINVAL, "ctx is NULL");
    ON_DEVICE(ctx->device);
    std::lock_guard<std::mutex> g(ctx->tr_mu);
    if (enable) {
        for (auto &m : ctx->marks) {
            ctx->spare.push_back(m.a);
            ctx->spare.push_back(m.b);
        }
        ctx->marks.clear();
        // the subspace-batched join's step counters restart too
        SNAPS_CHECK_CUDA(cudaDeviceSynchronize());
        SNAPS_CHECK_CUDA(cudaMemset(&ctx->ctrl->steps_loaded, 0, 2 * sizeof(unsigned long long)));
        SNAPS_CHECK_CUDA(cudaDeviceSynchronize());
    }
    ctx->tracing = enable != 0;
    return SNAPS_OK;
}

snaps_status snaps_trace_steps(snaps_ctx *ctx, int64_t *steps_loaded, int64_t *steps_total)
{
    clear_error();
    if (!ctx) FAIL(SNAPS_EINVAL, "ctx is NULL");
    ON_DEVICE(ctx->device);
    unsigned long long v[2] = {0ull, 0ull};
    SNAPS_CHECK_CUDA(cudaDeviceSynchronize());
    SNAPS_CHECK_CUDA(cudaMemcpy(v, &ctx->ctrl->steps_loaded, sizeof(v), cudaMemcpyDeviceToHost));
    if (steps_loaded) *steps_loaded = (int64_t)v[0];
    if (steps_total) *steps_total = (int64_t)v[1];
    return SNAPS_OK;
}

snaps_status snaps_trace_read(snaps_ctx *ctx, double *ms, int64_t *launches)
{
    clear_error();
    if (!ctx) FAIL(SNAPS_EINVAL, "ctx is NULL");
    ON_DEVICE(ctx->device);
    std::vector<snaps_ctx::Mark> marks;
    {
        std::lock_guard<std::mutex> g(ctx->tr_mu);
        marks.swap(ctx->marks);
    }
    double acc[SNAPS_N_PHASES] = {0};
    int64_t cnt[SNAPS_N_PHASES] = {0};
    snaps_status st = SNAPS_OK;
    for (auto &m : marks) {
        if (cudaEventSynchronize(m.b) != cudaSuccess) st = SNAPS_ECUDA;
        float t = 0.f;
        if (cudaEventElapsedTime(&t, m.a, m.b) == cudaSuccess) {
            acc[m.phase] += t;
            cnt[m.phase] += m.kernels;
        } else {
            cudaGetLastError();
        }
    }
    {
        std::lock_guard<std::mutex> g(ctx->tr_mu);
        for (auto &m : marks) {
            ctx->spare.push_back(m.a);
            ctx->spare.push_back(m.b);
        }
    }
    for (int p = 0; p < SNAPS_N_PHASES; ++p) {
        if (ms) ms[p] = acc[p];
        if (launches) launches[p] = cnt[p];
    }
    if (st != SNAPS_OK) FAIL(st, "waiting for trace events failed");
    return SNAPS_OK;
}

}  // extern "C"
