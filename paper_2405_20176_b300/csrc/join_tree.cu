// Subspace-batched self-join: DSSJ (Sec. 3.5) and kNNSJ (Sec. 3.6) for the 32
// subspaces (H << 5) | L, L = 0..31, that share one high part H.
//
// Why batching pays: in the fixed order the library uses, the squared
// distance of subspace S is the FMA fold of the squared feature differences
// from the highest feature index down.  The subspaces H|L therefore form a
// tree rooted at the fold over H's features, and node L is one FMA away from
// node L minus its lowest bit.  A warp evaluates all 32 subspaces of a
// (query, candidate) pair with 15 subtractions, <= 10 root FMAs and 31 tree
// FMAs -- about one FMA per subspace instead of one per feature.
//
// Mapping: a warp owns one work item, one query of one chunk, which it
// claims from an atomic counter.  Each lane owns two candidates per step of
// 64 rows, packed so that the f32x2 instructions (FADD2/FFMA2) process both;
// the rows are read straight from global memory (the population stays in L2),
// the next live step's while the current one is walked.  The walk spends, per
// subspace, one FFMA2, one FADD2 against the negated pass threshold,
// max(current k-th distance, eps), read from shared memory (warp-uniform,
// broadcast), and a sign-bit OR and shift.  On steps where some lane's
// candidates pass somewhere, an out-of-line handler lists the warp's
// triggered (lane, subspace) pairs and processes them 32 at a time with every
// lane busy: it recomputes each pair's distances, counts the eps-neighbours
// and sums their exact fixed-point distances by shared-memory atomics, and
// appends the kNN candidates as (squared distance, subspace, candidate)
// tuples to the warp's buffer.  Once enough tuples wait, a flush offers them
// to the kNN lists (max-heaps), lanes holding different subspaces inserting
// into their lists at the same time.
//
// Skipping: every node of a chunk's tree is at least its root, the fold over
// the high features, so a step none of whose roots is below the chunk's
// largest pass threshold cannot produce an event.  Each step of a chunk's row
// copy carries the box (min, max) of its rows' high features; the warp bounds
// 32 steps at a time from the boxes, one lane per step, and only loads and
// walks the steps whose bound stays under the threshold.  Loaded steps are
// then tested on their exact roots before the walk.
//
// Row order: each chunk gets its own copy of the rows, sorted by a Morton key
// over the chunk's high features (the features all 32 of its subspaces share)
// and stored pair-planar (common.cuh); every row carries its original index in
// float 15, and lists, ties and outputs use original indices, so results do
// not depend on the order.  A query's stream starts at its own tile -- its
// neighbourhood in those features -- and wraps around.  A set-up phase (out
// of line) first bounds every subspace's k-th distance from the first 768
// candidates of the stream: each lane keeps, per subspace, the smallest of its
// own candidates' distances, and the k-th smallest of those 32 group minima
// is an upper bound (k distinct candidates lie at or below it).  Each list
// starts as k placeholder entries at that bound, so the thresholds start
// tight, and the main loop then walks the whole stream, the set-up's steps
// included; only candidates at or below the bound become kNN events.  This
// costs a fold and a minimum per node and one 32-value sort per subspace,
// where inserting the early candidates one by one into the lists cost a
// serial list update for each of the many that improved an early list.
//
// Two CTAs share an SM (16 warps with k <= 16), with no barriers between
// warps: every warp streams at its own pace.

#include <math_constants.h>

#include <algorithm>

#include "device.cuh"
#include "join.cuh"

namespace snaps {
namespace {

constexpr int kLB = kTreeLowBits;  // 5
constexpr int kW = kTreeWidth;     // 32 subspaces per chunk
constexpr int kTile = 256;
constexpr int kInit = 768;         // candidates that bound the k-th distances in the set-up phase
constexpr int kTBuf = 1024;        // event tuples buffered per warp
// The buffer's tail stages an append's candidates (7 x 32 float2) and its
// list of (lane, subspace) pairs (at most 32 x 32 halfwords): 480 tuples' room.
constexpr int kTStage = kTBuf - 480;
constexpr int kTFlushAt = kTStage - 64;  // a round of appends adds at most 64 tuples
constexpr int kFlushMin = 32;      // tuples that trigger an end-of-step flush

// Depth-first order of the subset tree over the low kLB bits: node L's parent
// is L with its lowest set bit cleared, and its children add a bit below that.
struct DfsTable {
    int node[kW];    // L at DFS position p
    int parent[kW];  // DFS position of the parent (p = 0 is the root)
    int bit[kW];     // feature (low-bit index) the node adds to its parent
};

constexpr DfsTable make_dfs() {
    DfsTable t{};
    int stack_node[kW] = {};
    int stack_pos[kW] = {};
    int cursor[kW] = {};
    int top = 1, pos = 1;
    t.node[0] = 0;
    t.parent[0] = 0;
    t.bit[0] = 0;
    stack_node[0] = 0;
    stack_pos[0] = 0;
    cursor[0] = kLB - 1;
    while (top > 0) {
        const int s = top - 1;
        if (cursor[s] < 0) {
            --top;
            continue;
        }
        const int b = cursor[s]--;
        const int child = stack_node[s] | (1 << b);
        t.node[pos] = child;
        t.parent[pos] = stack_pos[s];
        t.bit[pos] = b;
        stack_node[top] = child;
        stack_pos[top] = pos;
        cursor[top] = b - 1;
        ++top;
        ++pos;
    }
    return t;
}
constexpr DfsTable kDfs = make_dfs();

static_assert(kTBuf * 2 >= kW * (kW + 1), "the set-up transpose fits the tuple buffer");
static_assert((kTBuf - kTStage) * 8 >= 7 * 32 * 8 + 32 * 32 * 2, "an append's staging fits the buffer's tail");
static_assert(64ull * ((1u << 20) + 1u) < (1ull << 32), "an append's eps partial sums fit 32 bits");
static_assert(kDfs.node[1] == 16 && kDfs.parent[kW / 2] > 0, "DFS order as expected");

// The walk visits node L = 8 j + m at position P = j + 4 m (j = 0..3, m =
// 0..7): a parent (L with its lowest set bit cleared) always comes first.
__host__ __device__ constexpr int walk_pos(int L) { return (L >> 3) + 4 * (L & 7); }
__host__ __device__ constexpr int low_bit(int L) { return (L & 1) ? 0 : (L & 2) ? 1 : (L & 4) ? 2 : (L & 8) ? 3 : 4; }
constexpr bool walk_order_valid()
{
    bool seen[kW] = {};
    for (int L = 0; L < kW; ++L) {
        if (walk_pos(L) < 0 || walk_pos(L) >= kW || seen[walk_pos(L)]) return false;  // a permutation
        seen[walk_pos(L)] = true;
        if (L > 0 && !(walk_pos(L & (L - 1)) < walk_pos(L))) return false;  // parents first
    }
    return true;
}
static_assert(walk_order_valid(), "the walk visits every node once, each after its parent");

// Per consumer warp: the state of its query across the chunk's 32 subspaces.
template <int KMAX>
struct WarpState {
    uint2 tbuf[kTBuf];              // pending kNN candidates: (d2 bits, L << 24 | candidate);
                                    // its tail stages an append's candidates and pairs;
                                    // during the set-up phase, the transpose buffer
    float ld[kW][KMAX + 1];         // kNN lists by L; +1 keeps both access patterns
    int lj[kW][KMAX + 1];           // free of bank conflicts
    unsigned long long esum[kW];    // exact quantised eps distance sums
    unsigned epart[kW];             // an append's partial sums (<= 64 terms of <= 2^20 + 1)
    float T[kW];                    // current k-th squared distance: the heap's root
    int Tj[kW];                     // its original index
    float tc[kW];                   // pass threshold max(T, eps) by L
    alignas(16) float tcw[kW];      // the same negated, in the walk's order, read four at a time
    float tcmax;                    // the largest of them: a bound for the whole tree
    int cnt[kW];                    // eps-neighbour counts
    float eps2[kW];                 // radii of this chunk
    int claim[kW];                  // flush: the lane that inserts into list L this round
    float escale[kW];               // 2^20 / eps
    float2 nxq[16];                 // the query's negated features, as (a, b) pairs
    unsigned long long stat_loaded; // steps loaded and steps in the streams of this warp's items
    unsigned long long stat_total;
};

// Two CTAs share an SM: 2 x 8 warps (k <= 16, 128 registers a thread) or
// 2 x 6 warps (k <= 32, whose lists need more shared memory; 168 registers).
template <int CW>
constexpr int kCtasPerSm = 2;

template <int KMAX, int CW>
struct TreeSmem {
    WarpState<KMAX> ws[CW];
};

// The kernel's dynamic shared memory, declared here so that device functions
// outside the kernel address it as shared memory.
extern __shared__ __align__(128) unsigned char tree_smem[];

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }

__device__ __forceinline__ float eps_up(float e2) {
    // d2 < eps_up(e2)  <=>  d2 <= e2 for finite e2 >= 0; disabled radii never pass
    return e2 >= 0.f ? __uint_as_float(__float_as_uint(e2) + 1u) : -CUDART_INF_F;
}

__device__ __forceinline__ float next_up(float t) {
    // d2 < next_up(t)  <=>  d2 <= t for finite t >= 0 (a tie with the k-th
    // distance may still enter through a smaller original index); +-inf stay as they are
    return (t >= 0.f && t < CUDART_INF_F) ? __uint_as_float(__float_as_uint(t) + 1u) : t;
}

// tcmax <- the largest pass threshold of the chunk's subspaces (lane L holds
// subspace L's).  Thresholds are floats >= 0 or -inf, whose bit patterns order
// like their values as signed integers.
template <int KMAX>
__device__ __forceinline__ void update_tcmax(WarpState<KMAX> &ws)
{
    __syncwarp();
    const int mx = __reduce_max_sync(dev::kFull, __float_as_int(ws.tc[dev::lane_id()]));
    if (dev::lane_id() == 0) ws.tcmax = __int_as_float(mx);
    __syncwarp();
}

// A kNN list is a max-heap of k entries by (distance, index) (dev::heap_sink_root):
// entry 0 is the largest, the current k-th nearest, and T / Tj mirror it.
__device__ __forceinline__ void list_offer(float *ld, int *lj, int k, float d2, int j, float &T, int &Tj)
{
    if (!(d2 < T || (d2 == T && j < Tj))) return;
    dev::heap_sink_root(ld, lj, 1, k, d2, j);
    T = ld[0];
    Tj = lj[0];
}

// Process the buffered kNN candidates (the appends count the eps-neighbours
// themselves), 32 at a time: lanes holding candidates of different subspaces
// insert at the same time (each into its own list); of the lanes that share a
// subspace, one per round claims the list (the last writer of a shared slot),
// the others retry.  A candidate that a list no longer admits (its k-th
// distance fell since the append) is turned away by the offer.  The k
// smallest (distance, original index) pairs do not depend on the order of
// insertion.  Returns true when a kNN list changed.
template <int KMAX>
__device__ __noinline__ bool flush_tuples(int ws_off, int count, int k)
{
    WarpState<KMAX> &ws = *reinterpret_cast<WarpState<KMAX> *>(tree_smem + ws_off);
    const unsigned lane = dev::lane_id();
    unsigned changed = 0;  // bit L: list L changed
    __syncwarp();
    for (int b = 0; b < count; b += 32) {
        const int idx = b + (int)lane;
        const bool ok = idx < count;
        const uint2 t = ok ? ws.tbuf[idx] : make_uint2(0x7f800000u, 0u);
        const int L = (int)(t.y >> 24);
        const int j = (int)(t.y & 0xffffffu);
        const float d2 = __uint_as_float(t.x);
        bool w = ok;
        unsigned pend = __ballot_sync(dev::kFull, w);
        while (pend) {
            // one of the lanes that hold list L inserts this round
            if (w) ws.claim[L] = (int)lane;
            __syncwarp();
            const bool mine = w && ws.claim[L] == (int)lane;
            if (mine) {
                float T = ws.T[L];
                int Tj = ws.Tj[L];
                list_offer(ws.ld[L], ws.lj[L], k, d2, j, T, Tj);
                ws.T[L] = T;
                ws.Tj[L] = Tj;
                changed |= 1u << L;
            }
            w = w && !mine;
            pend = __ballot_sync(dev::kFull, w);
        }
    }
    changed = __reduce_or_sync(dev::kFull, changed);
    __syncwarp();
    ws.esum[lane] += ws.epart[lane];  // an interrupted append's eps sums so far
    ws.epart[lane] = 0u;
    if ((changed >> lane) & 1u) {
        const float t = fmaxf(next_up(ws.T[lane]), eps_up(ws.eps2[lane]));
        ws.tc[lane] = t;
        ws.tcw[walk_pos(lane)] = -t;
    }
    update_tcmax(ws);
    return changed != 0u;
}

// The walk: the 32 subspace distances of this lane's two candidates (one
// FFMA2 per node) and the set of subspaces L in which either candidate fell
// below its pass threshold.  The test is the sign of d2 - threshold (an FADD2
// with the negated thresholds, exact in sign: the difference of two floats is
// 0 only when they are equal), shifted into one of four partial masks, node
// m of partial j at bit 7 - m; walk_bits turns them into bit L.  No branches.
template <int P>
__device__ __forceinline__ void walk(float2 (&v)[kW], const float2 (&d)[15], const float4 *tcw, float4 tq,
                                     unsigned (&part)[4])
{
    if constexpr (P < kW) {
        constexpr int j = P & 3, m = P >> 2;
        constexpr int L = 8 * j + m;
        if constexpr (P > 0) {
            constexpr int par = L & (L - 1);           // parent: the lowest set bit cleared
            constexpr int b = low_bit(L);              // the low feature it adds
            v[P] = __ffma2_rn(d[b], d[b], v[walk_pos(par)]);
        }
        if constexpr (j == 0) tq = tcw[P >> 2];  // negated thresholds of positions P .. P + 3
        const float tn = j == 0 ? tq.x : j == 1 ? tq.y : j == 2 ? tq.z : tq.w;
        const float2 w = __fadd2_rn(v[P], make_float2(tn, tn));
        part[j] = __funnelshift_l(__float_as_uint(w.x) | __float_as_uint(w.y), part[j], 1);
        walk<P + 1>(v, d, tcw, tq, part);
    }
}

__device__ __forceinline__ unsigned walk_bits(const unsigned (&part)[4])
{
    return (__brev(part[0]) >> 24) | (__brev(part[1]) >> 16) | (__brev(part[2]) >> 8) | __brev(part[3]);
}

// Handle this lane's triggered subspaces (bit L of `bits`: either candidate
// fell below subspace L's pass threshold in the walk), with the work spread
// evenly over the warp.  Each lane stages its two candidates (root, the low
// features' differences and the original indices) in the tail of the tuple
// buffer and lists its (lane, L) pairs there at its offset of the warp's
// prefix sum; then every lane takes one pair per round, so the rounds number
// the warp's pairs over 32, not the most any one lane triggered.  A node's
// distances are recomputed from the root with the walk's own FFMA2 chain (the
// low features of L folded from the highest down), so they are bit-identical
// to the walk's.  eps-neighbours are counted and their quantised distances
// summed right here (shared-memory atomics, merged into the exact totals when
// the call ends); candidates at or below the subspace's k-th distance are
// appended as tuples for the next flush.  A round appends at most 64 tuples,
// and a nearly full buffer is flushed.  Out of line: it runs on a minority of
// steps, and inlined its registers would count against the walk's.  Returns
// the new tuple count.
__device__ __forceinline__ float2 node_of(float2 v, int L, float2 d0, float2 d1, float2 d2, float2 d3, float2 d4)
{
    if (L & 16) v = __ffma2_rn(d4, d4, v);
    if (L & 8) v = __ffma2_rn(d3, d3, v);
    if (L & 4) v = __ffma2_rn(d2, d2, v);
    if (L & 2) v = __ffma2_rn(d1, d1, v);
    if (L & 1) v = __ffma2_rn(d0, d0, v);
    return v;
}

template <int KMAX>
__device__ __noinline__ int append_hits(int ws_off, unsigned bits, float2 root, float2 d0, float2 d1,
                                        float2 d2, float2 d3, float2 d4, int count, int ja, int jb, int k)
{
    WarpState<KMAX> &ws = *reinterpret_cast<WarpState<KMAX> *>(tree_smem + ws_off);
    const unsigned lane = dev::lane_id();
    const unsigned lower = (1u << lane) - 1u;
    float2 *stg = reinterpret_cast<float2 *>(&ws.tbuf[kTStage]);
    unsigned short *pairs = reinterpret_cast<unsigned short *>(stg + 7 * 32);
    __syncwarp();  // a previous call's readers of the staging area are done
    stg[0 * 32 + lane] = root;
    stg[1 * 32 + lane] = d0;
    stg[2 * 32 + lane] = d1;
    stg[3 * 32 + lane] = d2;
    stg[4 * 32 + lane] = d3;
    stg[5 * 32 + lane] = d4;
    stg[6 * 32 + lane] = make_float2(__int_as_float(ja), __int_as_float(jb));
    const int c = __popc(bits);
    int inc = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(dev::kFull, inc, o);
        if ((int)lane >= o) inc += v;
    }
    const int total = __shfl_sync(dev::kFull, inc, 31);
    int pos = inc - c;
    for (unsigned m = bits; m; m &= m - 1u) pairs[pos++] = (unsigned short)((lane << 5) | (unsigned)(__ffs(m) - 1));
    __syncwarp();
    for (int e0 = 0; e0 < total; e0 += 32) {
        const int e = e0 + (int)lane;
        const bool has = e < total;
        const unsigned pr = has ? pairs[e] : 0u;
        const int o = (int)(pr >> 5), L = (int)(pr & 31u);
        const float2 jj = stg[6 * 32 + o];
        const float2 v = node_of(stg[o], L, stg[1 * 32 + o], stg[2 * 32 + o], stg[3 * 32 + o], stg[4 * 32 + o],
                                 stg[5 * 32 + o]);
        // eps-neighbours are counted here; only kNN candidates become tuples
        const float e2 = ws.eps2[L];
        const bool ia = has && v.x <= e2, ib = has && v.y <= e2;
        if (ia || ib) {
            const float es = ws.escale[L];
            atomicAdd(&ws.cnt[L], (ia ? 1 : 0) + (ib ? 1 : 0));
            atomicAdd(&ws.epart[L], (ia ? dev::eps_quant(v.x, es) : 0u) + (ib ? dev::eps_quant(v.y, es) : 0u));
        }
        const float t = ws.T[L];  // -inf for inactive subspaces and k = 0
        const bool pa = has && v.x <= t, pb = has && v.y <= t;
        const unsigned ba = __ballot_sync(dev::kFull, pa);
        const unsigned bb = __ballot_sync(dev::kFull, pb);
        const int ob = count + __popc(ba);
        if (pa) ws.tbuf[count + __popc(ba & lower)] = make_uint2(__float_as_uint(v.x), (L << 24) | (__float_as_int(jj.x) & 0xffffff));
        if (pb) ws.tbuf[ob + __popc(bb & lower)] = make_uint2(__float_as_uint(v.y), (L << 24) | (__float_as_int(jj.y) & 0xffffff));
        count = ob + __popc(bb);
        if (count > kTFlushAt) {
            flush_tuples<KMAX>(ws_off, count, k);
            count = 0;
        }
    }
    // this call's eps sums (<= 64 terms a subspace) into the exact totals
    __syncwarp();
    ws.esum[lane] += ws.epart[lane];
    ws.epart[lane] = 0u;
    __syncwarp();
    return count;
}

// One step's candidates in the pair-planar layout: lane l's 8 float4 hold
// the 16 floats of rows a = 64s + l and b = 64s + 32 + l, feature pairs (a, b)
// adjacent.  Loaded straight from global memory (the rows stay in L2).
struct StepRows {
    float4 r[8];
};

__device__ __forceinline__ void load_step(const float4 *__restrict__ x, int step, unsigned lane,
                                          StepRows &r)
{
#pragma unroll
    for (int q = 0; q < 8; ++q) r.r[q] = __ldg(&x[(step * 8 + q) * 32 + lane]);
}

// (a, b) pair of feature f.
__device__ __forceinline__ float2 feat_pair(const StepRows &r, int f)
{
    const float4 v = r.r[f >> 1];
    return (f & 1) ? make_float2(v.z, v.w) : make_float2(v.x, v.y);
}

// The root of a step's two candidates: the fold over the chunk's high
// features, the highest first.  In a compacted copy those sit in floats 5..
// in that order, followed by zeros whose FMAs leave the fold unchanged, so the
// fold needs no branches.
template <bool CMP>
__device__ __forceinline__ float2 root_fold(const float2 (&d)[15], uint32_t high)
{
    float2 v = f2(0.f, 0.f);
    if constexpr (CMP) {
#pragma unroll
        for (int f = kLB; f < 15; ++f) v = __ffma2_rn(d[f], d[f], v);
    } else {
#pragma unroll
        for (int f = 14; f >= kLB; --f)
            if ((high >> (f - kLB)) & 1u) v = __ffma2_rn(d[f], d[f], v);
    }
    return v;
}

// Sorts a[0..N) ascending (bitonic network, N a power of two).
template <int N>
__device__ __forceinline__ void sort_net(float (&a)[N])
{
#pragma unroll
    for (int size = 2; size <= N; size <<= 1)
#pragma unroll
        for (int stride = size >> 1; stride > 0; stride >>= 1)
#pragma unroll
            for (int e = 0; e < N; ++e) {
                const int f = e ^ stride;
                if (f > e) {
                    const float x = a[e], y = a[f];
                    const bool up = (e & size) == 0;
                    a[e] = up ? fminf(x, y) : fmaxf(x, y);
                    a[f] = up ? fmaxf(x, y) : fminf(x, y);
                }
            }
}

// The walk with a running minimum per node (set-up phase): mn[L] <- min(mn[L],
// both candidates' squared distances in subspace L).
template <int P>
__device__ __forceinline__ void fold_min(float2 (&v)[kW], const float2 (&d)[15], float (&mn)[kW])
{
    if constexpr (P < kW) {
        if constexpr (P > 0) {
            constexpr int b = kDfs.bit[P];
            constexpr int par = kDfs.parent[P];
            v[P] = __ffma2_rn(d[b], d[b], v[par]);
        }
        constexpr int L = kDfs.node[P];
        mn[L] = fminf(mn[L], fminf(v[P].x, v[P].y));
        fold_min<P + 1>(v, d, mn);
    }
}

// Set-up phase (see the kernel), kept out of line so that its registers do
// not add to the main loop's.  Each lane folds its candidates of the first
// steps and keeps, per subspace, the smallest squared distance among them: 32
// groups of candidates (one per lane) and their 32 minima per subspace.  The
// k-th smallest of those minima bounds the subspace's k-th distance from
// above -- k distinct candidates lie at or below it -- and its list starts as
// k entries (bound, largest index), which any candidate at or below the bound
// displaces.  The steps themselves are walked again by the main loop.
template <int KMAX, bool CMP>
__device__ __noinline__ void setup_phase(int ws_off, const float4 *__restrict__ x, int64_t i, int64_t n,
                                         uint32_t high, uint32_t active, int64_t s0, int64_t n_steps, int k)
{
    WarpState<KMAX> &ws = *reinterpret_cast<WarpState<KMAX> *>(tree_smem + ws_off);
    const unsigned lane = dev::lane_id();
    const float2 *nxq = ws.nxq;
    float mn[kW];
#pragma unroll
    for (int L = 0; L < kW; ++L) mn[L] = CUDART_INF_F;
    const int64_t init_steps = std::min<int64_t>(kInit / 64, n_steps);
    for (int64_t u = 0; u < init_steps; ++u) {
        const int64_t step = (s0 + u) % n_steps;
        StepRows r;
        load_step(x, step, lane, r);
        float2 d[15];
#pragma unroll
        for (int f = 0; f < 15; ++f) d[f] = __fadd2_rn(feat_pair(r, f), nxq[f]);
        if ((i >> 6) == step) {
            // the query itself is in this step: make it infinitely far
            const int64_t ja = step * 64 + lane, jb = ja + 32;
#pragma unroll
            for (int f = 0; f < 15; ++f) {
                if (ja == i) d[f].x = CUDART_INF_F;
                if (jb == i) d[f].y = CUDART_INF_F;
            }
        }
        // (padding rows are +inf and fold to +inf)
        float2 v[kW];
        v[0] = root_fold<CMP>(d, high);
        fold_min<0>(v, d, mn);
    }
    // transpose: row L <- the 32 lanes' minima of subspace L
    float *stg = reinterpret_cast<float *>(ws.tbuf);  // [32][33]
    __syncwarp();
#pragma unroll
    for (int L = 0; L < kW; ++L) stg[L * 33 + lane] = mn[L];
    __syncwarp();
    const uint32_t L = lane;
    float g[kW];
#pragma unroll
    for (int c = 0; c < kW; ++c) g[c] = stg[L * 33 + c];
    sort_net<kW>(g);
    float bound = g[0];
#pragma unroll
    for (int c = 1; c < kW; ++c) bound = (c == k - 1) ? g[c] : bound;
    __syncwarp();
    const bool mine = (active >> L) & 1u;
    const float e2 = ws.eps2[L];
    if (mine && k > 0) {
        for (int p = 0; p < k; ++p) {
            ws.ld[L][p] = bound;
            ws.lj[L][p] = 0x7fffffff;
        }
        ws.T[L] = bound;
        ws.Tj[L] = 0x7fffffff;
    }
    ws.tc[L] = mine ? fmaxf(next_up(ws.T[L]), eps_up(e2)) : -CUDART_INF_F;
    ws.tcw[walk_pos(L)] = -ws.tc[L];
    update_tcmax(ws);
}

template <int KMAX, int CW, bool CMP>
__global__ void __launch_bounds__(CW * 32, kCtasPerSm<CW>)
    join_tree_kernel(JoinShape s, const TreeChunk *__restrict__ chunks, int n_chunks, JoinOut o,
                     DeviceControl *ctrl)
{
    TreeSmem<KMAX, CW> &sm = *reinterpret_cast<TreeSmem<KMAX, CW> *>(tree_smem);
    const int warp = threadIdx.x >> 5;
    const unsigned lane = threadIdx.x & 31u;
    const int64_t n = s.n;
    const int k = s.k;
    const long long total = n * (long long)n_chunks;
    const int n_tiles = (int)(s.n_pad / kTile);
    WarpState<KMAX> &ws = sm.ws[warp];
    const int ws_off = (int)((const unsigned char *)&sm.ws[warp] - tree_smem);

    if (lane == 0) {
        ws.stat_loaded = 0ull;
        ws.stat_total = 0ull;
    }
    for (;;) {
        // ---- next work item (one query of one chunk), claimed by the warp -----------
        unsigned long long wc = 0;
        if (lane == 0) wc = atomicAdd(&ctrl->next_work, 1ull);
        const long long w = (long long)__shfl_sync(dev::kFull, wc, 0);
        if (w >= total) {
            if (lane == 0) {
                atomicAdd(&ctrl->steps_loaded, ws.stat_loaded);
                atomicAdd(&ctrl->steps_total, ws.stat_total);
            }
            return;
        }
        const TreeChunk *ch = &chunks[w / n];
        // the chunk's rows (in the chunk's own order when each chunk has a copy)
        const float4 *__restrict__ x = s.x + (w / n) * s.chunk_stride;
        const int i = (int)(w % n);  // the query's row in that order (n <= 2^24)
        const uint32_t high = ch->high;
        const uint32_t active = ch->active;
        float xq[16];
        const float *xf = reinterpret_cast<const float *>(x);
#pragma unroll
        for (int f = 0; f < 16; ++f) xq[f] = xf[pair_float(i, f)];
        const int orig_i = __float_as_int(xq[15]);  // the query's original index
        if (orig_i < 0 || orig_i >= n) {
            // rows that do not carry their index: report, write nothing
            if (lane == 0) atomicOr(&ctrl->error, kErrBadRow);
            continue;
        }
        if (lane < 15) ws.nxq[lane] = f2(-xq[lane], -xq[lane]);
        __syncwarp();
        const float2 *nxq = ws.nxq;
        // the candidate stream starts at the query's own tile (in cell order, its
        // neighbourhood) and wraps around
        const int t0 = (int)(i / kTile);
        {
            const uint32_t L = lane;
            const float e2 = ch->eps2[L];
            ws.eps2[L] = e2;
            ws.escale[L] = dev::eps_scale(e2).scale;
            for (int p = 0; p < KMAX; ++p) {
                ws.ld[L][p] = CUDART_INF_F;
                ws.lj[L][p] = 0x7fffffff;
            }
            ws.esum[L] = 0ull;
            ws.epart[L] = 0u;
            ws.cnt[L] = 0;
            ws.T[L] = (((active >> L) & 1u) && k > 0) ? CUDART_INF_F : -CUDART_INF_F;
            ws.Tj[L] = 0x7fffffff;
        }
        __syncwarp();
        // The candidate stream: all steps of 64 rows, starting at the query's own
        // tile (in the chunk's order, its neighbourhood) and wrapping around.
        constexpr int kSteps = kTile / 64;  // steps per tile
        const int n_steps = n_tiles * kSteps;
        const int s0 = t0 * kSteps;
        setup_phase<KMAX, CMP>(ws_off, x, i, n, high, active, s0, n_steps, k);
        __syncwarp();

        // ---- main loop: the rest of the stream, 64 candidates a step -----------------
        // Steps go in windows of 32.  Lane l bounds the roots of window step l from
        // below by the box of its rows' high features (folded in the root's order,
        // so the bound is <= every row's FP32 root); a step whose bound reaches the
        // chunk's largest pass threshold cannot pass anywhere and is neither loaded
        // nor walked.  The next live step's rows load while one is walked.
        int tcount = 0;  // buffered event tuples (warp-uniform)
        const int init_steps = std::min(kInit / 64, n_steps);
        const float2 *box = s.box ? s.box + (w / n) * s.box_stride : nullptr;
        const int n_high = __popc(high);
        int wbase = 0, next_w = 0;  // the set-up's steps are walked again
        unsigned live = 0u;
        int taken = 0;  // steps of the stream loaded by the main loop
        auto take = [&]() -> int {
            while (live == 0u) {
                if (next_w >= n_steps) return -1;
                const int u = next_w + (int)lane;
                bool ok = u < n_steps;
                if (ok && box) {
                    const int step = (s0 + u) % n_steps;
                    float lb = 0.f;
                    if constexpr (CMP) {
                        for (int b = 0; b < n_high; ++b) {
                            const float2 mm = box[(int64_t)b * n_steps + step];
                            const float q = -nxq[kLB + b].x;
                            const float g = fmaxf(fmaxf(mm.x - q, q - mm.y), 0.f);
                            lb = fmaf(g, g, lb);
                        }
                    } else {
#pragma unroll
                        for (int b = 9; b >= 0; --b)
                            if ((high >> b) & 1u) {
                                const float2 mm = box[(int64_t)b * n_steps + step];
                                const float q = -nxq[kLB + b].x;
                                const float g = fmaxf(fmaxf(mm.x - q, q - mm.y), 0.f);
                                lb = fmaf(g, g, lb);
                            }
                    }
                    ok = lb < ws.tcmax;
                }
                live = __ballot_sync(dev::kFull, ok);
                wbase = next_w;
                next_w += 32;
            }
            const int b = __ffs(live) - 1;
            live &= live - 1u;
            ++taken;
            return wbase + b;
        };
        StepRows cur;
        int u = take();
        if (u >= 0) load_step(x, (s0 + u) % n_steps, lane, cur);
        while (u >= 0) {
            const int step = (s0 + u) % n_steps;
            const int ja = step * 64 + (int)lane;
            const int jb = ja + 32;
            float2 d[15];
#pragma unroll
            for (int f = 0; f < 15; ++f) d[f] = __fadd2_rn(feat_pair(cur, f), nxq[f]);
            // original indices of the two candidates
            const int oa = __float_as_int(cur.r[7].z);
            const int ob = __float_as_int(cur.r[7].w);
            if ((i >> 6) == step) {
                // the query itself is in this step: make it infinitely far
#pragma unroll
                for (int f = 0; f < 15; ++f) {
                    if (ja == i) d[f].x = CUDART_INF_F;
                    if (jb == i) d[f].y = CUDART_INF_F;
                }
            }
            float2 v[kW];
            v[0] = root_fold<CMP>(d, high);
            // the next live step's rows load while this one is walked
            const int un = take();
            if (un >= 0) load_step(x, (s0 + un) % n_steps, lane, cur);
            // Every node of the tree is >= its root, the fold over the high features.
            // When no root of the step's 64 candidates is below the chunk's largest pass
            // threshold, no subspace can pass and the walk is skipped.
            const float tmax = ws.tcmax;
            if (!__all_sync(dev::kFull, (v[0].x >= tmax) & (v[0].y >= tmax))) {
                unsigned part[4] = {0u, 0u, 0u, 0u};
                walk<0>(v, d, reinterpret_cast<const float4 *>(ws.tcw), make_float4(0.f, 0.f, 0.f, 0.f), part);
                const unsigned bits = walk_bits(part);
                if (__any_sync(dev::kFull, bits != 0u)) {
                    tcount = append_hits<KMAX>(ws_off, bits, v[0], d[0], d[1], d[2], d[3], d[4], tcount, oa, ob,
                                               k);
                    // flushing once a batch is waiting keeps the kNN thresholds fresh
                    // without paying a flush per step
                    if (tcount >= kFlushMin) {
                        flush_tuples<KMAX>(ws_off, tcount, k);
                        tcount = 0;
                    }
                }
            }
            u = un;
        }
        if (tcount > 0) flush_tuples<KMAX>(ws_off, tcount, k);
        if (lane == 0) {
            ws.stat_loaded += (unsigned long long)(taken + init_steps);  // the set-up's loads included
            ws.stat_total += (unsigned long long)n_steps;
        }

        // ---- end of the work item: lane L reports subspace L ---------------------------
        {
            const uint32_t L = lane;
            if ((active >> L) & 1u) {
                const int slot = ch->slot[L];
                float *sc = o.scores + (int64_t)slot * 4 * n;
                const int cnt = ws.cnt[L];
                sc[orig_i] = (float)cnt;
                sc[n + orig_i] = dev::eps_mean(ws.esum[L], cnt, ws.escale[L]);
                if (o.eps_count) o.eps_count[(int64_t)slot * n + orig_i] = cnt;
                if (k > 0) {
                    // sort the list by (distance, index); the mean is summed in that order
                    float *ld = ws.ld[L];
                    int *lj = ws.lj[L];
                    for (int p = 1; p < k; ++p) {
                        const float v = ld[p];
                        const int j = lj[p];
                        int q = p;
                        while (q > 0 && (ld[q - 1] > v || (ld[q - 1] == v && lj[q - 1] > j))) {
                            ld[q] = ld[q - 1];
                            lj[q] = lj[q - 1];
                            --q;
                        }
                        ld[q] = v;
                        lj[q] = j;
                    }
                    float msum = 0.f;
                    for (int p = 0; p < k; ++p) {
                        const float dd = sqrtf(ws.ld[L][p]);
                        const int j = ws.lj[L][p];
                        msum += dd;
                        if (j >= 0 && j < n) atomicAdd(&sc[2 * n + j], 1.f);
                        if (o.knn_idx) o.knn_idx[((int64_t)slot * n + orig_i) * k + p] = j;
                        if (o.knn_dist) o.knn_dist[((int64_t)slot * n + orig_i) * k + p] = dd;
                    }
                    sc[3 * n + orig_i] = msum / (float)k;
                }
            }
            __syncwarp();
        }
    }
}

template <int KMAX, int CW, bool CMP>
snaps_status launch_tree(const JoinShape &s, const TreeChunk *chunks, int n_chunks,
                         const JoinOut &o, DeviceControl *ctrl, cudaStream_t st)
{
    const size_t smem = sizeof(TreeSmem<KMAX, CW>);
    auto kern = join_tree_kernel<KMAX, CW, CMP>;
    SNAPS_CHECK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int dev = 0, sms = 0, per_sm = 0;
    SNAPS_CHECK_CUDA(cudaGetDevice(&dev));
    SNAPS_CHECK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    SNAPS_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, CW * 32, smem));
    if (per_sm < 1) {
        set_error("subspace-batched join does not fit on an SM (smem %zu)", smem);
        return SNAPS_ECUDA;
    }
    const long long warps = s.n * (long long)n_chunks;
    const long long grid = std::min<long long>((warps + CW - 1) / CW, (long long)sms * per_sm);
    SNAPS_CHECK_CUDA(cudaMemsetAsync(&ctrl->next_work, 0, sizeof(unsigned long long), st));
    kern<<<(unsigned)grid, CW * 32, smem, st>>>(s, chunks, n_chunks, o, ctrl);
    SNAPS_CHECK_CUDA(cudaGetLastError());
    return SNAPS_OK;
}

}  // namespace

snaps_status launch_join_tree(const JoinShape &s, const TreeChunk *chunks, int n_chunks,
                              const JoinOut &o, DeviceControl *ctrl, cudaStream_t st)
{
    if (n_chunks <= 0) return SNAPS_OK;
    if (s.k <= 16)
        return s.compact ? launch_tree<16, 8, true>(s, chunks, n_chunks, o, ctrl, st)
                         : launch_tree<16, 8, false>(s, chunks, n_chunks, o, ctrl, st);
    return s.compact ? launch_tree<32, 6, true>(s, chunks, n_chunks, o, ctrl, st)
                     : launch_tree<32, 6, false>(s, chunks, n_chunks, o, ctrl, st);
}

}  // namespace snaps
