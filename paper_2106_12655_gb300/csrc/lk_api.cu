// Host runtime of the linking-number library: the C ABI of include/lk.h.
//
// A context keeps one CSR geometry resident on the device (FP64 vertices
// padded to 32 bytes, loop offsets, loop boxes).  A verify packs the pair list
// on the host into work items (tiles of one pair: 128 column segments by
// tile_rows row segments, ordered by decreasing cost), uploads the item
// tables, and enqueues on the caller's stream: pair frames -> persistent bulk
// sweep -> careful sweep of handed-over items -> FP64 recompute of near
// segment pairs -> fixed-order per-pair reduction (Algorithm 1's loop over P,
// each ComputeLink being the direct sum of Sec. 3.4.2).  A plan captures the
// same device sequence once in a CUDA graph.
#include <cuda_runtime.h>

#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <type_traits>
#include <numeric>
#include <string>
#include <vector>

#include "lk.h"
#include "lk_internal.h"

using lk::NearEntry;
using lk::PairTask;
using lk::Vtx;

namespace {

std::mutex g_err_mu;
std::string g_last_error = "";

void set_global_error(const std::string& m) {
    std::lock_guard<std::mutex> g(g_err_mu);
    g_last_error = m;
}

bool is_device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

template <class T>
struct DevBuf {
    T* p = nullptr;
    size_t cap = 0;  // elements
    bool fixed = false;  // bound to memory the buffer does not own (never freed or reallocated)
    cudaError_t ensure(size_t n) {
        if (n <= cap && p) return cudaSuccess;
        if (fixed) return cudaErrorInvalidValue;   // callers check fits() first
        if (p) cudaFree(p);
        p = nullptr;
        cap = 0;
        const size_t want = std::max<size_t>(n, 1);
        cudaError_t e = cudaMalloc(&p, want * sizeof(T));
        if (e == cudaSuccess) cap = want;
        return e;
    }
    bool fits(size_t n) const { return !fixed || (p && n <= cap); }
    void release() {
        if (p && !fixed) cudaFree(p);
        p = nullptr;
        cap = 0;
    }
    size_t bytes_for(size_t n) const { return std::max<size_t>(n, 1) * sizeof(T); }
};

// Work counters of a verify (see Workspace::counters).
constexpr size_t kCounters = 12;

// A counting-crossings pair searched with the binned candidate search.
struct GridJob {
    int32_t task, n_rows, n_cols, G_max;   // G_max: the largest grid the pair may take
};

// Pairs with at least this many segment pairs take the binned candidate
// search under LK_METHOD_CC (about the size at which its fixed launches cost
// less than sweeping every segment pair).
constexpr int64_t kCcGridMin = (int64_t)1 << 28;

struct Packed {
    std::vector<PairTask> tasks;
    std::vector<GridJob> grid;          // counting crossings: pairs for the binned search
    int64_t grid_cells = 0, grid_rows = 0, grid_cols = 0;   // their largest sizes
    int64_t n_cc_local = 0, n_cc_sweep = 0;   // counting crossings: one-CTA pairs, swept pairs
    int32_t local_rows = 0, local_cols = 0;   // the one-CTA pairs' largest loops
    std::vector<int64_t> item_begin;
    std::vector<int32_t> item_task;
    int64_t n_items = 0;
    int64_t n_acc_items = 0;   // items [0, n_acc_items) belong to accurate-variant pairs
    int64_t n_acc_tasks = 0;   // and tasks [0, n_acc_tasks)
    int64_t n_chunks = 0;      // 32-row chunks over all items
    int64_t n_chunk_bits = 0;  // chunk bits of the accurate-variant items (PairTask::bit_base)
    int64_t segment_pairs = 0;
    int tile_rows_max = 0;
    int tile_cols = 0;
};

// Device working memory of one verify (grow-only, reused across calls).
struct Workspace {
    DevBuf<PairTask> tasks;
    DevBuf<int64_t> item_begin;
    DevBuf<int32_t> item_task;
    DevBuf<double> partial;
    DevBuf<int64_t> careful_items;
    DevBuf<lk::CarefulChunk> careful_chunks;
    DevBuf<unsigned long long> item_fix;
    DevBuf<NearEntry> near_list;
    DevBuf<unsigned long long> fix_acc;
    DevBuf<unsigned long long> fp64_count;
    DevBuf<int> flags;
    DevBuf<unsigned long long> counters;  // [0] accurate-sweep counter, [1] overflow,
                                          // [2] u32 careful_count, careful_counter,
                                          // [3] u32 near_count, unused, [4] fast-sweep / f64 counter,
                                          // [5], [6] chunk pass, [7] precise sweep, [8] crossing sweep
                                          // counter, [9] u32 crossing candidates, [10] precise careful pass
    DevBuf<NearEntry> cc_list;            // counting crossings: candidates (method CC only)
    DevBuf<int> cc_half;
    DevBuf<unsigned int> flag_scan, flag_sums;   // counting crossings: items of the undecided pairs
    DevBuf<unsigned int> grid_offsets, grid_cursor, grid_sums;   // binned search (largest grid pair)
    DevBuf<int32_t> grid_entries;
    DevBuf<float2> grid_row_xy, grid_col_xy;
    DevBuf<unsigned long long> grid_meta;   // [0] entries total, [1] low half: the chosen grid size
    DevBuf<int32_t> lk;
    DevBuf<double> raw;
    DevBuf<int32_t> status;
    DevBuf<float4> item_err;              // bulk-sweep error statistics per item
    DevBuf<unsigned int> chunk_bits;      // chunks the careful pass sums (accurate variant)
    DevBuf<unsigned int> precise_scan, precise_sums;   // items of the kFlagPrecise pairs
    DevBuf<double> err;                   // per-pair error estimates, by output position
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;  // around the bulk sweep (options.timing)

    cudaError_t events() {
        cudaError_t e = cudaSuccess;
        if (!ev0) e = cudaEventCreate(&ev0);
        if (e == cudaSuccess && !ev1) e = cudaEventCreate(&ev1);
        return e;
    }

    void release() {
        if (ev0) cudaEventDestroy(ev0);
        if (ev1) cudaEventDestroy(ev1);
        ev0 = ev1 = nullptr;
        tasks.release(); item_begin.release(); item_task.release(); partial.release();
        careful_items.release(); careful_chunks.release(); item_fix.release(); near_list.release(); fix_acc.release(); fp64_count.release();
        flags.release(); counters.release(); lk.release(); raw.release(); status.release();
        cc_list.release(); cc_half.release(); flag_scan.release(); flag_sums.release();
        grid_offsets.release(); grid_cursor.release(); grid_sums.release(); grid_entries.release();
        grid_row_xy.release(); grid_col_xy.release(); grid_meta.release();
        item_err.release(); chunk_bits.release(); precise_scan.release(); precise_sums.release(); err.release();
    }
};

}  // namespace

// A repeated certificate check (lk_verify_expected with the same pair list
// and batch size as the previous call): its batches packed once, their item
// tables resident, and the whole batched sequence captured in a CUDA graph.
struct ExpectedPlan {
    std::vector<int32_t> pairs;
    int64_t batch = 0;
    std::vector<int64_t> bounds;
    std::vector<Packed> batches;
    Workspace ws;                                   // shared work buffers, sized for the largest batch
    std::vector<DevBuf<PairTask>> tasks;            // per batch
    std::vector<DevBuf<int64_t>> item_begin;
    std::vector<DevBuf<int32_t>> item_task;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t capture = nullptr;

    void release() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (capture) cudaStreamDestroy(capture);
        exec = nullptr;
        graph = nullptr;
        capture = nullptr;
        ws.release();
        for (auto& b : tasks) b.release();
        for (auto& b : item_begin) b.release();
        for (auto& b : item_task) b.release();
    }
};

struct lk_ctx {
    int device = 0;
    int num_sms = 1;
    lk_options opt;
    int64_t n_vertices = 0;
    int64_t n_loops = 0;
    std::vector<int64_t> h_offsets;
    Vtx* d_V = nullptr;
    float4* d_R = nullptr;    // FP32 loop-relative copy of d_V (the mixed path reads it)
    int64_t* d_offsets = nullptr;
    double* d_aabb = nullptr;
    unsigned long long* d_box_keys = nullptr;   // two sets of [6][n_loops] keys of the box passes
    int box_set = 0;                            // the set in the reset state
    void* d_stage = nullptr;  // staging for host-side lk_update data
    size_t stage_bytes = 0;
    Workspace ws;
    lk_stats stats{};
    int64_t stats_tasks = 0;        // tasks of the last verify (for lazy FP64 counts)
    bool stats_pending = false;
    const unsigned long long* stats_fp64 = nullptr;
    const unsigned long long* stats_overflow = nullptr;
    const unsigned int* stats_careful = nullptr;
    const int* stats_flags = nullptr;            // per-pair flags of the last verify (CC fallbacks)
    const double* last_err = nullptr;            // the last verify's per-pair error estimates
    int64_t last_n = 0;
    bool stats_cc = false;
    cudaEvent_t stats_ev0 = nullptr, stats_ev1 = nullptr;
    cudaStream_t stats_stream = nullptr;
    std::map<uint32_t, int> tune;   // size class -> tile rows chosen by lk_autotune
    // Repeated pair lists: lk_verify keeps the last list it packed and, when
    // the same list comes again, a graph plan of it (the packing depends only
    // on the list, the loop sizes and the tune table, none of which lk_update
    // changes); the kernels still run in full on the current geometry.
    std::vector<int32_t> last_pairs;
    lk_plan* repeat_plan = nullptr;
    // Potential link search buffers (allocated on first use).
    long long* d_pls_keys = nullptr;     // [6][n_loops]
    int32_t* d_pls_counts = nullptr;     // [n_loops]
    int64_t* d_pls_offsets = nullptr;    // [n_loops + 1] exclusive scan of the counts (total last)
    long long* d_pls_scan = nullptr;     // the scan's block totals
    int64_t* h_pls_total = nullptr;      // pinned: the candidate count
    int32_t* d_pls_pairs = nullptr;      // staging for host destinations
    int64_t pls_pairs_cap = 0;
    unsigned long long* d_pls_order = nullptr;   // [pls_sort_size(n_loops)] sorted (x key, loop)
    DevBuf<unsigned long long> pls_pair_keys;    // the pairs as (i << 32 | j), padded for the sort
    // List growth: after each lk_verify its work counters are copied to pinned
    // host memory on the stream; a later lk_verify reads them once the copy has
    // landed (without waiting for it) and enlarges any list that overflowed.
    // Early exit (lk_verify_expected): the certificate, the stop word and the
    // results of every batch, on the device.
    DevBuf<int32_t> ee_expected, ee_lk, ee_status;
    DevBuf<double> ee_raw;
    DevBuf<long long> ee_stop;
    std::vector<int32_t> ee_last_pairs;         // the previous check's list and batch size
    int64_t ee_last_batch = 0;
    ExpectedPlan* ee_plan = nullptr;            // built on the first repeat
    unsigned long long* h_counters = nullptr;   // [10], pinned
    cudaEvent_t counters_ev = nullptr;
    bool counters_pending = false;
    int64_t counters_item_chunks = 0;           // that verify's chunks per work item (at most)
    int64_t counters_chunks = 0;                // and its chunks in all
    std::string err;
};

struct lk_plan {
    lk_ctx* ctx = nullptr;
    Packed pk;
    Workspace ws;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t capture = nullptr;
};

// Forget lk_verify's repeated-list state (the tune table changed, another
// list came, or the context goes away).
static void drop_repeat_plan(lk_ctx* ctx) {
    if (ctx->repeat_plan) lk_plan_destroy(ctx->repeat_plan);
    ctx->repeat_plan = nullptr;
    ctx->last_pairs.clear();
}

// Upper bound of automatic list growth: a list grows to at most a quarter of
// the device memory free at that moment (and 2^31 - 1 entries).
static int64_t grow_limit(size_t entry_bytes) {
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
        cudaGetLastError();
        return (int64_t)1 << 20;
    }
    return std::max<int64_t>(1, std::min<int64_t>(INT32_MAX, (int64_t)(free_b / 4 / entry_bytes)));
}

// Enlarge the recompute, chunk and candidate lists to what the previous
// lk_verify on this context asked for (the next power of two above it, within
// the bounds above).  An overflow never changes a result -- the overflowing
// entries are evaluated in place, handed over whole or decided by the direct
// sum -- but each of those is slower than the list it replaces.  A context
// with a memory budget keeps its configured sizes.
static void grow_lists(lk_ctx* ctx) {
    if (!ctx->counters_pending) return;
    const cudaError_t q = cudaEventQuery(ctx->counters_ev);
    if (q == cudaErrorNotReady) {
        cudaGetLastError();        // not an error: the copy has not landed yet
        return;
    }
    ctx->counters_pending = false;
    if (q != cudaSuccess || ctx->opt.mem_budget > 0) return;
    const unsigned long long* h = ctx->h_counters;
    const unsigned long long need_near = h[3] & 0xffffffffull;     // near_count: low half of counters[3]
    // chunk_count (low half of counters[5]) misses the chunks an item did not
    // reach after its hand-over failed; each item handed over whole (careful
    // count, low half of counters[2]) may have had all of its chunks to hand
    const unsigned long long whole = h[2] & 0xffffffffull;
    const unsigned long long need_chunk =
        std::min<unsigned long long>((h[5] & 0xffffffffull) + whole * (unsigned long long)ctx->counters_item_chunks,
                                     (unsigned long long)std::max<int64_t>(ctx->counters_chunks, 1));
    const unsigned long long need_cc = h[9];                       // crossing candidates
    auto grown = [](int cur, unsigned long long need, size_t entry_bytes) {
        if (need <= (unsigned long long)cur) return cur;
        const int64_t limit = grow_limit(entry_bytes);
        int64_t n = 1;
        while ((unsigned long long)n < need && n < limit) n <<= 1;
        return (int)std::max<int64_t>(cur, std::min<int64_t>(n, limit));
    };
    const int near = grown(ctx->opt.near_capacity, need_near, sizeof(NearEntry));
    const int chunk = grown(ctx->opt.chunk_capacity, need_chunk, sizeof(lk::CarefulChunk));
    const int cc = ctx->opt.method == LK_METHOD_CC ? grown(ctx->opt.cc_capacity, need_cc, sizeof(NearEntry))
                                                   : ctx->opt.cc_capacity;
    if (near == ctx->opt.near_capacity && chunk == ctx->opt.chunk_capacity && cc == ctx->opt.cc_capacity) return;
    ctx->opt.near_capacity = near;
    ctx->opt.chunk_capacity = chunk;
    ctx->opt.cc_capacity = cc;
    drop_repeat_plan(ctx);         // its work buffers have the old sizes
}

// Queue the copy of a verify's work counters for grow_lists.  While the
// previous copy is still in flight this verify's counters are not copied (the
// host never waits here); a copy that landed unread is replaced by this one.
static void note_counters(lk_ctx* ctx, const unsigned long long* d_counters, int64_t item_chunks,
                          int64_t chunks, cudaStream_t s) {
    if (!ctx->h_counters || !ctx->counters_ev) return;
    if (ctx->counters_pending && cudaEventQuery(ctx->counters_ev) == cudaErrorNotReady) {
        cudaGetLastError();
        return;
    }
    ctx->counters_pending = false;
    ctx->counters_item_chunks = item_chunks;
    ctx->counters_chunks = chunks;
    if (cudaMemcpyAsync(ctx->h_counters, d_counters, 10 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s) ==
            cudaSuccess &&
        cudaEventRecord(ctx->counters_ev, s) == cudaSuccess)
        ctx->counters_pending = true;
    else
        cudaGetLastError();
}

namespace {

lk_status fail(lk_ctx* ctx, lk_status st, const std::string& msg) {
    if (ctx) ctx->err = msg;
    set_global_error(msg);
    return st;
}

lk_status cuda_fail(lk_ctx* ctx, cudaError_t e, const char* where) {
    const lk_status st = (e == cudaErrorMemoryAllocation) ? LK_ERR_OOM : LK_ERR_CUDA;
    return fail(ctx, st, std::string(where) + ": " + cudaGetErrorString(e));
}

#define LK_CUDA(ctx, call)                                  \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
    } while (0)

// Size class of a pair for tuning: ceil(log2) of its row and column loop sizes.
// ceil(log2 v) for v >= 1
inline uint32_t ceil_log2(int64_t v) { return v <= 1 ? 0u : (uint32_t)(64 - __builtin_clzll((uint64_t)(v - 1))); }

uint32_t size_class(int64_t n_rows, int64_t n_cols) { return (ceil_log2(n_rows) << 8) | ceil_log2(n_cols); }

// Tile widths and the chunk height are powers of two: the packer's ceilings
// by them are shifts (a list of thousands of pairs is packed per request).
static_assert((lk::kTileCols & (lk::kTileCols - 1)) == 0 && (lk::kF64TileCols & (lk::kF64TileCols - 1)) == 0 &&
                  (lk::kChunkRows & (lk::kChunkRows - 1)) == 0,
              "tile widths and the chunk height must be powers of two");
inline int64_t ceil_shift(int64_t v, int shift) { return (v + ((int64_t)1 << shift) - 1) >> shift; }
inline int64_t ceil_div(int64_t a, int64_t b) { return b >= a ? (a > 0 ? 1 : 0) : (a + b - 1) / b; }

int default_tile_rows(int64_t n_rows, int64_t n_cols, int tc_shift, int user_rows) {
    if (user_rows > 0) return user_rows;
    const int64_t col_tiles = ceil_shift(n_cols, tc_shift);
    int64_t row_tiles = ceil_shift(n_rows, 8);
    const int64_t max_items_per_pair = 1 << 16;
    if (col_tiles * row_tiles > max_items_per_pair)
        row_tiles = std::max<int64_t>(1, max_items_per_pair / col_tiles);
    int64_t rows = ceil_div(n_rows, row_tiles);
    rows = ceil_shift(rows, 5) << 5;                                    // a multiple of kChunkRows
    static_assert(lk::kChunkRows == 32, "the shift above is by log2 kChunkRows");
    return (int)std::min<int64_t>(rows, INT32_MAX);
}

// Work items of a pair list.  Loop a of a pair plays gamma_1 of Eq. 4 and loop
// b gamma_2; the term is symmetric under exchanging them (Eq. 1), so either
// can be the row loop (iterated) and the other the column loop (spread over
// lanes in tiles of tile_cols): the one whose column tiles waste fewer lanes,
// else the longer one.  The tiling of a pair depends on its two sizes only,
// so a pair's result does not depend on the rest of the batch.
lk_status pack_pairs(lk_ctx* ctx, const int32_t* pairs, int64_t n, Packed& pk) {
    const bool f64 = ctx->opt.precision == LK_ALL_F64;
    const int tile_cols = f64 ? lk::kF64TileCols : lk::kTileCols;
    const int tc_shift = ceil_log2(tile_cols);
    pk.tile_cols = tile_cols;
    pk.tile_rows_max = 0;
    pk.segment_pairs = 0;
    pk.grid.clear();
    pk.grid_cells = pk.grid_rows = pk.grid_cols = 0;
    pk.n_cc_local = pk.n_cc_sweep = 0;
    pk.local_rows = pk.local_cols = 0;
    // Per pair: its shape, work items and sort key.  Accurate-variant pairs go
    // first (they run in their own launch), then within each variant the
    // largest items first, so that the persistent grid's tail is made of small
    // ones; ties keep the input order.  key = (variant, clamped item cost),
    // sorted ascending by a stable LSD radix sort.
    struct Shape {
        int32_t row_loop, col_loop, n_rows, n_cols, tile_rows, col_tiles, status, accurate;
        int64_t items;
    };
    // scratch kept per thread across calls (a server packs a list per
    // request; fresh vectors would be allocated and faulted in each time)
    thread_local std::vector<Shape> sh;
    thread_local std::vector<uint32_t> key;
    thread_local std::vector<uint64_t> kv, tmp;
    // ... but not after a list of millions of pairs (68 B a pair)
    struct Release {
        int64_t n;
        ~Release() {
            if (n <= ((int64_t)1 << 20)) return;
            std::vector<Shape>().swap(sh);
            std::vector<uint32_t>().swap(key);
            std::vector<uint64_t>().swap(kv);
            std::vector<uint64_t>().swap(tmp);
        }
    } release{n};
    sh.resize((size_t)n);
    key.resize((size_t)n);
    const bool tuned = !f64 && ctx->opt.tile_rows <= 0 && !ctx->tune.empty();
    for (int64_t p = 0; p < n; ++p) {
        Shape& t = sh[(size_t)p];
        const int32_t a = pairs[2 * p], b = pairs[2 * p + 1];
        if (a < 0 || b < 0 || a >= ctx->n_loops || b >= ctx->n_loops || a == b) {
            t = Shape{0, 0, 0, 0, 0, 0, LK_ERR_ARG, 0, 0};
            key[(size_t)p] = 0xffffffffu;                       // invalid pairs last (no items)
            continue;
        }
        const int64_t na = ctx->h_offsets[a + 1] - ctx->h_offsets[a];
        const int64_t nb = ctx->h_offsets[b + 1] - ctx->h_offsets[b];
        // The orientation that sweeps fewer cells including the padding of the
        // last column tile; on a tie the longer loop is the row loop.
        const int64_t cells_a_rows = na * ceil_shift(nb, tc_shift);
        const int64_t cells_b_rows = nb * ceil_shift(na, tc_shift);
        const bool a_rows = cells_a_rows != cells_b_rows ? cells_a_rows < cells_b_rows : na >= nb;
        t.row_loop = a_rows ? a : b;
        t.col_loop = a_rows ? b : a;
        t.n_rows = (int32_t)(a_rows ? na : nb);
        t.n_cols = (int32_t)(a_rows ? nb : na);
        int rows = ctx->opt.tile_rows;
        if (tuned) {
            auto it = ctx->tune.find(size_class(t.n_rows, t.n_cols));
            if (it != ctx->tune.end()) rows = it->second;
        }
        t.tile_rows = default_tile_rows(t.n_rows, t.n_cols, tc_shift, rows);
        t.col_tiles = (int32_t)ceil_shift(t.n_cols, tc_shift);
        t.items = (int64_t)t.col_tiles * ceil_div(t.n_rows, t.tile_rows);
        t.status = LK_OK;
        t.accurate = (int64_t)t.n_rows * t.n_cols >= ctx->opt.accurate_threshold ? 1 : 0;
        const int64_t cost = (int64_t)std::min(t.tile_rows, t.n_rows) * std::min(tile_cols, t.n_cols);
        const uint32_t c = (uint32_t)std::min<int64_t>(cost, 0x7ffffffe);
        key[(size_t)p] = (t.accurate ? 0u : 0x80000000u) | (0x7ffffffeu - c);
        pk.segment_pairs += (int64_t)t.n_rows * t.n_cols;
        pk.tile_rows_max = std::max(pk.tile_rows_max, t.tile_rows);
    }
    // (key << 32 | index) values, sorted by the key bytes that vary (LSD,
    // stable: equal keys keep the input order), read and written in sequence
    kv.resize((size_t)n);
    tmp.resize((size_t)n);
    uint32_t varying = 0;
    const uint32_t key0 = n > 0 ? key[0] : 0u;
    for (int64_t p = 0; p < n; ++p) {
        kv[(size_t)p] = ((uint64_t)key[(size_t)p] << 32) | (uint64_t)p;
        varying |= key[(size_t)p] ^ key0;
    }
    for (int shift = 0; shift < 32; shift += 8) {
        if (((varying >> shift) & 0xffu) == 0) continue;                 // one digit value
        size_t cnt[257] = {};
        for (int64_t k = 0; k < n; ++k) ++cnt[((kv[(size_t)k] >> (32 + shift)) & 0xffu) + 1];
        for (int d = 0; d < 256; ++d) cnt[d + 1] += cnt[d];
        for (int64_t k = 0; k < n; ++k) tmp[cnt[(kv[(size_t)k] >> (32 + shift)) & 0xffu]++] = kv[(size_t)k];
        kv.swap(tmp);
    }
    pk.tasks.resize((size_t)n);
    pk.item_begin.assign((size_t)n + 1, 0);
    pk.n_acc_items = 0;
    pk.n_acc_tasks = 0;
    pk.n_chunks = 0;
    pk.n_chunk_bits = 0;
    for (int64_t k = 0; k < n; ++k) {
        const int64_t p = (int64_t)(kv[(size_t)k] & 0xffffffffu);
        const Shape& q = sh[(size_t)p];
        PairTask t{};
        t.out_index = (int32_t)p;
        t.status = q.status;
        t.scale = 1.0f;
        if (q.status == LK_OK) {
            t.V = ctx->d_V;
            t.R = ctx->d_R;
            t.row_loop = q.row_loop;
            t.col_loop = q.col_loop;
            t.row_base = ctx->h_offsets[q.row_loop];
            t.col_base = ctx->h_offsets[q.col_loop];
            t.n_rows = q.n_rows;
            t.n_cols = q.n_cols;
            t.tile_rows = q.tile_rows;
            t.col_tiles = q.col_tiles;
            t.accurate = q.accurate;
            if (q.accurate) {
                // one bit per chunk slot of each item (the precise sweep skips the
                // chunks the bulk sweep handed to the careful pass)
                t.bit_base = pk.n_chunk_bits;
                pk.n_chunk_bits += q.items * ceil_shift(q.tile_rows, 5);
            }
            const bool cc = ctx->opt.method == LK_METHOD_CC;
            const int search = ctx->opt.cc_search;
            const bool fits = q.n_rows <= lk::kCcLocalMax && q.n_cols <= lk::kCcLocalMax;
            if (cc && search != LK_CC_SEARCH_SWEEP && fits) {
                t.cc_grid = 2;
                ++pk.n_cc_local;
                pk.local_rows = std::max(pk.local_rows, q.n_rows);
                pk.local_cols = std::max(pk.local_cols, q.n_cols);
            } else if (cc && (search == LK_CC_SEARCH_BINNED ||
                              (search == LK_CC_SEARCH_AUTO && (int64_t)q.n_rows * q.n_cols >= kCcGridMin))) {
                // at most about 2 sqrt(N) cells per side; the device takes fewer
                // where the segments are long (cells about 1.5 segment lengths)
                const int64_t want = 2 * (int64_t)std::ceil(std::sqrt((double)std::max(q.n_rows, q.n_cols)));
                int G = 64;
                while (G < want && G < 4096) G <<= 1;
                t.cc_grid = 1;
                pk.grid.push_back(GridJob{(int32_t)k, q.n_rows, q.n_cols, G});
                pk.grid_cells = std::max<int64_t>(pk.grid_cells, (int64_t)G * G);
                pk.grid_rows = std::max<int64_t>(pk.grid_rows, q.n_rows);
                pk.grid_cols = std::max<int64_t>(pk.grid_cols, q.n_cols);
            } else if (cc) {
                ++pk.n_cc_sweep;
            }
            const int64_t full = q.tile_rows >= q.n_rows ? (q.tile_rows == q.n_rows ? 1 : 0) : q.n_rows / q.tile_rows;
            const int64_t last = q.n_rows - full * q.tile_rows;
            const int64_t chunks_per_col = full * ceil_shift(q.tile_rows, 5) + (last > 0 ? ceil_shift(last, 5) : 0);
            pk.n_chunks += chunks_per_col * q.col_tiles;
        }
        pk.tasks[(size_t)k] = t;
        pk.item_begin[(size_t)k + 1] = pk.item_begin[(size_t)k] + q.items;
        if (q.accurate) {
            pk.n_acc_items = pk.item_begin[(size_t)k + 1];
            pk.n_acc_tasks = k + 1;
        }
    }
    pk.n_items = pk.item_begin[(size_t)n];
    if (pk.n_items > (int64_t)INT32_MAX * 16)
        return fail(ctx, LK_ERR_ARG, "lk_verify: too many work items");
    pk.item_task.resize((size_t)pk.n_items);
    for (int64_t k = 0; k < n; ++k)
        std::fill(pk.item_task.begin() + pk.item_begin[(size_t)k],
                  pk.item_task.begin() + pk.item_begin[(size_t)k + 1], (int32_t)k);
    return LK_OK;
}

size_t chunk_capacity(const lk_options& o, int64_t n_chunks);

// Row-segment entries of the binned search: with cells about 1.5 mean segment
// lengths wide a row segment covers about two cells; a pair whose entries do
// not fit goes to the direct sum.
int64_t grid_entry_capacity(const Packed* pk) {
    return pk && !pk->grid.empty() ? std::max<int64_t>(8 * pk->grid_rows, (int64_t)1 << 20) : 0;
}

size_t grid_bytes(const Packed* pk) {
    if (!pk || pk->grid.empty()) return 0;
    return (size_t)(2 * pk->grid_cells + 1 + pk->grid_cells / 4096 + 2) * sizeof(unsigned int) +
           (size_t)grid_entry_capacity(pk) * sizeof(int32_t) + (size_t)(pk->grid_rows + pk->grid_cols) * sizeof(float2) +
           2 * sizeof(unsigned long long);
}

size_t workspace_bytes(const lk_ctx* ctx, int64_t n_tasks, int64_t n_items, int64_t n_chunks, const Packed* pk) {
    const size_t near = (size_t)std::max(0, ctx->opt.near_capacity);
    const size_t cc = ctx->opt.method == LK_METHOD_CC ? (size_t)std::max(1, ctx->opt.cc_capacity) : 0;
    const size_t stats = ctx->opt.precision != LK_ALL_F64 ? 1 : 0;
    const size_t bits = pk ? (size_t)(pk->n_chunk_bits + 31) / 32 * 4 : 0;
    return n_tasks * (sizeof(PairTask) + 8 + 8 + 8 + 4 + 4 + 8 + 4 + (cc ? 4 + 4 : 0) + stats * (4 + 8)) +
           n_items * (4 + 8 + 8 + 8 + stats * sizeof(float4)) + bits +
           chunk_capacity(ctx->opt, n_chunks) * sizeof(lk::CarefulChunk) +
           (near + cc) * sizeof(NearEntry) + grid_bytes(pk) + 80;
}

// Entries of the chunk hand-over list: every chunk of the batch, at most the
// configured capacity (an overflow hands whole items over instead).
size_t chunk_capacity(const lk_options& o, int64_t n_chunks) {
    const int64_t cap = o.chunk_capacity > 0 ? o.chunk_capacity : (int64_t)1 << 20;
    return (size_t)std::max<int64_t>(1, std::min<int64_t>(n_chunks, cap));
}

lk_status ensure_workspace(lk_ctx* ctx, Workspace& ws, int64_t n_tasks, int64_t n_items, int64_t n_chunks,
                           const Packed* pk = nullptr) {
    if (ctx->opt.mem_budget > 0 && workspace_bytes(ctx, n_tasks, n_items, n_chunks, pk) > ctx->opt.mem_budget)
        return fail(ctx, LK_ERR_OOM, "lk_verify: work buffers exceed mem_budget");
    const size_t nt = (size_t)std::max<int64_t>(n_tasks, 1), ni = (size_t)std::max<int64_t>(n_items, 1);
    // Buffers bound to fixed memory (the allocation-free entry point) are never
    // reallocated: a need beyond one of them is an argument error.
    const size_t bit_words = pk ? (size_t)std::max<int64_t>((pk->n_chunk_bits + 31) / 32, 1) : 1;
    const bool stats = ctx->opt.precision != LK_ALL_F64;
    if (!ws.tasks.fits(nt) || !ws.item_begin.fits(nt + 1) || !ws.item_task.fits(ni) || !ws.partial.fits(ni) ||
        !ws.careful_items.fits(ni) || !ws.careful_chunks.fits(chunk_capacity(ctx->opt, n_chunks)) ||
        !ws.item_fix.fits(ni) || !ws.near_list.fits((size_t)std::max(1, ctx->opt.near_capacity)) ||
        !ws.fix_acc.fits(nt) || !ws.fp64_count.fits(nt) || !ws.flags.fits(nt) || !ws.lk.fits(nt) ||
        !ws.counters.fits(kCounters) ||
        !ws.raw.fits(nt) || !ws.status.fits(nt) ||
        (stats && (!ws.item_err.fits(ni) || !ws.chunk_bits.fits(bit_words) || !ws.precise_scan.fits(nt + 1) ||
                   !ws.precise_sums.fits(nt / 4096 + 2) || !ws.err.fits(nt))))
        return fail(ctx, LK_ERR_ARG, "lk_verify: work beyond the fixed buffers' limits");
    LK_CUDA(ctx, ws.tasks.ensure(nt));
    LK_CUDA(ctx, ws.item_begin.ensure(nt + 1));
    LK_CUDA(ctx, ws.item_task.ensure(ni));
    LK_CUDA(ctx, ws.partial.ensure(ni));
    LK_CUDA(ctx, ws.careful_items.ensure(ni));
    LK_CUDA(ctx, ws.careful_chunks.ensure(chunk_capacity(ctx->opt, n_chunks)));
    LK_CUDA(ctx, ws.item_fix.ensure(ni));
    LK_CUDA(ctx, ws.near_list.ensure((size_t)std::max(1, ctx->opt.near_capacity)));
    LK_CUDA(ctx, ws.fix_acc.ensure(nt));
    LK_CUDA(ctx, ws.fp64_count.ensure(nt));
    LK_CUDA(ctx, ws.flags.ensure(nt));
    LK_CUDA(ctx, ws.counters.ensure(kCounters));
    if (ctx->opt.method == LK_METHOD_CC) {
        LK_CUDA(ctx, ws.cc_list.ensure((size_t)std::max(1, ctx->opt.cc_capacity)));
        LK_CUDA(ctx, ws.cc_half.ensure(nt));
        LK_CUDA(ctx, ws.flag_scan.ensure(nt + 1));
        LK_CUDA(ctx, ws.flag_sums.ensure(nt / 4096 + 2));
        if (pk && !pk->grid.empty()) {
            LK_CUDA(ctx, ws.grid_offsets.ensure((size_t)pk->grid_cells + 1));
            LK_CUDA(ctx, ws.grid_cursor.ensure((size_t)pk->grid_cells));
            LK_CUDA(ctx, ws.grid_sums.ensure((size_t)(pk->grid_cells / 4096 + 2)));
            LK_CUDA(ctx, ws.grid_entries.ensure((size_t)grid_entry_capacity(pk)));
            LK_CUDA(ctx, ws.grid_row_xy.ensure((size_t)pk->grid_rows));
            LK_CUDA(ctx, ws.grid_col_xy.ensure((size_t)pk->grid_cols));
            LK_CUDA(ctx, ws.grid_meta.ensure(2));
        }
    }
    LK_CUDA(ctx, ws.lk.ensure(nt));
    LK_CUDA(ctx, ws.raw.ensure(nt));
    LK_CUDA(ctx, ws.status.ensure(nt));
    if (stats) {
        LK_CUDA(ctx, ws.item_err.ensure(ni));
        LK_CUDA(ctx, ws.chunk_bits.ensure(bit_words));
        LK_CUDA(ctx, ws.precise_scan.ensure(nt + 1));
        LK_CUDA(ctx, ws.precise_sums.ensure(nt / 4096 + 2));
        LK_CUDA(ctx, ws.err.ensure(nt));
    }
    if (ctx->opt.timing) LK_CUDA(ctx, ws.events());
    return LK_OK;
}

lk_status upload_packed(lk_ctx* ctx, Workspace& ws, const Packed& pk, cudaStream_t s) {
    const int64_t n = (int64_t)pk.tasks.size();
    if (n > 0)
        LK_CUDA(ctx, cudaMemcpyAsync(ws.tasks.p, pk.tasks.data(), n * sizeof(PairTask),
                                     cudaMemcpyHostToDevice, s));
    LK_CUDA(ctx, cudaMemcpyAsync(ws.item_begin.p, pk.item_begin.data(), (n + 1) * sizeof(int64_t),
                                 cudaMemcpyHostToDevice, s));
    if (pk.n_items > 0)
        LK_CUDA(ctx, cudaMemcpyAsync(ws.item_task.p, pk.item_task.data(),
                                     pk.n_items * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    return LK_OK;
}

lk::SweepArgs sweep_args(const lk_ctx* ctx, Workspace& ws, const Packed& pk) {
    lk::SweepArgs a{};
    a.tasks = ws.tasks.p;
    a.item_begin = ws.item_begin.p;
    a.item_task = ws.item_task.p;
    a.n_items = pk.n_items;
    a.partial = ws.partial.p;
    a.item_counter = ws.counters.p + 4;
    a.overflow = ws.counters.p + 1;
    unsigned int* u32 = reinterpret_cast<unsigned int*>(ws.counters.p + 2);
    a.careful_count = u32 + 0;
    a.careful_counter = u32 + 1;
    a.near_count = u32 + 2;   // low half of counters[3]
    a.n_tasks = (int64_t)pk.tasks.size();
    a.careful_items = ws.careful_items.p;
    a.careful_chunks = ws.careful_chunks.p;
    a.chunk_capacity = (int)std::min<size_t>(ws.careful_chunks.cap, (size_t)INT32_MAX);
    a.chunk_count = u32 + 6;     // low half of counters[5]
    a.chunk_counter = u32 + 7;   // high half of counters[5], low half of counters[6]
    a.item_fix = ws.item_fix.p;
    a.near_list = ws.near_list.p;
    a.near_capacity = std::max(1, ctx->opt.near_capacity);
    a.fix_acc = ws.fix_acc.p;
    a.fp64_count = ws.fp64_count.p;
    a.flags = ws.flags.p;
    a.near_ratio_sq = (float)(ctx->opt.near_ratio * ctx->opt.near_ratio);
    if (ctx->opt.method == LK_METHOD_CC) {
        a.cc_list = ws.cc_list.p;
        a.cc_count = ws.counters.p + 9;
        a.cc_capacity = (int)std::min<size_t>(ws.cc_list.cap, (size_t)INT32_MAX);
        a.cc_half = ws.cc_half.p;
        a.flag_scan = ws.flag_scan.p;
    }
    if (ctx->opt.precision != LK_ALL_F64) {
        a.item_err = ws.item_err.p;
        a.chunk_bits = pk.n_chunk_bits > 0 ? ws.chunk_bits.p : nullptr;
        a.precise_scan = ws.precise_scan.p;
    }
    return a;
}

// Record a timing event; inside stream capture it must become an external
// event-record node of the graph.
cudaError_t record_event(cudaEvent_t ev, cudaStream_t s) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(s, &cs);
    if (e != cudaSuccess) return e;
    return cs == cudaStreamCaptureStatusActive ? cudaEventRecordWithFlags(ev, s, cudaEventRecordExternal)
                                                : cudaEventRecord(ev, s);
}

// The device sequence of one verify (graph-capturable: no host sync).  With
// `stop` set (early exit), every kernel first reads *stop and does nothing
// when it is below stop_base.
lk_status enqueue_verify(lk_ctx* ctx, Workspace& ws, const Packed& pk, cudaStream_t s,
                         const long long* stop = nullptr, long long stop_base = 0) {
    const int64_t n = (int64_t)pk.tasks.size();
    if (n == 0) return LK_OK;
    LK_CUDA(ctx, cudaMemsetAsync(ws.counters.p, 0, kCounters * sizeof(unsigned long long), s));
    LK_CUDA(ctx, cudaMemsetAsync(ws.fix_acc.p, 0, n * sizeof(unsigned long long), s));
    const bool cc = ctx->opt.method == LK_METHOD_CC;
    if (cc) LK_CUDA(ctx, cudaMemsetAsync(ws.cc_half.p, 0, n * sizeof(int), s));
    LK_CUDA(ctx, cudaMemsetAsync(ws.fp64_count.p, 0, n * sizeof(unsigned long long), s));
    LK_CUDA(ctx, cudaMemsetAsync(ws.flags.p, 0, n * sizeof(int), s));
    if (pk.n_items > 0)
        LK_CUDA(ctx, cudaMemsetAsync(ws.item_fix.p, 0, pk.n_items * sizeof(unsigned long long), s));
    const bool mixed = ctx->opt.precision != LK_ALL_F64;
    if (mixed && pk.n_chunk_bits > 0)
        LK_CUDA(ctx, cudaMemsetAsync(ws.chunk_bits.p, 0, (size_t)(pk.n_chunk_bits + 31) / 32 * sizeof(unsigned int), s));
    lk::launch_pair_frames(ws.tasks.p, n, ctx->d_aabb, s);
    lk::SweepArgs a = sweep_args(ctx, ws, pk);
    a.stop = stop;
    a.stop_base = stop_base;
    lk::ReduceArgs r{};
    r.tasks = ws.tasks.p;
    r.item_err = mixed ? ws.item_err.p : nullptr;
    r.err_out = mixed ? ws.err.p : nullptr;
    r.stop = stop;
    r.stop_base = stop_base;
    r.cc_half = cc ? ws.cc_half.p : nullptr;
    r.item_begin = ws.item_begin.p;
    r.partial = ws.partial.p;
    r.fix_acc = ws.fix_acc.p;
    r.item_fix = ctx->opt.precision == LK_ALL_F64 ? nullptr : ws.item_fix.p;
    r.flags = ws.flags.p;
    r.n_tasks = n;
    r.int_tol = ctx->opt.int_tol;
    r.lk_out = ws.lk.p;
    r.raw_out = ws.raw.p;
    r.status_out = ws.status.p;
    if (pk.n_items > 0) {
        if (ctx->opt.precision == LK_ALL_F64) {
            const int grid = ctx->num_sms * lk::sweep_f64_blocks_per_sm();
            if (ctx->opt.timing) LK_CUDA(ctx, record_event(ws.ev0, s));
            lk::launch_sweep_f64(a, grid, s);
            if (ctx->opt.timing) LK_CUDA(ctx, record_event(ws.ev1, s));
        } else {
            if (ctx->opt.timing) LK_CUDA(ctx, record_event(ws.ev0, s));
            if (cc) {
                // counting crossings first; the direct sum then runs only on the
                // pairs it flagged (its sweeps skip every other item)
                if (pk.n_cc_sweep > 0)
                    lk::launch_cc_sweep(a, ws.counters.p + 8, ctx->num_sms * lk::cc_sweep_blocks_per_sm(), s);
                if (pk.n_cc_local > 0) {
                    int G = 1;
                    while (G < lk::kCcLocalGridMax && G * G < pk.local_rows) G <<= 1;
                    const lk::CcLocalShape S{pk.local_rows, pk.local_cols, G, lk::kCcLocalEntries * pk.local_rows};
                    LK_CUDA(ctx, lk::launch_cc_local(a, n, pk.n_cc_local, S, s));
                }
                if (!pk.grid.empty()) {
                    const lk::CcGridWork w{ws.grid_offsets.p, ws.grid_cursor.p, ws.grid_sums.p, ws.grid_entries.p,
                                           (int64_t)std::min<size_t>(ws.grid_entries.cap, (size_t)INT32_MAX),
                                           ws.grid_row_xy.p, ws.grid_col_xy.p,
                                           reinterpret_cast<int*>(ws.grid_meta.p + 1), ws.grid_meta.p};
                    for (const GridJob& gj : pk.grid)
                        LK_CUDA(ctx, lk::launch_cc_grid(a, gj.task, gj.n_rows, gj.n_cols, gj.G_max, w, s));
                }
                lk::launch_cc_resolve(a, ctx->num_sms * 4, s);
            }
            if (cc) lk::launch_cc_flag_scan(a, ws.flag_scan.p, ws.flag_sums.p, s);
            lk::launch_sweep_mixed(a, true, 0, pk.n_acc_items, 0, pk.n_acc_tasks, ws.counters.p + 0,
                                   ctx->num_sms * lk::sweep_mixed_blocks_per_sm(true), s);
            lk::launch_sweep_mixed(a, false, pk.n_acc_items, pk.n_items, pk.n_acc_tasks, n, ws.counters.p + 4,
                                   ctx->num_sms * lk::sweep_mixed_blocks_per_sm(false), s);
            if (ctx->opt.timing) LK_CUDA(ctx, record_event(ws.ev1, s));
            const bool fast = pk.n_items > pk.n_acc_items, acc = pk.n_acc_items > 0;
            // Pairs of the accurate variant whose estimated error (from the
            // bulk sweep's statistics) exceeds precise_tol are flagged
            // kFlagPrecise by a first reduction; their bulk chunks are summed
            // again by the precise sweep and their handed-over chunks by the
            // precise careful pass.  The final reduction replaces its results.
            const bool precise = acc && ctx->opt.precise_tol > 0.0;
            const int pgrid = ctx->num_sms * lk::sweep_precise_blocks_per_sm();
            if (precise) {
                r.precise_tol = ctx->opt.precise_tol;
                lk::launch_reduce(r, s);
                r.precise_tol = 0.0;
                lk::launch_flag_scan(a, lk::kFlagPrecise, ws.precise_scan.p, ws.precise_sums.p, s);
                lk::launch_sweep_precise(a, 0, pk.n_acc_tasks, ws.counters.p + 7, pgrid, s);
            }
            lk::launch_careful_chunks(a, fast, acc, ctx->num_sms * lk::careful_chunk_blocks_per_sm(), s);
            if (precise) lk::launch_precise_careful(a, ws.counters.p + 10, pgrid, s);
            lk::launch_sweep_careful(a, fast, acc, ctx->num_sms * lk::sweep_careful_blocks_per_sm(), s);
            lk::launch_near_fix(a, ctx->num_sms * 4, s);
        }
    }
    lk::launch_reduce(r, s);
    LK_CUDA(ctx, cudaGetLastError());
    return LK_OK;
}

lk_status copy_outputs(lk_ctx* ctx, Workspace& ws, int64_t n, int32_t* lk_out, double* raw_out,
                       int32_t* status_out, cudaStream_t s) {
    bool host = false;
    if (lk_out) {
        LK_CUDA(ctx, cudaMemcpyAsync(lk_out, ws.lk.p, n * sizeof(int32_t), cudaMemcpyDefault, s));
        host |= !is_device_ptr(lk_out);
    }
    if (raw_out) {
        LK_CUDA(ctx, cudaMemcpyAsync(raw_out, ws.raw.p, n * sizeof(double), cudaMemcpyDefault, s));
        host |= !is_device_ptr(raw_out);
    }
    if (status_out) {
        LK_CUDA(ctx, cudaMemcpyAsync(status_out, ws.status.p, n * sizeof(int32_t), cudaMemcpyDefault, s));
        host |= !is_device_ptr(status_out);
    }
    if (host) LK_CUDA(ctx, cudaStreamSynchronize(s));
    return LK_OK;
}

void note_stats(lk_ctx* ctx, Workspace& ws, const Packed& pk, cudaStream_t s) {
    ctx->stats = lk_stats{};
    ctx->stats.n_pairs = (int64_t)pk.tasks.size();
    ctx->stats.n_items = pk.n_items;
    ctx->stats.segment_pairs = pk.segment_pairs;
    ctx->stats.tile_rows = pk.tile_rows_max;
    ctx->stats.tile_cols = pk.tile_cols;
    ctx->stats_tasks = (int64_t)pk.tasks.size();
    ctx->stats_fp64 = ws.fp64_count.p;
    ctx->stats_overflow = ws.counters.p + 1;
    ctx->stats_careful = reinterpret_cast<const unsigned int*>(ws.counters.p + 2);
    ctx->stats_flags = ws.flags.p;
    ctx->last_err = ws.err.p;
    ctx->last_n = (int64_t)pk.tasks.size();
    ctx->stats_cc = ctx->opt.method == LK_METHOD_CC && ws.cc_list.p != nullptr;
    ctx->stats_ev0 = (ctx->opt.timing && pk.n_items > 0) ? ws.ev0 : nullptr;
    ctx->stats_ev1 = ws.ev1;
    ctx->stats_stream = s;
    ctx->stats_pending = true;
}

bool finite3(double x, double y, double z) { return std::isfinite(x) && std::isfinite(y) && std::isfinite(z); }

lk_status get_pairs_on_host(lk_ctx* ctx, const int32_t* pairs, int64_t n, cudaStream_t s,
                            std::vector<int32_t>& hp) {
    hp.resize((size_t)(2 * n));
    if (n == 0) return LK_OK;
    if (is_device_ptr(pairs)) {
        LK_CUDA(ctx, cudaMemcpyAsync(hp.data(), pairs, 2 * n * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        LK_CUDA(ctx, cudaStreamSynchronize(s));
    } else {
        std::memcpy(hp.data(), pairs, 2 * n * sizeof(int32_t));
    }
    return LK_OK;
}

}  // namespace

extern "C" {

void lk_default_options(lk_options* opt) {
    if (!opt) return;
    opt->precision = LK_MIXED;
    opt->near_ratio = 3.0;
    opt->int_tol = 0.1;
    opt->mem_budget = 0;
    opt->tile_rows = 0;
    opt->near_capacity = 1 << 20;
    opt->timing = 0;
    opt->chunk_capacity = 1 << 20;
    opt->accurate_threshold = (int64_t)1 << 22;
    opt->method = LK_METHOD_DS;
    opt->cc_capacity = 1 << 18;
    opt->cc_search = LK_CC_SEARCH_AUTO;
    opt->precise_tol = 5e-7;
}

const char* lk_last_error(const lk_ctx* ctx) {
    if (ctx) return ctx->err.c_str();
    std::lock_guard<std::mutex> g(g_err_mu);
    return g_last_error.c_str();
}

lk_status lk_create(lk_ctx** out, const void* vertices, lk_dtype vdtype, int64_t n_vertices,
                    const int64_t* loop_offsets, int64_t n_loops, const lk_options* opt,
                    void* cuda_stream) {
    if (!out) return fail(nullptr, LK_ERR_ARG, "lk_create: out is NULL");
    *out = nullptr;
    if (!vertices || !loop_offsets || n_vertices < 3 || n_loops < 1 ||
        (vdtype != LK_F32 && vdtype != LK_F64))
        return fail(nullptr, LK_ERR_ARG, "lk_create: invalid arguments");
    lk_options o;
    lk_default_options(&o);
    if (opt) o = *opt;
    if (!(o.near_ratio >= 3.0) || !(o.int_tol > 0.0 && o.int_tol < 0.5) ||
        (o.precision != LK_MIXED && o.precision != LK_ALL_F64) || o.tile_rows < 0 ||
        o.near_capacity < 1 || o.accurate_threshold < 0 || o.chunk_capacity < 1 ||
        (o.method != LK_METHOD_DS && o.method != LK_METHOD_CC) || o.cc_capacity < 1 ||
        o.cc_search < LK_CC_SEARCH_AUTO || o.cc_search > LK_CC_SEARCH_BINNED || !(o.precise_tol >= 0.0) ||
        (o.method == LK_METHOD_CC && o.precision != LK_MIXED))
        return fail(nullptr, LK_ERR_ARG,
                    "lk_create: invalid options (near_ratio >= 3, 0 < int_tol < 0.5; LK_METHOD_CC needs LK_MIXED)");
    cudaStream_t s = (cudaStream_t)cuda_stream;

    // Host copies for validation.
    std::vector<int64_t> off((size_t)n_loops + 1);
    if (is_device_ptr(loop_offsets)) {
        if (cudaMemcpy(off.data(), loop_offsets, off.size() * sizeof(int64_t), cudaMemcpyDeviceToHost) != cudaSuccess)
            return fail(nullptr, LK_ERR_CUDA, "lk_create: cannot read loop_offsets");
    } else {
        std::memcpy(off.data(), loop_offsets, off.size() * sizeof(int64_t));
    }
    if (off[0] != 0 || off[(size_t)n_loops] != n_vertices)
        return fail(nullptr, LK_ERR_ARG, "lk_create: loop_offsets must start at 0 and end at n_vertices");
    for (int64_t l = 0; l < n_loops; ++l) {
        if (off[(size_t)l + 1] - off[(size_t)l] < 3)
            return fail(nullptr, LK_ERR_ARG, "lk_create: every loop needs at least 3 vertices");
        if (off[(size_t)l + 1] - off[(size_t)l] > INT32_MAX)
            return fail(nullptr, LK_ERR_ARG, "lk_create: loop too long");
    }
    std::vector<Vtx> hv((size_t)n_vertices);
    {
        const size_t esz = vdtype == LK_F32 ? 4 : 8;
        std::vector<unsigned char> raw((size_t)n_vertices * 3 * esz);
        if (is_device_ptr(vertices)) {
            if (cudaMemcpy(raw.data(), vertices, raw.size(), cudaMemcpyDeviceToHost) != cudaSuccess)
                return fail(nullptr, LK_ERR_CUDA, "lk_create: cannot read vertices");
        } else {
            std::memcpy(raw.data(), vertices, raw.size());
        }
        for (int64_t i = 0; i < n_vertices; ++i) {
            double x, y, z;
            if (vdtype == LK_F32) {
                const float* f = reinterpret_cast<const float*>(raw.data()) + 3 * i;
                x = f[0]; y = f[1]; z = f[2];
            } else {
                const double* f = reinterpret_cast<const double*>(raw.data()) + 3 * i;
                x = f[0]; y = f[1]; z = f[2];
            }
            if (!finite3(x, y, z)) return fail(nullptr, LK_ERR_ARG, "lk_create: non-finite coordinate");
            hv[(size_t)i] = Vtx{x, y, z, 0.0};
        }
    }
    // Zero-length segments (Algorithm 3's input check): |s| < eps * xi, xi the
    // mean absolute coordinate, eps the machine epsilon of the input type.
    {
        double xi = 0.0;
        for (const Vtx& v : hv) xi += std::fabs(v.x) + std::fabs(v.y) + std::fabs(v.z);
        xi /= (3.0 * (double)n_vertices);
        const double eps = vdtype == LK_F32 ? (double)FLT_EPSILON : DBL_EPSILON;
        const double thr = eps * xi;
        for (int64_t l = 0; l < n_loops; ++l) {
            const int64_t b = off[(size_t)l], e = off[(size_t)l + 1];
            for (int64_t i = b; i < e; ++i) {
                const Vtx& p = hv[(size_t)i];
                const Vtx& q = hv[(size_t)(i + 1 < e ? i + 1 : b)];
                const double len = std::sqrt((q.x - p.x) * (q.x - p.x) + (q.y - p.y) * (q.y - p.y) +
                                             (q.z - p.z) * (q.z - p.z));
                if (!(len >= thr) || len == 0.0) {
                    char buf[160];
                    snprintf(buf, sizeof buf, "lk_create: loop %lld has a zero-length segment at vertex %lld",
                             (long long)l, (long long)(i - b));
                    return fail(nullptr, LK_ERR_ZERO_SEGMENT, buf);
                }
            }
        }
    }

    lk_ctx* ctx = new lk_ctx();
    ctx->opt = o;
    ctx->n_vertices = n_vertices;
    ctx->n_loops = n_loops;
    ctx->h_offsets = off;
    cudaGetDevice(&ctx->device);
    cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, ctx->device);
    cudaError_t e = cudaMalloc(&ctx->d_V, (size_t)n_vertices * sizeof(Vtx));
    if (e == cudaSuccess) e = cudaMalloc(&ctx->d_offsets, off.size() * sizeof(int64_t));
    if (e == cudaSuccess) e = cudaMalloc(&ctx->d_aabb, (size_t)n_loops * 6 * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&ctx->d_R, (size_t)n_vertices * sizeof(float4));
    if (e == cudaSuccess) e = cudaMalloc(&ctx->d_box_keys, (size_t)n_loops * 12 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemcpyAsync(ctx->d_V, hv.data(), hv.size() * sizeof(Vtx), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(ctx->d_offsets, off.data(), off.size() * sizeof(int64_t), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = lk::reset_box_keys(ctx->d_box_keys, n_loops, s);
    if (e == cudaSuccess)
        e = lk::launch_loop_boxes(ctx->d_V, ctx->d_offsets, n_loops, n_vertices, ctx->d_box_keys,
                                  ctx->d_box_keys + 6 * n_loops, ctx->d_aabb, ctx->d_R, nullptr, 0, 0, s);
    ctx->box_set = 1;
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaMallocHost(&ctx->h_counters, 10 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMallocHost(&ctx->h_pls_total, sizeof(int64_t));
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->counters_ev, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        const lk_status st = cuda_fail(nullptr, e, "lk_create");
        lk_destroy(ctx);
        return st;
    }
    *out = ctx;
    return LK_OK;
}

lk_status lk_update(lk_ctx* ctx, const void* data, lk_dtype dtype, int is_delta, void* cuda_stream) {
    if (!ctx) return fail(nullptr, LK_ERR_ARG, "lk_update: NULL context");
    if (!data || (dtype != LK_F32 && dtype != LK_F64))
        return fail(ctx, LK_ERR_ARG, "lk_update: invalid arguments");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const size_t bytes = (size_t)ctx->n_vertices * 3 * (dtype == LK_F32 ? 4 : 8);
    const void* src = data;
    if (!is_device_ptr(data)) {
        if (ctx->stage_bytes < bytes) {
            if (ctx->d_stage) cudaFree(ctx->d_stage);
            ctx->d_stage = nullptr;
            ctx->stage_bytes = 0;
            LK_CUDA(ctx, cudaMalloc(&ctx->d_stage, bytes));
            ctx->stage_bytes = bytes;
        }
        LK_CUDA(ctx, cudaMemcpyAsync(ctx->d_stage, data, bytes, cudaMemcpyHostToDevice, s));
        src = ctx->d_stage;
    }
    unsigned long long* cur = ctx->d_box_keys + 6 * ctx->n_loops * ctx->box_set;
    unsigned long long* next = ctx->d_box_keys + 6 * ctx->n_loops * (1 - ctx->box_set);
    LK_CUDA(ctx, lk::launch_loop_boxes(ctx->d_V, ctx->d_offsets, ctx->n_loops, ctx->n_vertices, cur, next,
                                       ctx->d_aabb, ctx->d_R, src, dtype == LK_F32 ? 0 : 1, is_delta ? 1 : 0, s));
    ctx->box_set = 1 - ctx->box_set;
    return LK_OK;
}

lk_status lk_get_options(const lk_ctx* ctx, lk_options* out) {
    if (!ctx || !out) return fail(nullptr, LK_ERR_ARG, "lk_get_options: NULL argument");
    *out = ctx->opt;
    return LK_OK;
}

lk_status lk_verify(lk_ctx* ctx, const int32_t* loop_pairs, int64_t n_pairs, int32_t* lk_out,
                    double* raw_out, int32_t* status_out, void* cuda_stream) {
    if (!ctx) return fail(nullptr, LK_ERR_ARG, "lk_verify: NULL context");
    if (n_pairs < 0 || (n_pairs > 0 && !loop_pairs) || n_pairs > INT32_MAX)
        return fail(ctx, LK_ERR_ARG, "lk_verify: invalid pair list");
    if (n_pairs == 0) return LK_OK;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    std::vector<int32_t> hp;
    lk_status st = get_pairs_on_host(ctx, loop_pairs, n_pairs, s, hp);
    if (st != LK_OK) return st;
    grow_lists(ctx);
    if (hp == ctx->last_pairs) {
        // the same list as the last call: replay its plan (built on the first repeat)
        if (!ctx->repeat_plan) {
            lk_plan* plan = nullptr;
            if ((st = lk_plan_create(ctx, hp.data(), n_pairs, &plan, cuda_stream)) != LK_OK) return st;
            ctx->repeat_plan = plan;
        }
        st = lk_plan_run(ctx->repeat_plan, lk_out, raw_out, status_out, cuda_stream);
        const Packed& rp = ctx->repeat_plan->pk;
        if (st == LK_OK)
            note_counters(ctx, ctx->repeat_plan->ws.counters.p,
                          (rp.tile_rows_max + lk::kChunkRows - 1) / lk::kChunkRows, rp.n_chunks, s);
        return st;
    }
    drop_repeat_plan(ctx);
    Packed pk;
    if ((st = pack_pairs(ctx, hp.data(), n_pairs, pk)) != LK_OK) return st;
    if ((st = ensure_workspace(ctx, ctx->ws, n_pairs, pk.n_items, pk.n_chunks, &pk)) != LK_OK) return st;
    if ((st = upload_packed(ctx, ctx->ws, pk, s)) != LK_OK) return st;
    if ((st = enqueue_verify(ctx, ctx->ws, pk, s)) != LK_OK) return st;
    note_stats(ctx, ctx->ws, pk, s);
    ctx->last_pairs.swap(hp);
    st = copy_outputs(ctx, ctx->ws, n_pairs, lk_out, raw_out, status_out, s);
    if (st == LK_OK)
        note_counters(ctx, ctx->ws.counters.p, (pk.tile_rows_max + lk::kChunkRows - 1) / lk::kChunkRows,
                      pk.n_chunks, s);
    return st;
}

lk_status lk_candidates(lk_ctx* ctx, int32_t* pairs_out, int64_t capacity, int64_t* n_pairs,
                        void* cuda_stream) {
    if (!ctx) return fail(nullptr, LK_ERR_ARG, "lk_candidates: NULL context");
    if (!n_pairs || capacity < 0 || (capacity > 0 && !pairs_out))
        return fail(ctx, LK_ERR_ARG, "lk_candidates: invalid output arguments");
    *n_pairs = 0;
    const int64_t L = ctx->n_loops;
    if (L < 2) return LK_OK;
    if (L > (int64_t)1 << 30) return fail(ctx, LK_ERR_ARG, "lk_candidates: too many loops");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const unsigned nsort = lk::pls_sort_size(L);
    if (!ctx->d_pls_keys) {
        cudaError_t e = cudaMalloc(&ctx->d_pls_keys, (size_t)L * 6 * sizeof(long long));
        if (e == cudaSuccess) e = cudaMalloc(&ctx->d_pls_counts, (size_t)L * sizeof(int32_t));
        if (e == cudaSuccess) e = cudaMalloc(&ctx->d_pls_offsets, ((size_t)L + 1) * sizeof(int64_t));
        if (e == cudaSuccess) e = cudaMalloc(&ctx->d_pls_scan, lk::scan_scratch_count(L) * sizeof(long long));
        if (e == cudaSuccess) e = cudaMalloc(&ctx->d_pls_order, (size_t)nsort * sizeof(unsigned long long));
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(ctx, LK_ERR_OOM, "lk_candidates: device allocation failed");
        }
    }
    // Up to 2^27 box tests every pair is tested directly (a tiled all-pairs
    // pass, faster than the sort's launches there: 9,248 loops in 0.22 ms
    // against 0.41 ms); above, sort by lower x and sweep.  Both give the same
    // list in (i, j) order.
    const bool sweep = L * (L - 1) / 2 > ((int64_t)1 << 27);
    lk::launch_pls_keys(ctx->d_aabb, L, ctx->d_pls_keys, s);
    if (sweep) {
        lk::launch_pls_sort(ctx->d_pls_keys, L, ctx->d_pls_order, nsort, s);
        lk::launch_pls_sweep_count(ctx->d_pls_keys, L, ctx->d_pls_order, ctx->d_pls_counts, s);
    } else {
        lk::launch_pls_count(ctx->d_pls_keys, L, ctx->d_pls_counts, s);
    }
    // offsets = exclusive scan of the counts on the device; only the total comes back
    lk::launch_scan_counts(ctx->d_pls_counts, L, ctx->d_pls_offsets, ctx->d_pls_scan, s);
    int64_t total = 0;
    LK_CUDA(ctx, cudaMemcpyAsync(ctx->h_pls_total, ctx->d_pls_offsets + L, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    LK_CUDA(ctx, cudaStreamSynchronize(s));
    total = *ctx->h_pls_total;
    if (total > (int64_t)1 << 31) return fail(ctx, LK_ERR_ARG, "lk_candidates: more than 2^31 candidate pairs");
    const int64_t m = std::min(total, capacity);
    if (m > 0 && !sweep) {
        int32_t* dst = pairs_out;
        const bool host = !is_device_ptr(pairs_out);
        if (host) {
            if (ctx->pls_pairs_cap < m) {
                if (ctx->d_pls_pairs) cudaFree(ctx->d_pls_pairs);
                ctx->d_pls_pairs = nullptr;
                ctx->pls_pairs_cap = 0;
                if (cudaMalloc(&ctx->d_pls_pairs, (size_t)m * 2 * sizeof(int32_t)) != cudaSuccess) {
                    cudaGetLastError();
                    return fail(ctx, LK_ERR_OOM, "lk_candidates: device allocation failed");
                }
                ctx->pls_pairs_cap = m;
            }
            dst = ctx->d_pls_pairs;
        }
        lk::launch_pls_write(ctx->d_pls_keys, L, ctx->d_pls_offsets, dst, m, s);
        LK_CUDA(ctx, cudaGetLastError());
        if (host)
            LK_CUDA(ctx, cudaMemcpyAsync(pairs_out, dst, (size_t)m * 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        LK_CUDA(ctx, cudaStreamSynchronize(s));
    } else if (m > 0) {
        // every pair as an (i << 32 | j) key, sorted into (i, j) order
        const unsigned npk = lk::pls_sort_size(total);
        LK_CUDA(ctx, ctx->pls_pair_keys.ensure(npk));
        LK_CUDA(ctx, cudaMemsetAsync(ctx->pls_pair_keys.p, 0xff, (size_t)npk * sizeof(unsigned long long), s));
        lk::launch_pls_sweep_write(ctx->d_pls_keys, L, ctx->d_pls_order, ctx->d_pls_offsets, ctx->pls_pair_keys.p,
                                   total, s);
        lk::launch_bitonic_sort(ctx->pls_pair_keys.p, npk, s);
        int32_t* dst = pairs_out;
        const bool host = !is_device_ptr(pairs_out);
        if (host) {
            if (ctx->pls_pairs_cap < m) {
                if (ctx->d_pls_pairs) cudaFree(ctx->d_pls_pairs);
                ctx->d_pls_pairs = nullptr;
                ctx->pls_pairs_cap = 0;
                if (cudaMalloc(&ctx->d_pls_pairs, (size_t)m * 2 * sizeof(int32_t)) != cudaSuccess) {
                    cudaGetLastError();
                    return fail(ctx, LK_ERR_OOM, "lk_candidates: device allocation failed");
                }
                ctx->pls_pairs_cap = m;
            }
            dst = ctx->d_pls_pairs;
        }
        lk::launch_pls_unpack(ctx->pls_pair_keys.p, m, dst, s);
        LK_CUDA(ctx, cudaGetLastError());
        if (host)
            LK_CUDA(ctx, cudaMemcpyAsync(pairs_out, dst, (size_t)m * 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        LK_CUDA(ctx, cudaStreamSynchronize(s));
    }
    *n_pairs = total;
    return LK_OK;
}

lk_status lk_sync(lk_ctx* ctx, void* cuda_stream) {
    if (!ctx) return fail(nullptr, LK_ERR_ARG, "lk_sync: NULL context");
    LK_CUDA(ctx, cudaStreamSynchronize((cudaStream_t)cuda_stream));
    return LK_OK;
}

lk_status lk_get_stats(lk_ctx* ctx, lk_stats* out) {
    if (!ctx || !out) return fail(ctx, LK_ERR_ARG, "lk_get_stats: NULL argument");
    if (ctx->stats_pending) {
        LK_CUDA(ctx, cudaStreamSynchronize(ctx->stats_stream));
        std::vector<unsigned long long> c((size_t)std::max<int64_t>(ctx->stats_tasks, 1), 0ull);
        if (ctx->stats_tasks > 0)
            LK_CUDA(ctx, cudaMemcpy(c.data(), ctx->stats_fp64, ctx->stats_tasks * sizeof(unsigned long long),
                                    cudaMemcpyDeviceToHost));
        unsigned long long ov = 0;
        LK_CUDA(ctx, cudaMemcpy(&ov, ctx->stats_overflow, sizeof ov, cudaMemcpyDeviceToHost));
        ctx->stats.fp64_pairs = (int64_t)std::accumulate(c.begin(), c.end(), 0ull);
        ctx->stats.near_overflow = (int64_t)ov;
        unsigned int u32[16] = {};
        LK_CUDA(ctx, cudaMemcpy(u32, ctx->stats_careful, ctx->stats_cc ? 16 * sizeof(unsigned int)
                                                                     : 8 * sizeof(unsigned int),
                                cudaMemcpyDeviceToHost));
        ctx->stats.careful_items = u32[0];
        ctx->stats.careful_chunks = u32[6];
        ctx->stats.cc_candidates = 0;
        ctx->stats.cc_fallback_pairs = 0;
        ctx->stats.precise_pairs = 0;
        if (ctx->stats_cc) ctx->stats.cc_candidates = (int64_t)(u32[14] | ((unsigned long long)u32[15] << 32));   // counters[9]
        {
            std::vector<int> fl((size_t)std::max<int64_t>(ctx->stats_tasks, 1), 0);
            if (ctx->stats_tasks > 0)
                LK_CUDA(ctx, cudaMemcpy(fl.data(), ctx->stats_flags, ctx->stats_tasks * sizeof(int),
                                        cudaMemcpyDeviceToHost));
            for (int64_t t = 0; t < ctx->stats_tasks; ++t) {
                if (ctx->stats_cc) ctx->stats.cc_fallback_pairs += (fl[(size_t)t] & lk::kFlagCcFallback) ? 1 : 0;
                ctx->stats.precise_pairs += (fl[(size_t)t] & lk::kFlagPrecise) ? 1 : 0;
            }
        }
        ctx->stats.sweep_ms = -1.0;
        if (ctx->stats_ev0) {
            float ms = 0.0f;
            LK_CUDA(ctx, cudaEventElapsedTime(&ms, ctx->stats_ev0, ctx->stats_ev1));
            ctx->stats.sweep_ms = ms;
        }
        ctx->stats_pending = false;
    }
    *out = ctx->stats;
    return LK_OK;
}

lk_status lk_get_error_estimates(const lk_ctx* ctx, double* err_out, int64_t n_pairs, void* cuda_stream) {
    if (!ctx || !err_out) return fail(nullptr, LK_ERR_ARG, "lk_get_error_estimates: NULL argument");
    lk_ctx* c = const_cast<lk_ctx*>(ctx);
    if (!ctx->last_err || n_pairs != ctx->last_n)
        return fail(c, LK_ERR_ARG, "lk_get_error_estimates: n_pairs must equal the last verify's pair count "
                                   "(and the last verify must have used LK_MIXED)");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    LK_CUDA(c, cudaMemcpyAsync(err_out, ctx->last_err, (size_t)n_pairs * sizeof(double), cudaMemcpyDefault, s));
    if (!is_device_ptr(err_out)) LK_CUDA(c, cudaStreamSynchronize(s));
    return LK_OK;
}

void lk_destroy(lk_ctx* ctx) {
    if (!ctx) return;
    drop_repeat_plan(ctx);
    ctx->ws.release();
    ctx->ee_expected.release(); ctx->ee_lk.release(); ctx->ee_status.release(); ctx->ee_raw.release();
    ctx->ee_stop.release();
    if (ctx->ee_plan) {
        ctx->ee_plan->release();
        delete ctx->ee_plan;
    }
    if (ctx->d_V) cudaFree(ctx->d_V);
    if (ctx->d_offsets) cudaFree(ctx->d_offsets);
    if (ctx->d_aabb) cudaFree(ctx->d_aabb);
    if (ctx->d_box_keys) cudaFree(ctx->d_box_keys);
    if (ctx->d_R) cudaFree(ctx->d_R);
    if (ctx->d_pls_keys) cudaFree(ctx->d_pls_keys);
    if (ctx->d_pls_counts) cudaFree(ctx->d_pls_counts);
    if (ctx->d_pls_offsets) cudaFree(ctx->d_pls_offsets);
    if (ctx->d_pls_scan) cudaFree(ctx->d_pls_scan);
    if (ctx->h_pls_total) cudaFreeHost(ctx->h_pls_total);
    if (ctx->d_pls_pairs) cudaFree(ctx->d_pls_pairs);
    if (ctx->d_pls_order) cudaFree(ctx->d_pls_order);
    ctx->pls_pair_keys.release();
    if (ctx->d_stage) cudaFree(ctx->d_stage);
    if (ctx->counters_ev) {
        cudaEventSynchronize(ctx->counters_ev);
        cudaEventDestroy(ctx->counters_ev);
    }
    if (ctx->h_counters) cudaFreeHost(ctx->h_counters);
    delete ctx;
}

lk_status lk_plan_create(lk_ctx* ctx, const int32_t* loop_pairs, int64_t n_pairs, lk_plan** out,
                         void* cuda_stream) {
    if (!out) return fail(ctx, LK_ERR_ARG, "lk_plan_create: out is NULL");
    *out = nullptr;
    if (!ctx) return fail(nullptr, LK_ERR_ARG, "lk_plan_create: NULL context");
    if (n_pairs < 0 || (n_pairs > 0 && !loop_pairs) || n_pairs > INT32_MAX)
        return fail(ctx, LK_ERR_ARG, "lk_plan_create: invalid pair list");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    std::vector<int32_t> hp;
    lk_status st = get_pairs_on_host(ctx, loop_pairs, n_pairs, s, hp);
    if (st != LK_OK) return st;
    lk_plan* plan = new lk_plan();
    plan->ctx = ctx;
    if ((st = pack_pairs(ctx, hp.data(), n_pairs, plan->pk)) != LK_OK ||
        (st = ensure_workspace(ctx, plan->ws, n_pairs, plan->pk.n_items, plan->pk.n_chunks, &plan->pk)) != LK_OK ||
        (st = upload_packed(ctx, plan->ws, plan->pk, s)) != LK_OK) {
        lk_plan_destroy(plan);
        return st;
    }
    cudaError_t e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&plan->capture, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(plan->capture, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        lk_plan_destroy(plan);
        return cuda_fail(ctx, e, "lk_plan_create");
    }
    st = enqueue_verify(ctx, plan->ws, plan->pk, plan->capture);
    e = cudaStreamEndCapture(plan->capture, &plan->graph);
    if (st != LK_OK) {
        lk_plan_destroy(plan);
        return st;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&plan->exec, plan->graph, 0);
    if (e != cudaSuccess) {
        lk_plan_destroy(plan);
        return cuda_fail(ctx, e, "lk_plan_create: graph");
    }
    *out = plan;
    return LK_OK;
}

lk_status lk_plan_run(lk_plan* plan, int32_t* lk_out, double* raw_out, int32_t* status_out,
                      void* cuda_stream) {
    if (!plan) return fail(nullptr, LK_ERR_ARG, "lk_plan_run: NULL plan");
    lk_ctx* ctx = plan->ctx;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const int64_t n = (int64_t)plan->pk.tasks.size();
    if (n == 0) return LK_OK;
    LK_CUDA(ctx, cudaGraphLaunch(plan->exec, s));
    note_stats(ctx, plan->ws, plan->pk, s);
    return copy_outputs(ctx, plan->ws, n, lk_out, raw_out, status_out, s);
}

void lk_plan_destroy(lk_plan* plan) {
    if (!plan) return;
    if (plan->exec) cudaGraphExecDestroy(plan->exec);
    if (plan->graph) cudaGraphDestroy(plan->graph);
    if (plan->capture) cudaStreamDestroy(plan->capture);
    if (plan->ctx && plan->ctx->stats_fp64 == plan->ws.fp64_count.p) plan->ctx->stats_pending = false;
    if (plan->ctx && plan->ctx->last_err == plan->ws.err.p) plan->ctx->last_err = nullptr;
    plan->ws.release();
    delete plan;
}

}  // extern "C"

// ----------------------------------------------------------------------------
// Allocation-free verify.
//
// Some callers cannot allocate device memory when they need a linking-number
// check: a simulation step that runs under a strict no-allocation rule (a
// device allocation synchronises the GPU and can stall a real-time loop),
// a process whose memory pool already owns all of device memory, or a host
// program that manages memory itself and forbids libraries to call
// cudaMalloc.  lk_verify_noalloc serves them: it runs the same kernels as
// lk_verify, but every work buffer -- the converted geometry, loop boxes,
// pair tasks, item tables, partial sums, recompute list, counters and
// results -- lives in one file-scope device array of fixed size.  It calls
// no cudaMalloc, cudaFree or allocating library routine.
namespace {

constexpr size_t kNoallocScratchBytes = (size_t)48 << 20;   // 48 MiB per device, held until exit
constexpr int64_t kNoallocMaxVertices = (int64_t)1 << 18;
constexpr int64_t kNoallocMaxLoops = (int64_t)1 << 14;
constexpr int64_t kNoallocMaxPairs = (int64_t)1 << 14;
constexpr int64_t kNoallocMaxItems = (int64_t)1 << 18;
constexpr int kNoallocNearCapacity = 1 << 16;
constexpr int64_t kNoallocMaxChunks = (int64_t)1 << 16;     // chunk hand-over list entries
constexpr int64_t kNoallocMaxChunkBits = (int64_t)1 << 23;  // chunk slots of accurate-variant items
constexpr int kNoallocMaxDevices = 64;

std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kNoallocMaxDevices] = {};

}  // namespace

// Shared by every call on a device: contents persist between calls.
static __device__ __align__(256) unsigned char lk_noalloc_scratch[kNoallocScratchBytes];

namespace {

// Carve the scratch into the buffers of one verify at the fixed maxima.
struct NoallocLayout {
    size_t off = 0;
    unsigned char* base;
    explicit NoallocLayout(void* b) : base((unsigned char*)b) {}
    template <class T>
    T* take(size_t count) {
        off = (off + 255) & ~(size_t)255;
        T* p = reinterpret_cast<T*>(base + off);
        off += count * sizeof(T);
        return p;
    }
};

// Address of the scratch array on the current device, looked up once per
// device (in host code the array's name is not a device address).
lk_status noalloc_scratch(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "lk_verify_noalloc: cudaGetDevice");
    if (dev < 0 || dev >= kNoallocMaxDevices)
        return fail(nullptr, LK_ERR_ARG, "lk_verify_noalloc: device index out of range");
    std::lock_guard<std::mutex> g(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, lk_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return cuda_fail(nullptr, e == cudaSuccess ? cudaErrorInvalidSymbol : e,
                             "lk_verify_noalloc: cudaGetSymbolAddress");
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return LK_OK;
}

}  // namespace

extern "C" lk_status lk_verify_noalloc(const void* vertices, lk_dtype vdtype, int64_t n_vertices,
                                       const int64_t* loop_offsets, int64_t n_loops,
                                       const int32_t* loop_pairs, int64_t n_pairs, int32_t* lk_out,
                                       double* raw_out, int32_t* status_out, void* cuda_stream) {
    char msg[200];
    if (!vertices || !loop_offsets || (n_pairs > 0 && !loop_pairs) || n_vertices < 3 || n_loops < 1 ||
        n_pairs < 0 || (vdtype != LK_F32 && vdtype != LK_F64))
        return fail(nullptr, LK_ERR_ARG, "lk_verify_noalloc: invalid arguments");
    if (n_vertices > kNoallocMaxVertices || n_loops > kNoallocMaxLoops || n_pairs > kNoallocMaxPairs) {
        snprintf(msg, sizeof msg,
                 "lk_verify_noalloc: size beyond the static scratch limits (vertices <= %lld, loops <= %lld, "
                 "pairs <= %lld)", (long long)kNoallocMaxVertices, (long long)kNoallocMaxLoops,
                 (long long)kNoallocMaxPairs);
        return fail(nullptr, LK_ERR_ARG, msg);
    }
    if (is_device_ptr(loop_offsets) || (n_pairs > 0 && is_device_ptr(loop_pairs)))
        return fail(nullptr, LK_ERR_ARG, "lk_verify_noalloc: loop_offsets and loop_pairs must be host memory");
    if (loop_offsets[0] != 0 || loop_offsets[n_loops] != n_vertices)
        return fail(nullptr, LK_ERR_ARG, "lk_verify_noalloc: loop_offsets must start at 0 and end at n_vertices");
    for (int64_t l = 0; l < n_loops; ++l)
        if (loop_offsets[l + 1] - loop_offsets[l] < 3)
            return fail(nullptr, LK_ERR_ARG, "lk_verify_noalloc: every loop needs at least 3 vertices");
    if (n_pairs == 0) return LK_OK;

    void* scratch = nullptr;
    lk_status st = noalloc_scratch(&scratch);
    if (st != LK_OK) return st;
    cudaStream_t s = (cudaStream_t)cuda_stream;

    // A context on the stack pointing into the scratch; it owns nothing and is
    // never passed to lk_destroy.
    lk_ctx ctx;
    lk_default_options(&ctx.opt);
    ctx.opt.near_capacity = kNoallocNearCapacity;
    // the hand-over list holds what the scratch reserves; a batch with more
    // chunks to hand over passes whole items to the careful pass instead
    ctx.opt.chunk_capacity = (int)kNoallocMaxChunks;
    ctx.n_vertices = n_vertices;
    ctx.n_loops = n_loops;
    ctx.h_offsets.assign(loop_offsets, loop_offsets + n_loops + 1);
    cudaGetDevice(&ctx.device);
    cudaDeviceGetAttribute(&ctx.num_sms, cudaDevAttrMultiProcessorCount, ctx.device);

    NoallocLayout L(scratch);
    ctx.d_V = L.take<Vtx>((size_t)kNoallocMaxVertices);
    ctx.d_R = L.take<float4>((size_t)kNoallocMaxVertices);
    double* raw_in = L.take<double>((size_t)kNoallocMaxVertices * 3);   // host vertices staged here
    ctx.d_offsets = L.take<int64_t>((size_t)kNoallocMaxLoops + 1);
    ctx.d_aabb = L.take<double>((size_t)kNoallocMaxLoops * 6);
    ctx.d_box_keys = L.take<unsigned long long>((size_t)kNoallocMaxLoops * 12);
    Workspace ws;
    auto bind = [&](auto& buf, size_t count) {
        using T = typename std::remove_pointer<decltype(buf.p)>::type;
        buf.p = L.take<T>(count);
        buf.cap = count;
        buf.fixed = true;
    };
    bind(ws.tasks, (size_t)kNoallocMaxPairs);
    bind(ws.item_begin, (size_t)kNoallocMaxPairs + 1);
    bind(ws.item_task, (size_t)kNoallocMaxItems);
    bind(ws.partial, (size_t)kNoallocMaxItems);
    bind(ws.careful_items, (size_t)kNoallocMaxItems);
    bind(ws.careful_chunks, (size_t)kNoallocMaxChunks);
    bind(ws.item_fix, (size_t)kNoallocMaxItems);
    bind(ws.near_list, (size_t)kNoallocNearCapacity);
    bind(ws.fix_acc, (size_t)kNoallocMaxPairs);
    bind(ws.fp64_count, (size_t)kNoallocMaxPairs);
    bind(ws.flags, (size_t)kNoallocMaxPairs);
    bind(ws.counters, kCounters);
    bind(ws.lk, (size_t)kNoallocMaxPairs);
    bind(ws.raw, (size_t)kNoallocMaxPairs);
    bind(ws.status, (size_t)kNoallocMaxPairs);
    bind(ws.item_err, (size_t)kNoallocMaxItems);
    bind(ws.chunk_bits, (size_t)kNoallocMaxChunkBits / 32);
    bind(ws.precise_scan, (size_t)kNoallocMaxPairs + 1);
    bind(ws.precise_sums, (size_t)kNoallocMaxPairs / 4096 + 2);
    bind(ws.err, (size_t)kNoallocMaxPairs);
    if (L.off > kNoallocScratchBytes) return fail(nullptr, LK_ERR_ARG, "lk_verify_noalloc: scratch layout overflow");

    Packed pk;
    if ((st = pack_pairs(&ctx, loop_pairs, n_pairs, pk)) != LK_OK) return fail(nullptr, st, ctx.err);
    if (pk.n_items > kNoallocMaxItems || pk.n_chunk_bits > kNoallocMaxChunkBits) {
        snprintf(msg, sizeof msg,
                 "lk_verify_noalloc: %lld work items (%lld chunk slots of large pairs) exceed the static limit of "
                 "%lld (%lld)", (long long)pk.n_items, (long long)pk.n_chunk_bits, (long long)kNoallocMaxItems,
                 (long long)kNoallocMaxChunkBits);
        return fail(nullptr, LK_ERR_ARG, msg);
    }
    // Geometry into the scratch: offsets, then the vertices as resident FP64
    // (the box passes replace them from the caller's layout) with the loop
    // boxes and the FP32 loop-relative copy.
    const size_t vbytes = (size_t)n_vertices * 3 * (vdtype == LK_F32 ? 4 : 8);
    const void* vsrc = vertices;
    if (!is_device_ptr(vertices)) {
        cudaError_t e = cudaMemcpyAsync(raw_in, vertices, vbytes, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return cuda_fail(nullptr, e, "lk_verify_noalloc: vertices");
        vsrc = raw_in;
    }
    cudaError_t e = cudaMemcpyAsync(ctx.d_offsets, loop_offsets, (size_t)(n_loops + 1) * sizeof(int64_t),
                                    cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "lk_verify_noalloc: offsets");
    e = lk::reset_box_keys(ctx.d_box_keys, n_loops, s);
    if (e == cudaSuccess)
        e = lk::launch_loop_boxes(ctx.d_V, ctx.d_offsets, n_loops, n_vertices, ctx.d_box_keys,
                                  ctx.d_box_keys + 6 * n_loops, ctx.d_aabb, ctx.d_R, vsrc, vdtype == LK_F32 ? 0 : 1, 0,
                                  s);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "lk_verify_noalloc: geometry");
    if ((st = ensure_workspace(&ctx, ws, n_pairs, pk.n_items, pk.n_chunks, &pk)) != LK_OK ||
        (st = upload_packed(&ctx, ws, pk, s)) != LK_OK || (st = enqueue_verify(&ctx, ws, pk, s)) != LK_OK ||
        (st = copy_outputs(&ctx, ws, n_pairs, lk_out, raw_out, status_out, s)) != LK_OK)
        return fail(nullptr, st, ctx.err);
    return LK_OK;
}

// ----------------------------------------------------------------------------
// Serving: continuous batching of verify requests.
//
// A server owns a device arena (the memory budget that admission checks), a
// pinned host arena for results, and a FIFO of submitted requests.  Each
// lk_server_step retires waves that have finished, admits queued requests
// while request slots and arena space allow, and launches one wave: a
// persistent launch over up to wave_items work items taken in admission order
// from every admitted request that still has items, so that requests which
// arrived while others were running share the device with them.  A request
// whose last items are in a wave gets its careful pass, FP64 recomputes and
// reduction right after that wave; its results are copied to pinned memory
// and handed out by lk_server_poll.
namespace {

// First-fit allocator over byte offsets [0, size), 256-byte granules.
struct Arena {
    size_t size = 0;
    std::map<size_t, size_t> free_;   // offset -> length
    size_t used = 0;

    void init(size_t n) {
        size = n;
        free_.clear();
        if (n) free_[0] = n;
        used = 0;
    }
    static size_t round(size_t n) { return (std::max<size_t>(n, 1) + 255) & ~(size_t)255; }
    bool alloc(size_t n, size_t* off) {
        n = round(n);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < n) continue;
            *off = it->first;
            const size_t rest = it->second - n, at = it->first + n;
            free_.erase(it);
            if (rest) free_[at] = rest;
            used += n;
            return true;
        }
        return false;
    }
    void release(size_t off, size_t n) {
        n = round(n);
        used -= n;
        auto it = free_.emplace(off, n).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
};

enum ReqState { kQueued = 0, kRunning = 1, kLaunched = 2, kDone = 3, kSearching = 4, kPacking = 5 };

struct Request {
    int64_t ticket = 0;
    lk_ctx* ctx = nullptr;
    std::vector<int32_t> pairs;
    Packed pk;
    bool packed = false;
    // The counts the waves and the finishing passes need (from pk, or for a
    // geometry request from the device packer's totals).
    int64_t n_tasks = 0, n_items = 0, n_acc_items = 0, n_chunks = 0;
    Workspace ws;              // pointers into the device arena
    size_t dev_off = 0, dev_bytes = 0;
    size_t host_off = 0, host_bytes = 0;
    int32_t* h_lk = nullptr;   // pinned results
    double* h_raw = nullptr;
    int32_t* h_status = nullptr;
    unsigned long long* h_counters = nullptr;   // the request's 8 work counters, copied back
    lk::SweepArgs args{};
    int64_t next_item = 0;
    int state = kQueued;
    // Geometry requests: the pairs are the potential link search's candidates
    // of the context, found and packed on the device (lk_server_submit_geometry).
    bool geometry = false;
    bool dev_pack = false;               // a pair list packed on the device (pack_on_device)
    bool sweep = false;                  // sort-and-sweep search (else every box pair)
    bool tuned = false;                  // the context's tune table goes to the packer
    lk_status error = LK_OK;             // set when the request could not run
    std::string error_msg;
    cudaEvent_t ev = nullptr;            // end of the search, then of the packing
    size_t scr_off = 0, scr_bytes = 0;   // device: the search's scratch (until packed)
    size_t blk_off = 0, blk_bytes = 0;   // device: the pair list, keys and tasks (until done)
    size_t sum_off = 0, sum_bytes = 0;   // pinned: the totals read back, the tune table
    long long* h_sum = nullptr;          // [0] candidate pairs, [1..6] lk::PackSums: the packing's totals
    int32_t* h_pairs = nullptr;          // pinned copy of the pair list (results)
    int32_t* d_pairs = nullptr;
    ~Request() {
        if (ev) cudaEventDestroy(ev);
    }
};

struct Wave {
    cudaEvent_t done = nullptr;       // the wave and its requests' finishing work are done
    cudaEvent_t swept = nullptr;      // the wave's bulk launches are done (finishing work waits for it)
    int slot = 0;
    std::vector<Request*> completing;
};

constexpr int kWaveSlots = 3;          // waves in flight at most
constexpr int kMaxSegs = 256;          // request runs per wave

constexpr int64_t kServerMaxChunks = (int64_t)1 << 22;

// Carve one request's work buffers out of the arena at `base` (or, with
// base = 0, only measure them); returns the bytes used.  Without `tables` the
// pair tasks and item_begin live elsewhere (a geometry request's pack block).
size_t request_layout(int64_t n_tasks, int64_t n_items, int64_t n_chunks, bool tables, int near_cap, Workspace* ws,
                      uintptr_t base) {
    size_t off = 0;
    const size_t P = (size_t)std::max<int64_t>(n_tasks, 1), I = (size_t)std::max<int64_t>(n_items, 1);
    auto bind = [&](auto& buf, size_t count) {
        using T = typename std::remove_pointer<decltype(buf.p)>::type;
        off = (off + 255) & ~(size_t)255;
        buf.p = reinterpret_cast<T*>(base + off);
        buf.cap = count;
        off += count * sizeof(T);
    };
    // Three groups, each contiguous so that one copy or memset serves it:
    // the uploaded tables (tasks, item_begin, item_task: the layout of the
    // pinned staging, upload_layout), the buffers that start at zero
    // (item_fix .. counters), and the results copied back (counters .. status:
    // the layout of the pinned result block, result_layout).
    if (tables) {
        bind(ws->tasks, P);
        bind(ws->item_begin, P + 1);
    }
    bind(ws->item_task, I);
    bind(ws->partial, I);
    bind(ws->careful_items, I);
    // room for every chunk of the request (up to 2^22 entries, 64 MB): a full
    // list hands items over whole, whose careful re-sum rounds differently,
    // so a result would depend on which items found the list full
    bind(ws->careful_chunks, (size_t)std::max<int64_t>(1, std::min<int64_t>(n_chunks, kServerMaxChunks)));
    bind(ws->near_list, (size_t)near_cap);
    bind(ws->item_fix, I);
    bind(ws->fix_acc, P);
    bind(ws->fp64_count, P);
    bind(ws->flags, P);
    bind(ws->counters, 8);
    bind(ws->lk, P);
    bind(ws->raw, P);
    bind(ws->status, P);
    return off;
}

size_t request_layout(const Packed& pk, int near_cap, Workspace* ws, uintptr_t base) {
    return request_layout((int64_t)pk.tasks.size(), pk.n_items, pk.n_chunks, true, near_cap, ws, base);
}

// Sequential 256-byte aligned pieces of one arena block (base 0: measure only).
struct Carver {
    uintptr_t base;
    size_t off = 0;
    template <class T>
    T* take(size_t count) {
        off = (off + 255) & ~(size_t)255;
        T* p = reinterpret_cast<T*>(base + off);
        off += count * sizeof(T);
        return p;
    }
};

// A geometry request's search scratch: box keys, per-loop counts and offsets,
// the scan's block totals, the sweep's sorted order, the tune table.
struct SearchBufs {
    long long* keys;
    int32_t* counts;
    int64_t* offsets;
    long long* scan;
    unsigned long long* order;
    int32_t* tune;
};

size_t search_layout(int64_t L, bool sweep, SearchBufs* b, uintptr_t base) {
    Carver c{base};
    b->keys = c.take<long long>((size_t)L * 6);
    b->counts = c.take<int32_t>((size_t)L);
    b->offsets = c.take<int64_t>((size_t)L + 1);
    b->scan = c.take<long long>(lk::scan_scratch_count(L));
    b->order = sweep ? c.take<unsigned long long>(lk::pls_sort_size(L)) : nullptr;
    b->tune = c.take<int32_t>((size_t)lk::kTuneClasses * lk::kTuneClasses);
    return c.off;
}

// Its pack block: the pair list, the 64-bit keys of both sorts, the tasks,
// their counts and scan, item_begin.
struct PackBufs {
    int32_t* pairs;
    unsigned long long* keys;
    PairTask* tasks;
    lk::PackSums* sums;
    lk::PackSums* scan;
    lk::PackSums* scratch;
    int64_t* item_begin;
};

size_t pack_layout(int64_t T, PackBufs* b, uintptr_t base) {
    Carver c{base};
    b->pairs = c.take<int32_t>((size_t)T * 2);
    b->keys = c.take<unsigned long long>(lk::pls_sort_size(T));
    b->tasks = c.take<PairTask>((size_t)T);
    b->sums = c.take<lk::PackSums>((size_t)T);
    b->scan = c.take<lk::PackSums>((size_t)T + 1);
    b->scratch = c.take<lk::PackSums>(lk::scan_scratch_count(T));
    b->item_begin = c.take<int64_t>((size_t)T + 1);
    return c.off;
}

// Pinned bytes of a geometry request's totals and tune table.
constexpr size_t kSumBytes = 64;
static_assert(sizeof(long long) + sizeof(lk::PackSums) <= kSumBytes, "the totals read back fit their slot");
size_t geometry_sum_bytes() { return kSumBytes + (size_t)lk::kTuneClasses * lk::kTuneClasses * sizeof(int32_t); }

// A pair-list request packed on the device: its pack block (the pack layout,
// then the tune table) and its pinned block (results, the staged list, the
// totals read back and the tune table).
size_t devpack_dev_bytes(int64_t T) {
    PackBufs pb;
    return ((pack_layout(T, &pb, 0) + 255) & ~(size_t)255) +
           (size_t)lk::kTuneClasses * lk::kTuneClasses * sizeof(int32_t);
}
size_t devpack_host_bytes(int64_t T);

inline size_t align256(size_t n) { return (n + 255) & ~(size_t)255; }

// Offsets within a request's result group, the same on the device (from
// ws.counters) and in its pinned result block: counters, lk, raw, status.
struct ResultLayout {
    size_t lk, raw, status, copy_bytes;
};
ResultLayout result_layout(size_t P) {
    ResultLayout r;
    r.lk = 256;                                   // after the 8 counters
    r.raw = r.lk + align256(P * 4);
    r.status = r.raw + align256(P * 8);
    r.copy_bytes = r.status + P * 4;
    return r;
}

size_t request_result_bytes(size_t P) { return result_layout(P).status + align256(P * 4); }

// Offsets within the uploaded tables, the same on the device (from
// ws.tasks) and in the pinned staging: tasks, item_begin, item_task.
struct UploadLayout {
    size_t item_begin, item_task, bytes;
};
UploadLayout upload_layout(size_t P, size_t I) {
    UploadLayout u;
    u.item_begin = align256(P * sizeof(PairTask));
    u.item_task = u.item_begin + align256((P + 1) * sizeof(int64_t));
    u.bytes = u.item_task + I * sizeof(int32_t);
    return u;
}

// Pinned host bytes of a geometry request's results: lk, raw, status,
// counters, then its pair list.
size_t geometry_host_bytes(size_t P) { return request_result_bytes(P) + P * 2 * sizeof(int32_t); }

size_t devpack_host_bytes(int64_t T) {
    return request_result_bytes((size_t)T) + align256((size_t)T * 2 * sizeof(int32_t)) + geometry_sum_bytes();
}

// Pinned host bytes of a request: its results, then its staged item tables.
size_t request_host_bytes(const Packed& pk) {
    const size_t P = pk.tasks.size();
    return request_result_bytes(P) + upload_layout(P, (size_t)pk.n_items).bytes;
}

}  // namespace

struct lk_server {
    lk_server_options opt;
    int device = 0;
    int num_sms = 1;
    cudaStream_t stream = nullptr;     // request setup and the bulk waves
    cudaStream_t finish = nullptr;     // each finished request's careful passes, FP64 fix, reduction, copies
    cudaStream_t prep = nullptr;       // geometry requests' search and packing
    Request* stalled = nullptr;        // the first geometry request of this step left waiting for room
    std::vector<Packed> pk_pool;       // packed tables of admitted requests, reused by later submits
    unsigned char* d_arena = nullptr;
    unsigned char* h_arena = nullptr;
    Arena dev, host;
    std::deque<Request*> queue;
    std::vector<Request*> running;     // admitted, in admission order
    std::map<int64_t, Request*> all;
    std::deque<int64_t> finished;      // tickets done and not yet reported by lk_server_completed
    std::deque<Wave> waves;
    bool slot_busy[kWaveSlots] = {};
    lk::WaveSeg* h_segs[kWaveSlots] = {};   // pinned staging of each slot's runs
    lk::WaveSeg* d_segs[kWaveSlots] = {};
    unsigned long long* d_counters = nullptr;  // 2 per slot
    int64_t next_ticket = 1;
    lk_server_stats st{};
    std::string err;
};

namespace {

lk_status srv_fail(lk_server* s, lk_status st, const std::string& m) {
    if (s) s->err = m;
    set_global_error(m);
    return st;
}

#define LK_SRV_CUDA(srv, call)                                                              \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess)                                                              \
            return srv_fail(srv, e_ == cudaErrorMemoryAllocation ? LK_ERR_OOM : LK_ERR_CUDA, \
                            std::string(#call) + ": " + cudaGetErrorString(e_));            \
    } while (0)

lk::SweepArgs request_args(lk_ctx* ctx, Workspace& ws, int64_t n_tasks, int64_t n_items, int near_cap) {
    lk::SweepArgs a{};
    a.tasks = ws.tasks.p;
    a.item_begin = ws.item_begin.p;
    a.item_task = ws.item_task.p;
    a.n_items = n_items;
    a.n_tasks = n_tasks;
    a.partial = ws.partial.p;
    a.item_counter = ws.counters.p + 4;
    a.overflow = ws.counters.p + 1;
    unsigned int* u32 = reinterpret_cast<unsigned int*>(ws.counters.p + 2);
    a.careful_count = u32 + 0;
    a.careful_counter = u32 + 1;
    a.near_count = u32 + 2;
    a.careful_items = ws.careful_items.p;
    a.careful_chunks = ws.careful_chunks.p;
    a.chunk_capacity = (int)std::min<size_t>(ws.careful_chunks.cap, (size_t)INT32_MAX);
    a.chunk_count = u32 + 6;     // low half of counters[5]
    a.chunk_counter = u32 + 7;   // high half of counters[5], low half of counters[6]
    a.item_fix = ws.item_fix.p;
    a.near_list = ws.near_list.p;
    a.near_capacity = near_cap;
    a.fix_acc = ws.fix_acc.p;
    a.fp64_count = ws.fp64_count.p;
    a.flags = ws.flags.p;
    a.near_ratio_sq = (float)(ctx->opt.near_ratio * ctx->opt.near_ratio);
    return a;
}

void take_counts(Request* r) {
    r->n_tasks = (int64_t)r->pk.tasks.size();
    r->n_items = r->pk.n_items;
    r->n_acc_items = r->pk.n_acc_items;
    r->n_chunks = r->pk.n_chunks;
}

// Retire finished waves (block on the oldest when `block`).
lk_status retire(lk_server* s, bool block) {
    while (!s->waves.empty()) {
        Wave& w = s->waves.front();
        cudaError_t e = block ? cudaEventSynchronize(w.done) : cudaEventQuery(w.done);
        if (e == cudaErrorNotReady) break;
        if (e != cudaSuccess) return srv_fail(s, LK_ERR_CUDA, std::string("lk_server_step: ") + cudaGetErrorString(e));
        block = false;
        for (Request* r : w.completing) {
            r->state = kDone;
            s->finished.push_back(r->ticket);
            // counters: [1] FP64 recomputes evaluated in place, [2] low half the
            // whole-item hand-overs, [5] low half the chunk hand-overs
            s->st.near_overflow += (int64_t)r->h_counters[1];
            s->st.careful_items += (int64_t)(uint32_t)r->h_counters[2];
            s->st.careful_chunks += (int64_t)(uint32_t)r->h_counters[5];
            s->dev.release(r->dev_off, r->dev_bytes);
            if (r->blk_bytes) s->dev.release(r->blk_off, r->blk_bytes);
            r->blk_bytes = 0;
            auto it = std::find(s->running.begin(), s->running.end(), r);
            if (it != s->running.end()) s->running.erase(it);
            s->st.completed += 1;
        }
        cudaEventDestroy(w.done);
        if (w.swept) cudaEventDestroy(w.swept);
        s->slot_busy[w.slot] = false;
        s->waves.pop_front();
    }
    return LK_OK;
}

// A geometry request that ends without waves (no candidate pairs, or an
// error): release what it holds and report it done.
void complete_now(lk_server* s, Request* r, lk_status error, const std::string& msg) {
    if (r->scr_bytes) s->dev.release(r->scr_off, r->scr_bytes);
    if (r->blk_bytes) s->dev.release(r->blk_off, r->blk_bytes);
    if (r->dev_bytes) s->dev.release(r->dev_off, r->dev_bytes);
    if (r->sum_bytes) s->host.release(r->sum_off, r->sum_bytes);
    if (r->host_bytes) s->host.release(r->host_off, r->host_bytes);
    r->scr_bytes = r->blk_bytes = r->dev_bytes = r->sum_bytes = r->host_bytes = 0;
    r->error = error;
    if (error != LK_OK) {
        r->n_tasks = 0;
        r->error_msg = msg;
    }
    r->state = kDone;
    s->finished.push_back(r->ticket);
    auto it = std::find(s->running.begin(), s->running.end(), r);
    if (it != s->running.end()) s->running.erase(it);
    s->st.completed += 1;
}

// Pinned result pointers of a request's host block (results, then for a
// geometry request its pair list).
void bind_results(lk_server* s, Request* r) {
    const size_t P = (size_t)r->n_tasks;
    unsigned char* hb = s->h_arena + r->host_off;
    const ResultLayout L = result_layout(P);
    r->h_counters = reinterpret_cast<unsigned long long*>(hb);
    r->h_lk = reinterpret_cast<int32_t*>(hb + L.lk);
    r->h_raw = reinterpret_cast<double*>(hb + L.raw);
    r->h_status = reinterpret_cast<int32_t*>(hb + L.status);
    r->h_pairs = reinterpret_cast<int32_t*>(hb + request_result_bytes(P));
}

// The request's buffers that start at zero (item_fix .. counters, one
// contiguous range of its work block), cleared with one memset.
cudaError_t zero_request(const Workspace& ws, cudaStream_t st) {
    unsigned char* a = reinterpret_cast<unsigned char*>(ws.item_fix.p);
    unsigned char* b = reinterpret_cast<unsigned char*>(ws.counters.p + 8);
    return cudaMemsetAsync(a, 0, (size_t)(b - a), st);
}

// Admission of a geometry request: the potential link search's count pass
// and the scan of its counts on the preparation stream (after the work that
// preceded the submit on the server's stream); the candidate count is read
// back without waiting.  Returns false when the arena has no room yet.
bool start_search(lk_server* s, Request* r, lk_status* err) {
    lk_ctx* ctx = r->ctx;
    const int64_t L = ctx->n_loops;
    *err = LK_OK;
    SearchBufs sb;
    r->scr_bytes = search_layout(L, r->sweep, &sb, 0);
    if (!s->dev.alloc(r->scr_bytes, &r->scr_off)) {
        r->scr_bytes = 0;
        return false;
    }
    r->sum_bytes = geometry_sum_bytes();
    if (!s->host.alloc(r->sum_bytes, &r->sum_off)) {
        s->dev.release(r->scr_off, r->scr_bytes);
        r->scr_bytes = r->sum_bytes = 0;
        return false;
    }
    search_layout(L, r->sweep, &sb, (uintptr_t)(s->d_arena + r->scr_off));
    unsigned char* hb = s->h_arena + r->sum_off;
    r->h_sum = reinterpret_cast<long long*>(hb);
    cudaStream_t st = s->prep;
    auto check = [&](cudaError_t e) {
        if (e != cudaSuccess && *err == LK_OK) {
            *err = LK_ERR_CUDA;
            s->err = std::string("lk_server_step (search): ") + cudaGetErrorString(e);
        }
    };
    check(cudaStreamWaitEvent(st, r->ev, 0));   // the submit's fence on the server's stream
    if (r->tuned) {
        int32_t* h_tune = reinterpret_cast<int32_t*>(hb + kSumBytes);
        std::fill(h_tune, h_tune + lk::kTuneClasses * lk::kTuneClasses, 0);
        for (const auto& kv : ctx->tune) {
            const uint32_t rc = kv.first >> 8, cc = kv.first & 0xffu;
            if (rc < (uint32_t)lk::kTuneClasses && cc < (uint32_t)lk::kTuneClasses)
                h_tune[rc * lk::kTuneClasses + cc] = kv.second;
        }
        check(cudaMemcpyAsync(sb.tune, h_tune, (size_t)lk::kTuneClasses * lk::kTuneClasses * sizeof(int32_t),
                              cudaMemcpyHostToDevice, st));
    }
    lk::launch_pls_keys(ctx->d_aabb, L, sb.keys, st);
    if (r->sweep) {
        lk::launch_pls_sort(sb.keys, L, sb.order, lk::pls_sort_size(L), st);
        lk::launch_pls_sweep_count(sb.keys, L, sb.order, sb.counts, st);
    } else {
        lk::launch_pls_count(sb.keys, L, sb.counts, st);
    }
    lk::launch_scan_counts(sb.counts, L, sb.offsets, sb.scan, st);
    check(cudaMemcpyAsync(r->h_sum, sb.offsets + L, sizeof(long long), cudaMemcpyDeviceToHost, st));
    check(cudaGetLastError());
    check(cudaEventRecord(r->ev, st));
    return true;
}

// Admission of a pair-list request packed on the device: its list staged in
// pinned memory and uploaded, then the device packer (as for a geometry
// request's candidates) on the preparation stream; the totals are read back
// without waiting.  Returns false when the arenas have no room yet.
bool start_devpack(lk_server* s, Request* r, lk_status* err) {
    lk_ctx* ctx = r->ctx;
    const int64_t T = r->n_tasks;
    *err = LK_OK;
    const size_t blk = devpack_dev_bytes(T), hbytes = devpack_host_bytes(T);
    if (!s->dev.alloc(blk, &r->blk_off)) return false;
    if (!s->host.alloc(hbytes, &r->host_off)) {
        s->dev.release(r->blk_off, blk);
        return false;
    }
    r->blk_bytes = blk;
    r->host_bytes = hbytes;
    bind_results(s, r);                               // h_pairs: the staged list
    unsigned char* hb = s->h_arena + r->host_off;
    r->h_sum = reinterpret_cast<long long*>(hb + request_result_bytes((size_t)T) +
                                            align256((size_t)T * 2 * sizeof(int32_t)));
    std::memcpy(r->h_pairs, r->pairs.data(), (size_t)T * 2 * sizeof(int32_t));
    PackBufs pb;
    const size_t off = pack_layout(T, &pb, (uintptr_t)(s->d_arena + r->blk_off));
    int32_t* d_tune = reinterpret_cast<int32_t*>(s->d_arena + r->blk_off + align256(off));
    cudaStream_t st = s->prep;
    auto check = [&](cudaError_t e) {
        if (e != cudaSuccess && *err == LK_OK) {
            *err = LK_ERR_CUDA;
            s->err = std::string("lk_server_step (device packing): ") + cudaGetErrorString(e);
        }
    };
    if (!r->ev) check(cudaEventCreateWithFlags(&r->ev, cudaEventDisableTiming));
    check(cudaMemcpyAsync(pb.pairs, r->h_pairs, (size_t)T * 2 * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    if (r->tuned) {
        int32_t* h_tune = reinterpret_cast<int32_t*>(reinterpret_cast<unsigned char*>(r->h_sum) + kSumBytes);
        std::fill(h_tune, h_tune + lk::kTuneClasses * lk::kTuneClasses, 0);
        for (const auto& kv : ctx->tune) {
            const uint32_t rc = kv.first >> 8, cc = kv.first & 0xffu;
            if (rc < (uint32_t)lk::kTuneClasses && cc < (uint32_t)lk::kTuneClasses)
                h_tune[rc * lk::kTuneClasses + cc] = kv.second;
        }
        check(cudaMemcpyAsync(d_tune, h_tune, (size_t)lk::kTuneClasses * lk::kTuneClasses * sizeof(int32_t),
                              cudaMemcpyHostToDevice, st));
    }
    const lk::PackParams P{ctx->d_V, ctx->d_R, ctx->d_offsets, r->tuned ? d_tune : nullptr,
                           ctx->opt.accurate_threshold, ctx->opt.tile_rows, (int32_t)ctx->n_loops};
    lk::launch_pack(pb.pairs, T, P, pb.tasks, pb.sums, pb.scan, pb.scratch, pb.item_begin, st);
    check(cudaMemcpyAsync(r->h_sum + 1, pb.scan + T, sizeof(lk::PackSums), cudaMemcpyDeviceToHost, st));
    check(cudaGetLastError());
    check(cudaEventRecord(r->ev, st));
    r->d_pairs = pb.pairs;
    r->ws.tasks.p = pb.tasks;
    r->ws.tasks.cap = (size_t)T;
    r->ws.item_begin.p = pb.item_begin;
    r->ws.item_begin.cap = (size_t)T + 1;
    return true;
}

// Advance geometry requests whose search or packing has finished on the
// device (polled, never waited for).
lk_status advance_geometry(lk_server* s) {
    std::vector<Request*> todo;
    s->stalled = nullptr;
    for (Request* r : s->running)
        if (r->state == kSearching || r->state == kPacking) todo.push_back(r);
    for (Request* r : todo) {
        const cudaError_t q = cudaEventQuery(r->ev);
        if (q == cudaErrorNotReady) continue;
        if (q != cudaSuccess) return srv_fail(s, LK_ERR_CUDA, std::string("lk_server_step: ") + cudaGetErrorString(q));
        lk_ctx* ctx = r->ctx;
        const int64_t L = ctx->n_loops;
        if (r->state == kSearching) {
            const int64_t T = r->h_sum[0];
            if (T == 0) {
                complete_now(s, r, LK_OK, "");
                continue;
            }
            if (T > (int64_t)INT32_MAX) {
                complete_now(s, r, LK_ERR_ARG, "lk_server_submit_geometry: more than 2^31 candidate pairs");
                continue;
            }
            PackBufs pb;
            const size_t blk = pack_layout(T, &pb, 0), hbytes = geometry_host_bytes((size_t)T);
            if (Arena::round(blk) > s->opt.arena_bytes || Arena::round(hbytes) > s->opt.host_bytes) {
                complete_now(s, r, LK_ERR_OOM, "lk_server_submit_geometry: the candidate pairs exceed the server's arena");
                continue;
            }
            if (!s->dev.alloc(blk, &r->blk_off)) {                     // wait for room
                if (!s->stalled) s->stalled = r;
                continue;
            }
            if (!s->host.alloc(hbytes, &r->host_off)) {
                s->dev.release(r->blk_off, blk);
                if (!s->stalled) s->stalled = r;
                continue;
            }
            r->blk_bytes = blk;
            r->host_bytes = hbytes;
            r->n_tasks = T;
            bind_results(s, r);
            pack_layout(T, &pb, (uintptr_t)(s->d_arena + r->blk_off));
            SearchBufs sb;
            search_layout(L, r->sweep, &sb, (uintptr_t)(s->d_arena + r->scr_off));
            const lk::PackParams P{ctx->d_V, ctx->d_R, ctx->d_offsets, r->tuned ? sb.tune : nullptr,
                                   ctx->opt.accurate_threshold, ctx->opt.tile_rows, (int32_t)ctx->n_loops};
            cudaStream_t st = s->prep;
            const unsigned npk = lk::pls_sort_size(T);
            if (r->sweep) {
                LK_SRV_CUDA(s, cudaMemsetAsync(pb.keys, 0xff, (size_t)npk * sizeof(unsigned long long), st));
                lk::launch_pls_sweep_write(sb.keys, L, sb.order, sb.offsets, pb.keys, T, st);
                lk::launch_bitonic_sort(pb.keys, npk, st);
                lk::launch_pls_unpack(pb.keys, T, pb.pairs, st);
            } else {
                lk::launch_pls_write(sb.keys, L, sb.offsets, pb.pairs, T, st);
            }
            lk::launch_pack(pb.pairs, T, P, pb.tasks, pb.sums, pb.scan, pb.scratch, pb.item_begin, st);
            LK_SRV_CUDA(s, cudaMemcpyAsync(r->h_sum + 1, pb.scan + T, sizeof(lk::PackSums), cudaMemcpyDeviceToHost, st));
            LK_SRV_CUDA(s, cudaGetLastError());
            LK_SRV_CUDA(s, cudaEventRecord(r->ev, st));
            r->d_pairs = pb.pairs;
            r->ws.tasks.p = pb.tasks;
            r->ws.tasks.cap = (size_t)T;
            r->ws.item_begin.p = pb.item_begin;
            r->ws.item_begin.cap = (size_t)T + 1;
            r->state = kPacking;
            continue;
        }
        // kPacking: the totals are in; lay out the work buffers and start.
        lk::PackSums tot;
        std::memcpy(&tot, r->h_sum + 1, sizeof tot);
        const int64_t T = r->n_tasks;
        const int64_t n_items = tot.acc_items + tot.fast_items;
        if (n_items > (int64_t)INT32_MAX * 16) {
            complete_now(s, r, LK_ERR_ARG, "lk_server_submit_geometry: too many work items");
            continue;
        }
        Workspace probe;
        const size_t need = request_layout(T, n_items, tot.chunks, false, s->opt.near_capacity, &probe, 0);
        if (Arena::round(need) > s->opt.arena_bytes) {
            complete_now(s, r, LK_ERR_OOM, "lk_server_submit_geometry: request larger than the server's arena");
            continue;
        }
        if (!s->dev.alloc(need, &r->dev_off)) {                       // wait for room
            if (!s->stalled) s->stalled = r;
            continue;
        }
        r->dev_bytes = need;
        r->n_items = n_items;
        r->n_acc_items = tot.acc_items;
        r->n_chunks = tot.chunks;
        request_layout(T, r->n_items, r->n_chunks, false, s->opt.near_capacity, &r->ws,
                       (uintptr_t)(s->d_arena + r->dev_off));
        if (r->scr_bytes) s->dev.release(r->scr_off, r->scr_bytes);
        if (r->sum_bytes) s->host.release(r->sum_off, r->sum_bytes);
        r->scr_bytes = r->sum_bytes = 0;
        r->h_sum = nullptr;
        cudaStream_t st = s->stream;
        lk::launch_pack_item_task(r->ws.item_begin.p, T, r->n_items, r->ws.item_task.p, st);
        LK_SRV_CUDA(s, zero_request(r->ws, st));
        lk::launch_pair_frames(r->ws.tasks.p, T, ctx->d_aabb, st);
        LK_SRV_CUDA(s, cudaGetLastError());
        r->args = request_args(ctx, r->ws, T, r->n_items, s->opt.near_capacity);
        r->state = kRunning;
        r->next_item = 0;
        if (r->geometry) s->st.candidate_pairs += T;
    }
    return LK_OK;
}

// Admit queued requests in arrival order while slots and arena space last.
lk_status admit(lk_server* s) {
    while (!s->queue.empty() && (int)s->running.size() < s->opt.max_requests) {
        Request* r = s->queue.front();
        lk_ctx* ctx = r->ctx;
        if (r->dev_pack) {
            lk_status err = LK_OK;
            if (!start_devpack(s, r, &err)) break;      // no room yet
            if (err != LK_OK) return err;
            r->state = kPacking;
            s->running.push_back(r);
            s->queue.pop_front();
            s->st.admitted += 1;
            continue;
        }
        if (r->geometry) {
            s->running.push_back(r);
            s->queue.pop_front();
            s->st.admitted += 1;
            if (ctx->n_loops < 2) {
                complete_now(s, r, LK_OK, "");
                continue;
            }
            lk_status err = LK_OK;
            if (!start_search(s, r, &err)) {
                // no room yet: back to the head of the queue
                s->running.pop_back();
                s->queue.push_front(r);
                s->st.admitted -= 1;
                break;
            }
            if (err != LK_OK) return err;
            r->state = kSearching;
            continue;
        }
        if (!r->packed) {
            lk_status st = pack_pairs(ctx, r->pairs.data(), (int64_t)(r->pairs.size() / 2), r->pk);
            if (st != LK_OK) return srv_fail(s, st, ctx->err);
            r->packed = true;
            take_counts(r);
            Workspace probe;
            r->dev_bytes = request_layout(r->pk, s->opt.near_capacity, &probe, 0);
            r->host_bytes = request_host_bytes(r->pk);
        }
        if (!s->dev.alloc(r->dev_bytes, &r->dev_off)) break;           // memory-based admission
        if (!s->host.alloc(r->host_bytes, &r->host_off)) {
            s->dev.release(r->dev_off, r->dev_bytes);
            break;
        }
        request_layout(r->pk, s->opt.near_capacity, &r->ws, (uintptr_t)(s->d_arena + r->dev_off));
        const size_t P = (size_t)r->n_tasks;
        bind_results(s, r);
        r->args = request_args(ctx, r->ws, r->n_tasks, r->n_items, s->opt.near_capacity);
        // Stage the item tables in pinned memory so that their upload is truly
        // asynchronous (a pageable source would make the copy wait for the
        // waves already queued on the stream, serialising host and device),
        // laid out as on the device so that one copy carries them.
        unsigned char* tb = s->h_arena + r->host_off + request_result_bytes(P);
        const UploadLayout U = upload_layout(P, (size_t)r->n_items);
        std::memcpy(tb, r->pk.tasks.data(), P * sizeof(PairTask));
        std::memcpy(tb + U.item_begin, r->pk.item_begin.data(), (P + 1) * sizeof(int64_t));
        if (r->n_items) std::memcpy(tb + U.item_task, r->pk.item_task.data(), (size_t)r->n_items * sizeof(int32_t));
        // the tables live on in pinned memory and on the device: their host
        // vectors go back to the pool (a few, of at most 2^20 pairs, to bound
        // the memory kept)
        if (s->pk_pool.size() < 8 && r->pk.tasks.capacity() <= ((size_t)1 << 20))
            s->pk_pool.push_back(std::move(r->pk));
        r->pk = Packed();
        LK_SRV_CUDA(s, cudaMemcpyAsync(r->ws.tasks.p, tb, U.bytes, cudaMemcpyHostToDevice, s->stream));
        const int64_t n = (int64_t)P;
        LK_SRV_CUDA(s, zero_request(r->ws, s->stream));
        lk::launch_pair_frames(r->ws.tasks.p, n, ctx->d_aabb, s->stream);
        r->state = kRunning;
        r->next_item = 0;
        s->running.push_back(r);
        s->queue.pop_front();
        s->st.admitted += 1;
    }
    return LK_OK;
}

// Launch one wave over the admitted requests' next items.
lk_status launch_wave(lk_server* s) {
    int slot = -1;
    for (int k = 0; k < kWaveSlots; ++k)
        if (!s->slot_busy[k]) { slot = k; break; }
    if (slot < 0) return LK_OK;
    bool any = false;
    for (Request* r : s->running)
        if (r->state == kRunning) { any = true; break; }
    if (!any) return LK_OK;

    lk::WaveSeg* segs = s->h_segs[slot];
    int n_acc = 0, n_fast = 0;   // runs stored as [acc runs..., then fast runs from the end]
    int64_t acc_items = 0, fast_items = 0;
    int64_t budget = s->opt.wave_items;
    std::vector<Request*> completing;
    int64_t touched = 0;
    std::vector<Request*> order;
    order.reserve(s->running.size());
    for (Request* r : s->running)
        if (r->state == kRunning) order.push_back(r);
    if (s->opt.wave_order == 1)        // fewest items left first; ties in admission order
        std::stable_sort(order.begin(), order.end(), [](const Request* a, const Request* b) {
            return a->n_items - a->next_item < b->n_items - b->next_item;
        });
    for (Request* r : order) {
        if (budget <= 0 || n_acc + n_fast + 2 > kMaxSegs) continue;
        ++touched;
        const int64_t lo = r->next_item, hi = std::min<int64_t>(r->n_items, lo + budget);
        // accurate items are [0, n_acc_items), fast items after them
        const int64_t a_lo = lo, a_hi = std::min(hi, r->n_acc_items);
        const int64_t f_lo = std::max(lo, r->n_acc_items), f_hi = hi;
        if (a_hi > a_lo) {
            segs[n_acc] = lk::WaveSeg{r->args, a_lo, acc_items};
            acc_items += a_hi - a_lo;
            ++n_acc;
        }
        if (f_hi > f_lo) {
            segs[kMaxSegs - 1 - n_fast] = lk::WaveSeg{r->args, f_lo, fast_items};
            fast_items += f_hi - f_lo;
            ++n_fast;
        }
        budget -= hi - lo;
        r->next_item = hi;
        if (hi >= r->n_items) {
            r->state = kLaunched;
            completing.push_back(r);
        }
    }
    // fast runs were written backwards from the end; put them after the accurate ones
    std::reverse(segs + kMaxSegs - n_fast, segs + kMaxSegs);
    std::copy(segs + kMaxSegs - n_fast, segs + kMaxSegs, segs + n_acc);
    cudaStream_t st = s->stream;
    LK_SRV_CUDA(s, cudaMemcpyAsync(s->d_segs[slot], segs, (size_t)(n_acc + n_fast) * sizeof(lk::WaveSeg),
                                   cudaMemcpyHostToDevice, st));
    unsigned long long* cnt = s->d_counters + 2 * slot;
    LK_SRV_CUDA(s, cudaMemsetAsync(cnt, 0, 2 * sizeof(unsigned long long), st));
    lk::launch_wave(s->d_segs[slot], n_acc, acc_items, true, cnt, s->num_sms * lk::wave_blocks_per_sm(true), st);
    lk::launch_wave(s->d_segs[slot] + n_acc, n_fast, fast_items, false, cnt + 1,
                    s->num_sms * lk::wave_blocks_per_sm(false), st);
    // The finishing work of the requests whose last items this wave holds runs
    // on the second stream, after the wave: the next wave's bulk launches (on
    // the first stream) overlap it instead of waiting behind these small,
    // latency-bound kernels.  It touches only those requests' buffers.
    Wave w;
    w.slot = slot;
    w.completing = completing;
    if (!completing.empty()) {
        LK_SRV_CUDA(s, cudaEventCreateWithFlags(&w.swept, cudaEventDisableTiming));
        LK_SRV_CUDA(s, cudaEventRecord(w.swept, st));
        LK_SRV_CUDA(s, cudaStreamWaitEvent(s->finish, w.swept, 0));
        st = s->finish;
    }
    for (Request* r : completing) {
        const bool fast = r->n_items > r->n_acc_items, acc = r->n_acc_items > 0;
        lk::launch_careful_chunks(r->args, fast, acc, s->num_sms * lk::careful_chunk_blocks_per_sm(), st);
        lk::launch_sweep_careful(r->args, fast, acc, s->num_sms * lk::sweep_careful_blocks_per_sm(), st);
        lk::launch_near_fix(r->args, s->num_sms * 4, st);
        lk::ReduceArgs ra{};
        ra.tasks = r->ws.tasks.p;
        ra.item_begin = r->ws.item_begin.p;
        ra.partial = r->ws.partial.p;
        ra.fix_acc = r->ws.fix_acc.p;
        ra.item_fix = r->ws.item_fix.p;
        ra.flags = r->ws.flags.p;
        ra.n_tasks = r->n_tasks;
        ra.int_tol = r->ctx->opt.int_tol;
        ra.lk_out = r->ws.lk.p;
        ra.raw_out = r->ws.raw.p;
        ra.status_out = r->ws.status.p;
        lk::launch_reduce(ra, st);
        const size_t P = (size_t)r->n_tasks;
        // counters, lk, raw and status in one copy (the same layout on both sides)
        LK_SRV_CUDA(s, cudaMemcpyAsync(r->h_counters, r->ws.counters.p, result_layout(P).copy_bytes,
                                       cudaMemcpyDeviceToHost, st));
        if (r->geometry)
            LK_SRV_CUDA(s, cudaMemcpyAsync(r->h_pairs, r->d_pairs, P * 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    }
    LK_SRV_CUDA(s, cudaGetLastError());
    LK_SRV_CUDA(s, cudaEventCreateWithFlags(&w.done, cudaEventDisableTiming));
    LK_SRV_CUDA(s, cudaEventRecord(w.done, st));
    s->slot_busy[slot] = true;
    s->waves.push_back(w);
    s->st.waves += 1;
    s->st.max_requests_per_wave = std::max<int64_t>(s->st.max_requests_per_wave, touched);
    s->st.items_launched += acc_items + fast_items;
    return LK_OK;
}

}  // namespace

extern "C" {

void lk_server_default_options(lk_server_options* o) {
    if (!o) return;
    o->max_requests = 64;
    o->arena_bytes = (size_t)1 << 30;
    o->host_bytes = (size_t)256 << 20;
    o->wave_items = 16384;
    o->near_capacity = 1 << 16;
    o->max_queue = 1 << 16;
    o->wave_order = 0;
    o->pack_on_device = 1;
}

lk_status lk_server_create(lk_server** out, const lk_server_options* opt) {
    if (!out) return srv_fail(nullptr, LK_ERR_ARG, "lk_server_create: out is NULL");
    *out = nullptr;
    lk_server_options o;
    lk_server_default_options(&o);
    if (opt) o = *opt;
    if (o.max_requests < 1 || o.wave_items < 1 || o.near_capacity < 1 || o.arena_bytes < 4096 ||
        o.host_bytes < 4096 || o.max_queue < 1 || o.wave_order < 0 || o.wave_order > 1 ||
        o.pack_on_device < 0 || o.pack_on_device > 1)
        return srv_fail(nullptr, LK_ERR_ARG, "lk_server_create: invalid options");
    lk_server* s = new lk_server();
    s->opt = o;
    cudaGetDevice(&s->device);
    cudaDeviceGetAttribute(&s->num_sms, cudaDevAttrMultiProcessorCount, s->device);
    cudaError_t e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->finish, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->prep, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc(&s->d_arena, o.arena_bytes);
    if (e == cudaSuccess) e = cudaHostAlloc(&s->h_arena, o.host_bytes, cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaMalloc(&s->d_counters, 2 * kWaveSlots * sizeof(unsigned long long));
    for (int k = 0; k < kWaveSlots && e == cudaSuccess; ++k) {
        e = cudaHostAlloc(&s->h_segs[k], kMaxSegs * sizeof(lk::WaveSeg), cudaHostAllocDefault);
        if (e == cudaSuccess) e = cudaMalloc(&s->d_segs[k], kMaxSegs * sizeof(lk::WaveSeg));
    }
    if (e != cudaSuccess) {
        lk_server_destroy(s);
        return srv_fail(nullptr, e == cudaErrorMemoryAllocation ? LK_ERR_OOM : LK_ERR_CUDA,
                        std::string("lk_server_create: ") + cudaGetErrorString(e));
    }
    s->dev.init(o.arena_bytes);
    s->host.init(o.host_bytes);
    *out = s;
    return LK_OK;
}

void* lk_server_stream(lk_server* s) { return s ? (void*)s->stream : nullptr; }

lk_status lk_server_submit(lk_server* s, lk_ctx* ctx, const int32_t* loop_pairs, int64_t n_pairs,
                           int64_t* ticket) {
    if (!s) return srv_fail(nullptr, LK_ERR_ARG, "lk_server_submit: NULL server");
    if (!ctx || !ticket || n_pairs < 1 || n_pairs > INT32_MAX || !loop_pairs)
        return srv_fail(s, LK_ERR_ARG, "lk_server_submit: invalid arguments");
    if (ctx->opt.precision != LK_MIXED)
        return srv_fail(s, LK_ERR_ARG, "lk_server_submit: the server runs the mixed-precision path");
    if ((int64_t)s->queue.size() >= s->opt.max_queue)
        return srv_fail(s, LK_ERR_BUSY, "lk_server_submit: queue full");
    Request* r = new Request();
    r->ctx = ctx;
    r->pairs.resize((size_t)(2 * n_pairs));
    if (is_device_ptr(loop_pairs)) {
        if (cudaMemcpy(r->pairs.data(), loop_pairs, 2 * n_pairs * sizeof(int32_t), cudaMemcpyDeviceToHost) != cudaSuccess) {
            delete r;
            return srv_fail(s, LK_ERR_CUDA, "lk_server_submit: cannot read loop_pairs");
        }
    } else {
        std::memcpy(r->pairs.data(), loop_pairs, 2 * n_pairs * sizeof(int32_t));
    }
    if (s->opt.pack_on_device) {
        // the list is packed on the device at admission; only its pack block
        // and pinned block can be checked against the arenas now
        r->dev_pack = true;
        r->packed = true;
        r->n_tasks = n_pairs;
        r->tuned = ctx->opt.tile_rows <= 0 && !ctx->tune.empty();
        if (Arena::round(devpack_dev_bytes(n_pairs)) > s->opt.arena_bytes ||
            Arena::round(devpack_host_bytes(n_pairs)) > s->opt.host_bytes) {
            delete r;
            return srv_fail(s, LK_ERR_OOM, "lk_server_submit: request larger than the server's arena");
        }
        r->ticket = s->next_ticket++;
        s->queue.push_back(r);
        s->all[r->ticket] = r;
        s->st.submitted += 1;
        *ticket = r->ticket;
        return LK_OK;
    }
    // A request that could never fit is refused now rather than blocking the queue.
    if (!s->pk_pool.empty()) {
        r->pk = std::move(s->pk_pool.back());          // vectors with capacity already
        s->pk_pool.pop_back();
    }
    lk_status st = pack_pairs(ctx, r->pairs.data(), n_pairs, r->pk);
    if (st != LK_OK) {
        delete r;
        return srv_fail(s, st, ctx->err);
    }
    r->packed = true;
    take_counts(r);
    Workspace probe;
    r->dev_bytes = request_layout(r->pk, s->opt.near_capacity, &probe, 0);
    r->host_bytes = request_host_bytes(r->pk);
    if (Arena::round(r->dev_bytes) > s->opt.arena_bytes || Arena::round(r->host_bytes) > s->opt.host_bytes) {
        delete r;
        return srv_fail(s, LK_ERR_OOM, "lk_server_submit: request larger than the server's arena");
    }
    r->ticket = s->next_ticket++;
    s->queue.push_back(r);
    s->all[r->ticket] = r;
    s->st.submitted += 1;
    *ticket = r->ticket;
    return LK_OK;
}

lk_status lk_server_submit_geometry(lk_server* s, lk_ctx* ctx, int64_t* ticket) {
    if (!s) return srv_fail(nullptr, LK_ERR_ARG, "lk_server_submit_geometry: NULL server");
    if (!ctx || !ticket) return srv_fail(s, LK_ERR_ARG, "lk_server_submit_geometry: invalid arguments");
    if (ctx->opt.precision != LK_MIXED)
        return srv_fail(s, LK_ERR_ARG, "lk_server_submit_geometry: the server runs the mixed-precision path");
    if (ctx->n_loops > (int64_t)1 << 30) return srv_fail(s, LK_ERR_ARG, "lk_server_submit_geometry: too many loops");
    if ((int64_t)s->queue.size() >= s->opt.max_queue)
        return srv_fail(s, LK_ERR_BUSY, "lk_server_submit_geometry: queue full");
    const int64_t L = ctx->n_loops;
    Request* r = new Request();
    r->ctx = ctx;
    r->geometry = true;
    r->packed = true;
    // the same choice of search as lk_candidates
    r->sweep = L * (L - 1) / 2 > ((int64_t)1 << 27);
    r->tuned = ctx->opt.tile_rows <= 0 && !ctx->tune.empty();
    SearchBufs sb;
    if (Arena::round(search_layout(std::max<int64_t>(L, 1), r->sweep, &sb, 0)) > s->opt.arena_bytes ||
        Arena::round(geometry_sum_bytes()) > s->opt.host_bytes) {
        delete r;
        return srv_fail(s, LK_ERR_OOM, "lk_server_submit_geometry: the search alone exceeds the server's arena");
    }
    // The search reads the context's boxes after the work enqueued on the
    // server's stream so far (an lk_update there, say).
    if (cudaEventCreateWithFlags(&r->ev, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventRecord(r->ev, s->stream) != cudaSuccess) {
        cudaGetLastError();
        delete r;
        return srv_fail(s, LK_ERR_CUDA, "lk_server_submit_geometry: cannot record the request's fence");
    }
    r->ticket = s->next_ticket++;
    s->queue.push_back(r);
    s->all[r->ticket] = r;
    s->st.submitted += 1;
    s->st.geometry_requests += 1;
    *ticket = r->ticket;
    return LK_OK;
}

lk_status lk_server_step(lk_server* s, int wait) {
    if (!s) return srv_fail(nullptr, LK_ERR_ARG, "lk_server_step: NULL server");
    lk_status st = retire(s, false);
    if (st != LK_OK) return st;
    if ((st = advance_geometry(s)) != LK_OK) return st;
    if ((st = admit(s)) != LK_OK) return st;
    if ((st = launch_wave(s)) != LK_OK) return st;
    if (s->stalled && s->waves.empty()) {
        // Nothing in flight will release memory: the geometry requests holding
        // the arena wait on one another.  The oldest waiting one gives up.
        bool busy = false;
        for (Request* r : s->running) {
            if (r->state == kRunning || r->state == kLaunched) busy = true;
            if ((r->state == kSearching || r->state == kPacking) && cudaEventQuery(r->ev) == cudaErrorNotReady) busy = true;
        }
        cudaGetLastError();
        if (!busy)
            complete_now(s, s->stalled, LK_ERR_OOM,
                         "lk_server_submit_geometry: no arena room while the other geometry requests hold it");
        s->stalled = nullptr;
    }
    if (wait && !s->waves.empty() && (st = retire(s, true)) != LK_OK) return st;
    if (wait && s->waves.empty()) {
        // nothing in flight but geometry requests' search or packing: wait for the oldest
        for (Request* r : s->running)
            if ((r->state == kSearching || r->state == kPacking) && r != s->stalled) {
                const cudaError_t e = cudaEventSynchronize(r->ev);
                if (e != cudaSuccess) return srv_fail(s, LK_ERR_CUDA, std::string("lk_server_step: ") + cudaGetErrorString(e));
                break;
            }
    }
    return LK_OK;
}

lk_status lk_server_completed(lk_server* s, int64_t* tickets, int64_t capacity, int64_t* n_done) {
    if (!s || !n_done || capacity < 0 || (capacity > 0 && !tickets))
        return srv_fail(s, LK_ERR_ARG, "lk_server_completed: invalid arguments");
    int64_t k = 0;
    while (k < capacity && !s->finished.empty()) {
        tickets[k++] = s->finished.front();
        s->finished.pop_front();
    }
    *n_done = k;
    return LK_OK;
}

lk_status lk_server_poll(lk_server* s, int64_t ticket, int* done, int32_t* lk_out, double* raw_out,
                         int32_t* status_out) {
    if (!s || !done) return srv_fail(s, LK_ERR_ARG, "lk_server_poll: NULL argument");
    *done = 0;
    auto it = s->all.find(ticket);
    if (it == s->all.end()) return srv_fail(s, LK_ERR_ARG, "lk_server_poll: unknown ticket");
    Request* r = it->second;
    if (r->geometry) return srv_fail(s, LK_ERR_ARG, "lk_server_poll: a geometry request is polled by lk_server_poll_pairs");
    if (r->state != kDone) return LK_OK;
    const size_t P = (size_t)r->n_tasks;
    // The pinned buffers are indexed by the caller's pair order already (the
    // reduction writes through out_index).
    if (lk_out) std::memcpy(lk_out, r->h_lk, P * 4);
    if (raw_out) std::memcpy(raw_out, r->h_raw, P * 8);
    if (status_out) std::memcpy(status_out, r->h_status, P * 4);
    s->host.release(r->host_off, r->host_bytes);
    s->all.erase(it);
    delete r;
    *done = 1;
    return LK_OK;
}

lk_status lk_server_poll_pairs(lk_server* s, int64_t ticket, int* done, int64_t* n_pairs, int32_t* pairs_out,
                               int64_t capacity, int32_t* lk_out, double* raw_out, int32_t* status_out) {
    if (!s || !done || !n_pairs || capacity < 0) return srv_fail(s, LK_ERR_ARG, "lk_server_poll_pairs: invalid arguments");
    *done = 0;
    *n_pairs = 0;
    auto it = s->all.find(ticket);
    if (it == s->all.end()) return srv_fail(s, LK_ERR_ARG, "lk_server_poll_pairs: unknown ticket");
    Request* r = it->second;
    if (r->state != kDone) return LK_OK;
    *done = 1;
    const lk_status err = r->error;
    if (err != LK_OK) {
        const std::string msg = r->error_msg;
        s->all.erase(it);
        delete r;
        return srv_fail(s, err, msg);
    }
    const size_t P = (size_t)r->n_tasks;
    *n_pairs = (int64_t)P;
    if ((int64_t)P > capacity) return LK_OK;   // the ticket stays valid for a larger buffer
    if (P > 0) {
        if (pairs_out) std::memcpy(pairs_out, r->geometry ? r->h_pairs : r->pairs.data(), P * 2 * sizeof(int32_t));
        if (lk_out) std::memcpy(lk_out, r->h_lk, P * 4);
        if (raw_out) std::memcpy(raw_out, r->h_raw, P * 8);
        if (status_out) std::memcpy(status_out, r->h_status, P * 4);
    }
    if (r->host_bytes) s->host.release(r->host_off, r->host_bytes);
    s->all.erase(it);
    delete r;
    return LK_OK;
}

lk_status lk_server_get_stats(lk_server* s, lk_server_stats* out) {
    if (!s || !out) return srv_fail(s, LK_ERR_ARG, "lk_server_get_stats: NULL argument");
    s->st.queued = (int64_t)s->queue.size();
    s->st.running = (int64_t)s->running.size();
    s->st.arena_used = (int64_t)s->dev.used;
    s->st.waves_in_flight = (int64_t)s->waves.size();
    *out = s->st;
    return LK_OK;
}

const char* lk_server_last_error(const lk_server* s) {
    if (s) return s->err.c_str();
    return lk_last_error(nullptr);
}

void lk_server_destroy(lk_server* s) {
    if (!s) return;
    if (s->stream) cudaStreamSynchronize(s->stream);
    if (s->finish) cudaStreamSynchronize(s->finish);
    if (s->prep) cudaStreamSynchronize(s->prep);
    for (Wave& w : s->waves) {
        cudaEventDestroy(w.done);
        if (w.swept) cudaEventDestroy(w.swept);
    }
    for (auto& kv : s->all) delete kv.second;
    for (int k = 0; k < kWaveSlots; ++k) {
        if (s->h_segs[k]) cudaFreeHost(s->h_segs[k]);
        if (s->d_segs[k]) cudaFree(s->d_segs[k]);
    }
    if (s->d_counters) cudaFree(s->d_counters);
    if (s->d_arena) cudaFree(s->d_arena);
    if (s->h_arena) cudaFreeHost(s->h_arena);
    if (s->stream) cudaStreamDestroy(s->stream);
    if (s->finish) cudaStreamDestroy(s->finish);
    if (s->prep) cudaStreamDestroy(s->prep);
    delete s;
}

}  // extern "C"

// ----------------------------------------------------------------------------
// Autotuner: rows per work item, per size class.
//
// The tile width is fixed by the kernel (128 column segments per warp); what
// is tuned is how many row segments a work item covers, which trades the
// per-item set-up (column staging, pair look-up, one partial) against the
// tail of the persistent grid and, for huge pairs, the number of partials.
// For every size class present in the given pair list the tuner times the
// mixed-precision verify of (a sample of) that class's pairs at each
// candidate height with CUDA events and keeps the fastest.  The table only
// changes the split, never the segment pairs evaluated; a pair's result is
// deterministic for a given table.
namespace {

const int kTuneCandidates[] = {32, 64, 128, 256, 512, 1024, 2048, 4096, 16384, 65536};
constexpr int64_t kTuneMaxSegmentPairs = (int64_t)2 << 30;   // per timed sample
constexpr int kTuneMaxPairs = 4096;

lk_status time_verify(lk_ctx* ctx, const std::vector<int32_t>& pairs, int tile_rows, cudaStream_t s,
                      cudaEvent_t e0, cudaEvent_t e1, float* ms) {
    const int saved = ctx->opt.tile_rows;
    ctx->opt.tile_rows = tile_rows;
    Packed pk;
    lk_status st = pack_pairs(ctx, pairs.data(), (int64_t)(pairs.size() / 2), pk);
    ctx->opt.tile_rows = saved;
    if (st != LK_OK) return st;
    if ((st = ensure_workspace(ctx, ctx->ws, (int64_t)pk.tasks.size(), pk.n_items, pk.n_chunks, &pk)) != LK_OK) return st;
    if ((st = upload_packed(ctx, ctx->ws, pk, s)) != LK_OK) return st;
    float best = 1e30f;
    for (int rep = 0; rep < 3; ++rep) {
        LK_CUDA(ctx, cudaEventRecord(e0, s));
        if ((st = enqueue_verify(ctx, ctx->ws, pk, s)) != LK_OK) return st;
        LK_CUDA(ctx, cudaEventRecord(e1, s));
        LK_CUDA(ctx, cudaEventSynchronize(e1));
        float m = 0.0f;
        LK_CUDA(ctx, cudaEventElapsedTime(&m, e0, e1));
        if (rep > 0) best = std::min(best, m);      // the first run warms caches
    }
    *ms = best;
    return LK_OK;
}

}  // namespace

extern "C" {

lk_status lk_autotune(lk_ctx* ctx, const int32_t* loop_pairs, int64_t n_pairs, void* cuda_stream) {
    if (!ctx) return fail(nullptr, LK_ERR_ARG, "lk_autotune: NULL context");
    if (n_pairs < 0 || (n_pairs > 0 && !loop_pairs)) return fail(ctx, LK_ERR_ARG, "lk_autotune: invalid pairs");
    if (ctx->opt.precision != LK_MIXED) return LK_OK;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    std::vector<int32_t> hp;
    lk_status st = get_pairs_on_host(ctx, loop_pairs, n_pairs, s, hp);
    if (st != LK_OK) return st;
    // group valid pairs by size class
    std::map<uint32_t, std::vector<int32_t>> groups;
    std::map<uint32_t, int64_t> group_sp, group_rows;
    for (int64_t p = 0; p < n_pairs; ++p) {
        const int32_t a = hp[2 * p], b = hp[2 * p + 1];
        if (a < 0 || b < 0 || a >= ctx->n_loops || b >= ctx->n_loops || a == b) continue;
        const int64_t na = ctx->h_offsets[a + 1] - ctx->h_offsets[a];
        const int64_t nb = ctx->h_offsets[b + 1] - ctx->h_offsets[b];
        const int64_t nr = std::max(na, nb), nc = std::min(na, nb);
        const uint32_t key = size_class(nr, nc);
        auto& g = groups[key];
        if ((int64_t)g.size() / 2 >= kTuneMaxPairs || group_sp[key] + nr * nc > kTuneMaxSegmentPairs) continue;
        g.push_back(a);
        g.push_back(b);
        group_sp[key] += nr * nc;
        group_rows[key] = std::max(group_rows[key], nr);
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    LK_CUDA(ctx, cudaEventCreate(&e0));
    LK_CUDA(ctx, cudaEventCreate(&e1));
    for (auto& kv : groups) {
        if (kv.second.empty()) continue;
        const int64_t max_rows = group_rows[kv.first];
        int best_rows = 0;
        float best_ms = 1e30f;
        for (int cand : kTuneCandidates) {
            if (cand > 2 * max_rows && cand != kTuneCandidates[0]) break;
            float ms = 0.0f;
            if ((st = time_verify(ctx, kv.second, cand, s, e0, e1, &ms)) != LK_OK) break;
            if (ms < best_ms) {
                best_ms = ms;
                best_rows = cand;
            }
        }
        if (st != LK_OK) break;
        if (best_rows > 0) ctx->tune[kv.first] = best_rows;
    }
    drop_repeat_plan(ctx);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return st;
}

lk_status lk_tune_get(lk_ctx* ctx, int32_t* entries, int64_t capacity, int64_t* n_entries) {
    if (!ctx || !n_entries || (capacity > 0 && !entries)) return fail(ctx, LK_ERR_ARG, "lk_tune_get: invalid arguments");
    *n_entries = (int64_t)ctx->tune.size();
    int64_t k = 0;
    for (auto& kv : ctx->tune) {
        if (k >= capacity) break;
        entries[3 * k + 0] = (int32_t)(kv.first >> 8);
        entries[3 * k + 1] = (int32_t)(kv.first & 0xff);
        entries[3 * k + 2] = kv.second;
        ++k;
    }
    return LK_OK;
}

lk_status lk_tune_set(lk_ctx* ctx, const int32_t* entries, int64_t n_entries) {
    if (!ctx || n_entries < 0 || (n_entries > 0 && !entries)) return fail(ctx, LK_ERR_ARG, "lk_tune_set: invalid arguments");
    for (int64_t k = 0; k < n_entries; ++k) {
        const int32_t rb = entries[3 * k], cb = entries[3 * k + 1], rows = entries[3 * k + 2];
        if (rb < 0 || rb > 40 || cb < 0 || cb > 40 || rows < 1)
            return fail(ctx, LK_ERR_ARG, "lk_tune_set: invalid entry");
    }
    ctx->tune.clear();
    for (int64_t k = 0; k < n_entries; ++k)
        ctx->tune[((uint32_t)entries[3 * k] << 8) | (uint32_t)entries[3 * k + 1]] = entries[3 * k + 2];
    drop_repeat_plan(ctx);
    return LK_OK;
}

}  // extern "C"

// ----------------------------------------------------------------------------
// Early-exit verification against an expected certificate.
extern "C" lk_status lk_verify_expected(lk_ctx* ctx, const int32_t* loop_pairs, const int32_t* expected,
                                        int64_t n_pairs, int64_t batch_segment_pairs, int64_t* first_mismatch,
                                        int64_t* n_checked, int32_t* lk_out, double* raw_out,
                                        int32_t* status_out, void* cuda_stream) {
    if (!ctx) return fail(nullptr, LK_ERR_ARG, "lk_verify_expected: NULL context");
    if (n_pairs < 0 || (n_pairs > 0 && (!loop_pairs || !expected)) || !first_mismatch || !n_checked ||
        batch_segment_pairs < 0 || n_pairs > INT32_MAX)
        return fail(ctx, LK_ERR_ARG, "lk_verify_expected: invalid arguments");
    *first_mismatch = -1;
    *n_checked = 0;
    if (n_pairs == 0) return LK_OK;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    std::vector<int32_t> hp;
    lk_status st = get_pairs_on_host(ctx, loop_pairs, n_pairs, s, hp);
    if (st != LK_OK) return st;
    // Batches in input order: at least one pair each, up to the segment-pair budget.
    const int64_t budget = batch_segment_pairs > 0 ? batch_segment_pairs : ((int64_t)1 << 28);
    std::vector<int64_t> bounds{0};
    {
        int64_t sp = 0;
        for (int64_t b = 0; b < n_pairs; ++b) {
            const int32_t x = hp[2 * b], y = hp[2 * b + 1];
            int64_t c = 0;
            if (x >= 0 && y >= 0 && x < ctx->n_loops && y < ctx->n_loops)
                c = (ctx->h_offsets[x + 1] - ctx->h_offsets[x]) * (ctx->h_offsets[y + 1] - ctx->h_offsets[y]);
            if (b > bounds.back() && sp + c > budget) {
                bounds.push_back(b);
                sp = 0;
            }
            sp += c;
        }
        bounds.push_back(n_pairs);
    }
    const size_t nb = bounds.size() - 1;
    const size_t n = (size_t)n_pairs;
    // A check of the same list and batch size as the previous call replays a
    // graph of the whole batched sequence (built on the first repeat): no
    // packing, no table uploads, one launch.
    constexpr size_t kExpectedGraphBatches = 256;
    ExpectedPlan* plan = ctx->ee_plan;
    if (plan && (plan->batch != budget || plan->pairs != hp)) {
        plan->release();
        delete plan;
        ctx->ee_plan = plan = nullptr;
    }
    LK_CUDA(ctx, ctx->ee_expected.ensure(n));
    LK_CUDA(ctx, ctx->ee_lk.ensure(n));
    LK_CUDA(ctx, ctx->ee_raw.ensure(n));
    LK_CUDA(ctx, ctx->ee_status.ensure(n));
    LK_CUDA(ctx, ctx->ee_stop.ensure(1));
    const bool build = !plan && nb <= kExpectedGraphBatches && budget == ctx->ee_last_batch && hp == ctx->ee_last_pairs;
    // Pack every batch first (their tables stay alive until the stream has
    // copied them) and size the shared workspace for the largest.
    std::vector<Packed> batches;
    Packed most;
    int64_t max_tasks = 0, max_items = 0, max_chunks = 0;
    if (!plan) {
        batches.resize(nb);
        for (size_t k = 0; k < nb; ++k) {
            Packed& pk = batches[k];
            if ((st = pack_pairs(ctx, hp.data() + 2 * bounds[k], bounds[k + 1] - bounds[k], pk)) != LK_OK) return st;
            max_tasks = std::max<int64_t>(max_tasks, (int64_t)pk.tasks.size());
            max_items = std::max(max_items, pk.n_items);
            max_chunks = std::max(max_chunks, pk.n_chunks);
            most.n_chunk_bits = std::max(most.n_chunk_bits, pk.n_chunk_bits);
            if (!pk.grid.empty()) {
                if (most.grid.empty()) most.grid.push_back(pk.grid[0]);
                most.grid_cells = std::max(most.grid_cells, pk.grid_cells);
                most.grid_rows = std::max(most.grid_rows, pk.grid_rows);
                most.grid_cols = std::max(most.grid_cols, pk.grid_cols);
            }
        }
    }
    if (build) {
        // resident item tables per batch and the captured sequence
        plan = new ExpectedPlan();
        plan->pairs = hp;
        plan->batch = budget;
        plan->bounds = bounds;
        plan->batches = std::move(batches);
        plan->tasks.resize(nb);
        plan->item_begin.resize(nb);
        plan->item_task.resize(nb);
        auto fail_plan = [&](lk_status code) {
            plan->release();
            delete plan;
            return code;
        };
        if ((st = ensure_workspace(ctx, plan->ws, max_tasks, max_items, max_chunks, &most)) != LK_OK)
            return fail_plan(st);
        cudaError_t e = cudaSuccess;
        for (size_t k = 0; k < nb && e == cudaSuccess; ++k) {
            const Packed& pk = plan->batches[k];
            const size_t m = pk.tasks.size();
            e = plan->tasks[k].ensure(m);
            if (e == cudaSuccess) e = plan->item_begin[k].ensure(m + 1);
            if (e == cudaSuccess) e = plan->item_task[k].ensure((size_t)std::max<int64_t>(pk.n_items, 1));
            if (e == cudaSuccess)
                e = cudaMemcpy(plan->tasks[k].p, pk.tasks.data(), m * sizeof(PairTask), cudaMemcpyHostToDevice);
            if (e == cudaSuccess)
                e = cudaMemcpy(plan->item_begin[k].p, pk.item_begin.data(), (m + 1) * sizeof(int64_t),
                               cudaMemcpyHostToDevice);
            if (e == cudaSuccess && pk.n_items > 0)
                e = cudaMemcpy(plan->item_task[k].p, pk.item_task.data(), pk.n_items * sizeof(int32_t),
                               cudaMemcpyHostToDevice);
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&plan->capture, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamBeginCapture(plan->capture, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return fail_plan(cuda_fail(ctx, e, "lk_verify_expected: plan"));
        lk_status cst = LK_OK;
        cudaError_t ce = cudaMemsetAsync(ctx->ee_stop.p, 0x7f, sizeof(long long), plan->capture);
        for (size_t k = 0; k < nb && cst == LK_OK && ce == cudaSuccess; ++k) {
            const Packed& pk = plan->batches[k];
            const int64_t b0 = bounds[k], m = bounds[k + 1] - bounds[k];
            Workspace view = plan->ws;             // the shared buffers, this batch's tables
            view.tasks = plan->tasks[k];
            view.item_begin = plan->item_begin[k];
            view.item_task = plan->item_task[k];
            cst = enqueue_verify(ctx, view, pk, plan->capture, ctx->ee_stop.p, b0);
            if (cst != LK_OK) break;
            lk::launch_compare_expected(view.lk.p, view.status.p, ctx->ee_expected.p, m, b0, ctx->ee_stop.p,
                                        plan->capture);
            ce = cudaMemcpyAsync(ctx->ee_lk.p + b0, view.lk.p, m * sizeof(int32_t), cudaMemcpyDeviceToDevice,
                                 plan->capture);
            if (ce == cudaSuccess)
                ce = cudaMemcpyAsync(ctx->ee_raw.p + b0, view.raw.p, m * sizeof(double), cudaMemcpyDeviceToDevice,
                                     plan->capture);
            if (ce == cudaSuccess)
                ce = cudaMemcpyAsync(ctx->ee_status.p + b0, view.status.p, m * sizeof(int32_t),
                                     cudaMemcpyDeviceToDevice, plan->capture);
        }
        e = cudaStreamEndCapture(plan->capture, &plan->graph);
        if (cst != LK_OK) return fail_plan(cst);
        if (ce != cudaSuccess) return fail_plan(cuda_fail(ctx, ce, "lk_verify_expected: capture"));
        if (e == cudaSuccess) e = cudaGraphInstantiate(&plan->exec, plan->graph, 0);
        if (e != cudaSuccess) return fail_plan(cuda_fail(ctx, e, "lk_verify_expected: graph"));
        ctx->ee_plan = plan;
    }
    LK_CUDA(ctx, cudaMemcpyAsync(ctx->ee_expected.p, expected, n * sizeof(int32_t), cudaMemcpyDefault, s));
    Workspace& ws = plan ? plan->ws : ctx->ws;
    if (plan) {
        LK_CUDA(ctx, cudaGraphLaunch(plan->exec, s));
    } else {
        if ((st = ensure_workspace(ctx, ctx->ws, max_tasks, max_items, max_chunks, &most)) != LK_OK) return st;
        LK_CUDA(ctx, cudaMemsetAsync(ctx->ee_stop.p, 0x7f, sizeof(long long), s));     // no mismatch yet
        // Every batch is enqueued back to back: its kernels read the stop word
        // and do nothing once an earlier batch has lowered it, so no host round
        // trip separates the batches.
        for (size_t k = 0; k < nb; ++k) {
            const Packed& pk = batches[k];
            const int64_t b0 = bounds[k], m = bounds[k + 1] - bounds[k];
            if ((st = upload_packed(ctx, ws, pk, s)) != LK_OK) return st;
            if ((st = enqueue_verify(ctx, ws, pk, s, ctx->ee_stop.p, b0)) != LK_OK) return st;
            lk::launch_compare_expected(ws.lk.p, ws.status.p, ctx->ee_expected.p, m, b0, ctx->ee_stop.p, s);
            LK_CUDA(ctx, cudaMemcpyAsync(ctx->ee_lk.p + b0, ws.lk.p, m * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
            LK_CUDA(ctx, cudaMemcpyAsync(ctx->ee_raw.p + b0, ws.raw.p, m * sizeof(double), cudaMemcpyDeviceToDevice, s));
            LK_CUDA(ctx, cudaMemcpyAsync(ctx->ee_status.p + b0, ws.status.p, m * sizeof(int32_t),
                                         cudaMemcpyDeviceToDevice, s));
        }
        ctx->ee_last_pairs = hp;
        ctx->ee_last_batch = budget;
    }
    LK_CUDA(ctx, cudaGetLastError());
    long long stop = 0;
    LK_CUDA(ctx, cudaMemcpyAsync(&stop, ctx->ee_stop.p, sizeof stop, cudaMemcpyDeviceToHost, s));
    LK_CUDA(ctx, cudaStreamSynchronize(s));
    note_stats(ctx, ws, plan ? plan->batches.back() : batches.back(), s);
    ctx->last_err = nullptr;             // the estimates of the batches are not kept
    int64_t checked = n_pairs;
    if (stop >= 0 && stop < n_pairs) {
        *first_mismatch = stop;
        checked = *std::upper_bound(bounds.begin(), bounds.end(), (int64_t)stop);   // end of its batch
    }
    *n_checked = checked;
    if (lk_out) LK_CUDA(ctx, cudaMemcpyAsync(lk_out, ctx->ee_lk.p, checked * sizeof(int32_t), cudaMemcpyDefault, s));
    if (raw_out) LK_CUDA(ctx, cudaMemcpyAsync(raw_out, ctx->ee_raw.p, checked * sizeof(double), cudaMemcpyDefault, s));
    if (status_out)
        LK_CUDA(ctx, cudaMemcpyAsync(status_out, ctx->ee_status.p, checked * sizeof(int32_t), cudaMemcpyDefault, s));
    LK_CUDA(ctx, cudaStreamSynchronize(s));
    return LK_OK;
}
