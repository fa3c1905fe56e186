// Internal types shared by the host runtime (lk_api.cu) and the kernels
// (lk_kernels.cu).  Nothing here is part of the C ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace lk {

// A resident vertex: FP64 coordinates padded to 32 bytes (w unused).
struct __align__(32) Vtx {
    double x, y, z, w;
};

// Mixed-precision tile sweep: one warp owns a work item of kTileCols columns
// (segments i of the column loop, kLaneCols per lane) by tile_rows rows
// (segments j of the row loop), streamed in chunks of kChunkRows rows.
constexpr int kLaneCols = 4;
constexpr int kTileCols = 32 * kLaneCols;
constexpr int kChunkRows = 32;
constexpr int kSweepWarps = 4;
constexpr int kSweepThreads = 32 * kSweepWarps;

// All-FP64 baseline sweep: one column per lane.
constexpr int kF64TileCols = 32;

// FP64 recomputes of near segment pairs are accumulated as fixed-point
// integers of 2^-38 rad, so that their sum is independent of the order in
// which threads add them.
constexpr double kFixScale = 274877906944.0;  // 2^38

// Careful-pass results of single chunks are added to their item as
// fixed-point integers of 2^-32 rad (order-independent; an item holds at most
// a few thousand chunks, so the sum cannot overflow).
constexpr double kChunkFixScale = 4294967296.0;  // 2^32

// Per-pair flag bits.
constexpr int kFlagIntersect = 1;
constexpr int kFlagCcFallback = 2;   // counting crossings could not decide the pair: direct sum
constexpr int kFlagPrecise = 4;      // the pair's bulk chunks are summed again by the precise sweep

// Error statistics of a work item's bulk sweep (SweepArgs::item_err), in units
// of the FP32 unit roundoff u = 2^-24 where they scale with it:
//   x: sum over its chunk columns of (a theta_c)^2 + 32 (b kq)^2 -- the variance
//      of the item's rounding errors over u^2 (theta_c a column's angle over one
//      32-row chunk, kq = L^2 / m^2 its lane's longest segment over nearest
//      grid distance, squared; a, b below);
//   y: sum of |theta_c| (radians);
//   z: the largest kq;  w: unused.
constexpr float kErrAcc = 3.0f;      // a: the running sum of a chunk column (FP32 emulation: about 2)
constexpr float kErrCell = 0.5f;     // b: a cell's rounding relative to L^2 / m^2 (analysis: about 1/4)

// One loop pair of a verify call, laid out for the device.
//
// The mixed path reads an FP32 copy of the geometry, R[v] = (float)(v -
// centre of v's loop box), refreshed with the boxes whenever the FP64
// vertices change.  The pair's frame has its origin at the centre of the union of the two loop
// boxes and a power-of-two scale that maps the union into [-1, 1]^3.  Every
// kernel of the mixed path sees a vertex of the pair as the FP32 value
//     fmaf(R[v], scale, off)   (per coordinate)
// with off = (float)((loop centre - origin) * scale) of the vertex's loop.
// Because the scale is a power of two, R[v] * scale is exact and this is the
// single rounding of (R[v] + loop centre - origin) * scale; the FP32 sweep and
// the FP64 recompute both use these values, so a pair's sum is the linking
// integral of one closed polyline pair.
struct PairTask {
    const Vtx* V;        // FP64 geometry (read by the all-FP64 path)
    const float4* R;     // FP32 loop-relative geometry (read by the mixed path)
    int64_t row_base;    // first vertex of the row loop (segments j, iterated)
    int64_t col_base;    // first vertex of the column loop (segments i, across lanes)
    int32_t n_rows;      // segments (= vertices) of the row loop
    int32_t n_cols;      // segments of the column loop
    int32_t tile_rows;   // rows per work item
    int32_t col_tiles;   // column tiles of this pair
    int32_t row_loop;    // loop indices, for the pair's frame
    int32_t col_loop;
    int32_t out_index;   // position of the pair in the caller's list
    int32_t status;      // LK_OK, or LK_ERR_ARG for an invalid pair (then it has no items)
    int32_t accurate;    // 1: bias-free FP32 arithmetic variant (large pairs)
    int32_t cc_grid;     // counting crossings: 1 when the pair's candidates come from the binned
                         // search over the device grid, 2 from the one-CTA search, else 0
    float row_off[4];    // frame offset of the row loop's vertices ([3] unused)
    float col_off[4];    // frame offset of the column loop's vertices ([3] unused)
    float scale;         // power of two
    int32_t pad2;
    int64_t bit_base;    // accurate variant: first bit of the pair's chunks in SweepArgs::chunk_bits
};

// A segment pair queued for FP64 recompute.
struct NearEntry {
    int32_t task;
    int32_t j;   // segment index in the row loop
    int32_t i;   // segment index in the column loop
    int32_t pad;
};

// A 32-row chunk handed from the bulk sweep to the careful pass.
struct CarefulChunk {
    int64_t item;
    int32_t chunk;   // chunk index within the item
    int32_t pad;
};

struct SweepArgs {
    const PairTask* tasks;
    const int64_t* item_begin;     // [n_tasks+1] first item of each task
    const int32_t* item_task;      // [n_items] task of each item
    int64_t n_items;
    int64_t n_tasks;
    double* partial;               // [n_items] radians: sum of (atan2 + atan2) over the item
    unsigned long long* item_counter;
    int64_t* careful_items;        // [n_items] items handed to the careful pass
    unsigned int* careful_count;   // [1] entries of careful_items
    unsigned int* careful_counter; // [1] work counter of the careful pass (fast items);
                                   // careful_counter + 2: accurate items
    NearEntry* near_list;
    unsigned int* near_count;
    int near_capacity;
    unsigned long long* fix_acc;   // [n_tasks] fixed-point radians of FP64 recomputes
    unsigned long long* fp64_count;// [n_tasks] segment pairs recomputed in FP64
    unsigned long long* overflow;  // [1] recomputes evaluated in place (list full)
    CarefulChunk* careful_chunks;  // chunks handed over by the bulk sweep
    unsigned int* chunk_count;     // [1] entries of careful_chunks (may exceed capacity)
    unsigned int* chunk_counter;   // [2] work counters of the chunk pass (fast, accurate)
    int chunk_capacity;
    unsigned long long* item_fix;  // [n_items] fixed-point 2^-32 rad: careful chunk sums
    int* flags;                    // [n_tasks] kFlag* bits
    float near_ratio_sq;           // tau^2
    // Counting crossings (lk_options.method = LK_METHOD_CC).
    NearEntry* cc_list;            // candidate crossings (task, j, i) for the FP64 resolve
    unsigned long long* cc_count;  // [1] candidates found (may exceed the list's capacity)
    int cc_capacity;
    int* cc_half;                  // [n_tasks] twice the linking number by crossings
    const unsigned int* flag_scan; // [n_tasks+1] exclusive scan of the item counts of pairs flagged
                                   // kFlagCcFallback; set: the direct-sum sweeps visit only those items
    // Error statistics and the precise re-sweep (accurate-variant pairs).
    float4* item_err;              // [n_items] bulk-sweep error statistics (see kErrAcc), or null
    unsigned int* chunk_bits;      // bit per chunk of accurate-variant items (PairTask::bit_base):
                                   // set when the bulk sweep handed the chunk to the careful pass
                                   // (every chunk of an item handed over whole), or null
    const unsigned int* precise_scan;  // [n_tasks+1] exclusive scan of the item counts of pairs flagged
                                       // kFlagPrecise (read by the precise sweep)
    // Early exit (lk_verify_expected): when *stop < stop_base, a pair before
    // this batch already differs from its expected linking number and every
    // kernel of the batch returns without work (the sweeps check before each
    // item they take).  Null: no early exit.
    const long long* stop;
    long long stop_base;
};

__device__ __forceinline__ bool stopped(const long long* stop, long long base) {
    return stop && *(volatile const long long*)stop < base;
}

// One request's contiguous run of items inside a serving wave.
struct WaveSeg {
    SweepArgs args;        // the request's arrays
    int64_t item_lo;       // first request-local item of the run
    int64_t wave_base;     // wave-global index of that item
};

struct ReduceArgs {
    const PairTask* tasks;
    const float4* item_err;        // bulk-sweep error statistics, or null
    double* err_out;               // [n_tasks] by out_index: estimated error of raw (see lk.h), or null
    double precise_tol;            // flag accurate pairs whose estimate exceeds it kFlagPrecise (0: never)
    const long long* stop;         // early exit, as in SweepArgs
    long long stop_base;
    const int* cc_half;            // counting crossings: non-null selects it for unflagged pairs
    const int64_t* item_begin;
    const double* partial;
    const unsigned long long* item_fix;   // may be null
    const unsigned long long* fix_acc;
    int* flags;                    // kFlagPrecise is set here (precise_tol)
    int64_t n_tasks;
    double int_tol;
    int32_t* lk_out;               // indexed by out_index
    double* raw_out;
    int32_t* status_out;
};

// Kernel launchers (lk_kernels.cu).
// Loop boxes (FP64, [n_loops][6]) and the FP32 loop-relative copy R, after
// applying `data` (if not null: [n_vertices][3] FP32 (dtype 0) or FP64, added
// when is_delta, else replacing) to V.  keys and next_keys are two sets of
// 6 * n_loops words: keys must be in the reset state (reset_box_keys, or a
// previous call's next_keys); the call leaves next_keys reset for the next.
cudaError_t reset_box_keys(unsigned long long* keys, int64_t n_loops, cudaStream_t s);
cudaError_t launch_loop_boxes(Vtx* V, const int64_t* offsets, int64_t n_loops, int64_t n_vertices,
                              unsigned long long* keys, unsigned long long* next_keys, double* aabb, float4* R,
                              const void* data, int dtype, int is_delta, cudaStream_t s);
void launch_pair_frames(PairTask* tasks, int64_t n_tasks, const double* aabb, cudaStream_t s);
void launch_sweep_mixed(const SweepArgs& a, bool accurate, int64_t item_lo, int64_t item_hi, int64_t task_lo,
                        int64_t task_hi, unsigned long long* counter, int grid, cudaStream_t s);
void launch_sweep_f64(const SweepArgs& a, int grid, cudaStream_t s);
// The careful passes of each arithmetic variant; a variant without work items
// in the call is not launched.
void launch_sweep_careful(const SweepArgs& a, bool fast, bool accurate, int grid, cudaStream_t s);
void launch_careful_chunks(const SweepArgs& a, bool fast, bool accurate, int grid, cudaStream_t s);
int careful_chunk_blocks_per_sm();
void launch_near_fix(const SweepArgs& a, int grid, cudaStream_t s);
void launch_wave(const WaveSeg* segs, int n_segs, int64_t n_items, bool accurate,
                 unsigned long long* counter, int grid, cudaStream_t s);
int wave_blocks_per_sm(bool accurate);
void launch_reduce(const ReduceArgs& a, cudaStream_t s);
int sweep_mixed_blocks_per_sm(bool accurate);

// Counting crossings (lk_kernels.cu): the FP32 candidate sweep over all items
// and the FP64 resolve of the candidates.
void launch_cc_sweep(const SweepArgs& a, unsigned long long* counter, int grid, cudaStream_t s);
// Binned candidate search of one counting-crossings pair (the pairs with
// cc_grid set): a G x G grid over the pair's mapped frame.
struct CcGridWork {
    unsigned int* offsets;     // [G*G + 1]: cell counts, then their exclusive scan (total last)
    unsigned int* cursor;      // [G*G]: fill positions
    unsigned int* block_sums;  // [G*G / 4096 + 2]: scan scratch
    int32_t* entries;          // [capacity]: row segments grouped by cell
    int64_t capacity;
    float2* row_xy;            // [n_rows]: mapped (x, y) of the row loop's vertices
    float2* col_xy;            // [n_cols]
    int* G;                    // [1]: the pair's grid size, chosen on the device
    unsigned long long* total; // [1]: the pair's entries, counted in 64 bits
};
// Counting crossings of pairs whose loops both have at most kCcLocalMax
// segments (cc_grid == 2): one CTA per pair, everything in shared memory.
constexpr int kCcLocalMax = 2048;
constexpr int kCcLocalGridMax = 64;     // grid cells per side at most
constexpr int kCcLocalEntries = 4;      // row-segment entries per row segment
struct CcLocalShape {
    int max_rows, max_cols;             // the largest loops among the pairs
    int G_max;                          // power of two <= kCcLocalGridMax
    int entry_cap;                      // kCcLocalEntries * max_rows
};
size_t cc_local_smem_bytes(const CcLocalShape& S);
// Counting crossings: scan[0..n_tasks] = exclusive scan of the item counts of
// the pairs flagged kFlagCcFallback (block_sums: n_tasks / 4096 + 2 entries).
void launch_cc_flag_scan(const SweepArgs& a, unsigned int* scan, unsigned int* block_sums, cudaStream_t s);
// scan[0..n_tasks] = exclusive scan of the item counts of the pairs whose flags have a bit of `mask`.
void launch_flag_scan(const SweepArgs& a, int mask, unsigned int* scan, unsigned int* block_sums, cudaStream_t s);
// The precise (compensated double-float) re-sweep of the bulk chunks of the
// pairs flagged kFlagPrecise (a.precise_scan, a.chunk_bits set), and the
// careful pass of their handed-over chunks (before launch_near_fix).
void launch_sweep_precise(const SweepArgs& a, int64_t task_lo, int64_t task_hi, unsigned long long* counter,
                          int grid, cudaStream_t s);
void launch_precise_careful(const SweepArgs& a, unsigned long long* counter, int grid, cudaStream_t s);
int sweep_precise_blocks_per_sm();
// Early exit: *stop = min(*stop, base + k) for the first k in [0, n) whose
// status is not LK_OK or whose linking number differs from expected[base + k]
// (skipped when *stop < base already).
void launch_compare_expected(const int32_t* lk, const int32_t* status, const int32_t* expected, int64_t n,
                             long long base, long long* stop, cudaStream_t s);
cudaError_t launch_cc_local(const SweepArgs& a, int64_t n_tasks, int64_t n_local, const CcLocalShape& S,
                            cudaStream_t s);
// G_max: the allocated grid size (offsets hold G_max^2 + 1 counts).
cudaError_t launch_cc_grid(const SweepArgs& a, int task, int n_rows, int n_cols, int G_max, const CcGridWork& w,
                           cudaStream_t s);
void launch_cc_resolve(const SweepArgs& a, int grid, cudaStream_t s);
int cc_sweep_blocks_per_sm();

// Potential link search (lk_pls.cu).
void launch_pls_keys(const double* aabb, int64_t n_loops, long long* keys, cudaStream_t s);
// Sort and sweep: pls_sort_size(n) is the padded length (a power of two) of
// the 64-bit key arrays the bitonic sort takes.
unsigned pls_sort_size(int64_t n);
void launch_bitonic_sort(unsigned long long* a, unsigned n, cudaStream_t s);
void launch_pls_sort(const long long* keys, int64_t n_loops, unsigned long long* order, unsigned n, cudaStream_t s);
void launch_pls_sweep_count(const long long* keys, int64_t n_loops, const unsigned long long* order,
                            int32_t* counts, cudaStream_t s);
void launch_pls_sweep_write(const long long* keys, int64_t n_loops, const unsigned long long* order,
                            const int64_t* offsets, unsigned long long* pairs, int64_t capacity, cudaStream_t s);
void launch_pls_unpack(const unsigned long long* keys, int64_t n, int32_t* pairs, cudaStream_t s);
void launch_pls_count(const long long* keys, int64_t n_loops, int32_t* counts, cudaStream_t s);
void launch_pls_write(const long long* keys, int64_t n_loops, const int64_t* offsets, int32_t* pairs,
                      int64_t capacity, cudaStream_t s);
// Device-side packing of a pair list that lives on the device (lk_pack.cu).
constexpr int kTuneClasses = 41;   // size classes ceil(log2 n) 0..40 per loop
struct PackParams {
    const Vtx* V;
    const float4* R;
    const int64_t* offsets;        // [n_loops + 1] first vertex of each loop
    const int32_t* tune;           // [kTuneClasses^2] tile rows per (row, column) size class, 0 = none; or null
    int64_t accurate_threshold;    // segment pairs from which a pair takes the accurate variant
    int32_t user_rows;             // fixed tile rows (> 0), else the tune table or the default
    int32_t n_loops;               // pairs outside [0, n_loops) or of one loop get status LK_ERR_ARG
};
struct PackSums {
    long long acc_n, acc_items;     // accurate-variant pairs and their items
    long long fast_n, fast_items;   // fast-variant (and invalid) pairs and their items
    long long chunks, segment_pairs;
};
// Entries of the scratch a scan of n values takes (block totals, grand total).
size_t scan_scratch_count(int64_t n);
// offsets[0..n] = exclusive scan of counts[0..n-1] (total at [n]).
void launch_scan_counts(const int32_t* counts, int64_t n, int64_t* offsets, long long* scratch, cudaStream_t s);
// tasks[0..n) and item_begin[0..n] of the pair list pairs[0..n) (device);
// scan_out[n] receives the totals.  vals, scan_out ([n + 1]) and scratch
// (scan_scratch_count(n)) are work space.
void launch_pack(const int32_t* pairs, int64_t n, const PackParams& P, PairTask* tasks, PackSums* vals,
                 PackSums* scan_out, PackSums* scratch, int64_t* item_begin, cudaStream_t s);
void launch_pack_item_task(const int64_t* item_begin, int64_t n_tasks, int64_t n_items, int32_t* item_task,
                           cudaStream_t s);
int sweep_f64_blocks_per_sm();
int sweep_careful_blocks_per_sm();

}  // namespace lk
