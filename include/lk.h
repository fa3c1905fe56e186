/*
 * lk.h -- C ABI of the GB300 linking-number library.
 *
 * The library computes Gauss linking numbers of closed polylines by direct
 * summation of the closed-form segment-pair term over every segment pair of
 * each requested loop pair, then rounds each per-pair sum to an integer
 * (Qu & James, "Fast Linking Numbers for Topology Verification of Loopy
 * Structures", SIGGRAPH 2021: Sec. 2.1 Eq. 3 and Eq. 4; Sec. 3.4.2,
 * Algorithm 5; the certificate matrix of Algorithm 1).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Geometry is CSR: vertices[n_vertices][3] (x,y,z interleaved, float32 or
 *    float64) and loop_offsets[n_loops+1] (int64, offsets[0] = 0,
 *    offsets[n_loops] = n_vertices, strictly increasing by >= 3).  Loop l owns
 *    vertices offsets[l] .. offsets[l+1]-1 and closes implicitly: its last
 *    vertex joins its first (Algorithm 5 indexes l_{j+1} with wrap-around).
 *    Orientation is the vertex order.
 *  - A loop pair is two int32 loop indices (a, b), a != b.  Loop a plays
 *    gamma_1 (vertices l_j) and loop b gamma_2 (vertices k_i) of Eq. 4; the
 *    linking number is symmetric in a and b.
 *  - Pointers may be host memory or device memory of the current device; the
 *    library tells them apart by CUDA unified addressing.  The caller owns
 *    every buffer it passes; the library copies what it keeps.
 *  - `cuda_stream` is a cudaStream_t (NULL = the legacy default stream).  Work
 *    is ordered on that stream.
 *  - Whole-call failures return a non-zero lk_status and set a message that
 *    lk_last_error() returns; per-pair outcomes go to status_out[].
 *  - Nothing in this library spins on device memory; no kernel waits for
 *    another, so no call can hang on a missing peer.
 */
#ifndef LK_H_
#define LK_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LK_OK = 0,
    LK_ERR_ARG = 1,          /* invalid argument (whole call) or invalid pair (per pair) */
    LK_ERR_ZERO_SEGMENT = 2, /* a segment shorter than eps*xi (Sec. 3.3, Algorithm 3 input check) */
    LK_ERR_INTERSECT = 3,    /* the loops meet: Eq. 4 is singular there (Sec. 4.1, robustness) */
    LK_ERR_NONINTEGER = 4,   /* |raw - round(raw)| > int_tol: result not trustworthy */
    LK_ERR_OOM = 5,          /* device allocation failed or the memory budget is exceeded */
    LK_ERR_TIMEOUT = 6,      /* reserved: no call waits on the device, so none returns it */
    LK_ERR_CUDA = 7,         /* a CUDA runtime error (message in lk_last_error) */
    LK_ERR_BUSY = 8          /* the server has no free slot / memory for this request now */
} lk_status;

typedef enum { LK_F32 = 0, LK_F64 = 1 } lk_dtype;

typedef enum {
    /* FP32 bulk sweep with FP64 accumulation; segment pairs closer than
     * near_ratio segment lengths are recomputed in FP64. */
    LK_MIXED = 0,
    /* every segment pair's term of Eq. 4 in FP64 with two atan2 (one per
     * triangle of the cell): the plain all-FP64 GPU direct sum. */
    LK_ALL_F64 = 1
} lk_precision;

typedef enum {
    /* direct summation of Eq. 4 over every segment pair (the default) */
    LK_METHOD_DS = 0,
    /* counting crossings of a projection (Sec. 3.4, Method 1; Algorithm 4): an
     * FP32 candidate search (binned, or a sweep over every segment pair: see
     * lk_cc_search) finds candidate crossings, FP64
     * decides them, and the count of signed crossings gives the linking
     * number exactly; a pair whose projection is not regular within FP64
     * rounding (or whose candidates overflow cc_capacity) is computed by the
     * direct sum in the same call.  raw_out then holds the exact integer.
     * Requires precision LK_MIXED; the server always uses LK_METHOD_DS. */
    LK_METHOD_CC = 1
} lk_method;

/* How LK_METHOD_CC finds its candidate crossings (Algorithm 4 queries a
 * hierarchy of one loop's projected segments with the other's).  Every
 * choice returns the same results; they differ only in speed. */
typedef enum lk_cc_search {
    LK_CC_SEARCH_AUTO = 0,    /* binned where it pays: pairs whose loops both have at most 2,048
                                 segments in one CTA each, pairs of at least 2^28 segment pairs
                                 on a device-wide grid, the rest by the all-pairs sweep */
    LK_CC_SEARCH_SWEEP = 1,   /* every pair by the all-pairs FP32 sweep */
    LK_CC_SEARCH_BINNED = 2   /* every pair binned: one CTA where both loops fit, else the grid */
} lk_cc_search;

typedef struct lk_options {
    int precision;       /* lk_precision, default LK_MIXED */
    double near_ratio;   /* tau >= 3: a segment pair whose nearest corner distance (the smallest
                            of |l_j-k_i|, |l_j-k_{i+1}|, |l_{j+1}-k_i|, |l_{j+1}-k_{i+1}|) is below
                            tau*max(|s_j|,|s_i|) is evaluated in FP64 (default 3.0) */
    double int_tol;      /* per-pair status LK_ERR_NONINTEGER when |raw - lk| > int_tol (default 0.1) */
    size_t mem_budget;   /* device bytes one verify may use for its work buffers, 0 = unlimited */
    int tile_rows;       /* rows per work item; 0 = chosen by the built-in tuner */
    int near_capacity;   /* entries of the FP64 recompute list (default 1<<20); overflow is
                            evaluated in place, results are unchanged.  This and the two
                            list sizes below are starting sizes: when a plain lk_verify
                            overflowed a list, a later lk_verify on the context grows it
                            to the next power of two above that call's need (at most a
                            quarter of the device memory then free, and 2^31 - 1 entries)
                            -- unless mem_budget is set.  The context then holds the grown
                            size (lk_get_options shows it). */
    int timing;          /* 1: time the bulk sweep kernel with CUDA events on the launch stream
                            (read back by lk_get_stats as sweep_ms); default 0 */
    int chunk_capacity;  /* entries of the chunk hand-over list (default 1<<20); an overflow
                            hands whole items to the careful pass instead, results unchanged */
    int64_t accurate_threshold; /* LK_MIXED: loop pairs with at least this many segment pairs use
                            the bias-free FP32 arithmetic (refined sqrt and division, shifted
                            denominators); smaller pairs use the hardware approximations,
                            whose relative bias (~5e-9) is negligible for them.  Both sum a
                            cell column's terms over a 32-row chunk by angle summation
                            (Appendix B: one arctangent per column and chunk); a chunk whose
                            nearest corner is within 4.5 segment lengths is swept per pair
                            instead.  0 = always accurate; default 1<<22 */
    int method;          /* lk_method, default LK_METHOD_DS */
    int cc_capacity;     /* LK_METHOD_CC: candidate crossings per verify (default 1<<18); pairs
                            whose candidates do not fit are computed by the direct sum */
    int cc_search;       /* lk_cc_search, default LK_CC_SEARCH_AUTO */
    double precise_tol;  /* LK_MIXED: the bulk sweep records its rounding-error statistics, and a
                            pair of the accurate variant whose estimated error of raw (see
                            lk_get_error_estimates) exceeds precise_tol has its bulk sum formed
                            again with compensated FP32 arithmetic (every quantity an unevaluated
                            sum of two floats, errors near 1e-10 where FP32 terms reach 1e-5; about
                            7 times the accurate variant's work), in the same call.  0 = never;
                            default 5e-7, half of the 1e-6 raw tolerance. */
} lk_options;

typedef struct lk_stats {
    int64_t n_pairs;          /* pairs in the last verify */
    int64_t n_items;          /* work items (tiles) of the last verify */
    int64_t segment_pairs;    /* segment pairs evaluated by the last verify */
    int64_t fp64_pairs;       /* of those, recomputed in FP64 (LK_MIXED) */
    int64_t near_overflow;    /* FP64 recomputes that did not fit the list */
    int32_t tile_rows;        /* rows per work item used */
    int32_t tile_cols;        /* columns per work item used */
    int64_t careful_items;    /* whole items swept again with per-pair tests (chunk list full) */
    double sweep_ms;          /* bulk sweep kernel time (options.timing = 1), else -1 */
    int64_t careful_chunks;   /* 32-row chunks swept again with per-pair tests */
    int64_t cc_candidates;    /* LK_METHOD_CC: candidate crossings found by the FP32 search */
    int64_t cc_fallback_pairs;/* LK_METHOD_CC: pairs the crossings could not decide (direct sum) */
    int64_t precise_pairs;    /* pairs summed again by the compensated sweep (options.precise_tol) */
} lk_stats;

typedef struct lk_ctx lk_ctx;
typedef struct lk_plan lk_plan;
typedef struct lk_server lk_server;

/* Fill *opt with the defaults listed above. */
void lk_default_options(lk_options* opt);

/*
 * Create a context holding one CSR geometry resident in device memory (the
 * loops Gamma_i of Algorithm 1, already discretised into polylines).
 *  out          : receives the context (caller destroys it with lk_destroy).
 *  vertices     : [n_vertices][3] of vdtype, host or device.
 *  loop_offsets : [n_loops+1] int64, host or device.
 *  opt          : NULL for defaults.
 * Errors: LK_ERR_ARG (bad sizes, offsets, fewer than 3 vertices in a loop,
 * non-finite coordinates), LK_ERR_ZERO_SEGMENT (a segment of length < eps*xi,
 * xi the mean absolute coordinate and eps the machine epsilon of vdtype:
 * Algorithm 3's input check), LK_ERR_OOM, LK_ERR_CUDA.  On error *out is NULL.
 * The call returns after the geometry is on the device.  Device memory: 48
 * bytes per vertex (FP64 coordinates plus an FP32 copy relative to each
 * loop's box centre, which the mixed-precision sweep reads) and 48 bytes per
 * loop (its box).
 */
lk_status lk_create(lk_ctx** out, const void* vertices, lk_dtype vdtype, int64_t n_vertices,
                    const int64_t* loop_offsets, int64_t n_loops, const lk_options* opt,
                    void* cuda_stream);

/*
 * Replace the resident vertices (is_delta = 0) or add a displacement to each
 * (is_delta = 1), keeping the loop structure: one simulation step of the
 * verification loop of Sec. 4.3 (a linking certificate before and after a
 * deformation).
 *  data : [n_vertices][3] of dtype, host or device.
 * Enqueued on cuda_stream; later work on that stream sees the new geometry.
 * Errors: LK_ERR_ARG, LK_ERR_CUDA.  No zero-length check is made here; a
 * degenerate step shows up as LK_ERR_INTERSECT in the verify that follows.
 */
lk_status lk_update(lk_ctx* ctx, const void* data, lk_dtype dtype, int is_delta, void* cuda_stream);

/*
 * Linking numbers of n_pairs loop pairs (the loop over P in Algorithm 1, every
 * pair by the direct sum of Sec. 3.4.2) in one batched persistent launch.
 *  loop_pairs : [n_pairs][2] int32, host or device.
 *  lk_out     : [n_pairs] int32, the rounded linking numbers (may be NULL).
 *  raw_out    : [n_pairs] double, the unrounded FP64 sums (may be NULL).
 *  status_out : [n_pairs] int32 lk_status per pair (may be NULL): LK_OK,
 *               LK_ERR_ARG (a == b or out of range), LK_ERR_INTERSECT,
 *               LK_ERR_NONINTEGER.  A pair that is not LK_OK has lk_out = 0.
 * Outputs may be host or device memory.  When any output is host memory the
 * call returns with the results written; otherwise it returns after enqueueing
 * and the results are valid once cuda_stream has reached the call's end
 * (lk_sync).  n_pairs = 0 is allowed and does nothing.
 * Repeated lists: the work decomposition depends only on the pair list, the
 * loop sizes and the tune table.  When a call passes the same list as the
 * previous call on this context, the context builds (once) and then replays
 * a graph plan of it, as lk_plan_create/lk_plan_run would, skipping the host
 * packing and table uploads; every kernel still runs on the current geometry.
 * A different list, lk_autotune or lk_tune_set drops that plan.
 * Errors: LK_ERR_ARG, LK_ERR_OOM (mem_budget exceeded or allocation failed),
 * LK_ERR_CUDA.
 */
lk_status lk_verify(lk_ctx* ctx, const int32_t* loop_pairs, int64_t n_pairs, int32_t* lk_out,
                    double* raw_out, int32_t* status_out, void* cuda_stream);

/*
 * Potential link search (Sec. 3.2, Algorithm 2) on the device: the loop pairs
 * (i, j), i < j, whose axis-aligned bounding boxes (closed, from the current
 * resident geometry, i.e. after any lk_update) overlap on all three axes.
 * Every pair with a nonzero linking number is among them.  The list is sorted
 * by (i, j) and feeds lk_verify directly.
 *  pairs_out : [capacity][2] int32, host or device; receives the first
 *              min(n, capacity) pairs (may be NULL when capacity = 0).
 *  n_pairs   : receives n, the number of candidate pairs (call with
 *              capacity 0 to size the output).
 * Synchronous: returns after the pairs are written.  The test is exact (FP64
 * box bounds).  Up to 2^27 box pairs (L(L-1)/2 for L loops, about 16,000
 * loops) every pair is tested; above, the loops are sorted by their lower x
 * bound and each is tested only against those whose lower x bound falls in
 * its x extent (a sort and sweep: work proportional to the pairs that overlap
 * in x).  Device memory: 68 bytes per loop (plus 8 bytes per loop rounded up
 * to a power of two for the sort), 8 bytes per candidate pair (rounded up
 * likewise) in the sweep, plus 8 bytes per pair written to a host
 * destination.
 * Errors: LK_ERR_ARG, LK_ERR_OOM, LK_ERR_CUDA.
 */
lk_status lk_candidates(lk_ctx* ctx, int32_t* pairs_out, int64_t capacity, int64_t* n_pairs,
                        void* cuda_stream);

/* Wait until all work the context enqueued on cuda_stream has finished. */
lk_status lk_sync(lk_ctx* ctx, void* cuda_stream);

/* Statistics of the most recent completed verify or plan run on this context. */
lk_status lk_get_stats(lk_ctx* ctx, lk_stats* out);

/*
 * Per-pair error estimates of the last verify or plan run on this context
 * (LK_MIXED): an estimate of |raw - exact| in units of the linking number,
 * where "exact" is the direct sum of the same staged polylines in exact
 * arithmetic (the integer linking number).  It is 4 standard deviations of
 * the bulk sweep's rounding errors (each work item records the sum of its
 * chunk columns' squared angles, a per-cell scale L^2/m^2 -- longest segment
 * over nearest grid distance -- and a share for each chunk it hands to the
 * careful pass), plus the part that a rounded |s|^2 shared by a whole row or
 * column adds coherently, plus a relative bias times the summed |angle|
 * (1e-8 for the fast variant's hardware approximations, 2e-10 for the
 * accurate variant); for a pair summed again by the compensated sweep, the
 * bulk estimate over 2^9.  Segment pairs recomputed in FP64 are not
 * included; pairs decided by counting crossings have 0; a pair whose status
 * is not LK_OK has NaN.  The estimate is not a bound.
 *  err_out : [n_pairs] double, host or device, in the order of the verify's
 *            pair list; n_pairs must equal that list's length.
 * Ordered on cuda_stream after the verify; returns after the copy when
 * err_out is host memory.  Errors: LK_ERR_ARG (no such verify, wrong
 * n_pairs, LK_ALL_F64), LK_ERR_CUDA.
 */
lk_status lk_get_error_estimates(const lk_ctx* ctx, double* err_out, int64_t n_pairs, void* cuda_stream);

/* The options the context runs with: those given to lk_create, with the
 * list sizes as grown by later verifies.  Errors: LK_ERR_ARG. */
lk_status lk_get_options(const lk_ctx* ctx, lk_options* out);

/* Free the context and its device memory.  NULL is ignored. */
void lk_destroy(lk_ctx* ctx);

/* The message of the last failed call on ctx (ctx may be NULL: the last
 * failure of lk_create or of a call given a NULL context). */
const char* lk_last_error(const lk_ctx* ctx);

/*
 * A plan fixes one pair list and captures the whole verify (pair set-up,
 * persistent tile sweep, FP64 recompute, per-pair reduction) as a CUDA graph,
 * so that a simulation loop re-verifies the same certificate after each
 * lk_update with one graph launch (Sec. 4.3 verification loop; Algorithm 1).
 *  loop_pairs : copied at creation; later changes to the caller's array are
 *               not seen.
 * lk_plan_run writes the same outputs as lk_verify (same rules for host and
 * device memory).  Plans hold device memory until lk_plan_destroy, and must
 * be destroyed before their context.
 */
lk_status lk_plan_create(lk_ctx* ctx, const int32_t* loop_pairs, int64_t n_pairs, lk_plan** out,
                         void* cuda_stream);
lk_status lk_plan_run(lk_plan* plan, int32_t* lk_out, double* raw_out, int32_t* status_out,
                      void* cuda_stream);
void lk_plan_destroy(lk_plan* plan);

/*
 * Early-exit verification of a certificate (Sec. 3.1, "Fast Verification":
 * exit as soon as any linking number differs from the input; Algorithm 1's
 * comparison of M_0 with M_t).  The pairs are verified in input order, in
 * batches of at most batch_segment_pairs segment pairs (0 = 2^28; every batch
 * holds at least one pair), all enqueued on cuda_stream back to back with no
 * host round trip between them.  expected[] ([n_pairs] int32, host or device)
 * is copied to the device; after each batch a kernel compares its rounded
 * linking numbers with it and records the first index that differs (a pair
 * whose status is not LK_OK also counts) in a device word.  Every kernel of
 * the later batches reads that word first -- the persistent sweeps before
 * each work item they take -- and does nothing once it is set, so the work
 * after the first differing batch costs only its launches.  No kernel waits
 * on the word.  A call with the same pair list and batch size as the previous
 * call on this context builds (once, up to 256 batches) a CUDA graph of the
 * whole batched sequence with the batches' item tables resident, and later
 * such calls upload the certificate and replay it: no host packing, one
 * launch.  A different list or batch size drops that graph.
 *  *first_mismatch : the smallest mismatching index of the first batch that
 *                    has one, or -1 if every pair matches.
 *  *n_checked      : pairs verified before stopping (a prefix of the list:
 *                    up to the end of the batch holding the mismatch).
 * lk_out / raw_out / status_out (may be NULL) receive the results of the
 * checked prefix; entries past it are left untouched.  Synchronises
 * cuda_stream once, at the end.  Device memory: 20 bytes per pair, plus the
 * work buffers of the largest batch.  Errors: as lk_verify.
 */
lk_status lk_verify_expected(lk_ctx* ctx, const int32_t* loop_pairs, const int32_t* expected,
                             int64_t n_pairs, int64_t batch_segment_pairs, int64_t* first_mismatch,
                             int64_t* n_checked, int32_t* lk_out, double* raw_out, int32_t* status_out,
                             void* cuda_stream);

/*
 * Autotuner for the work split (the batching of Algorithm 1's loop over P
 * into work items; the paper launches one kernel per pair, Sec. 3.4).
 * For each size class present in loop_pairs -- a class is the pair
 * (ceil(log2 N_rows), ceil(log2 N_cols)) of the row and column loop --
 * times the mixed-precision verify of up to 4096 of that class's pairs
 * (at most 2^31 segment pairs) at each candidate work-item height
 * (32 ... 65536 row segments) with CUDA events, and records the fastest in the
 * context.  Later verifies and plans of pairs in a tuned class use it unless
 * options.tile_rows is set.  The split changes the order of the FP64 sums, not
 * which segment pairs are evaluated: results agree with the untuned ones to
 * rounding, and are deterministic for a given table.  Synchronises
 * cuda_stream.  Errors: LK_ERR_ARG, LK_ERR_OOM, LK_ERR_CUDA.
 */
lk_status lk_autotune(lk_ctx* ctx, const int32_t* loop_pairs, int64_t n_pairs, void* cuda_stream);
/* The tuning table: entries[3k..3k+2] = (row class, column class, rows per
 * item).  lk_tune_get writes at most `capacity` entries and the total count to
 * *n_entries; lk_tune_set replaces the table (e.g. with one saved for this GPU). */
lk_status lk_tune_get(lk_ctx* ctx, int32_t* entries, int64_t capacity, int64_t* n_entries);
lk_status lk_tune_set(lk_ctx* ctx, const int32_t* entries, int64_t n_entries);

/*
 * Serving: continuous batching of verify requests over resident geometry
 * (the per-frame verification of Sec. 4.3's simulation examples, as a service).
 * A server owns a device arena of arena_bytes (requests are admitted only
 * while their work buffers fit in it), a pinned host arena of host_bytes for
 * results, and a FIFO of submitted requests.  lk_server_step retires finished
 * waves, admits queued requests while fewer than max_requests are admitted and
 * the arena has room, then launches one wave: a single persistent launch over
 * up to wave_items work items taken, in admission order, from every admitted
 * request with items left -- so a request that arrives while others run shares
 * the device with them.  A request's result does not depend on what shares
 * its waves (each pair's tiling and reduction order depend only on the pair).
 * All work of a server runs on its own streams: request setup and the bulk
 * waves on lk_server_stream, and each request's finishing passes (careful
 * re-sweeps, FP64 recompute, reduction, result copies) on a second internal
 * stream ordered after the request's last wave, so that the next wave
 * overlaps them.  A request is complete (lk_server_poll, lk_server_completed)
 * only when both are done.  The caller must not change (lk_update) a context
 * while it has unfinished requests; an update enqueued on lk_server_stream
 * after they are complete is ordered before every later wave.
 */
typedef struct lk_server_options {
    int max_requests;     /* requests admitted at once (default 64) */
    size_t arena_bytes;   /* device memory for request work buffers (default 1 GiB) */
    size_t host_bytes;    /* pinned host memory for staged item tables and results (default 256 MiB) */
    int64_t wave_items;   /* work items per wave (default 16384) */
    int near_capacity;    /* FP64 recompute list entries per request (default 65536, 1 MB of
                             arena; a request of chainmail piles with 64-256-segment rings
                             has ~1.5 near segment pairs per loop pair, and entries beyond
                             the list are evaluated in place, much more slowly) */
    int max_queue;        /* queued requests before submit returns LK_ERR_BUSY (default 65536) */
    int wave_order;       /* which admitted requests' items a wave takes first: 0 (default) in
                             admission order, 1 the requests with the fewest items left first
                             (shortest remaining work; a result never depends on the order) */
    int pack_on_device;   /* 1 (default): a pair-list request's list is uploaded as it is and laid
                             out as work items on the device (the packing geometry-only requests
                             use), so submit does not pack on the host; its work buffers are then
                             sized only once the packing is done, and a request whose work does
                             not fit the arena fails when polled (LK_ERR_OOM).  0: host packing
                             at submit, where a request too large for the arena is refused */
} lk_server_options;

typedef struct lk_server_stats {
    int64_t submitted, admitted, completed;
    int64_t queued, running;             /* now */
    int64_t waves, waves_in_flight;
    int64_t items_launched;
    int64_t max_requests_per_wave;       /* most requests that shared one wave */
    int64_t arena_used;                  /* bytes of the device arena in use now */
    int64_t near_overflow;               /* FP64 recomputes that did not fit a request's list
                                            (evaluated in place, slowly): raise near_capacity */
    int64_t careful_items;               /* whole items swept again per pair (chunk list full) */
    int64_t careful_chunks;              /* 32-row chunks swept again per pair */
    int64_t geometry_requests;           /* submitted by lk_server_submit_geometry */
    int64_t candidate_pairs;             /* pairs their potential link searches found */
} lk_server_stats;

void lk_server_default_options(lk_server_options* opt);
/* Errors: LK_ERR_ARG, LK_ERR_OOM (arena allocation), LK_ERR_CUDA. */
lk_status lk_server_create(lk_server** out, const lk_server_options* opt);
/* The server's CUDA stream (cudaStream_t). */
void* lk_server_stream(lk_server* srv);
/* Queue a request to verify n_pairs >= 1 pairs of ctx (host or device memory,
 * copied).  *ticket identifies it.  Errors: LK_ERR_ARG; LK_ERR_BUSY (queue
 * full); LK_ERR_OOM (the request alone exceeds the arena: with pack_on_device
 * its list and tables, the work buffers failing at poll instead). */
lk_status lk_server_submit(lk_server* srv, lk_ctx* ctx, const int32_t* loop_pairs, int64_t n_pairs,
                           int64_t* ticket);
/* Queue a request that carries geometry only: verify every potential link of
 * ctx, the loop pairs (i, j), i < j, whose bounding boxes overlap (Sec. 3.2,
 * Algorithm 2; every other pair has linking number 0).  The search, the
 * packing of its pairs into work items and the sweep all run on the device:
 * no pair list passes through the host, which reads back only the number of
 * candidates and of work items (polled by lk_server_step, never waited for).
 * The search runs on an internal stream after the work enqueued on
 * lk_server_stream before this call (an lk_update of ctx there, say).  The
 * pairs are the ones lk_candidates returns, in the same (i, j) order, and each
 * pair's result equals lk_verify's for that list.  Results:
 * lk_server_poll_pairs.  Errors: LK_ERR_ARG (not a mixed-precision context;
 * more than 2^30 loops); LK_ERR_BUSY (queue full); LK_ERR_OOM (the search
 * alone exceeds the arena).  A request whose candidates or work items do not
 * fit the arena fails when it is polled (LK_ERR_OOM). */
lk_status lk_server_submit_geometry(lk_server* srv, lk_ctx* ctx, int64_t* ticket);
/* Retire finished waves, admit, launch the next wave.  wait = 1 also blocks
 * until the oldest wave in flight has finished. */
lk_status lk_server_step(lk_server* srv, int wait);
/* *done = 1 and the results copied to the host buffers ([n_pairs] each, may
 * be NULL) once the request has finished; the ticket is then released.
 * *done = 0 while it is queued or running.  Not for geometry requests
 * (LK_ERR_ARG): their pair count is known only to lk_server_poll_pairs. */
lk_status lk_server_poll(lk_server* srv, int64_t ticket, int* done, int32_t* lk_out, double* raw_out,
                         int32_t* status_out);
/* Poll any request, with its pair list: once it has finished, *done = 1 and
 * *n_pairs receives its number of pairs.  If capacity >= *n_pairs the pairs
 * ([2 * n] int32: loop i, loop j) and their results ([n] each) are copied to
 * the non-NULL buffers and the ticket is released; otherwise nothing is
 * copied and the ticket stays valid for a call with a larger buffer.  A
 * geometry request's pairs are in (i, j) order, i < j.  Returns the request's
 * error (and releases the ticket) if it could not run. */
lk_status lk_server_poll_pairs(lk_server* srv, int64_t ticket, int* done, int64_t* n_pairs, int32_t* pairs_out,
                               int64_t capacity, int32_t* lk_out, double* raw_out, int32_t* status_out);
/* Tickets of requests that have finished (as seen by lk_server_step) and were
 * not reported before, in completion order: up to capacity of them are
 * written to tickets[], *n_done receives how many.  A reported ticket stays
 * valid for lk_server_poll, which copies its results and releases it. */
lk_status lk_server_completed(lk_server* srv, int64_t* tickets, int64_t capacity, int64_t* n_done);
lk_status lk_server_get_stats(lk_server* srv, lk_server_stats* out);
const char* lk_server_last_error(const lk_server* srv);
/* Waits for the server's stream, then frees everything it owns. */
void lk_server_destroy(lk_server* srv);

/*
 * Measurement support (the paper has no counterpart): the FP32 rate this GPU
 * reaches, reported beside the bulk sweep's roofline, measured by kernels of
 * independent fused multiply-adds on every SM (packed FP32x2 with eight
 * chains per thread, and scalar with sixteen; 2,048 threads per SM), timed
 * with CUDA events on `cuda_stream`: the faster form, each the fastest of
 * three launches after one warm-up (about 16-20 ms each).  *tflops receives
 * the rate (2 flops per FMA and lane), *ms (may be NULL) that launch's time.
 * It allocates and frees a small device buffer.
 * Errors: LK_ERR_ARG (tflops NULL), LK_ERR_OOM, LK_ERR_CUDA.
 */
lk_status lk_measure_fp32_peak(double* tflops, double* ms, void* cuda_stream);

/*
 * Allocation-free verify (the paper has no counterpart; this is a service of
 * this library).  For callers that cannot allocate device memory at the time
 * they verify: a simulation step under a strict no-allocation rule (a device
 * allocation synchronises the GPU and can stall a real-time loop), a process
 * whose memory pool already owns all of device memory, or a host program that
 * forbids libraries to call cudaMalloc.  It runs the same kernels as
 * lk_verify with the default options, but every work buffer lives in one
 * file-scope device array of 48 MiB that each GPU loading the library holds
 * until the process exits; it calls no cudaMalloc, cudaFree or allocating
 * library routine.
 *  vertices     : [n_vertices][3] of vdtype, host or device memory.
 *  loop_offsets : [n_loops+1] int64, HOST memory (CSR as for lk_create).
 *  loop_pairs   : [n_pairs][2] int32, HOST memory.
 *  lk_out, raw_out, status_out : as for lk_verify (host or device, may be NULL).
 * Limits: n_vertices <= 262144, n_loops <= 16384, n_pairs <= 16384, at most
 * 262144 work items (tiles of 128 x tile_rows segment pairs) and at most 2^23
 * 32-row chunk slots in the items of pairs of at least accurate_threshold
 * segment pairs; larger inputs return LK_ERR_ARG with a message naming the
 * limit, before any device work.  The chunk hand-over list holds 65536
 * chunks: a call with more chunks near enough for the careful pass hands
 * whole work items to it instead (the results are unchanged, only slower),
 * and its FP64 recompute list holds 65536 segment pairs (the rest are
 * evaluated in place).  None of these buffers ever grows.
 * The first call on each device looks up the array's device address once
 * (cudaGetSymbolAddress); make that first call before any stream capture.
 * Every call on a device shares the one array and leaves its contents behind
 * (each call clears what must start at zero), so calls whose work overlaps on
 * the GPU -- on different streams, or from different host threads -- race and
 * must be serialised by the caller.  The input checks of lk_create (finite
 * coordinates, zero-length segments) are not made; degenerate geometry shows
 * up as per-pair LK_ERR_INTERSECT or LK_ERR_NONINTEGER.
 */
lk_status lk_verify_noalloc(const void* vertices, lk_dtype vdtype, int64_t n_vertices,
                            const int64_t* loop_offsets, int64_t n_loops,
                            const int32_t* loop_pairs, int64_t n_pairs, int32_t* lk_out,
                            double* raw_out, int32_t* status_out, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* LK_H_ */
