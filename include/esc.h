/*
 * esc.h -- C ABI of the GB300 exact selectivity computation library (libesc).
 *
 * Exact selectivity computation (ESC; Shin, Rusu, Suhan, "Exact Selectivity
 * Computation for Modern In-Memory Database Query Optimization", CIDR 2019)
 * replaces a cardinality estimate by the answer of a selectivity sub-query
 * run during optimisation (Sec. 2): the number of rows of one table that
 * satisfy a complex selection predicate, and optionally those rows with a
 * pushed-down projection, materialised for reuse by the final plan
 * (Sec. 2, Sec. 2.1).  This library runs that sub-query on one GPU over
 * resident columns, and adds exact filtered-join counts over dense keys
 * (the COUNT(*) foreign-key join queries of Sec. 3.1) and batched execution
 * of many sub-queries (Sec. 2: the procedure is applied to every table that
 * has a selection).
 *
 * Conventions for every entry point
 *  - Every call returns an esc_status; ESC_OK is 0.  On any other status the
 *    outputs are undefined, except where a function says otherwise, and
 *    esc_last_error() returns a message for the calling thread.
 *  - Device pointers are CUDA device (or managed) addresses on the current
 *    device; host pointers are ordinary process memory.  The library never
 *    takes ownership of caller memory.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream).  Work is enqueued on it; functions that return host values
 *    synchronise that stream before returning, *_async functions do not.
 *  - Calls are thread-safe for distinct handles.  Handles are immutable after
 *    creation and may be shared by concurrent calls on different streams.
 *  - Device-side errors (a bounded wait that gave up) come back as
 *    ESC_ETIMEOUT from synchronous calls; no kernel traps or asserts.
 */
#ifndef ESC_H
#define ESC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum esc_status {
    ESC_OK = 0,
    ESC_EINVAL = 1,    /* bad argument, size, alignment, or predicate text */
    ESC_ETYPE = 2,     /* unsupported column type or a type mismatch */
    ESC_ENOMEM = 3,    /* device or host allocation failed */
    ESC_ETRUNC = 4,    /* output rows did not fit: count is exact, rows truncated */
    ESC_ETIMEOUT = 5,  /* a bounded device-side wait gave up */
    ESC_EBUSY = 6,     /* resource in use */
    ESC_ECUDA = 7,     /* a CUDA runtime call failed */
    ESC_EBOUNDS = 8    /* checked build only: a kernel found an index out of range (and skipped the access) */
} esc_status;

/* Column element types.  Values are widened to int64 for every comparison:
 * signed types sign-extend, unsigned types zero-extend. */
typedef enum esc_dtype { ESC_I32 = 0, ESC_I64 = 1, ESC_U8 = 2, ESC_U16 = 3 } esc_dtype;

/* One column of a table: `data` is a device array of nrows elements of
 * `dtype`, 16-byte aligned.  `name` is copied at table creation. */
typedef struct esc_column {
    const char *name;
    int32_t dtype;        /* esc_dtype */
    const void *data;     /* device pointer, borrowed */
} esc_column;

typedef struct esc_table esc_table;   /* opaque column-store table */
typedef struct esc_pred esc_pred;     /* opaque compiled predicate bound to a table */
typedef struct esc_batch esc_batch;   /* opaque prepared batch of sub-queries */

/* Caller-owned output buffers for the materialised sub-query result.
 * row_ids: device array of `capacity` uint32 row ids, written in ascending
 * order.  proj: host array of nproj device pointers, one per projected
 * column (in the order given to esc_predicate_compile), each an array of
 * `capacity` elements of that column's type.  `written` is set by
 * synchronous calls to min(count, capacity). */
typedef struct esc_rows {
    uint64_t capacity;
    uint32_t *row_ids;
    void *const *proj;
    uint64_t written;
} esc_rows;

/* ---------------------------------------------------------------- tables */

#define ESC_MAX_ROWS 4294901760ull /* 2^32 - 2^16 */

/* Columnar table store (Sec. 2: column-wise in-memory tables).  Registers
 * `ncols` (1..64) borrowed device columns of `nrows` rows each (0 to
 * ESC_MAX_ROWS = 2^32 - 2^16: row ids are uint32, and every extent rounded up
 * to a compaction unit, at most 65536 rows, stays below 2^32).  Column
 * names must be distinct identifiers.  Each `data` must be 16-byte aligned
 * (ESC_EINVAL otherwise) and stay valid until esc_table_destroy.  Unknown dtypes give ESC_ETYPE.  *out is owned by the
 * caller and released with esc_table_destroy. */
esc_status esc_table_create(const esc_column *cols, int32_t ncols, uint64_t nrows,
                            esc_table **out);
esc_status esc_table_destroy(esc_table *table);
uint64_t esc_table_nrows(const esc_table *table);

/* ---------------------------------------------------------------- predicates */

/* Compiles a selection predicate (the WHERE clause of the selectivity
 * sub-query, Sec. 1 and Sec. 2) over `table` into a flat postfix program,
 * and binds the projection pushed down with it (Sec. 2: the columns later
 * operators need).
 *
 * Language (keywords case-insensitive, column names case-sensitive):
 *   pred    := or;  or := and (OR and)*;  and := unary (AND unary)*
 *   unary   := NOT unary | '(' pred ')' | TRUE | FALSE | test
 *   test    := operand cmp INT | operand [NOT] BETWEEN INT AND INT
 *            | operand [NOT] IN '(' [INT (',' INT)*] ')'
 *   operand := column | udf '(' column ',' column ',' INT ')'
 *   cmp     := = | == | != | <> | < | <= | > | >=
 * INT is a decimal int64.  BETWEEN is inclusive (empty when lo > hi).
 * The compiled program is an exact simplification: comparisons become ranges
 * clamped to the operand's domain, and tests on one operand (a column, or a
 * udf with the same columns in either order and the same m) combine --
 * intersected under AND, united under OR -- so esc_predicate_explain may
 * list fewer tests than the text has; results never change.
 * udf(a, b, m) is (a * b) mod m with the product wrapping in 64-bit two's
 * complement and the remainder truncated toward zero; m must be > 0.
 * An IN list holds at most 16 values; an empty list is false.
 *
 * proj: `nproj` (0..16) column names to materialise.  Limits: at most 16
 * distinct columns read by the predicate, 64 program instructions, nesting
 * that needs at most 8 evaluation-stack entries; each violation, a syntax
 * error, an unknown column or m <= 0 gives ESC_EINVAL with a message.
 * *out is released with esc_predicate_destroy; the table must outlive it. */
esc_status esc_predicate_compile(const esc_table *table, const char *text,
                                 const char *const *proj, int32_t nproj, esc_pred **out);
esc_status esc_predicate_destroy(esc_pred *pred);

/* Compiles n predicates against one table, as esc_predicate_compile does for
 * each (same projection for all), on up to `nthreads` host threads
 * (<= 0: one per hardware thread; at least 64 predicates per thread).
 * out: host array of n handles, each released with esc_predicate_destroy.
 * If any text fails, every handle is released, out[] is all NULL, and the
 * status is that of the failing predicate of lowest index, whose index the
 * message names. */
esc_status esc_predicate_compile_many(const esc_table *table, const char *const *texts, int32_t n,
                                      const char *const *proj, int32_t nproj, esc_pred **out,
                                      int32_t nthreads);

/* Launch shape of a compiled predicate's scans (the autotuner's knobs; not
 * in the paper).  max_tile_rows: rows staged per tile (256..32768, a
 * multiple of 256; the stage size caps it further); max_unit_kb: staged
 * bytes per work unit (16..4096; a unit is a run of tiles claimed with one
 * ticket; the last tiles of a table always go out one per unit);
 * units_per_sm: work units to aim for per SM (1..64; more balances load,
 * fewer amortises per-unit work).  consumer_warps and rows_per_pass pick the
 * scan kernel's block shape: the warps per CTA that evaluate (the CTA has
 * one more, the copy warp) and the rows each lane evaluates per decoded
 * program instruction (8 per 256-row group, one, two or four groups per
 * pass).  The shapes compiled are (15, 16) and (19, 8), which run every
 * program, and (19, 16), (23, 8) and (15, 32), which run programs without a
 * udf.  (0, 0) is
 * automatic: a program reading more than 20 bytes per row runs (19, 8) if
 * it has a udf, else (23, 8); a narrower one (15, 16) or (19, 16).
 * Defaults: 32768, 512, 8, 0, 0.  A batch (esc_batch_prepare,
 * esc_selectivity_batch) uses its queries' tile and unit sizes, but its
 * queries share a launch, so each launch takes the automatic shape: with
 * the udf path if any of its programs has a udf, and the wide form if
 * programs reading more than 20 bytes per row hold most of its bytes.
 * Results never depend on any of these. */
typedef struct esc_tuning {
    uint32_t max_tile_rows;
    uint32_t max_unit_kb;
    int32_t units_per_sm;
    uint16_t consumer_warps;
    uint16_t rows_per_pass;
} esc_tuning;

/* Sets (tuning NULL: restores the defaults) or reads a predicate's launch
 * shape.  ESC_EINVAL for values outside the ranges above, for a block shape
 * that is not compiled, and for a shape without the udf path on a program
 * with a udf; the predicate's tuning is then unchanged.  Not thread-safe
 * against concurrent calls that use the same predicate. */
esc_status esc_predicate_set_tuning(esc_pred *pred, const esc_tuning *tuning);
esc_status esc_predicate_get_tuning(const esc_pred *pred, esc_tuning *out);

/* Writes a NUL-terminated listing of the compiled program (read columns,
 * projection, one line per instruction) into buf[0..buflen).  ESC_EINVAL if
 * it does not fit. */
esc_status esc_predicate_explain(const esc_pred *pred, char *buf, uint64_t buflen);

/* ---------------------------------------------------------------- sub-queries */

/* The selectivity sub-query (Sec. 2): *count (host) receives the exact
 * number of rows of `table` satisfying `pred`.  When `rows` is not NULL the
 * qualifying rows are also materialised (Sec. 2.1): their ids in ascending
 * order and their projected columns, in the caller's buffers.  If count >
 * rows->capacity, the first `capacity` rows are written, rows->written =
 * capacity, *count is still exact and the status is ESC_ETRUNC.
 * Synchronises `stream`.  `pred` must have been compiled against `table`. */
esc_status esc_selectivity(const esc_table *table, const esc_pred *pred, uint64_t *count,
                           esc_rows *rows, void *stream);

/* Same as esc_selectivity without synchronising: the exact count is written
 * to the device word *dev_count when the stream reaches that point, and
 * rows->written is not set (it is min(count, capacity)).  Truncation and
 * device-side timeouts are not reported by this call. */
esc_status esc_selectivity_async(const esc_table *table, const esc_pred *pred,
                                 uint64_t *dev_count, esc_rows *rows, void *stream);

/* Allocation-free form of esc_selectivity, for callers that must not
 * allocate device memory: code running inside an allocator of its own (a
 * buffer pool that owns the GPU's memory), code on a latency-critical path
 * where cudaMalloc and cudaFree would synchronise the device, or host code
 * that runs where CUDA allocation calls are not allowed.  The paper has no
 * counterpart; it is an interface convenience of this library.
 * Same arguments, results and status codes as esc_selectivity.  It calls no
 * cudaMalloc, cudaFree or other allocating routine: its scratch is a 12 MiB
 * array built into the library, reserved on every device that loads the
 * library until the process exits.  Counting alone fits any table; with
 * `rows` (materialisation) the table may have up to about 95 million rows
 * (the scratch needs about nrows/8 bytes); larger tables give ESC_EINVAL.
 * The first call on a device looks up the array's device address (no
 * allocation).  Every call
 * shares the one array: calls whose GPU work overlaps (different streams,
 * or host threads without ordering) race and give wrong results.
 * Synchronises `stream`. */
esc_status esc_selectivity_noalloc(const esc_table *table, const esc_pred *pred, uint64_t *count,
                                   esc_rows *rows, void *stream);

/* Batched sub-queries (Sec. 2: one per table that has a selection): the n
 * pairs (tables[i], preds[i]) run in one persistent kernel launch, captured
 * in a CUDA graph at prepare time.  rows may be NULL (counts only) or an
 * array of n esc_rows whose entries with capacity 0 and row_ids NULL are
 * count-only.  All buffers are borrowed and must stay valid until
 * esc_batch_destroy.  esc_batch_run writes n exact counts to the device
 * array dev_counts and, if dev_done_ns is not NULL, the device time
 * (%globaltimer, ns) at which each sub-query's last tile finished.  Runs
 * enqueued on one stream are ordered; concurrent runs of the same batch on
 * different streams are not allowed (ESC_EBUSY is not detected). */
esc_status esc_batch_prepare(const esc_table *const *tables, const esc_pred *const *preds,
                             int32_t n, const esc_rows *rows, esc_batch **out);

/* Same as esc_batch_prepare, in `waves` launches (1..16) instead of one, for
 * per-sub-query latency: the sub-queries are ordered by the bytes their
 * scans read, smallest first (esc_batch_prepare orders them the same way),
 * and cut into consecutive waves whose work doubles from one to the next
 * (the last about half of the batch).  Each wave is one persistent scan
 * launch and, when it materialises, one write launch, all captured in the
 * batch's CUDA graph; a sub-query completes with its wave, so small ones
 * complete early.  Results, completion times and status as for
 * esc_batch_prepare.  Not in the paper (the optimizer's sub-queries are
 * issued one per table with a selection, Sec. 2). */
esc_status esc_batch_prepare_waves(const esc_table *const *tables, const esc_pred *const *preds,
                                   int32_t n, const esc_rows *rows, int32_t waves, esc_batch **out);
esc_status esc_batch_run(esc_batch *batch, uint64_t *dev_counts, uint64_t *dev_done_ns,
                         void *stream);
esc_status esc_batch_destroy(esc_batch *batch);

/* Asynchronous batch without a prepared graph, for a stream of changing
 * sub-queries (the serving loop): enqueues the n sub-queries as one
 * persistent scan launch (plus one compaction write launch when any has
 * rows), with scratch from the library's stream-ordered pool.  Writes n exact
 * counts to dev_counts and, when dev_done_ns is not NULL, each sub-query's
 * completion time (%globaltimer).  Does not synchronise; `rows` entries with
 * capacity 0 and row_ids NULL are count-only; truncation is not reported
 * (written = min(count, capacity)).  Host arrays may be freed on return. */
esc_status esc_selectivity_batch_async(const esc_table *const *tables, const esc_pred *const *preds,
                                       int32_t n, const esc_rows *rows, uint64_t *dev_counts,
                                       uint64_t *dev_done_ns, void *stream);

/* Count-only sub-queries of many predicates on one table in one pass over
 * it (a shared scan; not in the paper): every tile of the union of the
 * columns the predicates read is staged once and each predicate evaluated on
 * it.  preds: n (>= 1) predicates compiled against `table` (projections are
 * ignored); dev_counts: device array receiving the n exact counts, in the
 * order of preds, when the stream reaches that point.  Predicates are taken
 * in passes whose read columns fit the 16 stage slots, at most 2048 per
 * pass.  Does not synchronise; host arrays may be freed on return.
 * ESC_EINVAL for a NULL argument or a predicate of another table. */
esc_status esc_selectivity_shared_async(const esc_table *table, const esc_pred *const *preds, int32_t n,
                                        uint64_t *dev_counts, void *stream);

/* One-shot form of the above: prepares, runs, synchronises and destroys.
 * counts is a host array of n entries. */
esc_status esc_selectivity_batch(const esc_table *const *tables, const esc_pred *const *preds,
                                 int32_t n, uint64_t *counts, esc_rows *rows, void *stream);

/* ---------------------------------------------------------------- joins */

/* Dense-key bitmap of a filtered dimension table: bit k of the device array
 * dev_bitmap (word k / 32, bit k % 32, little-endian bit order) is set when
 * row k -- the row whose dense key is k -- satisfies pred.  dev_bitmap holds
 * ceil(nrows / 32) uint32 words, all of which are written.  *count (host,
 * may be NULL) receives the number of set bits.  Synchronises `stream`. */
esc_status esc_bitmap_build(const esc_table *dim, const esc_pred *pred, uint32_t *dev_bitmap,
                            uint64_t *count, void *stream);

/* Exact semi-join cardinalities of a fact table against filtered dimensions
 * on dense keys (the COUNT(*) foreign-key join queries of Sec. 3.1):
 * for every subset S of the ndims (1..4) dimensions, subset_counts[S] (host,
 * 2^ndims entries, bit d of S = dimension d) receives
 *   |{ i : for all d in S, 0 <= fk_d[i] < dim_rows[d] and bit fk_d[i] of
 *          dev_bitmaps[d] is set }|,
 * which equals |fact JOIN_S sigma(dims)| when dimension keys are dense and
 * unique.  fk_cols names ndims distinct ESC_I32 columns of `fact`.
 * dev_bitmaps[d] (host array of device pointers) holds ceil(dim_rows[d]/32)
 * words.  Synchronises `stream`. */
esc_status esc_semijoin_counts(const esc_table *fact, const char *const *fk_cols, int32_t ndims,
                               const uint32_t *const *dev_bitmaps, const uint64_t *dim_rows,
                               uint64_t *subset_counts, void *stream);

/* ---------------------------------------------------------------- learned surrogate */

/* A learned selectivity estimator built on top of ESC (not in the paper; the
 * paper's counts are exact -- this network is trained on them and evaluated
 * against them): an MLP 64 -> 128 -> ReLU -> 128 -> ReLU -> 1 mapping encoded
 * predicate features to log10 selectivity.  Parameters are one flat array
 * of ESC_MLP_PARAMS floats: W1 [128][64] row-major, b1 [128], W2 [128][128],
 * b2 [128], w3 [128], b3.  `w_bf16` is a bfloat16 copy of the same array
 * (the weights the matrix products use; its bias entries are ignored).
 * All accumulation is float32.  Every pointer is a device pointer; nothing
 * is synchronised. */
#define ESC_MLP_PARAMS 24961

/* y[i] = network(x[i]) for `batch` rows of 64 bfloat16 features. */
esc_status esc_mlp_forward(const uint16_t *x_bf16, uint64_t batch, const uint16_t *w_bf16,
                           const float *params, float *y, void *stream);

/* Adds to grad[ESC_MLP_PARAMS] the gradient of mean_i (y_i - target_i)^2
 * over the batch, and to *loss_sum the sum of squared errors.  The caller
 * zeroes both beforehand. */
esc_status esc_mlp_grad(const uint16_t *x_bf16, const float *target, uint64_t batch,
                        const uint16_t *w_bf16, const float *params, float *grad, float *loss_sum,
                        void *stream);

/* One Adam step (Kingma & Ba 2015) on n float32 parameters with first and
 * second moments m, v; `step` counts from 1 (bias correction).  Also
 * refreshes the bfloat16 copy. */
esc_status esc_mlp_adam(float *params, uint16_t *w_bf16, const float *grad, float *m, float *v,
                        uint64_t n, float lr, float beta1, float beta2, float eps, int32_t step,
                        void *stream);

/* ---------------------------------------------------------------- misc */

/* Message for the last non-OK status returned to the calling thread. */
const char *esc_last_error(void);
const char *esc_status_string(esc_status status);

/* Multiplier and shifts used to divide by the udf modulus d (d >= 1) with a
 * multiply-high, after Granlund and Montgomery, "Division by Invariant
 * Integers using Multiplication" (PLDI 1994), Fig. 4.1: for every 64-bit n,
 * t = mulhi(mult, n), n / d = (t + ((n - t) >> sh1)) >> sh2. */
esc_status esc_udf_magic(uint64_t d, uint64_t *mult, int32_t *sh1, int32_t *sh2);

/* Writes the device's nanosecond clock (%globaltimer, the clock of the
 * per-sub-query completion times of esc_batch_run) to the device word
 * *dev_ns when the stream reaches this point.  Not in the paper: used to
 * measure per-sub-query latency from a common start. */
esc_status esc_timestamp(uint64_t *dev_ns, void *stream);

/* Runs a one-CTA kernel that waits on a device flag nothing sets, with the
 * same bounded wait the scan kernels use, giving up after about `limit_ns`
 * nanoseconds.  Returns ESC_ETIMEOUT when the wait gave up (the expected
 * outcome) and leaves the context usable.  Exercises failure detection
 * without faulting a GPU. */
esc_status esc_selftest_wait_timeout(uint64_t limit_ns, void *stream);

/* Test hooks (not in the paper; they exercise the error paths without a
 * GPU fault).  esc_debug_fail_allocs(n): the library's next n device
 * allocations (per-call scratch, batch memory) fail with ESC_ENOMEM as if
 * the device were out of memory, and the calls that make them return
 * ESC_ENOMEM having launched nothing; n = 0 turns the injection off.
 * esc_build_checked(&flag): *flag = 1 in the checked build
 * (libesc_checked.so), whose kernels test the indices they are about to use
 * and report ESC_EBOUNDS (with the site and the index in the message)
 * instead of touching memory out of range; 0 in the release build.
 * esc_debug_write_units(nrows, slots, ...): the compaction units a
 * materialising call on a table of nrows rows (<= ESC_MAX_ROWS) uses when
 * the GPU holds `slots` write-kernel blocks at once (slots = 0: the
 * full-size units of a batch); out (host, 3 entries): the groups of 256
 * rows per unit, the number of units, and the reciprocal that maps a group
 * to its unit (ceil(2^32 / groups per unit), 0 for one group). */
esc_status esc_debug_fail_allocs(int32_t n);
esc_status esc_build_checked(int32_t *flag);
esc_status esc_debug_write_units(uint64_t nrows, int32_t slots, uint32_t *out);

#ifdef __cplusplus
}
#endif
#endif /* ESC_H */
