/*
 * mdrq.h — C ABI of the GB300 multidimensional range query (MDRQ) scan library.
 *
 * Problem (Sec. 2.1 of "Multidimensional Range Queries on Modern Hardware",
 * arXiv 1801.03644): a table holds n objects with d attributes (dimensions). A query
 * gives closed intervals [lo_j, hi_j] on some or all dimensions; an object qualifies
 * iff lo_j <= x_j <= hi_j for every constrained dimension j, and a dimension the
 * query leaves out behaves as [-inf, +inf] (partial-match query). The answer is the
 * set of identifiers of the qualifying objects, where the identifier of an object is
 * its row index i (Sec. 2.2.4). This library returns it as an ascending uint32 list.
 *
 * Layout: the table is held column-wise on the GPU, one contiguous array per
 * dimension (the vertical layout of Sec. 3.2), so a query reads only the columns it
 * constrains. Columns are float32 or int32 (Sec. 7.2 uses float32 throughout).
 *
 * Conventions for every function below:
 *  - Return value: MDRQ_OK (0) or a negative mdrq_status. Nothing is thrown.
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream). Work is enqueued
 *    on it and the call returns once the status is known (it synchronises that
 *    stream), unless the function says otherwise.
 *  - Pointers marked "device" must be device-accessible memory of the current CUDA
 *    device; "host" pointers are plain host memory (pinned memory copies faster).
 *  - The caller owns every buffer it passes in; the library owns mdrq_table and the
 *    scratch memory inside it.
 *  - Calls on one table must not run concurrently (a table holds one scratch area).
 *  - Floating-point data and bounds never contain NaN: mdrq_load_columns rejects NaN
 *    data (MDRQ_E_NAN) and the query calls reject NaN bounds (MDRQ_E_INVAL). With NaN
 *    excluded, the closed-interval test of Sec. 2.1 (ordered IEEE compare, so
 *    -0.0 == +0.0; +-inf allowed as bounds) is the same under both of the paper's
 *    listings (Listing 1 and Listing 2), which otherwise disagree on NaN.
 */
#ifndef MDRQ_H
#define MDRQ_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Column element types. */
typedef enum { MDRQ_F32 = 0, MDRQ_I32 = 1 } mdrq_dtype;

/* Status codes. */
typedef enum {
    MDRQ_OK = 0,
    MDRQ_E_INVAL = -1,    /* bad argument: see each function */
    MDRQ_E_NOMEM = -2,    /* a device or host allocation failed */
    MDRQ_E_CUDA = -3,     /* a CUDA runtime call failed; the table may be unusable */
    MDRQ_E_CAPACITY = -4, /* the answer is longer than the caller's id buffer */
    MDRQ_E_TIMEOUT = -5,  /* a bounded device-side wait gave up; results are invalid */
    MDRQ_E_NAN = -6       /* a float32 column holds a NaN */
} mdrq_status;

/* Opaque table handle (library-owned). */
typedef struct mdrq_table mdrq_table;

/* One bound, read as float32 or int32 according to the type of the column. */
typedef union {
    float f;
    int32_t i;
} mdrq_value;

/*
 * One predicate p_j = [lo, hi] on dimension `dim` (Sec. 2.1). lo > hi is valid and
 * matches nothing. A dimension may appear in several predicates of one query; they
 * are ANDed. `reserved` must be 0.
 */
typedef struct {
    uint32_t dim;
    uint32_t reserved;
    mdrq_value lo;
    mdrq_value hi;
} mdrq_pred;

/* One query of a batch: `npreds` predicates at host address `preds`. */
typedef struct {
    const mdrq_pred *preds;
    uint32_t npreds;
    uint32_t reserved;
} mdrq_qdesc;

/*
 * mdrq_load_columns — make a table of n objects with d dimensions resident on the
 * current CUDA device (the vertical partitioning of Sec. 3.2: one array per dimension).
 *
 *  cols[j]        column j: n values of type types[j] (MDRQ_F32 / MDRQ_I32).
 *                 cols_on_device = 0: host pointers; the values are copied to the GPU.
 *                 cols_on_device = 1: device pointers, each 16-byte aligned; the table
 *                 refers to that memory, which must outlive the table and stay
 *                 unchanged while it is in use.
 *  d              number of dimensions, >= 1.
 *  n              number of objects, <= 2^32 - 1 (identifiers are uint32). n = 0 is a
 *                 valid empty table.
 *  stream         stream for the copies and checks.
 *  out            receives the handle; release it with mdrq_free.
 *
 * Loading also limits the L2 cache's fetch granularity of the current CUDA context
 * to 32 bytes (cudaLimitMaxL2FetchGranularity): the scan's early break reads isolated
 * 32-byte sectors, and larger fetches would bring in the sectors it skips. The limit
 * applies to every kernel of the context and ends with it; a caller who wants another
 * value sets it again after loading.
 *
 * Errors: MDRQ_E_INVAL (d = 0, n >= 2^32, a null pointer where n > 0, an unknown
 * type, a device column that is not 16-byte aligned, out == NULL); MDRQ_E_NAN (a
 * float32 column holds a NaN; nothing is kept); MDRQ_E_NOMEM; MDRQ_E_CUDA.
 */
int mdrq_load_columns(const void *const *cols, const int32_t *types, uint32_t d, uint64_t n,
                      int cols_on_device, void *stream, mdrq_table **out);

/*
 * mdrq_query — answer one MDRQ (Sec. 2.1) with a full parallel scan of the
 * constrained columns (Sec. 5.5), returning the qualifying row indices in ascending
 * order.
 *
 *  preds, npreds  host array of predicates; npreds = 0 is the full-domain query
 *                 (all n ids). At most 128 distinct dimensions may be constrained.
 *  ids            output, `capacity` uint32 slots; device memory when
 *                 ids_on_device = 1, host memory when 0. Host answers in page-locked
 *                 memory (cudaHostAlloc / cudaHostRegister, a pinned torch tensor) are
 *                 written by the scan kernels themselves over the CPU-GPU link, unless
 *                 the batch's output is staged (see mdrq_set_host_answers and
 *                 mdrq_set_output_order). Other host memory goes through a device
 *                 staging buffer of `capacity` ids that the table keeps; a plain batch
 *                 that scans at least 2 GiB of columns then runs as several launches
 *                 (up to 16, of equal query counts, on average at least 1 GiB of
 *                 columns each) and the ids of each are copied out (on a second
 *                 stream) while the next one runs; a smaller batch is one launch
 *                 followed by one copy.
 *  count          host; receives the length of the answer (also when it exceeds
 *                 capacity).
 *
 * Errors: MDRQ_E_INVAL (t or count NULL, dim >= d, a NaN float bound, nonzero
 * reserved field, ids NULL with capacity > 0, more than 128 constrained
 * dimensions); MDRQ_E_CAPACITY (*count > capacity: the first `capacity` ids are
 * written, nothing beyond); MDRQ_E_TIMEOUT; MDRQ_E_NOMEM; MDRQ_E_CUDA.
 */
int mdrq_query(mdrq_table *t, const mdrq_pred *preds, uint32_t npreds, uint32_t *ids,
               uint64_t capacity, uint64_t *count, int ids_on_device, void *stream);

/*
 * mdrq_query_batch — answer nq queries; the answers are concatenated in query order
 * into `ids` in CSR form: query q's ascending ids are ids[offsets[q] .. offsets[q+1]).
 *
 *  qs, nq         host array of nq query descriptors (nq = 0 is valid).
 *  ids, capacity  output as for mdrq_query, holding the concatenation.
 *  offsets        host, nq + 1 entries; offsets[0] = 0 and offsets[nq] is the total
 *                 length (also when it exceeds capacity).
 *
 * Errors: as mdrq_query; MDRQ_E_CAPACITY when offsets[nq] > capacity (every id at a
 * position below capacity is written, nothing beyond).
 */
int mdrq_query_batch(mdrq_table *t, const mdrq_qdesc *qs, uint32_t nq, uint32_t *ids,
                     uint64_t capacity, uint64_t *offsets, int ids_on_device, void *stream);

/*
 * mdrq_set_host_answers — how answers bound for host memory (ids_on_device = 0) get
 * there; the paper's answers stay in the memory of the machine that scans (Sec. 7.1).
 *  MDRQ_HOST_AUTO    (default) written by the scan itself when the buffer is page-locked
 *                    and mapped into the device's address space (on a GPU that shares a
 *                    coherent link with the CPU, as on GB300, the stores cross that link
 *                    at the scan's pace), staged otherwise. A plain batch whose output
 *                    is staged (mdrq_set_output_order) is ordered by a pass after each
 *                    scan launch, so its ids are always staged and copied, each
 *                    launch's while the next one runs;
 *  MDRQ_HOST_STAGED  always through the device staging buffer and copies;
 *  MDRQ_HOST_DIRECT  always written by the scan; calls with a buffer that is not
 *                    page-locked fail with MDRQ_E_INVAL.
 * Answers are identical in every mode. Errors: MDRQ_E_INVAL (t NULL, unknown mode).
 */
#define MDRQ_HOST_AUTO 0
#define MDRQ_HOST_STAGED 1
#define MDRQ_HOST_DIRECT 2
int mdrq_set_host_answers(mdrq_table *t, int mode);

/*
 * mdrq_set_output_order — how a plain scan launch puts the partial results of its
 * partitions (one row tile of one query each) into ascending order; the paper
 * concatenates its partitions' results in partition order (Sec. 3.1).
 *  MDRQ_ORDER_AUTO      (default) staged for a plain launch of at least 8 tiles per
 *                       resident thread block (on GB300 about 8,500 tiles, e.g. 100
 *                       queries of 1M rows or one query of 35M rows), look-back below
 *                       that and for windowed launches;
 *  MDRQ_ORDER_LOOKBACK  each tile finds its place in the answer while the scan runs
 *                       (single-pass decoupled look-back over the tiles' counts);
 *                       nothing beyond the scratch of mdrq_load_columns is allocated;
 *  MDRQ_ORDER_STAGED    each tile writes its ids to a device staging buffer of
 *                       `capacity` ids plus 3 per tile (a tile's run is padded to a
 *                       multiple of 4 ids) and an 8-byte record per tile (both kept by
 *                       the table and grown as needed), and an ordering pass of three
 *                       kernels after the scan copies every tile's ids into place: the
 *                       ids are written twice, but no tile of the scan waits on another.
 *                       A launch whose staging buffers cannot be allocated uses the
 *                       look-back instead.
 * Answers are identical in every order. It applies to the plain scan's launches (batch
 * mode PLAIN, AUTO when that scans plainly, single queries, prepared batches) and to
 * the windowed launches of tile pruning (mdrq_set_zone_maps) and of the learned
 * narrower (MDRQ_BATCH_LEARNED), which are staged only under MDRQ_ORDER_STAGED: they
 * read few rows per id they write, so the second write of the ids costs more than the
 * look-back saves. A staged windowed launch sizes its tile records by its upper bound
 * of tiles (every tile of every query plus one per window), since its tile count is
 * known only on the device. The shared and allocation-free
 * paths order their output their own way, and the serving loop's plain batches use
 * the look-back.
 * Errors: MDRQ_E_INVAL (t NULL, unknown mode).
 */
#define MDRQ_ORDER_AUTO 0
#define MDRQ_ORDER_LOOKBACK 1
#define MDRQ_ORDER_STAGED 2
int mdrq_set_output_order(mdrq_table *t, int mode);

/* mdrq_free — release a table and its device memory (not caller-owned columns). NULL is
 * a no-op. Synchronises the device work the table still has in flight. */
void mdrq_free(mdrq_table *t);

/* Short English description of a status code (static storage). */
const char *mdrq_status_string(int status);

/* Table shape: number of objects and of dimensions (0 for NULL). */
uint64_t mdrq_table_rows(const mdrq_table *t);
uint32_t mdrq_table_dims(const mdrq_table *t);

/*
 * mdrq_last_scan_stats — figures of the most recent query call on this table, for
 * measurement: the number of scan-kernel launches it made and the algorithmic bytes
 * they imply (4 bytes per row per constrained column, plus 4 bytes per id written).
 * Either pointer may be NULL.
 */
void mdrq_last_scan_stats(const mdrq_table *t, uint64_t *launches, uint64_t *bytes);

/*
 * mdrq_explain_query — the plan the scan follows for one query (query encoding, Sec.
 * 2.1 with Sec. 2.2.4's most-selective-first order): the predicates it evaluates, in
 * evaluation order, after predicates on one dimension are intersected (ANDed) and
 * predicates that every value of their column satisfies are dropped. *empty = 1 when
 * the query is answered as empty without a scan (an empty interval, or one that no
 * value of its column meets); the plan is then empty. Nothing runs on the GPU.
 *
 *  preds, npreds   host predicates, as mdrq_query.
 *  plan, max_plan  host output: plan[i].dim and its intersected bounds (column type).
 *  nplan, empty    host outputs.
 *
 * Errors: MDRQ_E_INVAL (t, nplan or empty NULL, plan NULL with max_plan > 0, a bad
 * predicate as for mdrq_query); MDRQ_E_CAPACITY (*nplan > max_plan: the first max_plan
 * entries are written).
 */
int mdrq_explain_query(const mdrq_table *t, const mdrq_pred *preds, uint32_t npreds, mdrq_pred *plan,
                       uint32_t max_plan, uint32_t *nplan, int *empty);

/*
 * mdrq_scan_timing — measurement aid: turn per-launch timing of the scan kernel on
 * (enable = 1) or off (0) for this table. While on, every scan launch is bracketed
 * by two CUDA events recorded on the stream it is launched on.
 * Errors: MDRQ_E_INVAL (t NULL).
 */
int mdrq_scan_timing(mdrq_table *t, int enable);

/*
 * mdrq_scan_timing_read — what the timed calls since the last reset measured:
 *  ms               summed device time between each timed launch's two events
 *  scan_launches    scan-kernel launches timed
 *  bytes            their algorithmic bytes (4 per row per constrained column, plus
 *                   4 per id written)
 *  kernel_launches  kernels of this library launched by the timed calls, all kinds
 * Any output pointer may be NULL. Waits for the last recorded event. reset = 1
 * clears the counters afterwards. Errors: MDRQ_E_INVAL (t NULL); MDRQ_E_CUDA.
 */
int mdrq_scan_timing_read(mdrq_table *t, double *ms, uint64_t *scan_launches, uint64_t *bytes,
                          uint64_t *kernel_launches, int reset);

/*
 * mdrq_set_batch_mode — how mdrq_query_batch answers a batch on this table.
 *  MDRQ_BATCH_PLAIN   every query is scanned on its own (one persistent launch for the
 *                     batch; the columns a query constrains are read once per query).
 *  MDRQ_BATCH_SHARED  shared scan: the queries are evaluated together, each constrained
 *                     column is read once per group of up to 128 queries, and every
 *                     row's set of matching queries comes from per-column tables of the
 *                     queries' interval end points (two passes: count, then write).
 *                     Between the passes the table keeps every row's query bits (16
 *                     bytes per row and group of 128 queries) when that fits 32 GB and
 *                     a quarter of the free device memory; the buffer stays with the
 *                     table for later batches. Otherwise the write pass evaluates the
 *                     columns again.
 *  MDRQ_BATCH_LEARNED every query scans only the rows its learned window allows (see
 *                     mdrq_learn); MDRQ_E_INVAL without a model.
 *  MDRQ_BATCH_AUTO    (default) shared when the batch has at least 32 queries that need
 *                     a scan and the table at least 4,000,000 rows, plain otherwise;
 *                     after mdrq_autotune, the faster of the two as measured there (for
 *                     batches of 32 or more queries).
 * Both modes return identical answers. The paper answers one query at a time (Sec.
 * 7.1.2); the shared scan is this library's extension for batches.
 * Errors: MDRQ_E_INVAL (t NULL or unknown mode).
 */
#define MDRQ_BATCH_AUTO 0
#define MDRQ_BATCH_PLAIN 1
#define MDRQ_BATCH_SHARED 2
#define MDRQ_BATCH_LEARNED 3 /* see mdrq_learn */
int mdrq_set_batch_mode(mdrq_table *t, int mode);

/*
 * mdrq_learn — build a learned range narrower for MDRQ_BATCH_LEARNED; the paper has no
 * learned component (its index structures are the R*-tree, kd-tree and VA-file, Sec.
 * 2.2); this narrows the full scan of Sec. 2.2.4 to the rows a query can match.
 *
 * The table's rows must already be sorted by the 32-bit Z-order (Morton) key of the
 * float32 columns dims[0 .. ndims) (1 <= ndims <= 4): key bit 4b + j is bit b of
 * cell(x_dims[j]), where cell(x) is the number of the column's 255 cell bounds at or
 * below x when mdrq_set_key_cells gave it bounds (for instance the column's quantiles,
 * so that every cell holds about as many rows), and clamp(floor(x * 256), 0, 255) in
 * float32 otherwise. The cells of a
 * query box then form key ranges, each one run of rows of the sorted table. Per batch
 * the GPU splits every query's box into at most 1024 such ranges (the key-bit tree
 * expanded level by level, largest runs first; the ranges left at the budget cover
 * some cells outside the box, whose rows the scan rejects), and the model predicts
 * each range's run from its end keys:
 *  MDRQ_MODEL_PLA  piecewise-linear, 4096 segments through evenly spaced (key, row)
 *                  pairs of the sorted keys, FP32;
 *  MDRQ_MODEL_MLP  two stages: a 1-32-32-1 ReLU network, FP32, trained on the GPU
 *                  (Adam, 3000 steps of 8192 pairs from a 2^20-pair sample) on the key
 *                  normalised over the column's key range, sends a key to one of 2^18
 *                  leaves (floor of its output times 2^18); the leaf's line through the
 *                  first and last (key, row) pair sent to it predicts the row;
 *  MDRQ_MODEL_NONE no model: every range's run is searched in the whole key column
 *                  (the ablation that measures what a model saves).
 * Its largest error over all n keys is measured exhaustively (mdrq_learn_info). Each
 * predicted window is proven against the key column (widened until the keys just
 * outside it lie outside the range) and narrowed to the range's exact run before it is
 * scanned with every predicate, so answers equal the full scan's whatever the model. Training and the key column (4
 * bytes per row) stay with the table; calling again replaces the model.
 *
 * Errors: MDRQ_E_INVAL (bad dims or model, a dim that is not float32, n = 0, or rows not
 * in key order); MDRQ_E_NOMEM; MDRQ_E_CUDA.
 */
#define MDRQ_MODEL_PLA 1
#define MDRQ_MODEL_MLP 2
#define MDRQ_MODEL_NONE 3

/* mdrq_set_key_cells — the cells of key dimension `dim` for later mdrq_learn calls:
 * bounds[0 .. 255) ascending (no NaN) split the values into 256 cells, cell(x) = the
 * number of bounds <= x; nbounds = 0 returns the column to equal-width cells. A model
 * keeps the cells it was trained with. The paper has no counterpart (its index
 * structures partition space by their own rules). Errors: MDRQ_E_INVAL (t NULL, dim >=
 * d, nbounds other than 0 or 255, bounds NULL, NaN or not ascending). */
int mdrq_set_key_cells(mdrq_table *t, uint32_t dim, const float *bounds, uint32_t nbounds);
int mdrq_learn(mdrq_table *t, const uint32_t *dims, uint32_t ndims, int model, void *stream);

/* mdrq_learn_info — the model's largest position error over all keys (n for
 * MDRQ_MODEL_NONE), its segments (PLA) or leaves (MLP; 0 for none) and the training time
 * in ms. Any pointer may be NULL. Errors: MDRQ_E_INVAL (t NULL or no model). */
int mdrq_learn_info(const mdrq_table *t, uint64_t *max_error, uint32_t *segments, double *train_ms);

/* mdrq_learn_window_rows — measurement aid: rows the last MDRQ_BATCH_LEARNED call's
 * windows covered (summed over its queries; of its last launch when the batch needed
 * several) and how many widening steps the window checks took (0 when every model
 * window already held its key run). Synchronous. Errors: MDRQ_E_INVAL (no model). */
int mdrq_learn_window_rows(mdrq_table *t, uint64_t *rows, uint64_t *widenings);

/* mdrq_learn_search_info — measurement aid: key ranges the last MDRQ_BATCH_LEARNED call
 * searched (of its last launch) and the keys its searches read in all (the two window
 * checks, the widening steps and both binary searches of every range). Synchronous.
 * Errors: MDRQ_E_INVAL (t NULL or no model); MDRQ_E_CUDA. */
int mdrq_learn_search_info(mdrq_table *t, uint64_t *ranges, uint64_t *probes);

/*
 * mdrq_learn_export — the trained model, for checking it away from the GPU (the paper
 * has no learned component; this serves tests and inspection).
 *  desc        kind, segments (PLA segments, MLP leaves, 0 for none), mlp_params, the
 *              MLP's input normalisation (u = (float)(key - key_min) * key_inv) and the
 *              largest error mdrq_learn_info reports.
 *  knot_key, knot_pos, slope   PLA: segments + 1 knots (the last is (max key + 1, n))
 *              and segments slopes; segment i predicts knot_pos[i] + (float)(key -
 *              knot_key[i]) * slope[i] (the product in float32) for the last i with
 *              knot_key[i] <= key (i = 0 below the first knot). MLP: the same per leaf
 *              (segments entries), for the leaf the network sends the key to.
 *  mlp         MLP: mlp_params float32 weights W1[32], b1[32], W2[32][32] (row = output
 *              unit), b2[32], W3[32], b3; output y, leaf = clamp(floor(y * segments)).
 *  capacity    entries knot_key / knot_pos / slope can hold.
 * Any array may be NULL. Synchronous. Errors: MDRQ_E_INVAL (t or desc NULL, no model);
 * MDRQ_E_CAPACITY (capacity below the entries of a non-NULL array); MDRQ_E_CUDA.
 */
typedef struct {
    int32_t kind;
    uint32_t segments;
    uint32_t mlp_params;
    uint32_t reserved;
    uint64_t key_min;
    float key_inv;
    float reserved2;
    uint64_t max_error;
} mdrq_model_desc;
int mdrq_learn_export(const mdrq_table *t, mdrq_model_desc *desc, uint64_t *knot_key, uint64_t *knot_pos,
                      float *slope, float *mlp, uint32_t capacity);

/*
 * Serving: continuous batching of queries that arrive over time; the paper has no
 * counterpart (it times a fixed workload of queries, Sec. 7.1.2).
 *
 * mdrq_server_start — start a server on table t. Callers submit queries from any
 * thread; a scheduler thread batches whatever has arrived (at most max_batch queries),
 * counts each query's answer with the shared scan, admits queries in arrival order
 * while their answers fit in the free part of a device arena of result_bytes (the
 * result-buffer budget), writes the admitted answers into their arena slots, and lets
 * the rest wait, ahead of later arrivals. Two batches may be on the GPU at once (two
 * streams), so arrivals are admitted as slots and memory free up and their work
 * overlaps the batch in flight. A batch of at most b queries is answered by the plain
 * scan into a per-stream scratch buffer of b * n ids and copied into its arena slots,
 * with b = min(12, 2^28 / n) (the buffer stays within 1 GiB; b = 0, no plain path, on
 * tables of more than 2^28 rows). While a server runs, t must not be used otherwise.
 * Errors: MDRQ_E_INVAL (t or out NULL, result_bytes < 4, max_batch 0); MDRQ_E_NOMEM;
 * MDRQ_E_CUDA.
 */
typedef struct mdrq_server mdrq_server;
int mdrq_server_start(mdrq_table *t, uint64_t result_bytes, uint32_t max_batch, mdrq_server **out);

/* mdrq_server_submit — enqueue one query (predicates as for mdrq_query, copied); a
 * ticket identifies it. Non-blocking. Errors: as mdrq_query's argument checks; a query
 * proven empty on the host is answered at once. */
int mdrq_server_submit(mdrq_server *s, const mdrq_pred *preds, uint32_t npreds, uint64_t *ticket);

/* mdrq_server_wait — wait (timeout_us < 0: without limit) until the query is answered.
 * ids receives a device pointer to its ascending ids in the arena (NULL when count is
 * 0), valid until mdrq_server_release; latency_us the time from submit to the end of
 * its batch. Returns the query's status: MDRQ_OK; MDRQ_E_CAPACITY (its answer, of
 * *count ids, can never fit the arena, or the server stopped while it waited for
 * memory); MDRQ_E_TIMEOUT (not answered within timeout_us; still queued); MDRQ_E_INVAL
 * (unknown or released ticket); the CUDA or allocation error (MDRQ_E_CUDA,
 * MDRQ_E_NOMEM, MDRQ_E_TIMEOUT from a device wait) that stopped the server, for the
 * queries of the failed batch and every query still queued behind it. After such a
 * failure mdrq_server_submit returns that error. */
int mdrq_server_wait(mdrq_server *s, uint64_t ticket, int64_t timeout_us, const uint32_t **ids, uint64_t *count,
                     double *latency_us);

/* mdrq_server_release — return an answered query's arena memory (its ids pointer dies). */
int mdrq_server_release(mdrq_server *s, uint64_t ticket);

/* mdrq_server_submit_batch — submit nq queries at once (one lock, one wake-up of the
 * scheduler); tickets (host, nq entries) receive their tickets in order. Every query is
 * encoded first: a bad one submits none of them. Errors: as mdrq_server_submit. */
int mdrq_server_submit_batch(mdrq_server *s, const mdrq_qdesc *qs, uint32_t nq, uint64_t *tickets);

/* mdrq_server_wait_many — wait until every one of the n tickets is answered (or
 * timeout_us, when >= 0, passes: MDRQ_E_TIMEOUT, nothing reported), then fill status,
 * counts and latency_us (host arrays of n entries, each may be NULL) as
 * mdrq_server_wait does per ticket; with release != 0 the answers are released as by
 * mdrq_server_release (for callers that need the sizes only, or that drain the server).
 * Errors: MDRQ_E_INVAL (s NULL, an unknown ticket); the per-ticket status otherwise. */
int mdrq_server_wait_many(mdrq_server *s, const uint64_t *tickets, uint32_t n, int64_t timeout_us, int *status,
                          uint64_t *counts, double *latency_us, int release);

/* mdrq_server_stats — answered queries, batches run, deferrals (a query sent back to
 * wait for memory counts once per time), and the median and 99th percentile of the
 * answered queries' latencies in microseconds. Any pointer may be NULL. */
int mdrq_server_stats(mdrq_server *s, uint64_t *completed, uint64_t *batches, uint64_t *deferred, double *p50_us,
                      double *p99_us);

/* mdrq_server_stop — stop accepting queries, answer the queued ones, free the server and
 * its arena (unreleased answers die with it). NULL is a no-op. Returns MDRQ_OK or the
 * error that stopped the server (a CUDA or allocation failure of a batch). */
int mdrq_server_stop(mdrq_server *s);

/*
 * mdrq_inject_fault — test hook for failure detection; the paper has no counterpart.
 * Arms one fault for the next query call on this table:
 *  MDRQ_FAULT_SKIP_TILES  the next scan launch never claims its first `arg` (>= 1) row
 *                         tiles, so the ordered compaction of the first claimed tile
 *                         waits on predecessor states that nothing will set. The
 *                         bounded wait runs out (about a second), the kernel records an
 *                         error bit and finishes, and the call returns MDRQ_E_TIMEOUT;
 *                         the table's scratch is then reset and stays usable.
 *  MDRQ_FAULT_NOMEM       the next query call, or the next batch of a server running
 *                         on this table, fails as if its scratch allocation had failed:
 *                         MDRQ_E_NOMEM, nothing launched. In a server that batch's
 *                         queries and every query queued behind it end with
 *                         MDRQ_E_NOMEM, mdrq_server_submit refuses new queries with it,
 *                         and mdrq_server_stop returns it.
 *  MDRQ_FAULT_STAGE_NOMEM the next scan launch that would stage its output (see
 *                         mdrq_set_output_order) finds its staging buffers unavailable,
 *                         as if their allocation had failed, and orders its output by
 *                         look-back instead: the call succeeds with the same answer.
 * Errors: MDRQ_E_INVAL (t NULL, unknown kind, SKIP_TILES with arg = 0).
 */
#define MDRQ_FAULT_SKIP_TILES 1
#define MDRQ_FAULT_NOMEM 2
#define MDRQ_FAULT_STAGE_NOMEM 3
int mdrq_inject_fault(mdrq_table *t, int kind, uint64_t arg);

/*
 * mdrq_query_static — answer one MDRQ like mdrq_query, but without allocating any
 * memory. The paper has no counterpart: it is an interface for callers that cannot
 * allocate device memory when they query, such as a serving loop whose device memory
 * belongs to another allocator's budget, a latency-critical path on which
 * cudaMalloc's implicit device-wide synchronisation would stall other streams, or
 * code that must not change the GPU's memory footprint after start-up.
 *
 * No table is made: the caller passes its device columns and receives the answer in
 * its own device buffer. The scan's scratch lives in a fixed array in device memory
 * inside the library, about 516 KiB on every GPU that loads the library, held
 * until the process exits; it limits the table to MDRQ_STATIC_MAX_ROWS rows.
 *
 *  cols[j], types[j], d, n   as mdrq_load_columns with cols_on_device = 1 (device
 *                            pointers, 16-byte aligned); n <= MDRQ_STATIC_MAX_ROWS.
 *  preds, npreds             host predicates, as mdrq_query.
 *  ids, capacity             device output buffer of `capacity` uint32 slots.
 *  count                     host; receives the length of the answer.
 *  stream                    the call synchronises it before returning.
 *
 * Every call on a device shares the scratch array and clears the part it uses before
 * its launch. Calls whose GPU work overlaps (several streams or host threads at once)
 * race on the array and give wrong answers: serialise them. The first call on a
 * device sets up that device (it looks up the array's device address, with the
 * device current): make it before any stream capture. Nothing in this call allocates
 * memory; in particular it calls neither cudaMalloc nor cudaFree.
 *
 * Errors: MDRQ_E_INVAL (n > MDRQ_STATIC_MAX_ROWS, d = 0, a null or misaligned
 * column, an unknown type, count NULL, ids NULL with capacity > 0, a bad predicate
 * as for mdrq_query); MDRQ_E_CAPACITY (*count > capacity: the first `capacity` ids
 * are written); MDRQ_E_TIMEOUT; MDRQ_E_CUDA.
 */
#define MDRQ_STATIC_MAX_ROWS 268435456ull /* 2^28 rows: 65536 tiles of 4096 rows */

int mdrq_query_static(const void *const *cols, const int32_t *types, uint32_t d, uint64_t n,
                      const mdrq_pred *preds, uint32_t npreds, uint32_t *ids, uint64_t capacity,
                      uint64_t *count, void *stream);

/*
 * Zone maps. At load the library records, for every column and every 4096-row tile,
 * the minimum and maximum value (8 bytes per 4096 rows). When a plain-mode batch has a
 * predicate whose column's zone map is in use, each query first lists the tiles whose
 * ranges meet all of its intervals — the others cannot hold an answer; this is the
 * VA-file's pruning of cells that miss the query (Sec. 2.2.3), applied to row tiles —
 * as runs of candidate tiles (at most 1024 per query, else one run from the first to
 * the last candidate), and the scan visits only those tiles. This pays where the row
 * order clusters values (a table sorted by a key, data loaded in time order).
 *
 * mdrq_set_zone_maps: MDRQ_ZONES_AUTO (default) uses a column's map when its zones'
 * mean width is below half of the column's range; MDRQ_ZONES_ALL uses every map;
 * MDRQ_ZONES_OFF none (every tile is read). Answers never change. Errors: MDRQ_E_INVAL.
 *
 * mdrq_zone_scan_info: rows and tiles the last zone-pruned launch visited (0 if none
 * ran). Synchronous. Errors: MDRQ_E_INVAL, MDRQ_E_CUDA.
 *
 * mdrq_zone_map_info: *used = 1 when queries on dimension `dim` read its zone map
 * under the current setting; *mean_width = the mean zone width over the column's
 * range (0..1). Either pointer may be NULL. Errors: MDRQ_E_INVAL (t NULL, dim >= d).
 */
#define MDRQ_ZONES_OFF 0
#define MDRQ_ZONES_AUTO 1
#define MDRQ_ZONES_ALL 2
int mdrq_set_zone_maps(mdrq_table *t, int mode);
int mdrq_zone_map_info(const mdrq_table *t, uint32_t dim, int *used, double *mean_width);
int mdrq_zone_scan_info(mdrq_table *t, uint64_t *rows, uint64_t *tiles);

/*
 * Shared-scan configuration and the autotuner. The shared scan (MDRQ_BATCH_SHARED)
 * has two shape parameters: the rows of one warp's work unit, and the shared-memory
 * budget of one chunk's search tables (which sets how many queries share one pass
 * over the columns and how many blocks fit on an SM).
 *
 * mdrq_set_shared_config sets them for the table: unit_rows (rounded up to a multiple
 * of 32; 0 = the built-in rule: enough units to fill the GPU, 256..8192 rows) and
 * image_kib (16..208; 0 = the built-in 56 KiB). Errors: MDRQ_E_INVAL (t NULL,
 * image_kib outside its range).
 *
 * mdrq_autotune times the given batch (synchronously, on `stream`, into a scratch
 * answer buffer it allocates and frees) with the plain scan, with the shared scan
 * under the built-in rule, and with the shared scan under a set of candidate
 * configurations (coordinate search: unit sizes first, then budgets), each the best of
 * two runs measured with CUDA events, host planning included. The table keeps the
 * fastest shared configuration, and MDRQ_BATCH_AUTO then takes the faster of the two
 * modes for batches of 32 or more live queries. The answers of every timed run are
 * discarded; the table's batch mode is left as it was. A batch with no live query
 * changes nothing. Errors: MDRQ_E_INVAL, MDRQ_E_NOMEM, MDRQ_E_TIMEOUT, MDRQ_E_CUDA.
 */
typedef struct {
    int32_t mode;              /* the faster mode for this batch: MDRQ_BATCH_PLAIN or _SHARED */
    uint32_t unit_rows;        /* the shared configuration kept (0: the built-in rule won) */
    uint32_t image_kib;        /* (0: the built-in default won) */
    uint32_t candidates;       /* shared-scan configurations timed */
    double plain_ms;           /* the batch with the plain scan */
    double shared_default_ms;  /* with the shared scan's built-in configuration */
    double shared_ms;          /* with the configuration kept */
} mdrq_tuning;

int mdrq_set_shared_config(mdrq_table *t, uint32_t unit_rows, uint32_t image_kib);

/* mdrq_set_shared_bits_budget — the most device memory (bytes) the shared scan may keep
 * for every row's query bits between its passes (16 bytes per row and group of 128
 * queries); a batch that needs more, or max_bytes = 0, evaluates the columns again in
 * the write pass. UINT64_MAX restores the default (32 GiB, and at most a quarter of the
 * free device memory). Memory already held is kept. Errors: MDRQ_E_INVAL (t NULL). */
int mdrq_set_shared_bits_budget(mdrq_table *t, uint64_t max_bytes);

/* mdrq_set_shared_codes — whether the shared scan may encode its columns (enable = 1,
 * the default): per batch, each column some query constrains is encoded once into
 * 16-bit codes, code(x) = the number of the batch's interval end points (over all
 * chunks) at or below x, and each chunk finds a row's elementary interval by a lookup
 * of its code instead of a search of the value. Used when every column has at most
 * 16,383 end points, each chunk's lookup tables fit its shared memory, and the codes
 * (2 bytes per row and encoded column, kept with the table) fit 32 GB and a quarter of
 * the free device memory; otherwise the values are searched. enable = 0 always
 * searches. Answers are identical either way. Errors: MDRQ_E_INVAL (t NULL). */
int mdrq_set_shared_codes(mdrq_table *t, int enable);
int mdrq_autotune(mdrq_table *t, const mdrq_qdesc *qs, uint32_t nq, void *stream, mdrq_tuning *out);

/*
 * Prepared batches — a fixed batch of queries answered again and again (a standing
 * report, a benchmark loop, a dashboard refresh) without per-call host work. The paper
 * answers each query from scratch (Sec. 7.1.2); this is a GPU-side addition.
 *
 * mdrq_prepare_batch encodes the batch once, runs it once (the answer and the offsets
 * are those of mdrq_query_batch with ids_on_device = 1, in the table's batch mode at
 * this call: MDRQ_BATCH_AUTO, _PLAIN or _SHARED), and records the batch's device work
 * (query-table copies, scan launches, offset copy-back) as one CUDA graph on a private
 * copy of the table's scratch state. mdrq_prepared_launch replays that graph on a
 * stream; mdrq_prepared_wait waits for the replay and returns its offsets.
 *
 *  t                 a loaded table; it must outlive the prepared batch (the batch
 *                    reads its columns); the batch keeps its own scratch, so calls on
 *                    t and replays of the batch do not share state. MDRQ_BATCH_LEARNED
 *                    batches cannot be prepared (MDRQ_E_INVAL).
 *  qs, nq            as mdrq_query_batch; copied, the caller may free them afterwards.
 *  ids, capacity     device buffer that every replay overwrites with the CSR answer.
 *  offsets           host, nq + 1 entries: the first run's CSR offsets. On
 *                    MDRQ_E_CAPACITY offsets[nq] is the size the buffer needs and no
 *                    batch is made (*out = NULL).
 *  stream            the first run and the graph build are ordered after the work on it.
 *  out               receives the prepared batch.
 *
 * Replays on one prepared batch must not overlap (they share its scratch): wait for
 * one before launching the next on another stream; on one stream they serialise.
 * Errors: MDRQ_E_INVAL, MDRQ_E_NOMEM, MDRQ_E_CAPACITY, MDRQ_E_TIMEOUT, MDRQ_E_CUDA.
 */
typedef struct mdrq_prepared mdrq_prepared;

int mdrq_prepare_batch(mdrq_table *t, const mdrq_qdesc *qs, uint32_t nq, uint32_t *ids, uint64_t capacity,
                       uint64_t *offsets, void *stream, mdrq_prepared **out);

/* Enqueue one replay on `stream` and return without waiting (MDRQ_E_CUDA if the launch
 * fails). */
int mdrq_prepared_launch(mdrq_prepared *p, void *stream);

/* Wait for the last replay enqueued on `stream`, then fill offsets (host, nq + 1) as
 * mdrq_query_batch does. MDRQ_E_TIMEOUT if a bounded device wait ran out (the batch's
 * scratch is reset and it stays usable). */
int mdrq_prepared_wait(mdrq_prepared *p, uint64_t *offsets, void *stream);

/* Number of kernel launches in one replay (the graph's kernel nodes) into *kernels. */
int mdrq_prepared_kernels(const mdrq_prepared *p, uint64_t *kernels);

/* Release the batch (NULL-safe). Waits for its replays to finish. */
void mdrq_prepared_free(mdrq_prepared *p);

#ifdef __cplusplus
}
#endif

#endif /* MDRQ_H */
