// Library-internal state of a table (the opaque mdrq_table of include/mdrq.h), shared by
// the translation units of the library.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "mdrq.h"
#include "scan_kernel.cuh"

namespace mdrq {

constexpr uint32_t kSampleRows = 4096;  // per-column sample for selectivity estimates

struct ColumnInfo {
    const void *ptr = nullptr;  // device
    int32_t type = MDRQ_F32;
    uint32_t min_bits = 0, max_bits = 0;  // exact column minimum / maximum (n > 0)
    std::vector<double> sample;           // sorted
    uint2 *zone = nullptr;                // zone map (device, owned): min / max bits per 4096 rows
    double zone_width = 1.0;              // mean zone width / column range
    bool zone_keep = false;               // MDRQ_ZONES_AUTO reads this column's map
    std::vector<float> key_cells;         // learned narrower: 255 ascending cell bounds, or
                                          // empty for equal-width cells (mdrq_set_key_cells)
};

// a2: one query after encoding
struct EncodedQuery {
    bool empty = false;          // proven empty on the host
    std::vector<DevPred> preds;  // non-trivial predicates, most selective first
    std::vector<uint32_t> dims;  // their dimensions
    uint64_t scanned_columns = 0;
};

struct SharedScanState;  // device buffers of the batched shared scan (batched.cu)
struct ZoneWindows;      // device buffers of the zone-pruned scan (zones.cu)

// A batch answering into host memory: the ids go to the device staging buffer and are
// copied to `host` on the copy stream, a finished launch's range while the next runs.
struct HostSink {
    uint32_t *host = nullptr;
    uint64_t capacity = 0;
    cudaStream_t copy = nullptr;
    unsigned long long *end_host = nullptr;  // pinned: a launch's CSR end, read back
    uint64_t copied = 0;                      // ids copied so far
    bool pending = false;                     // a launch whose ids are still to be copied
    cudaEvent_t pending_done = nullptr;
    uint32_t pending_last = 0;                // the caller's index of its last query
};
struct LearnedModel;     // learned range narrower (learned.cu)

}  // namespace mdrq

struct mdrq_table {
    int device = 0;
    uint64_t n = 0;
    uint32_t d = 0;
    std::vector<mdrq::ColumnInfo> cols;
    std::vector<void *> owned;  // device columns this table allocated

    // scratch: [0] claim counter, [1] error word, [2 .. 2 + ring) look-back states,
    // [2 + ring] the staged output's allocation counter
    unsigned long long *scratch = nullptr;
    unsigned long long *ticket = nullptr;
    int *error = nullptr;
    unsigned long long *tile_state = nullptr;
    uint32_t ring_bits = 16;
    uint32_t tag_next = 1;  // tag of the next launch's first ring lap (0: cleared slot)

    // per-batch query tables: device copies and their pinned staging
    mdrq::DevQuery *dq_dev = nullptr;
    size_t dq_dev_cap = 0;
    mdrq::DevPred *dp_dev = nullptr;
    size_t dp_dev_cap = 0;
    unsigned char *qstage_host = nullptr;  // pinned: DevQuery[] then DevPred[]
    size_t qstage_host_cap = 0;

    unsigned long long *offsets_dev = nullptr;  // nq + 1 entries
    size_t offsets_dev_cap = 0;
    unsigned long long *offsets_host = nullptr;  // pinned mirror
    size_t offsets_host_cap = 0;
    uint32_t *ids_stage = nullptr;  // device staging for host-side answers
    size_t ids_stage_cap = 0;
    uint32_t *tile_map = nullptr;   // windowed launches: the window of every tile
    size_t tile_map_cap = 0;
    // staged output of large plain launches (scan_kernel.cuh STAGED, concat.cu)
    int output_order = MDRQ_ORDER_AUTO;  // mdrq_set_output_order
    uint32_t *cat_ids = nullptr;          // staging runs of the tiles' ids
    size_t cat_ids_cap = 0;               // bytes
    unsigned long long *cat_rec = nullptr;  // per tile: staging position << 13 | id count
    size_t cat_rec_cap = 0;
    unsigned long long *cat_seg = nullptr;  // per segment of 2048 tiles: id count, then prefix
    size_t cat_seg_cap = 0;
    unsigned long long *cat_bump = nullptr;  // in scratch: ids staged so far by the launch
    cudaStream_t sink_copy = nullptr;  // copies of host answers out of the staging buffer
    cudaEvent_t sink_done = nullptr;
    unsigned long long *sink_end = nullptr;  // pinned
    size_t sink_end_cap = 0;
    int *error_host = nullptr;      // pinned

    int sm_count = 0;
    int blocks_per_sm[3] = {0, 0, 0};  // for U = 1, 2, 4
    int blocks_per_sm_window = 0;      // windowed scan

    uint64_t last_launches = 0;
    uint64_t last_bytes = 0;

    // optional per-launch event timing of the scan kernel
    bool timing = false;
    std::vector<cudaEvent_t> ev;  // pairs: [2i] before, [2i+1] after launch i
    size_t ev_used = 0;           // pairs recorded since the last reset
    uint64_t acc_scans = 0, acc_bytes = 0, acc_kernels = 0;

    // batched shared scan (mdrq_set_batch_mode, batched.cu)
    int batch_mode = MDRQ_BATCH_AUTO;
    mdrq::SharedScanState *shared = nullptr;
    uint32_t shared_unit_rows = 0;    // rows per warp unit (0: built-in rule)
    uint32_t shared_image_words = 0;  // shared-memory budget per chunk (0: built-in default)
    uint64_t shared_bits_budget = ~0ull;  // row bits kept between the passes, bytes (~0: default)
    int auto_mode = -1;               // mode AUTO takes for 32+ queries, once measured (-1: rule)
    bool shared_coded = true;         // shared scan may encode its columns (mdrq_set_shared_codes)
    mdrq::LearnedModel *learned = nullptr;

    int zone_mode = MDRQ_ZONES_AUTO;  // mdrq_set_zone_maps
    int host_answers = MDRQ_HOST_AUTO;  // mdrq_set_host_answers
    mdrq::HostSink *sink = nullptr;   // set while a batch answers into host memory (run_batch)
    mdrq::ZoneWindows *zwin = nullptr;

    // set on the private table of a prepared batch while its launches are captured
    bool graph_capture = false;

    // host-side fault injection for failure-detection tests (mdrq_inject_fault)
    uint64_t inject_skip_tiles = 0;  // next scan launch never claims its first tiles
    int inject_nomem = 0;            // next query call fails its scratch allocation
    int inject_stage_nomem = 0;      // next staged launch finds its staging buffers missing
};


#define MDRQ_TRY_STATUS(expr)                   \
    do {                                        \
        int _s = mdrq::cuda_status(expr);       \
        if (_s != MDRQ_OK) {                    \
            (void)cudaGetLastError();           \
            return _s;                          \
        }                                       \
    } while (0)

namespace mdrq {

int cuda_status(cudaError_t e);
double bound_value(uint32_t bits, int32_t type);
int encode_query(const mdrq_table *t, const mdrq_pred *preds, uint32_t npreds, EncodedQuery &q);
int grow_device(void **p, size_t *cap, size_t bytes);
int grow_pinned(void **p, size_t *cap, size_t bytes);

// mdrq.cu: the steps of a batch call (run_batch = encode, enqueue, finish)
int encode_batch(const mdrq_table *t, const mdrq_qdesc *qs, uint32_t nq, std::vector<EncodedQuery> &enc,
                 std::vector<uint32_t> &live, size_t &npreds);
int enqueue_batch(mdrq_table *t, const std::vector<EncodedQuery> &enc, const std::vector<uint32_t> &live,
                  uint32_t nq, size_t npreds, uint32_t *out, uint64_t capacity, cudaStream_t s);
int finish_batch(mdrq_table *t, const std::vector<uint32_t> &live, uint32_t nq, uint64_t *offsets, cudaStream_t s);
int alloc_scratch(mdrq_table *t, cudaStream_t s);
void reset_scratch(mdrq_table *t, cudaStream_t s);
void destroy(mdrq_table *t);
// a private table over t's columns (own scratch; borrows columns, statistics and zone
// maps), for prepared batches and the server's streams; released with free_shadow
int make_shadow(const mdrq_table *t, cudaStream_t s, mdrq_table **out);
void free_shadow(mdrq_table *sh);

// batched.cu: answer the live queries of a batch with the shared scan. enc/live as in
// run_batch; writes offsets_dev[orig + 1] for every live query.
int shared_scan_batch(mdrq_table *t, const std::vector<EncodedQuery> &enc, const std::vector<uint32_t> &live,
                      uint32_t *ids, uint64_t capacity, cudaStream_t s);
void shared_scan_free(mdrq_table *t);
// the two phases of the shared scan on an explicit state (the serving loop keeps two)
SharedScanState *shared_state_new();
void shared_state_free(SharedScanState *S);
unsigned long long *shared_state_qbase(SharedScanState *S);   // device, per live query
unsigned long long *shared_state_totals(SharedScanState *S);  // device, per live query
int shared_scan_count(mdrq_table *t, SharedScanState &S, const std::vector<EncodedQuery> &enc,
                      const std::vector<uint32_t> &live, cudaStream_t s);
int shared_scan_write(mdrq_table *t, SharedScanState &S, uint32_t *ids, uint64_t capacity, bool csr, cudaStream_t s);

// mdrq.cu: one windowed scan launch over nq live queries whose rows and tiles the device
// holds in windows / total_tiles (written by earlier kernels on the same stream).
// alg_bytes: the launch's algorithmic bytes for the timing counters; helper_kernels:
// kernels launched before it for its windows.
int launch_window_scan(mdrq_table *t, uint32_t q0, uint32_t nq, uint64_t max_windows,
                       const unsigned long long *nwindows, uint64_t alg_bytes, uint32_t helper_kernels,
                       uint32_t *ids, uint64_t capacity, const unsigned long long *base_in, const DevWindow *windows,
                       const unsigned long long *total_tiles, cudaStream_t s);

// learned.cu: the window list of nq queries from per-query slots (per_query windows
// each; counts[q] used, qtiles[q] tiles, tile_start local to the query): exclusive
// scans into wbase / tbase, totals[0] = tiles, totals[1] = windows, then compaction.
int window_list(uint32_t nq, uint32_t per_query, const uint32_t *counts, const uint32_t *qtiles,
                unsigned long long *wbase, unsigned long long *tbase, const DevWindow *slots, DevWindow *windows,
                unsigned long long *totals, cudaStream_t s);

// zones.cu: the plain scan of live queries q0 .. q0 + nlive restricted to the row tiles
// their zone maps do not rule out (one windowed launch)
int zone_batch(mdrq_table *t, uint32_t q0, uint32_t nlive, uint64_t scanned_columns, uint32_t *ids,
               uint64_t capacity, const unsigned long long *base_in, cudaStream_t s);
void zone_windows_free(mdrq_table *t);
int zone_window_rows(mdrq_table *t, uint64_t *rows, uint64_t *tiles);

// concat.cu: order the staged output of a launch (t->cat_rec, t->cat_ids) into ids (CSR
// from *base_in, or 0) and write the CSR end of every query of the launch (queries: the
// launch's query table). Plain launch: ntiles tiles of tile_rows rows, tiles_per_query
// per query; ntiles_dev, tile_map and windows null. Windowed launch: at most ntiles
// tiles, the count in *ntiles_dev, placed by tile_map and windows (device).
int concat_staged(mdrq_table *t, uint64_t ntiles, const unsigned long long *ntiles_dev, uint32_t tiles_per_query,
                  uint32_t tile_rows, const DevQuery *queries, const uint32_t *tile_map, const DevWindow *windows,
                  const unsigned long long *base_in, uint32_t *ids, uint64_t capacity, cudaStream_t s);
void concat_free(mdrq_table *t);

// learned.cu
int learn(mdrq_table *t, const uint32_t *dims, uint32_t ndims, int kind, cudaStream_t s);
int learned_batch(mdrq_table *t, const std::vector<EncodedQuery> &enc, const std::vector<uint32_t> &live,
                  uint32_t q0, uint32_t nlive, uint32_t *ids, uint64_t capacity, const unsigned long long *base_in,
                  cudaStream_t s);
int learned_info(const mdrq_table *t, uint64_t *max_error, uint32_t *segments, double *train_ms);
void learned_free(mdrq_table *t);
int learned_window_rows(mdrq_table *t, uint64_t *rows, uint64_t *widenings);
int learned_search_info(mdrq_table *t, uint64_t *ranges, uint64_t *probes);
int set_key_cells(mdrq_table *t, uint32_t dim, const float *bounds, uint32_t nbounds);
int learned_export(const mdrq_table *t, mdrq_model_desc *desc, uint64_t *knot_key, uint64_t *knot_pos, float *slope,
                   float *mlp, uint32_t capacity);

}  // namespace mdrq
