// C ABI of the MDRQ scan library: table residency, query encoding, launches and result
// hand-off. The operations are defined in include/mdrq.h; the scan itself is in
// scan_kernel.cuh.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <limits>
#include <map>
#include <new>
#include <vector>

#include "mdrq.h"
#include "scan_kernel.cuh"
#include "table.h"

using namespace mdrq;

// ---------------------------------------------------------------- small helper kernels

namespace mdrq {

// The window of every tile of a windowed launch: map[tile_start + i] = w for the tiles
// of window w (one warp per window, grid-stride; windows without tiles write nothing).
__global__ void __launch_bounds__(256) mdrq_tile_map_kernel(const DevWindow *windows,
                                                            const unsigned long long *nwindows, uint32_t *map)
{
    const int lane = threadIdx.x & 31;
    const unsigned long long nw = *nwindows;
    const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x / 32);
    for (uint64_t w = (uint64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5); w < nw; w += warps) {
        const unsigned long long t0 = windows[w].tile_start, nt = windows[w].tiles;
        for (unsigned long long i = lane; i < nt; i += 32)
            map[t0 + i] = (uint32_t)w;
    }
}

// The scan over per-query row windows (the learned range narrower's exact check, and
// the tiles the zone maps leave).
__global__ void __launch_bounds__(kScanThreads, 7) mdrq_scan_window_kernel(const __grid_constant__ ScanParams p)
{
    scan_cta<4, true>(p);
}

// The same with staged output (concat.cu orders it by the launch's tile map).
__global__ void __launch_bounds__(kScanThreads, 7)
    mdrq_scan_window_staged_kernel(const __grid_constant__ ScanParams p)
{
    scan_cta<4, true, true>(p);
}

// NaN count, minimum and maximum of a column. out[0] += NaNs; out[1] / out[2] hold the
// minimum / maximum as order-preserving keys (see key_of).
__device__ __forceinline__ unsigned long long key_of(uint32_t bits, uint32_t type)
{
    if (type == kTypeF32)
        return (bits & 0x80000000u) ? (unsigned long long)(~bits) : (unsigned long long)(bits | 0x80000000u);
    return (unsigned long long)(bits ^ 0x80000000u);
}

__global__ void __launch_bounds__(kBlock)
    mdrq_column_stats_kernel(const uint32_t *col, uint64_t n, uint32_t type, unsigned long long *out)
{
    unsigned long long nan = 0, mn = ~0ull, mx = 0;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const uint32_t b = col[i];
        if (type == kTypeF32 && (b & 0x7fffffffu) > 0x7f800000u) {
            ++nan;
            continue;
        }
        const unsigned long long k = key_of(b, type);
        mn = k < mn ? k : mn;
        mx = k > mx ? k : mx;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        nan += __shfl_xor_sync(0xffffffffu, nan, o);
        const unsigned long long a = __shfl_xor_sync(0xffffffffu, mn, o);
        const unsigned long long b = __shfl_xor_sync(0xffffffffu, mx, o);
        mn = a < mn ? a : mn;
        mx = b > mx ? b : mx;
    }
    if ((threadIdx.x & 31) == 0) {
        if (nan)
            atomicAdd(&out[0], nan);
        atomicMin(&out[1], mn);
        atomicMax(&out[2], mx);
    }
}

// Zone map of a column: zone[i] = bits of the minimum and maximum of rows
// [4096i, 4096i + 4096) (exact column values, ordered by key_of); width_sum += the
// zones' widths (max - min) * inv_range. One warp per zone, grid-stride.
__global__ void __launch_bounds__(256) mdrq_zone_kernel(const uint32_t *col, uint64_t n, uint32_t type, uint2 *zone,
                                                        double inv_range, double *width_sum)
{
    const int lane = threadIdx.x & 31;
    const uint64_t nz = (n + kZoneTileRows - 1) / kZoneTileRows;
    const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x / 32);
    double width = 0.0;
    for (uint64_t z = (uint64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5); z < nz; z += warps) {
        unsigned long long mn = ~0ull, mx = 0;
        const uint64_t r0 = z * kZoneTileRows, r1 = r0 + kZoneTileRows < n ? r0 + kZoneTileRows : n;
        for (uint64_t r = r0 + lane; r < r1; r += 32) {
            const unsigned long long key = key_of(col[r], type);
            mn = key < mn ? key : mn;
            mx = key > mx ? key : mx;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long a = __shfl_xor_sync(0xffffffffu, mn, o);
            const unsigned long long b = __shfl_xor_sync(0xffffffffu, mx, o);
            mn = a < mn ? a : mn;
            mx = b > mx ? b : mx;
        }
        // back from keys to the value bits
        uint32_t lo, hi;
        if (type == kTypeF32) {
            lo = (mn & 0x80000000ull) ? (uint32_t)mn ^ 0x80000000u : ~(uint32_t)mn;
            hi = (mx & 0x80000000ull) ? (uint32_t)mx ^ 0x80000000u : ~(uint32_t)mx;
        } else {
            lo = (uint32_t)mn ^ 0x80000000u;
            hi = (uint32_t)mx ^ 0x80000000u;
        }
        if (lane == 0) {
            zone[z] = make_uint2(lo, hi);
            const double w = type == kTypeF32 ? ((double)__uint_as_float(hi) - (double)__uint_as_float(lo)) * inv_range
                                              : ((double)(int)hi - (double)(int)lo) * inv_range;
            width += w <= 1.0 ? w : 1.0;  // (a non-finite width counts as the whole range)
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        width += __shfl_xor_sync(0xffffffffu, width, o);
    if (lane == 0 && width > 0.0)
        atomicAdd(width_sum, width);
}

// out[s] = col[floor(s * n / S)] for s < S: a strided sample for selectivity estimates
__global__ void mdrq_sample_kernel(const uint32_t *col, uint64_t n, uint32_t S, uint32_t *out)
{
    const uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < S)
        out[s] = col[(uint64_t)s * n / S];
}

}  // namespace mdrq

namespace mdrq {

constexpr size_t kAutoSharedMinQueries = 32;       // MDRQ_BATCH_AUTO: shared scan from this many
constexpr uint64_t kAutoSharedMinRows = 4000000;   // queries, on tables of at least this many rows
// Plain batches answering into host memory run as several launches, each one's ids
// copied out while the next one runs: at most kSinkLaunches, and each launch scans at
// least kSinkLaunchBytes of columns, so that its scan outlasts the host's wait for the
// previous launch (a small batch is one launch and one copy).
constexpr size_t kSinkLaunches = 16;
constexpr uint64_t kSinkLaunchBytes = 1ull << 30;

int cuda_status(cudaError_t e)
{
    if (e == cudaSuccess)
        return MDRQ_OK;
    if (e == cudaErrorMemoryAllocation)
        return MDRQ_E_NOMEM;
    return MDRQ_E_CUDA;
}

#define MDRQ_TRY(expr)                         \
    do {                                       \
        int _s = cuda_status(expr);            \
        if (_s != MDRQ_OK) {                   \
            (void)cudaGetLastError();          \
            return _s;                         \
        }                                      \
    } while (0)

inline cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

double bound_value(uint32_t bits, int32_t type)
{
    if (type == MDRQ_F32) {
        float f;
        std::memcpy(&f, &bits, 4);
        return (double)f;
    }
    return (double)(int32_t)bits;
}

uint32_t bits_from_key(unsigned long long key, int32_t type)
{
    const uint32_t k = (uint32_t)key;
    if (type == MDRQ_F32)
        return (k & 0x80000000u) ? (k ^ 0x80000000u) : ~k;
    return k ^ 0x80000000u;
}

// Sec. 2.1: a predicate is kept as an interval in the column's own type; the
// comparisons here are exact in double for both float32 and int32 values.
int encode_query(const mdrq_table *t, const mdrq_pred *preds, uint32_t npreds, EncodedQuery &q)
{
    q = EncodedQuery();
    if (npreds > 0 && !preds)
        return MDRQ_E_INVAL;
    std::map<uint32_t, std::pair<double, double>> iv;  // dim -> [lo, hi] intersected
    std::map<uint32_t, std::pair<uint32_t, uint32_t>> bits;
    for (uint32_t i = 0; i < npreds; ++i) {
        const mdrq_pred &p = preds[i];
        if (p.dim >= t->d || p.reserved != 0)
            return MDRQ_E_INVAL;
        const int32_t type = t->cols[p.dim].type;
        uint32_t lb, hb;
        std::memcpy(&lb, &p.lo, 4);
        std::memcpy(&hb, &p.hi, 4);
        const double lo = bound_value(lb, type), hi = bound_value(hb, type);
        if (std::isnan(lo) || std::isnan(hi))
            return MDRQ_E_INVAL;
        auto it = iv.find(p.dim);
        if (it == iv.end()) {
            iv[p.dim] = {lo, hi};
            bits[p.dim] = {lb, hb};
        } else {
            // a repeated dimension ANDs its predicates: intersect the intervals
            if (lo > it->second.first) {
                it->second.first = lo;
                bits[p.dim].first = lb;
            }
            if (hi < it->second.second) {
                it->second.second = hi;
                bits[p.dim].second = hb;
            }
        }
    }
    struct Cand {
        double est;
        uint32_t dim;
    };
    std::vector<Cand> keep;
    for (auto &kv : iv) {
        const uint32_t j = kv.first;
        const double lo = kv.second.first, hi = kv.second.second;
        const ColumnInfo &c = t->cols[j];
        if (lo > hi) {
            q.empty = true;  // an empty interval matches nothing
            continue;
        }
        if (t->n == 0)
            continue;
        const double mn = bound_value(c.min_bits, c.type), mx = bound_value(c.max_bits, c.type);
        if (hi < mn || lo > mx) {
            q.empty = true;  // no value of the column lies in the interval
            continue;
        }
        if (lo <= mn && mx <= hi)
            continue;  // every value lies in it: the predicate is always true
        const auto b = std::lower_bound(c.sample.begin(), c.sample.end(), lo);
        const auto e = std::upper_bound(c.sample.begin(), c.sample.end(), hi);
        keep.push_back({(double)(e - b), j});
    }
    if (q.empty) {
        q.preds.clear();
        return MDRQ_OK;
    }
    // Sec. 2.2.4: evaluating the most selective dimension first ends rows earliest
    std::stable_sort(keep.begin(), keep.end(),
                     [](const Cand &a, const Cand &b) { return a.est < b.est; });
    if (keep.size() > (size_t)kMaxPreds)
        return MDRQ_E_INVAL;
    for (const Cand &cd : keep) {
        q.dims.push_back(cd.dim);
        DevPred sp;
        sp.col = t->cols[cd.dim].ptr;
        sp.zone = t->zone_mode == MDRQ_ZONES_ALL || (t->zone_mode == MDRQ_ZONES_AUTO && t->cols[cd.dim].zone_keep)
                      ? t->cols[cd.dim].zone
                      : nullptr;
        sp.type = (uint32_t)t->cols[cd.dim].type;
        sp.lo = bits[cd.dim].first;
        sp.hi = bits[cd.dim].second;
        sp.pad = 0;
        q.preds.push_back(sp);
    }
    q.scanned_columns = q.preds.size();
    return MDRQ_OK;
}

int grow_device(void **p, size_t *cap, size_t bytes)
{
    if (*cap >= bytes)
        return MDRQ_OK;
    if (*p)
        cudaFree(*p);
    *p = nullptr;
    *cap = 0;
    MDRQ_TRY(cudaMalloc(p, bytes));
    *cap = bytes;
    return MDRQ_OK;
}

int grow_pinned(void **p, size_t *cap, size_t bytes)
{
    if (*cap >= bytes)
        return MDRQ_OK;
    if (*p)
        cudaFreeHost(*p);
    *p = nullptr;
    *cap = 0;
    MDRQ_TRY(cudaMallocHost(p, bytes));
    *cap = bytes;
    return MDRQ_OK;
}

template <int U>
constexpr uint64_t tile_rows()
{
    return (uint64_t)kWarps * U * 128;
}

// MDRQ_ORDER_AUTO stages a plain launch's output from this many tiles per resident block
constexpr uint64_t kStagedMinTilesPerBlock = 8;

// With event timing on (mdrq_scan_timing): the next event pair of the table, its first
// event recorded on s; *evp stays null when timing is off.
int timing_begin(mdrq_table *t, cudaStream_t s, cudaEvent_t **evp)
{
    *evp = nullptr;
    if (!t->timing)
        return MDRQ_OK;
    if (t->ev.size() < 2 * (t->ev_used + 1)) {
        cudaEvent_t a, b;
        MDRQ_TRY(cudaEventCreate(&a));
        MDRQ_TRY(cudaEventCreate(&b));
        t->ev.push_back(a);
        t->ev.push_back(b);
    }
    *evp = &t->ev[2 * t->ev_used];
    ++t->ev_used;
    MDRQ_TRY(cudaEventRecord((*evp)[0], s));
    return MDRQ_OK;
}

// Launch one scan over the queries qs[0 .. nq) (all non-empty), whose predicates are
// already in t->dp_dev and descriptors in t->dq_dev at offset q0.
int launch_scan(mdrq_table *t, uint32_t q0, uint32_t nq, uint64_t scanned_columns, uint32_t *ids,
                uint64_t capacity, const unsigned long long *base_in, cudaStream_t s)
{
    // 4096-row tiles unless the launch would leave SMs without work
    const uint64_t resident4 = (uint64_t)t->sm_count * t->blocks_per_sm[2];
    auto tiles_of = [&](uint64_t rows) { return (t->n + rows - 1) / rows; };
    int ui = 2;
    if (tiles_of(tile_rows<4>()) * nq < 2 * resident4)
        ui = tiles_of(tile_rows<2>()) * nq < 2 * resident4 ? 0 : 1;
    const uint64_t rows = ui == 2 ? tile_rows<4>() : ui == 1 ? tile_rows<2>() : tile_rows<1>();
    const uint64_t tiles_per_query = tiles_of(rows);
    const uint64_t total_tiles = tiles_per_query * nq;
    const uint64_t resident = (uint64_t)t->sm_count * t->blocks_per_sm[ui];
    const uint32_t grid = (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(resident, total_tiles));

    // tags: one per lap of the ring; restart from a cleared ring before they wrap, and
    // at every launch of a captured graph (its replays repeat the same tags)
    const uint32_t laps = (uint32_t)(total_tiles >> t->ring_bits) + 1;
    if (t->graph_capture || (uint64_t)t->tag_next + laps > kTagLimit) {
        MDRQ_TRY(cudaMemsetAsync(t->tile_state, 0, ((size_t)1 << t->ring_bits) * 8, s));
        t->tag_next = 1;
    }

    // every launch starts its tile claims from zero
    MDRQ_TRY(cudaMemsetAsync(t->ticket, 0, sizeof(unsigned long long), s));

    // Output order (mdrq_set_output_order): staged when the launch has many tiles in
    // flight behind each resident block, where the look-back's chain of inclusive
    // prefixes paces the whole launch; look-back when the staging buffers cannot be
    // had, and always under fault injection (whose failure is a look-back wait).
    bool staged = false;
    if (t->inject_skip_tiles == 0 && t->output_order != MDRQ_ORDER_LOOKBACK &&
        (t->output_order == MDRQ_ORDER_STAGED || total_tiles >= kStagedMinTilesPerBlock * resident)) {
        // (each tile's run is padded to a multiple of 4 ids)
        staged = !__atomic_exchange_n(&t->inject_stage_nomem, 0, __ATOMIC_ACQ_REL) &&
                 grow_device(reinterpret_cast<void **>(&t->cat_ids), &t->cat_ids_cap,
                             std::max<uint64_t>(16, (capacity + 3 * total_tiles) * 4)) == MDRQ_OK &&
                 grow_device(reinterpret_cast<void **>(&t->cat_rec), &t->cat_rec_cap, total_tiles * 8) == MDRQ_OK;
        if (!staged)
            (void)cudaGetLastError();
    }
    if (staged)
        MDRQ_TRY(cudaMemsetAsync(t->cat_bump, 0, sizeof(unsigned long long), s));

    ScanParams p;
    std::memset(&p, 0, sizeof(p));
    p.queries = t->dq_dev + q0;
    p.preds = t->dp_dev;
    p.nq = nq;
    p.tiles_per_query = (uint32_t)tiles_per_query;
    p.n = t->n;
    p.total_tiles = total_tiles;
    p.tile_state = t->tile_state;
    p.ring_bits = t->ring_bits;
    p.tag0 = t->tag_next;
    p.ticket = t->ticket;
    p.ticket_base = 0;
    p.ids = ids;
    p.capacity = capacity;
    p.base_in = base_in;
    p.offsets = t->offsets_dev;
    p.error = t->error;
    if (t->inject_skip_tiles) {
        // the first tiles are never claimed: the look-back of the first claimed tile
        // waits on states nobody sets and gives up after its bound
        p.ticket_base -= std::min<uint64_t>(t->inject_skip_tiles, total_tiles);
        t->inject_skip_tiles = 0;
    }

    cudaEvent_t *evp = nullptr;
    {
        const int st = timing_begin(t, s, &evp);
        if (st != MDRQ_OK)
            return st;
    }
    if (staged) {
        // the scan writes each tile's ids to a run of the staging buffer; concat_staged
        // below puts them in order into ids
        p.bump = t->cat_bump;
        p.tile_rec = t->cat_rec;
        p.ids = t->cat_ids;
        p.capacity = t->cat_ids_cap / 4;
        if (ui == 2)
            mdrq_scan_staged_kernel<4><<<grid, kScanThreads, 0, s>>>(p);
        else if (ui == 1)
            mdrq_scan_staged_kernel<2><<<grid, kScanThreads, 0, s>>>(p);
        else
            mdrq_scan_staged_kernel<1><<<grid, kScanThreads, 0, s>>>(p);
    } else if (ui == 2) {
        mdrq_scan_kernel<4><<<grid, kScanThreads, 0, s>>>(p);
    } else if (ui == 1) {
        mdrq_scan_kernel<2><<<grid, kScanThreads, 0, s>>>(p);
    } else {
        mdrq_scan_kernel<1><<<grid, kScanThreads, 0, s>>>(p);
    }
    MDRQ_TRY(cudaGetLastError());
    if (evp)
        MDRQ_TRY(cudaEventRecord(evp[1], s));
    if (staged) {
        const int st = concat_staged(t, total_tiles, nullptr, (uint32_t)tiles_per_query, (uint32_t)rows,
                                     t->dq_dev + q0, nullptr, nullptr, base_in, ids, capacity, s);
        if (st != MDRQ_OK)
            return st;
    }
    t->tag_next += laps;
    t->last_launches += 1;
    t->last_bytes += scanned_columns * 4ull * t->n;
    if (t->timing) {
        t->acc_scans += 1;
        t->acc_kernels += staged ? 4 : 1;  // the scan and the three ordering kernels
        t->acc_bytes += scanned_columns * 4ull * t->n;
    }
    return MDRQ_OK;
}

int launch_window_scan(mdrq_table *t, uint32_t q0, uint32_t nq, uint64_t max_windows,
                       const unsigned long long *nwindows, uint64_t alg_bytes, uint32_t helper_kernels,
                       uint32_t *ids, uint64_t capacity, const unsigned long long *base_in, const DevWindow *windows,
                       const unsigned long long *total_tiles, cudaStream_t s)
{
    if (t->blocks_per_sm_window == 0) {
        MDRQ_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&t->blocks_per_sm_window, mdrq_scan_window_kernel,
                                                               kScanThreads, 0));
        t->blocks_per_sm_window = std::max(1, t->blocks_per_sm_window);
    }
    // a query's windows are disjoint runs of the table; each adds at most one partial
    // tile (its start is rounded down)
    const uint64_t max_tiles = (uint64_t)nq * ((t->n + tile_rows<4>() - 1) / tile_rows<4>()) + max_windows;
    const uint32_t grid = (uint32_t)std::max<uint64_t>(
        1, std::min<uint64_t>((uint64_t)t->sm_count * t->blocks_per_sm_window, max_tiles));
    const uint32_t laps = (uint32_t)(max_tiles >> t->ring_bits) + 1;
    if (t->graph_capture || (uint64_t)t->tag_next + laps > kTagLimit) {
        MDRQ_TRY(cudaMemsetAsync(t->tile_state, 0, ((size_t)1 << t->ring_bits) * 8, s));
        t->tag_next = 1;
    }
    // the window of every tile, so that a claim finds its window with one load
    {
        const int st = grow_device((void **)&t->tile_map, &t->tile_map_cap, (size_t)max_tiles * 4);
        if (st != MDRQ_OK)
            return st;
    }
    mdrq_tile_map_kernel<<<(uint32_t)t->sm_count * 8, 256, 0, s>>>(windows, nwindows, t->tile_map);
    MDRQ_TRY(cudaMemsetAsync(t->ticket, 0, sizeof(unsigned long long), s));
    // Output order: staged only on request. A windowed launch reads few rows per id it
    // writes (the Z-sorted bench: 26.6 GB of ids for about 300 GB of column sectors), so
    // writing the ids a second time cost more than the look-back did (tile pruning 55.3
    // against 49.4 ms, learned windows 53.8 against 48.4 ms).
    bool staged = false;
    if (t->inject_skip_tiles == 0 && t->output_order == MDRQ_ORDER_STAGED) {
        staged = !__atomic_exchange_n(&t->inject_stage_nomem, 0, __ATOMIC_ACQ_REL) &&
                 grow_device(reinterpret_cast<void **>(&t->cat_ids), &t->cat_ids_cap,
                             std::max<uint64_t>(16, (capacity + 3 * max_tiles) * 4)) == MDRQ_OK &&
                 grow_device(reinterpret_cast<void **>(&t->cat_rec), &t->cat_rec_cap, max_tiles * 8) == MDRQ_OK;
        if (!staged)
            (void)cudaGetLastError();
    }
    if (staged)
        MDRQ_TRY(cudaMemsetAsync(t->cat_bump, 0, sizeof(unsigned long long), s));
    ScanParams p;
    std::memset(&p, 0, sizeof(p));
    p.queries = t->dq_dev + q0;
    p.tile_map = t->tile_map;
    p.preds = t->dp_dev;
    p.nq = nq;
    p.n = t->n;
    p.tile_state = t->tile_state;
    p.ring_bits = t->ring_bits;
    p.tag0 = t->tag_next;
    p.ticket = t->ticket;
    p.ticket_base = 0;
    p.ids = ids;
    p.capacity = capacity;
    p.base_in = base_in;
    p.offsets = t->offsets_dev;
    p.error = t->error;
    p.windows = windows;
    p.nwindows_dev = nwindows;
    p.total_tiles_dev = total_tiles;
    cudaEvent_t *evp = nullptr;
    {
        const int st = timing_begin(t, s, &evp);
        if (st != MDRQ_OK)
            return st;
    }
    if (staged) {
        p.bump = t->cat_bump;
        p.tile_rec = t->cat_rec;
        p.ids = t->cat_ids;
        p.capacity = t->cat_ids_cap / 4;
        mdrq_scan_window_staged_kernel<<<grid, kScanThreads, 0, s>>>(p);
    } else {
        mdrq_scan_window_kernel<<<grid, kScanThreads, 0, s>>>(p);
    }
    MDRQ_TRY(cudaGetLastError());
    if (evp)
        MDRQ_TRY(cudaEventRecord(evp[1], s));
    if (staged) {
        const int st = concat_staged(t, max_tiles, total_tiles, 0, (uint32_t)tile_rows<4>(), t->dq_dev + q0,
                                     t->tile_map, windows, base_in, ids, capacity, s);
        if (st != MDRQ_OK)
            return st;
    }
    t->tag_next += laps;
    t->last_launches += 1;
    t->last_bytes += alg_bytes;
    if (t->timing) {
        t->acc_scans += 1;
        t->acc_kernels += 2 + helper_kernels + (staged ? 3 : 0);  // tile map, scan, ordering pass
        t->acc_bytes += alg_bytes;
    }
    return MDRQ_OK;
}

// After an error the claim counter and ring may be inconsistent: reset them.
void reset_scratch(mdrq_table *t, cudaStream_t s)
{
    cudaStreamSynchronize(s);
    (void)cudaGetLastError();
    cudaMemset(t->scratch, 0, (size_t)(3 + ((size_t)1 << t->ring_bits)) * 8);
    cudaDeviceSynchronize();
    (void)cudaGetLastError();
    t->tag_next = 1;
}

// a2: every query of a batch encoded first, so that a bad argument launches nothing;
// live = the queries that need a scan, in order; npreds = their predicates
int encode_batch(const mdrq_table *t, const mdrq_qdesc *qs, uint32_t nq, std::vector<EncodedQuery> &enc,
                 std::vector<uint32_t> &live, size_t &npreds)
{
    for (uint32_t q = 0; q < nq; ++q)
        if (qs[q].reserved != 0)
            return MDRQ_E_INVAL;
    enc.assign(nq, EncodedQuery());
    live.clear();
    npreds = 0;
    for (uint32_t q = 0; q < nq; ++q) {
        int st = encode_query(t, qs[q].preds, qs[q].npreds, enc[q]);
        if (st != MDRQ_OK)
            return st;
        if (t->n > 0 && !enc[q].empty) {
            live.push_back(q);
            npreds += enc[q].preds.size();
        }
    }
    return MDRQ_OK;
}

// Host answers: copy the ids of the launch awaiting its copy (if any) to the host
// buffer, once it has finished; the launch after it may already be running.
static int sink_flush(mdrq_table *t)
{
    HostSink &k = *t->sink;
    if (!k.pending)
        return MDRQ_OK;
    k.pending = false;
    MDRQ_TRY(cudaStreamWaitEvent(k.copy, k.pending_done, 0));
    MDRQ_TRY(cudaMemcpyAsync(k.end_host, t->offsets_dev + k.pending_last + 1, 8, cudaMemcpyDeviceToHost, k.copy));
    MDRQ_TRY(cudaStreamSynchronize(k.copy));
    const uint64_t end = std::min<uint64_t>(*k.end_host, k.capacity);
    if (end > k.copied) {
        MDRQ_TRY(cudaMemcpyAsync(k.host + k.copied, t->ids_stage + k.copied, (end - k.copied) * 4,
                                 cudaMemcpyDeviceToHost, k.copy));
        k.copied = end;
    }
    return MDRQ_OK;
}

// Everything a batch does on the stream: the query tables to the device, the scan
// launches of the table's batch mode, and the offsets and error word back to pinned
// host memory. Asynchronous. It allocates nothing once the table's buffers have the
// batch's sizes, which is what lets a prepared batch capture it as a graph.
int enqueue_batch(mdrq_table *t, const std::vector<EncodedQuery> &enc, const std::vector<uint32_t> &live,
                  uint32_t nq, size_t npreds, uint32_t *out, uint64_t capacity, cudaStream_t s)
{
    const size_t nlive = live.size();
    const size_t dq_bytes = std::max<size_t>(1, nlive) * sizeof(DevQuery);
    const size_t dp_bytes = std::max<size_t>(1, npreds) * sizeof(DevPred);
    int st = grow_device((void **)&t->offsets_dev, &t->offsets_dev_cap, ((size_t)nq + 1) * 8);
    if (st == MDRQ_OK)
        st = grow_pinned((void **)&t->offsets_host, &t->offsets_host_cap, ((size_t)nq + 1) * 8);
    if (st == MDRQ_OK)
        st = grow_device((void **)&t->dq_dev, &t->dq_dev_cap, dq_bytes);
    if (st == MDRQ_OK)
        st = grow_device((void **)&t->dp_dev, &t->dp_dev_cap, dp_bytes);
    if (st == MDRQ_OK)
        st = grow_pinned((void **)&t->qstage_host, &t->qstage_host_cap, dq_bytes + dp_bytes);
    if (st != MDRQ_OK)
        return st;

    // the query tables go to the device in one copy (pinned staging)
    DevQuery *hq = reinterpret_cast<DevQuery *>(t->qstage_host);
    DevPred *hp = reinterpret_cast<DevPred *>(t->qstage_host + dq_bytes);
    uint64_t first = 0;
    for (size_t i = 0; i < nlive; ++i) {
        const EncodedQuery &e = enc[live[i]];
        hq[i].first = (uint32_t)first;
        hq[i].npred = (uint32_t)e.preds.size();
        hq[i].orig = live[i];
        hq[i].pad = 0;
        for (const DevPred &dp : e.preds)
            hp[first++] = dp;
    }
    // the offsets array and the query tables are written by this call only after the
    // previous call's kernels (same stream) have finished reading them
    MDRQ_TRY(cudaMemcpyAsync(t->dq_dev, hq, dq_bytes, cudaMemcpyHostToDevice, s));
    if (npreds)
        MDRQ_TRY(cudaMemcpyAsync(t->dp_dev, hp, npreds * sizeof(DevPred), cudaMemcpyHostToDevice, s));
    MDRQ_TRY(cudaMemsetAsync(t->offsets_dev, 0, ((size_t)nq + 1) * 8, s));
    MDRQ_TRY(cudaMemsetAsync(t->error, 0, sizeof(int), s));

    if (t->batch_mode == MDRQ_BATCH_LEARNED) {
        if (!t->learned)
            return MDRQ_E_INVAL;
        // windows and their scan, one launch per chunk whose ids fit the state values
        const uint64_t per = std::max<uint64_t>(1, kValueMask / std::max<uint64_t>(1, t->n));
        for (size_t c0 = 0; c0 < nlive; c0 += per) {
            const uint32_t cnt = (uint32_t)std::min<uint64_t>(per, nlive - c0);
            const unsigned long long *base = c0 == 0 ? nullptr : t->offsets_dev + live[c0 - 1] + 1;
            st = learned_batch(t, enc, live, (uint32_t)c0, cnt, out, capacity, base, s);
            if (st != MDRQ_OK) {
                reset_scratch(t, s);
                return st;
            }
        }
    }
    const bool learned_mode = t->batch_mode == MDRQ_BATCH_LEARNED;
    const bool shared = !learned_mode && (t->batch_mode == MDRQ_BATCH_SHARED ||
                        (t->batch_mode == MDRQ_BATCH_AUTO && nlive >= kAutoSharedMinQueries &&
                         (t->auto_mode >= 0 ? t->auto_mode == MDRQ_BATCH_SHARED : t->n >= kAutoSharedMinRows)));
    if (shared) {
        cudaEvent_t *evp = nullptr;
        if (t->timing) {
            if (t->ev.size() < 2 * (t->ev_used + 1)) {
                cudaEvent_t a, b;
                MDRQ_TRY(cudaEventCreate(&a));
                MDRQ_TRY(cudaEventCreate(&b));
                t->ev.push_back(a);
                t->ev.push_back(b);
            }
            evp = &t->ev[2 * t->ev_used];
            ++t->ev_used;
            MDRQ_TRY(cudaEventRecord(evp[0], s));
        }
        st = shared_scan_batch(t, enc, live, out, capacity, s);
        if (st != MDRQ_OK)
            return st;
        if (evp) {
            MDRQ_TRY(cudaEventRecord(evp[1], s));
            t->acc_scans += 1;
        }
    }
    // one launch per chunk of queries whose ids fit the 40-bit state values; with the
    // answers bound for host memory, up to kSinkLaunches launches of at least
    // kSinkLaunchBytes of columns each, each one's ids copied out while the next runs
    uint64_t per_launch = std::max<uint64_t>(1, kValueMask / std::max<uint64_t>(1, t->n));
    if (t->sink && !shared && !learned_mode) {
        uint64_t scan_bytes = 0;
        for (size_t i = 0; i < nlive; ++i)
            scan_bytes += enc[live[i]].scanned_columns * 4ull * t->n;
        const uint64_t launches =
            std::max<uint64_t>(1, std::min<uint64_t>(kSinkLaunches, scan_bytes / kSinkLaunchBytes));
        per_launch = std::min<uint64_t>(per_launch, std::max<uint64_t>(1, (nlive + launches - 1) / launches));
    }
    for (size_t c0 = 0; !shared && !learned_mode && c0 < nlive; c0 += per_launch) {
        const uint32_t cnt = (uint32_t)std::min<uint64_t>(per_launch, nlive - c0);
        uint64_t cols = 0;
        bool zones = false;
        for (size_t i = c0; i < c0 + cnt; ++i) {
            cols += enc[live[i]].scanned_columns;
            for (const DevPred &dp : enc[live[i]].preds)
                zones = zones || dp.zone != nullptr;
        }
        const unsigned long long *base = c0 == 0 ? nullptr : t->offsets_dev + live[c0 - 1] + 1;
        // zone maps in use: scan only the tiles they do not rule out
        st = zones ? zone_batch(t, (uint32_t)c0, cnt, cols, out, capacity, base, s)
                   : launch_scan(t, (uint32_t)c0, cnt, cols, out, capacity, base, s);
        if (st == MDRQ_OK && t->sink) {
            st = sink_flush(t);  // the previous launch's ids, while this one runs
            if (st == MDRQ_OK)
                st = cuda_status(cudaEventRecord(t->sink->pending_done, s));
            t->sink->pending = true;
            t->sink->pending_last = live[c0 + cnt - 1];
        }
        if (st != MDRQ_OK) {
            reset_scratch(t, s);
            return st;
        }
    }
    MDRQ_TRY(cudaMemcpyAsync(t->offsets_host, t->offsets_dev, ((size_t)nq + 1) * 8,
                             cudaMemcpyDeviceToHost, s));
    MDRQ_TRY(cudaMemcpyAsync(t->error_host, t->error, sizeof(int), cudaMemcpyDeviceToHost, s));
    return MDRQ_OK;
}

// Waits for a batch enqueued on s and fills the caller's offsets (nq + 1); a query
// answered on the host (empty) ends where the previous one ends.
int finish_batch(mdrq_table *t, const std::vector<uint32_t> &live, uint32_t nq, uint64_t *offsets, cudaStream_t s)
{
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        reset_scratch(t, s);
        return cuda_status(e);
    }
    if (*t->error_host != 0) {
        reset_scratch(t, s);
        return MDRQ_E_TIMEOUT;
    }
    std::memcpy(offsets, t->offsets_host, ((size_t)nq + 1) * 8);
    offsets[0] = 0;
    size_t li = 0;
    for (uint32_t q = 0; q < nq; ++q) {
        if (li < live.size() && live[li] == q)
            ++li;
        else
            offsets[q + 1] = offsets[q];
    }
    return MDRQ_OK;
}

// Whether a batch's live queries go to plain launches with staged output (the mode
// choice of enqueue_batch and the order rule of launch_scan, for a single launch).
static bool batch_output_staged(const mdrq_table *t, const std::vector<EncodedQuery> &enc,
                                const std::vector<uint32_t> &live)
{
    const size_t nlive = live.size();
    if (nlive == 0 || t->n == 0 || t->batch_mode == MDRQ_BATCH_LEARNED || t->output_order == MDRQ_ORDER_LOOKBACK)
        return false;
    const bool shared = t->batch_mode == MDRQ_BATCH_SHARED ||
                        (t->batch_mode == MDRQ_BATCH_AUTO && nlive >= kAutoSharedMinQueries &&
                         (t->auto_mode >= 0 ? t->auto_mode == MDRQ_BATCH_SHARED : t->n >= kAutoSharedMinRows));
    if (shared)
        return false;
    for (uint32_t q : live)
        for (const DevPred &dp : enc[q].preds)
            if (dp.zone)
                return false;  // tile pruning: a windowed launch
    if (t->output_order == MDRQ_ORDER_STAGED)
        return true;
    const uint64_t tiles = (uint64_t)nlive * ((t->n + tile_rows<4>() - 1) / tile_rows<4>());
    return tiles >= kStagedMinTilesPerBlock * (uint64_t)t->sm_count * t->blocks_per_sm[2];
}

int run_batch(mdrq_table *t, const mdrq_qdesc *qs, uint32_t nq, uint32_t *ids, uint64_t capacity,
              uint64_t *offsets, int ids_on_device, cudaStream_t s)
{
    if (!t || !offsets || (nq > 0 && !qs) || (capacity > 0 && !ids))
        return MDRQ_E_INVAL;
    std::vector<EncodedQuery> enc;
    std::vector<uint32_t> live;
    size_t npreds = 0;
    int st = encode_batch(t, qs, nq, enc, live, npreds);
    if (st != MDRQ_OK)
        return st;
    t->last_launches = 0;
    t->last_bytes = 0;
    MDRQ_TRY(cudaSetDevice(t->device));
    if (__atomic_exchange_n(&t->inject_nomem, 0, __ATOMIC_ACQ_REL))
        return MDRQ_E_NOMEM;
    // host answers: the scan writes a device staging buffer, and the ids of each finished
    // launch are copied to the host on a second stream while the next launch runs
    uint32_t *out = ids;
    HostSink sink;
    uint32_t *mapped = nullptr;  // the caller's page-locked buffer as the device sees it
    // AUTO: a batch whose plain output is staged is ordered by a pass after each scan;
    // its ids go through device staging and copies that overlap the next launch rather
    // than crossing the CPU-GPU link from the ordering pass, after the scan
    const bool via_copies = t->host_answers == MDRQ_HOST_STAGED ||
                            (t->host_answers == MDRQ_HOST_AUTO && batch_output_staged(t, enc, live));
    if (!ids_on_device && capacity > 0 && !via_copies) {
        cudaPointerAttributes a;
        if (cudaPointerGetAttributes(&a, ids) == cudaSuccess && a.type == cudaMemoryTypeHost && a.devicePointer)
            mapped = static_cast<uint32_t *>(a.devicePointer);
        (void)cudaGetLastError();
        if (!mapped && t->host_answers == MDRQ_HOST_DIRECT)
            return MDRQ_E_INVAL;
    }
    if (mapped) {
        // the scan writes the ids into host memory itself, over the CPU-GPU link: no
        // staging buffer, no copy engine competing with the scan for HBM
        out = mapped;
    } else if (!ids_on_device && capacity > 0) {
        st = grow_device((void **)&t->ids_stage, &t->ids_stage_cap, (size_t)capacity * 4);
        if (st == MDRQ_OK && !t->sink_copy) {
            st = cuda_status(cudaStreamCreateWithFlags(&t->sink_copy, cudaStreamNonBlocking));
            if (st == MDRQ_OK)
                st = cuda_status(cudaEventCreateWithFlags(&t->sink_done, cudaEventDisableTiming));
            if (st == MDRQ_OK)
                st = grow_pinned((void **)&t->sink_end, &t->sink_end_cap, 8);
        }
        if (st != MDRQ_OK)
            return st;
        out = t->ids_stage;
        sink.host = ids;
        sink.capacity = capacity;
        sink.copy = t->sink_copy;
        sink.end_host = t->sink_end;
        sink.pending_done = t->sink_done;
        t->sink = &sink;
    }
    st = enqueue_batch(t, enc, live, nq, npreds, out, capacity, s);
    if (st == MDRQ_OK)
        st = finish_batch(t, live, nq, offsets, s);
    const uint64_t total = st == MDRQ_OK ? offsets[nq] : 0;
    if (t->sink) {
        // the rest of the ids (the last launch's, or all of a shared or learned batch)
        sink.pending = false;
        if (st == MDRQ_OK && std::min<uint64_t>(total, capacity) > sink.copied) {
            const uint64_t end = std::min<uint64_t>(total, capacity);
            st = cuda_status(cudaMemcpyAsync(ids + sink.copied, t->ids_stage + sink.copied, (end - sink.copied) * 4,
                                             cudaMemcpyDeviceToHost, sink.copy));
        }
        const int cs = cuda_status(cudaStreamSynchronize(sink.copy));
        t->sink = nullptr;
        if (st == MDRQ_OK)
            st = cs;
    }
    if (st != MDRQ_OK)
        return st;
    // 4 bytes per id written
    t->last_bytes += 4ull * std::min<uint64_t>(total, capacity);
    if (t->timing)
        t->acc_bytes += 4ull * std::min<uint64_t>(total, capacity);
    return total > capacity ? MDRQ_E_CAPACITY : MDRQ_OK;
}

// scratch: claim counter, error word, a ring of 2^16 look-back states (512 KiB) and the
// staged output's allocation counter; and the pinned error word
int alloc_scratch(mdrq_table *t, cudaStream_t s)
{
    t->ring_bits = 16;
    const size_t scratch_words = 3 + ((size_t)1 << t->ring_bits);
    MDRQ_TRY(cudaMalloc(&t->scratch, scratch_words * 8));
    t->ticket = t->scratch;
    t->error = reinterpret_cast<int *>(t->scratch + 1);
    t->tile_state = t->scratch + 2;
    t->cat_bump = t->scratch + 2 + ((size_t)1 << t->ring_bits);
    MDRQ_TRY(cudaMemsetAsync(t->scratch, 0, scratch_words * 8, s));
    MDRQ_TRY(cudaMallocHost((void **)&t->error_host, sizeof(int)));
    return MDRQ_OK;
}

// A private table over t's columns: the same rows, statistics, zone maps, batch mode and
// shared-scan configuration, its own scratch and per-batch buffers. Owns nothing of t.
int make_shadow(const mdrq_table *t, cudaStream_t s, mdrq_table **out)
{
    *out = nullptr;
    mdrq_table *sh = new (std::nothrow) mdrq_table();
    if (!sh)
        return MDRQ_E_NOMEM;
    sh->device = t->device;
    sh->n = t->n;
    sh->d = t->d;
    sh->cols = t->cols;
    sh->sm_count = t->sm_count;
    for (int i = 0; i < 3; ++i)
        sh->blocks_per_sm[i] = t->blocks_per_sm[i];
    sh->blocks_per_sm_window = t->blocks_per_sm_window;
    sh->batch_mode = t->batch_mode;
    sh->shared_unit_rows = t->shared_unit_rows;
    sh->shared_image_words = t->shared_image_words;
    sh->shared_bits_budget = t->shared_bits_budget;
    sh->auto_mode = t->auto_mode;
    sh->zone_mode = t->zone_mode;
    sh->output_order = t->output_order;
    const int st = alloc_scratch(sh, s);
    if (st != MDRQ_OK) {
        free_shadow(sh);
        return st;
    }
    *out = sh;
    return MDRQ_OK;
}

void free_shadow(mdrq_table *sh)
{
    if (!sh)
        return;
    for (ColumnInfo &c : sh->cols)
        c.zone = nullptr;  // the parent's
    destroy(sh);
}

void destroy(mdrq_table *t)
{
    if (!t)
        return;
    cudaSetDevice(t->device);
    cudaDeviceSynchronize();
    for (void *p : t->owned)
        cudaFree(p);
    for (ColumnInfo &c : t->cols)
        cudaFree(c.zone);
    cudaFree(t->scratch);
    cudaFree(t->offsets_dev);
    shared_scan_free(t);
    zone_windows_free(t);
    learned_free(t);
    cudaFree(t->ids_stage);
    cudaFree(t->tile_map);
    concat_free(t);
    if (t->sink_copy)
        cudaStreamDestroy(t->sink_copy);
    if (t->sink_done)
        cudaEventDestroy(t->sink_done);
    cudaFreeHost(t->sink_end);
    cudaFree(t->dq_dev);
    cudaFree(t->dp_dev);
    cudaFreeHost(t->qstage_host);
    cudaFreeHost(t->offsets_host);
    cudaFreeHost(t->error_host);
    for (cudaEvent_t e : t->ev)
        cudaEventDestroy(e);
    (void)cudaGetLastError();
    delete t;
}

// Zone maps of every column (one read of the table) and their mean width relative to
// the column's range; MDRQ_ZONES_AUTO uses a column's map when that mean is below
// kZoneKeepWidth, i.e. when the row order clusters its values.
constexpr double kZoneKeepWidth = 0.5;

int build_zone_maps(mdrq_table *t, cudaStream_t s)
{
    const uint64_t nz = (t->n + kZoneTileRows - 1) / kZoneTileRows;
    double *sums = nullptr;
    MDRQ_TRY(cudaMalloc(&sums, (size_t)t->d * 8));
    int st = cuda_status(cudaMemsetAsync(sums, 0, (size_t)t->d * 8, s));
    for (uint32_t j = 0; j < t->d && st == MDRQ_OK; ++j) {
        ColumnInfo &c = t->cols[j];
        if ((st = cuda_status(cudaMalloc(&c.zone, (size_t)nz * sizeof(uint2)))))
            break;
        const double range = bound_value(c.max_bits, c.type) - bound_value(c.min_bits, c.type);
        const double inv = std::isfinite(range) && range > 0 ? 1.0 / range : 0.0;
        const uint32_t grid = (uint32_t)std::min<uint64_t>((nz + 7) / 8, (uint64_t)t->sm_count * 16);
        mdrq_zone_kernel<<<std::max(1u, grid), 256, 0, s>>>((const uint32_t *)c.ptr, t->n, (uint32_t)c.type, c.zone,
                                                             inv, sums + j);
        st = cuda_status(cudaGetLastError());
    }
    std::vector<double> h((size_t)t->d, 0.0);
    if (st == MDRQ_OK)
        st = cuda_status(cudaMemcpyAsync(h.data(), sums, (size_t)t->d * 8, cudaMemcpyDeviceToHost, s));
    if (st == MDRQ_OK)
        st = cuda_status(cudaStreamSynchronize(s));
    cudaFree(sums);
    if (st != MDRQ_OK)
        return st;
    for (uint32_t j = 0; j < t->d; ++j) {
        ColumnInfo &c = t->cols[j];
        const double range = bound_value(c.max_bits, c.type) - bound_value(c.min_bits, c.type);
        c.zone_width = nz ? h[j] / (double)nz : 1.0;
        c.zone_keep = std::isfinite(range) && c.zone_width < kZoneKeepWidth;
    }
    return MDRQ_OK;
}

int load(const void *const *cols, const int32_t *types, uint32_t d, uint64_t n, int cols_on_device,
         cudaStream_t s, mdrq_table *t)
{
    MDRQ_TRY(cudaGetDevice(&t->device));
    MDRQ_TRY(cudaDeviceGetAttribute(&t->sm_count, cudaDevAttrMultiProcessorCount, t->device));
    // The early break reads isolated 32-byte sectors of the later columns; fetching
    // more than a sector from DRAM per L2 miss brings in sectors the scan skips
    // (measured: 1.27x the early-break bytes at the default granularity, 0.99x at 32).
    // The limit is a property of the CUDA context and ends with it.
    MDRQ_TRY(cudaDeviceSetLimit(cudaLimitMaxL2FetchGranularity, 32));
    MDRQ_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&t->blocks_per_sm[0], mdrq_scan_kernel<1>, kScanThreads, 0));
    MDRQ_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&t->blocks_per_sm[1], mdrq_scan_kernel<2>, kScanThreads, 0));
    MDRQ_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&t->blocks_per_sm[2], mdrq_scan_kernel<4>, kScanThreads, 0));
    for (int i = 0; i < 3; ++i)
        t->blocks_per_sm[i] = std::max(1, t->blocks_per_sm[i]);
    t->n = n;
    t->d = d;
    t->cols.resize(d);

    for (uint32_t j = 0; j < d; ++j) {
        t->cols[j].type = types[j];
        if (n == 0)
            continue;
        if (cols_on_device) {
            t->cols[j].ptr = cols[j];
        } else {
            void *p = nullptr;
            MDRQ_TRY(cudaMalloc(&p, (size_t)((n * 4 + 15) & ~15ull)));
            t->owned.push_back(p);
            MDRQ_TRY(cudaMemcpyAsync(p, cols[j], (size_t)n * 4, cudaMemcpyHostToDevice, s));
            t->cols[j].ptr = p;
        }
    }

    {
        const int st = alloc_scratch(t, s);
        if (st != MDRQ_OK)
            return st;
    }

    if (n == 0)
        return cuda_status(cudaStreamSynchronize(s));

    // exact minimum / maximum, NaN count and a strided sample of every column
    unsigned long long *stats = nullptr;
    uint32_t *sample = nullptr;
    const uint32_t S = (uint32_t)std::min<uint64_t>(n, kSampleRows);
    MDRQ_TRY(cudaMalloc(&stats, (size_t)d * 3 * 8));
    MDRQ_TRY(cudaMalloc(&sample, (size_t)d * S * 4));
    std::vector<unsigned long long> init(3 * (size_t)d);
    for (uint32_t j = 0; j < d; ++j) {
        init[3 * j] = 0;
        init[3 * j + 1] = ~0ull;
        init[3 * j + 2] = 0;
    }
    int st = MDRQ_OK;
    std::vector<unsigned long long> h_stats(3 * (size_t)d);
    std::vector<uint32_t> h_sample((size_t)d * S);
    do {
        if ((st = cuda_status(cudaMemcpyAsync(stats, init.data(), init.size() * 8, cudaMemcpyHostToDevice, s))))
            break;
        const uint32_t grid = (uint32_t)std::min<uint64_t>((n + kBlock - 1) / kBlock, (uint64_t)t->sm_count * 8);
        for (uint32_t j = 0; j < d; ++j) {
            mdrq_column_stats_kernel<<<grid, kBlock, 0, s>>>((const uint32_t *)t->cols[j].ptr, n,
                                                             (uint32_t)types[j], stats + 3 * j);
            mdrq_sample_kernel<<<(S + 255) / 256, 256, 0, s>>>((const uint32_t *)t->cols[j].ptr, n, S,
                                                              sample + (size_t)j * S);
        }
        if ((st = cuda_status(cudaGetLastError())))
            break;
        if ((st = cuda_status(cudaMemcpyAsync(h_stats.data(), stats, h_stats.size() * 8, cudaMemcpyDeviceToHost, s))))
            break;
        if ((st = cuda_status(cudaMemcpyAsync(h_sample.data(), sample, h_sample.size() * 4, cudaMemcpyDeviceToHost, s))))
            break;
        st = cuda_status(cudaStreamSynchronize(s));
    } while (0);
    cudaFree(stats);
    cudaFree(sample);
    if (st != MDRQ_OK)
        return st;
    for (uint32_t j = 0; j < d; ++j) {
        if (h_stats[3 * j] != 0)
            return MDRQ_E_NAN;
        ColumnInfo &c = t->cols[j];
        c.min_bits = bits_from_key(h_stats[3 * j + 1], c.type);
        c.max_bits = bits_from_key(h_stats[3 * j + 2], c.type);
        c.sample.resize(S);
        for (uint32_t i = 0; i < S; ++i)
            c.sample[i] = bound_value(h_sample[(size_t)j * S + i], c.type);
        std::sort(c.sample.begin(), c.sample.end());
    }
    return build_zone_maps(t, s);
}

}  // namespace mdrq

extern "C" {

int mdrq_load_columns(const void *const *cols, const int32_t *types, uint32_t d, uint64_t n,
                      int cols_on_device, void *stream, mdrq_table **out)
{
    if (!out)
        return MDRQ_E_INVAL;
    *out = nullptr;
    if (d == 0 || n > 0xFFFFFFFFull || !types || (n > 0 && !cols))
        return MDRQ_E_INVAL;
    for (uint32_t j = 0; j < d; ++j) {
        if (types[j] != MDRQ_F32 && types[j] != MDRQ_I32)
            return MDRQ_E_INVAL;
        if (n > 0 && !cols[j])
            return MDRQ_E_INVAL;
        if (n > 0 && cols_on_device && (reinterpret_cast<uintptr_t>(cols[j]) & 15u))
            return MDRQ_E_INVAL;
    }
    mdrq_table *t = new (std::nothrow) mdrq_table();
    if (!t)
        return MDRQ_E_NOMEM;
    int st = load(cols, types, d, n, cols_on_device, as_stream(stream), t);
    if (st != MDRQ_OK) {
        destroy(t);
        return st;
    }
    *out = t;
    return MDRQ_OK;
}

int mdrq_query(mdrq_table *t, const mdrq_pred *preds, uint32_t npreds, uint32_t *ids,
               uint64_t capacity, uint64_t *count, int ids_on_device, void *stream)
{
    if (!t || !count)
        return MDRQ_E_INVAL;
    mdrq_qdesc q;
    q.preds = preds;
    q.npreds = npreds;
    q.reserved = 0;
    uint64_t off[2] = {0, 0};
    int st = run_batch(t, &q, 1, ids, capacity, off, ids_on_device, as_stream(stream));
    if (st == MDRQ_OK || st == MDRQ_E_CAPACITY)
        *count = off[1];
    return st;
}

int mdrq_query_batch(mdrq_table *t, const mdrq_qdesc *qs, uint32_t nq, uint32_t *ids,
                     uint64_t capacity, uint64_t *offsets, int ids_on_device, void *stream)
{
    return run_batch(t, qs, nq, ids, capacity, offsets, ids_on_device, as_stream(stream));
}

void mdrq_free(mdrq_table *t) { destroy(t); }

const char *mdrq_status_string(int status)
{
    switch (status) {
    case MDRQ_OK: return "ok";
    case MDRQ_E_INVAL: return "invalid argument";
    case MDRQ_E_NOMEM: return "out of memory";
    case MDRQ_E_CUDA: return "CUDA error";
    case MDRQ_E_CAPACITY: return "answer longer than the id buffer";
    case MDRQ_E_TIMEOUT: return "device wait timed out";
    case MDRQ_E_NAN: return "NaN in a float32 column";
    default: return "unknown status";
    }
}

uint64_t mdrq_table_rows(const mdrq_table *t) { return t ? t->n : 0; }
uint32_t mdrq_table_dims(const mdrq_table *t) { return t ? t->d : 0; }

int mdrq_scan_timing(mdrq_table *t, int enable)
{
    if (!t)
        return MDRQ_E_INVAL;
    t->timing = enable != 0;
    return MDRQ_OK;
}

int mdrq_scan_timing_read(mdrq_table *t, double *ms, uint64_t *scan_launches, uint64_t *bytes,
                          uint64_t *kernel_launches, int reset)
{
    if (!t)
        return MDRQ_E_INVAL;
    double total = 0.0;
    if (t->ev_used > 0) {
        MDRQ_TRY(cudaEventSynchronize(t->ev[2 * t->ev_used - 1]));
        for (size_t i = 0; i < t->ev_used; ++i) {
            float x = 0.f;
            MDRQ_TRY(cudaEventElapsedTime(&x, t->ev[2 * i], t->ev[2 * i + 1]));
            total += x;
        }
    }
    if (ms)
        *ms = total;
    if (scan_launches)
        *scan_launches = t->acc_scans;
    if (bytes)
        *bytes = t->acc_bytes;
    if (kernel_launches)
        *kernel_launches = t->acc_kernels;
    if (reset) {
        t->ev_used = 0;
        t->acc_scans = t->acc_bytes = t->acc_kernels = 0;
    }
    return MDRQ_OK;
}

int mdrq_set_batch_mode(mdrq_table *t, int mode)
{
    if (!t || (mode != MDRQ_BATCH_AUTO && mode != MDRQ_BATCH_PLAIN && mode != MDRQ_BATCH_SHARED &&
               mode != MDRQ_BATCH_LEARNED))
        return MDRQ_E_INVAL;
    t->batch_mode = mode;
    return MDRQ_OK;
}

int mdrq_learn(mdrq_table *t, const uint32_t *dims, uint32_t ndims, int model, void *stream)
{
    if (!t)
        return MDRQ_E_INVAL;
    const cudaError_t e = cudaSetDevice(t->device);
    if (e != cudaSuccess)
        return cuda_status(e);
    return learn(t, dims, ndims, model, as_stream(stream));
}

int mdrq_learn_info(const mdrq_table *t, uint64_t *max_error, uint32_t *segments, double *train_ms)
{
    return learned_info(t, max_error, segments, train_ms);
}

int mdrq_learn_window_rows(mdrq_table *t, uint64_t *rows, uint64_t *widenings)
{
    return learned_window_rows(t, rows, widenings);
}

int mdrq_set_key_cells(mdrq_table *t, uint32_t dim, const float *bounds, uint32_t nbounds)
{
    return set_key_cells(t, dim, bounds, nbounds);
}

int mdrq_learn_search_info(mdrq_table *t, uint64_t *ranges, uint64_t *probes)
{
    return learned_search_info(t, ranges, probes);
}

int mdrq_learn_export(const mdrq_table *t, mdrq_model_desc *desc, uint64_t *knot_key, uint64_t *knot_pos,
                      float *slope, float *mlp, uint32_t capacity)
{
    return learned_export(t, desc, knot_key, knot_pos, slope, mlp, capacity);
}

int mdrq_set_host_answers(mdrq_table *t, int mode)
{
    if (!t || (mode != MDRQ_HOST_AUTO && mode != MDRQ_HOST_STAGED && mode != MDRQ_HOST_DIRECT))
        return MDRQ_E_INVAL;
    t->host_answers = mode;
    return MDRQ_OK;
}

int mdrq_set_output_order(mdrq_table *t, int mode)
{
    if (!t || (mode != MDRQ_ORDER_AUTO && mode != MDRQ_ORDER_LOOKBACK && mode != MDRQ_ORDER_STAGED))
        return MDRQ_E_INVAL;
    t->output_order = mode;
    return MDRQ_OK;
}

int mdrq_set_zone_maps(mdrq_table *t, int mode)
{
    if (!t || (mode != MDRQ_ZONES_OFF && mode != MDRQ_ZONES_AUTO && mode != MDRQ_ZONES_ALL))
        return MDRQ_E_INVAL;
    t->zone_mode = mode;
    return MDRQ_OK;
}

int mdrq_zone_map_info(const mdrq_table *t, uint32_t dim, int *used, double *mean_width)
{
    if (!t || dim >= t->d)
        return MDRQ_E_INVAL;
    const mdrq::ColumnInfo &c = t->cols[dim];
    if (used)
        *used = t->n > 0 && (t->zone_mode == MDRQ_ZONES_ALL || (t->zone_mode == MDRQ_ZONES_AUTO && c.zone_keep));
    if (mean_width)
        *mean_width = c.zone_width;
    return MDRQ_OK;
}

int mdrq_inject_fault(mdrq_table *t, int kind, uint64_t arg)
{
    if (!t)
        return MDRQ_E_INVAL;
    switch (kind) {
    case MDRQ_FAULT_SKIP_TILES:
        if (arg == 0)
            return MDRQ_E_INVAL;
        t->inject_skip_tiles = arg;
        return MDRQ_OK;
    case MDRQ_FAULT_NOMEM:
        __atomic_store_n(&t->inject_nomem, 1, __ATOMIC_RELEASE);
        return MDRQ_OK;
    case MDRQ_FAULT_STAGE_NOMEM:
        __atomic_store_n(&t->inject_stage_nomem, 1, __ATOMIC_RELEASE);
        return MDRQ_OK;
    default:
        return MDRQ_E_INVAL;
    }
}

int mdrq_explain_query(const mdrq_table *t, const mdrq_pred *preds, uint32_t npreds, mdrq_pred *plan,
                       uint32_t max_plan, uint32_t *nplan, int *empty)
{
    if (!t || !nplan || !empty || (max_plan > 0 && !plan))
        return MDRQ_E_INVAL;
    EncodedQuery q;
    const int st = encode_query(t, preds, npreds, q);
    if (st != MDRQ_OK)
        return st;
    *empty = q.empty ? 1 : 0;
    *nplan = (uint32_t)q.preds.size();
    for (size_t i = 0; i < q.preds.size() && i < max_plan; ++i) {
        plan[i].dim = q.dims[i];
        plan[i].reserved = 0;
        std::memcpy(&plan[i].lo, &q.preds[i].lo, 4);
        std::memcpy(&plan[i].hi, &q.preds[i].hi, 4);
    }
    return q.preds.size() > max_plan ? MDRQ_E_CAPACITY : MDRQ_OK;
}

void mdrq_last_scan_stats(const mdrq_table *t, uint64_t *launches, uint64_t *bytes)
{
    if (launches)
        *launches = t ? t->last_launches : 0;
    if (bytes)
        *bytes = t ? t->last_bytes : 0;
}

}  // extern "C"
