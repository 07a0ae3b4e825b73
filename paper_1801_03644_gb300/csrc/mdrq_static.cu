// mdrq_query_static: the scan of one query with no memory allocation at all.
//
// Some callers cannot allocate device memory when they query: a serving loop that
// runs under a memory budget owned by another allocator, a latency-critical path
// where cudaMalloc's implicit device-wide synchronisation would stall other streams,
// or code that must not change the GPU's memory footprint after start-up. For them,
// the scan's scratch (tile claim counter, error word, answer length and the per-tile
// look-back states) lives in one fixed-size array in device global memory, declared
// in this file; the caller passes only its own inputs (device columns, predicates)
// and outputs (device id buffer, host count).
//
// Set-up: the host cannot use the array's name as a device address, so the first
// call on each device (with that device current) asks the runtime for the address
// with cudaGetSymbolAddress and caches it, together with the launch shape. Make
// that first call before any stream capture. Nothing here calls cudaMalloc,
// cudaFree, cudaMallocHost or any other allocating routine, on the host or the GPU.
//
// The array is shared by every call on a device and keeps the last call's contents,
// so each call clears the words that must start at zero (claim counter, error word,
// answer length, the look-back states it will use) before its launch. Calls whose
// work overlaps on the GPU (concurrent streams, several host threads) race on the
// array and give wrong answers: serialise them.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>

#include "mdrq.h"
#include "scan_kernel.cuh"

using namespace mdrq;

namespace {

constexpr uint64_t kTileRows = (uint64_t)kWarps * 4 * 128;  // 4096: the U = 4 tile
constexpr uint64_t kMaxTiles = MDRQ_STATIC_MAX_ROWS / kTileRows;
static_assert(kMaxTiles * kTileRows == MDRQ_STATIC_MAX_ROWS, "limit is a whole number of tiles");

// word layout: [0] claim counter, [1] error word, [2] answer start (0), [3] answer
// length, then the look-back states (one per tile, used as a ring that never wraps
// here), the query descriptor and its predicates
constexpr uint32_t kRingBits = 16;
static_assert((1ull << kRingBits) == kMaxTiles, "one state per tile of the largest table");
constexpr uint64_t kHeadWords = 4;
constexpr uint64_t kQueryWord = kHeadWords + kMaxTiles;
constexpr uint64_t kPredWord = kQueryWord + sizeof(DevQuery) / 8;
constexpr uint64_t kScratchWords = kPredWord + (uint64_t)kMaxPreds * sizeof(DevPred) / 8;
static_assert(sizeof(DevQuery) % 8 == 0 && sizeof(DevPred) % 8 == 0, "word-aligned tables");

constexpr int kMaxDevices = 64;

}  // namespace

// The fixed scratch: (4 + 65536 + 2 + 512) * 8 bytes = 516.1 KiB per device that loads
// the library, held until the process exits.
static __device__ __align__(256) unsigned long long g_scan_scratch[kScratchWords];

__global__ void __launch_bounds__(kScanThreads, 7) mdrq_scan_static_kernel(const __grid_constant__ ScanParams p)
{
    scan_cta<4>(p);
}

namespace {

struct DeviceSetup {
    bool ready = false;
    unsigned long long *scratch = nullptr;  // device address of g_scan_scratch
    int sm_count = 0;
    int blocks_per_sm = 0;
};

std::mutex g_setup_mutex;
DeviceSetup g_setup[kMaxDevices];  // by device ordinal; fixed storage, no allocation

int status_of(cudaError_t e)
{
    if (e == cudaSuccess)
        return MDRQ_OK;
    (void)cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? MDRQ_E_NOMEM : MDRQ_E_CUDA;
}

// once per device, with that device current
int device_setup(int dev, DeviceSetup *&out)
{
    if (dev < 0 || dev >= kMaxDevices)
        return MDRQ_E_INVAL;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    DeviceSetup &s = g_setup[dev];
    if (!s.ready) {
        void *ptr = nullptr;
        int st = status_of(cudaGetSymbolAddress(&ptr, g_scan_scratch));
        if (st != MDRQ_OK)
            return st;
        if ((st = status_of(cudaDeviceGetAttribute(&s.sm_count, cudaDevAttrMultiProcessorCount, dev))))
            return st;
        if ((st = status_of(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&s.blocks_per_sm, mdrq_scan_static_kernel,
                                                                           kScanThreads, 0))))
            return st;
        if (s.blocks_per_sm < 1)
            s.blocks_per_sm = 1;
        s.scratch = static_cast<unsigned long long *>(ptr);
        s.ready = true;
    }
    out = &s;
    return MDRQ_OK;
}

double value_of(uint32_t bits, int32_t type)
{
    if (type == MDRQ_F32) {
        float f;
        std::memcpy(&f, &bits, 4);
        return (double)f;
    }
    return (double)(int32_t)bits;
}

}  // namespace

extern "C" int mdrq_query_static(const void *const *cols, const int32_t *types, uint32_t d, uint64_t n,
                                 const mdrq_pred *preds, uint32_t npreds, uint32_t *ids, uint64_t capacity,
                                 uint64_t *count, void *stream)
{
    if (!count || !types || d == 0 || (n > 0 && !cols) || (npreds > 0 && !preds) || (capacity > 0 && !ids))
        return MDRQ_E_INVAL;
    if (n > MDRQ_STATIC_MAX_ROWS)
        return MDRQ_E_INVAL;  // the fixed scratch holds look-back states for at most this many rows
    for (uint32_t j = 0; j < d; ++j) {
        if (types[j] != MDRQ_F32 && types[j] != MDRQ_I32)
            return MDRQ_E_INVAL;
        if (n > 0 && (!cols[j] || (reinterpret_cast<uintptr_t>(cols[j]) & 15u)))
            return MDRQ_E_INVAL;
    }

    // Sec. 2.1: AND of closed intervals; a repeated dimension intersects its intervals.
    // Fixed storage: at most kMaxPreds distinct dimensions.
    DevPred pred[kMaxPreds];
    double lo_v[kMaxPreds], hi_v[kMaxPreds];
    uint32_t dim_of[kMaxPreds];
    uint32_t k = 0;
    bool empty = false;
    for (uint32_t i = 0; i < npreds; ++i) {
        const mdrq_pred &q = preds[i];
        if (q.dim >= d || q.reserved != 0)
            return MDRQ_E_INVAL;
        uint32_t lb, hb;
        std::memcpy(&lb, &q.lo, 4);
        std::memcpy(&hb, &q.hi, 4);
        const double lo = value_of(lb, types[q.dim]), hi = value_of(hb, types[q.dim]);
        if (std::isnan(lo) || std::isnan(hi))
            return MDRQ_E_INVAL;
        uint32_t slot = k;
        for (uint32_t s = 0; s < k; ++s)
            if (dim_of[s] == q.dim)
                slot = s;
        if (slot == k) {
            if (k == (uint32_t)kMaxPreds)
                return MDRQ_E_INVAL;
            dim_of[k] = q.dim;
            lo_v[k] = lo;
            hi_v[k] = hi;
            pred[k].col = n > 0 ? cols[q.dim] : nullptr;
            pred[k].zone = nullptr;
            pred[k].type = (uint32_t)types[q.dim];
            pred[k].lo = lb;
            pred[k].hi = hb;
            pred[k].pad = 0;
            ++k;
        } else {
            if (lo > lo_v[slot]) {
                lo_v[slot] = lo;
                pred[slot].lo = lb;
            }
            if (hi < hi_v[slot]) {
                hi_v[slot] = hi;
                pred[slot].hi = hb;
            }
        }
    }
    for (uint32_t s = 0; s < k; ++s)
        if (lo_v[s] > hi_v[s])
            empty = true;  // an empty interval matches nothing
    *count = 0;
    if (n == 0 || empty)
        return MDRQ_OK;

    int dev = 0;
    int st = status_of(cudaGetDevice(&dev));
    if (st != MDRQ_OK)
        return st;
    DeviceSetup *ds = nullptr;
    if ((st = device_setup(dev, ds)) != MDRQ_OK)
        return st;

    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const uint64_t n_tiles = (n + kTileRows - 1) / kTileRows;
    const uint64_t resident = (uint64_t)ds->sm_count * ds->blocks_per_sm;
    const uint32_t grid = (uint32_t)(resident < n_tiles ? resident : n_tiles);
    unsigned long long *scratch = ds->scratch;

    // clear the header and the states this launch uses (the array keeps old contents),
    // then copy the query in (from host stack memory: no staging buffer is allocated)
    DevQuery qd;
    qd.first = 0;
    qd.npred = k;
    qd.orig = 0;
    qd.pad = 0;
    if ((st = status_of(cudaMemsetAsync(scratch, 0, (size_t)(kHeadWords + n_tiles) * 8, s))))
        return st;
    if ((st = status_of(cudaMemcpyAsync(scratch + kQueryWord, &qd, sizeof(qd), cudaMemcpyHostToDevice, s))))
        return st;
    if (k > 0 && (st = status_of(cudaMemcpyAsync(scratch + kPredWord, pred, k * sizeof(DevPred),
                                                 cudaMemcpyHostToDevice, s))))
        return st;

    ScanParams p;
    std::memset(&p, 0, sizeof(p));
    p.queries = reinterpret_cast<const DevQuery *>(scratch + kQueryWord);
    p.preds = reinterpret_cast<const DevPred *>(scratch + kPredWord);
    p.nq = 1;
    p.tiles_per_query = (uint32_t)n_tiles;
    p.n = n;
    p.total_tiles = n_tiles;
    p.tile_state = scratch + kHeadWords;
    p.ring_bits = kRingBits;
    p.tag0 = 1;  // cleared states carry tag 0
    p.ticket = scratch;
    p.ticket_base = 0;
    p.ids = ids;
    p.capacity = capacity;
    p.base_in = nullptr;
    p.offsets = scratch + 2;  // offsets[1], the answer length, lands in word 3
    p.error = reinterpret_cast<int *>(scratch + 1);
    mdrq_scan_static_kernel<<<grid, kScanThreads, 0, s>>>(p);
    if ((st = status_of(cudaGetLastError())))
        return st;

    unsigned long long head[4] = {0, 0, 0, 0};  // claim counter, error word, 0, answer length
    if ((st = status_of(cudaMemcpyAsync(head, scratch, sizeof(head), cudaMemcpyDeviceToHost, s))))
        return st;
    if ((st = status_of(cudaStreamSynchronize(s))))
        return st;
    if ((int)head[1] != 0)
        return MDRQ_E_TIMEOUT;
    *count = head[3];
    return head[3] > capacity ? MDRQ_E_CAPACITY : MDRQ_OK;
}
