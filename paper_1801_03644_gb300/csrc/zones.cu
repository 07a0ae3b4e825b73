// Zone-pruned plain scan: the row tiles a query's zone maps rule out are never visited.
//
// Every column carries, per 4096-row tile, the minimum and maximum of its values (built
// at load). A tile can hold an answer of a query only if, for
// every predicate with a zone map, the tile's range meets [lo, hi] — the VA-file's
// pruning of cells that cannot meet the query (Sec. 2.2.3), applied to row blocks of
// the scan. One block per query turns its candidate tiles into runs (windows, at most
// kZoneWindowsPerQuery; beyond that one window from the first to the last candidate),
// and the windowed scan then evaluates every predicate on the windows' rows exactly.
// Answers equal the plain scan's.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <new>
#include <vector>

#include "mdrq.h"
#include "scan_kernel.cuh"
#include "table.h"

namespace mdrq {

struct ZoneWindows {
    DevWindow *slots = nullptr;  // kZoneWindowsPerQuery per query, uncompacted
    size_t slots_cap = 0;
    DevWindow *windows = nullptr;  // compacted
    size_t windows_cap = 0;
    unsigned char *qaux = nullptr;  // per query: count, tiles, window base, tile base
    size_t qaux_cap = 0;
    unsigned long long *totals = nullptr;  // [0] tiles, [1] windows of the last launch
    bool have = false;
};

namespace {

constexpr uint32_t kZoneWindowsPerQuery = 1024;
constexpr int kZwThreads = 256;
constexpr int kZwPer = 4;            // tiles per thread per step
constexpr uint32_t kZwMaxPreds = 32;  // zone predicates a query is pruned by (the first ones)
static_assert(kZoneTileRows == (uint32_t)kWarps * 4 * 128, "tile zones match the windowed scan's tiles");

struct ZPred {
    const uint2 *tz;  // tile zones of the column
    uint32_t type, lo, hi;
};

__device__ __forceinline__ bool candidate(const ZPred *zp, uint32_t np, uint64_t tile)
{
    for (uint32_t i = 0; i < np; ++i)
        if (zone_verdict(zp[i].tz[tile], zp[i].type, zp[i].lo, zp[i].hi) == 0u)
            return false;
    return true;
}

// inclusive scan of one value per thread over the block; *total = the block's sum
__device__ __forceinline__ uint32_t zw_scan(uint32_t v, uint32_t *s_warp, uint32_t *s_total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t x = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o)
            v += x;
    }
    if (lane == 31)
        s_warp[warp] = v;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < kZwThreads / 32 ? s_warp[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t x = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o)
                w += x;
        }
        if (lane < kZwThreads / 32)
            s_warp[lane] = w;
        if (lane == kZwThreads / 32 - 1)
            *s_total = w;
    }
    __syncthreads();
    const uint32_t r = v + (warp ? s_warp[warp - 1] : 0u);
    __syncthreads();
    return r;
}

// One block per query: its windows (runs of candidate tiles) in slots[q * cap ..], with
// tile_start local to the query; counts[q] windows, qtiles[q] tiles. A query with no
// candidate tile gets one empty window of one tile, which closes its answer.
__global__ void __launch_bounds__(kZwThreads) mdrq_zone_windows_kernel(const DevQuery *queries, const DevPred *preds,
                                                                       uint64_t n, uint64_t ntiles,
                                                                       DevWindow *slots, uint32_t *counts,
                                                                       uint32_t *qtiles)
{
    __shared__ ZPred s_zp[kZwMaxPreds];
    __shared__ uint32_t s_t0[kZoneWindowsPerQuery], s_t1[kZoneWindowsPerQuery];
    __shared__ uint32_t s_warp[kZwThreads / 32];
    __shared__ uint32_t s_np, s_total, s_first, s_last;
    const uint32_t q = blockIdx.x;
    if (threadIdx.x == 0) {
        const DevQuery dq = queries[q];
        uint32_t k = 0;
        for (uint32_t i = 0; i < dq.npred && k < kZwMaxPreds; ++i) {
            const DevPred pr = preds[dq.first + i];
            if (pr.zone)
                s_zp[k++] = ZPred{pr.zone, pr.type, pr.lo, pr.hi};
        }
        s_np = k;
        s_first = 0xffffffffu;
        s_last = 0;
    }
    __syncthreads();
    const uint32_t np = s_np;
    const uint64_t step = (uint64_t)kZwThreads * kZwPer;

    // pass 1: number of runs, first and last candidate
    uint32_t runs = 0, first = 0xffffffffu, last = 0;
    for (uint64_t b = 0; b < ntiles; b += step) {
        const uint64_t i0 = b + (uint64_t)threadIdx.x * kZwPer;
        bool prev = i0 > 0 && i0 - 1 < ntiles && candidate(s_zp, np, i0 - 1);
        for (int k = 0; k < kZwPer; ++k) {
            const uint64_t i = i0 + k;
            const bool c = i < ntiles && candidate(s_zp, np, i);
            if (c) {
                runs += !prev;
                first = min(first, (uint32_t)i);
                last = max(last, (uint32_t)i);
            }
            prev = c;
        }
    }
    zw_scan(runs, s_warp, &s_total);
    const uint32_t nruns = s_total;
    if (first != 0xffffffffu) {
        atomicMin(&s_first, first);
        atomicMax(&s_last, last);
    }
    __syncthreads();

    uint32_t nr;
    if (nruns == 0) {
        nr = 0;  // no candidate: the empty window below
    } else if (nruns > kZoneWindowsPerQuery) {
        nr = 1;  // too fragmented: one window over the candidate span
        if (threadIdx.x == 0) {
            s_t0[0] = s_first;
            s_t1[0] = s_last + 1;
        }
    } else {
        // pass 2: the runs' first and end tiles, numbered in row order
        nr = nruns;
        uint32_t carry = 0;
        for (uint64_t b = 0; b < ntiles; b += step) {
            const uint64_t i0 = b + (uint64_t)threadIdx.x * kZwPer;
            bool c[kZwPer + 2];  // c[0]: tile i0 - 1, c[k + 1]: tile i0 + k, c[kZwPer + 1]: tile i0 + kZwPer
            c[0] = i0 > 0 && i0 - 1 < ntiles && candidate(s_zp, np, i0 - 1);
            for (int k = 0; k <= kZwPer; ++k) {
                const uint64_t i = i0 + k;
                c[k + 1] = i < ntiles && candidate(s_zp, np, i);
            }
            uint32_t mine = 0;
            for (int k = 1; k <= kZwPer; ++k)
                mine += c[k] && !c[k - 1];
            const uint32_t incl = zw_scan(mine, s_warp, &s_total);
            uint32_t r = carry + incl - mine;  // runs started before this thread's tiles
            for (int k = 1; k <= kZwPer; ++k) {
                const uint32_t i = (uint32_t)(i0 + k - 1);
                if (c[k] && !c[k - 1])
                    s_t0[r++] = i;
                if (c[k] && !c[k + 1])
                    s_t1[r - 1] = i + 1;
            }
            carry += s_total;
            __syncthreads();
        }
    }
    __syncthreads();
    // windows and their tiles (4 per thread, in row order), tile prefix local to the query
    const uint32_t nw = nr ? nr : 1u;
    uint32_t tl[4], mine = 0;
    for (int k = 0; k < 4; ++k) {
        const uint32_t r = threadIdx.x * 4 + k;
        tl[k] = r < nr ? s_t1[r] - s_t0[r] : (r == 0 && nr == 0 ? 1u : 0u);
        mine += tl[k];
    }
    const uint32_t incl = zw_scan(mine, s_warp, &s_total);
    uint32_t pos = incl - mine;
    DevWindow *dst = slots + (size_t)q * kZoneWindowsPerQuery;
    for (int k = 0; k < 4; ++k) {
        const uint32_t r = threadIdx.x * 4 + k;
        if (r < nw) {
            DevWindow w;
            if (nr) {
                w.row_begin = (unsigned long long)s_t0[r] * kZoneTileRows;
                w.row_end = min((unsigned long long)s_t1[r] * kZoneTileRows, (unsigned long long)n);
            } else {
                w.row_begin = 0;
                w.row_end = 0;
            }
            w.row_first = w.row_begin;
            w.tile_start = pos;
            w.tiles = tl[k];
            w.query = q;
            w.last = r + 1 == nw;
            dst[r] = w;
        }
        pos += tl[k];
    }
    if (threadIdx.x == 0) {
        counts[q] = nw;
        qtiles[q] = s_total;
    }
}

}  // namespace

int zone_batch(mdrq_table *t, uint32_t q0, uint32_t nlive, uint64_t scanned_columns, uint32_t *ids,
               uint64_t capacity, const unsigned long long *base_in, cudaStream_t s)
{
    if (nlive == 0)
        return MDRQ_OK;
    if (!t->zwin) {
        t->zwin = new (std::nothrow) ZoneWindows();
        if (!t->zwin)
            return MDRQ_E_NOMEM;
        MDRQ_TRY_STATUS(cudaMalloc(&t->zwin->totals, 16));
    }
    ZoneWindows &Z = *t->zwin;
    const size_t max_windows = (size_t)nlive * kZoneWindowsPerQuery;
    int st = grow_device((void **)&Z.slots, &Z.slots_cap, max_windows * sizeof(DevWindow));
    if (st == MDRQ_OK)
        st = grow_device((void **)&Z.windows, &Z.windows_cap, max_windows * sizeof(DevWindow));
    if (st == MDRQ_OK)
        st = grow_device((void **)&Z.qaux, &Z.qaux_cap, (size_t)nlive * 24);
    if (st != MDRQ_OK)
        return st;
    uint32_t *counts = reinterpret_cast<uint32_t *>(Z.qaux);
    uint32_t *qtiles = counts + nlive;
    unsigned long long *wbase = reinterpret_cast<unsigned long long *>(qtiles + nlive);
    unsigned long long *tbase = wbase + nlive;
    const uint64_t ntiles = (t->n + kZoneTileRows - 1) / kZoneTileRows;
    mdrq_zone_windows_kernel<<<nlive, kZwThreads, 0, s>>>(t->dq_dev + q0, t->dp_dev, t->n, ntiles, Z.slots, counts,
                                                          qtiles);
    MDRQ_TRY_STATUS(cudaGetLastError());
    st = window_list(nlive, kZoneWindowsPerQuery, counts, qtiles, wbase, tbase, Z.slots, Z.windows, Z.totals, s);
    if (st != MDRQ_OK)
        return st;
    Z.have = true;
    return launch_window_scan(t, q0, nlive, max_windows, Z.totals + 1, scanned_columns * 4ull * t->n, 3, ids,
                              capacity, base_in, Z.windows, Z.totals, s);
}

void zone_windows_free(mdrq_table *t)
{
    if (!t || !t->zwin)
        return;
    cudaFree(t->zwin->slots);
    cudaFree(t->zwin->windows);
    cudaFree(t->zwin->qaux);
    cudaFree(t->zwin->totals);
    delete t->zwin;
    t->zwin = nullptr;
}

int zone_window_rows(mdrq_table *t, uint64_t *rows, uint64_t *tiles)
{
    unsigned long long tot[2] = {0, 0};
    if (t->zwin && t->zwin->have)
        MDRQ_TRY_STATUS(cudaMemcpy(tot, t->zwin->totals, 16, cudaMemcpyDeviceToHost));
    std::vector<DevWindow> w(tot[1]);
    if (tot[1])
        MDRQ_TRY_STATUS(cudaMemcpy(w.data(), t->zwin->windows, tot[1] * sizeof(DevWindow), cudaMemcpyDeviceToHost));
    uint64_t sum = 0;
    for (const DevWindow &x : w)
        sum += x.row_end - x.row_first;
    if (rows)
        *rows = sum;
    if (tiles)
        *tiles = tot[0];
    return MDRQ_OK;
}

}  // namespace mdrq

extern "C" int mdrq_zone_scan_info(mdrq_table *t, uint64_t *rows, uint64_t *tiles)
{
    if (!t)
        return MDRQ_E_INVAL;
    const cudaError_t e = cudaSetDevice(t->device);
    if (e != cudaSuccess)
        return mdrq::cuda_status(e);
    return mdrq::zone_window_rows(t, rows, tiles);
}
