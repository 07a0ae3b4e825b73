// Ordering pass of a plain launch with staged output (scan_kernel.cuh, STAGED).
//
// Method (arXiv 1801.03644, Sec. 3.1): the scan's partitions produce partial results
// that are concatenated in partition order, so that the answer lists object ids in
// ascending order. Here a partition is a row tile of one query; the scan wrote each
// tile's ids (ascending within the tile) to a run of a staging buffer in whatever order
// the tiles finished, and recorded per tile rec[t] = staging position << 13 | id count.
// Because the tiles of a launch are numbered query-major and ascending in rows (a
// windowed launch's tiles follow its windows, which run in query and row order), the
// answer is the concatenation of the tiles' runs in tile order:
//   dst(t) = base + sum of the counts of tiles 0 .. t-1,
//   offsets[orig(q) + 1] = dst(last tile of q) + its count  (the CSR end of query q).
// A tile whose run did not fit the staging buffer (the scan writes no position past its
// end) is recomputed in place by one warp of the ordering kernel: the same predicates
// over the tile's rows, in row order. So the answer never depends on the staging size,
// and on a short answer buffer every id below its capacity is still written.
// Three kernels, all HBM-bound on the ids they move:
//   mdrq_concat_count_kernel  one block per segment of kCatSeg tiles: its id count;
//   mdrq_concat_scan_kernel   one block: exclusive prefix over the segments;
//   mdrq_concat_kernel        one block per segment: the prefix of each tile in it, the
//                             CSR ends of the queries that end in it, and the copy of
//                             every tile's run from the staging buffer into place.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "scan_kernel.cuh"
#include "table.h"

namespace mdrq {

constexpr int kCatThreads = 256;
constexpr int kCatPerThread = 8;
constexpr int kCatSeg = kCatThreads * kCatPerThread;  // 2048 tiles per segment
constexpr unsigned long long kRecCountMask = (1ull << kRecCountBits) - 1;
constexpr uint32_t kSmallRun = 8;  // runs this short are copied by one lane

__device__ __forceinline__ uint64_t umin64(uint64_t a, uint64_t b) { return a < b ? a : b; }
__device__ __forceinline__ uint64_t umax64(uint64_t a, uint64_t b) { return a > b ? a : b; }

// sum over the block (every thread gets it)
__device__ __forceinline__ unsigned long long block_sum(unsigned long long v, unsigned long long *s_w)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0)
        s_w[warp] = v;
    __syncthreads();
    unsigned long long tot = 0;
#pragma unroll
    for (int w = 0; w < kCatThreads / 32; ++w)
        tot += s_w[w];
    __syncthreads();
    return tot;
}

// exclusive prefix over the block of v (thread order); *total <- the block's sum
__device__ __forceinline__ unsigned long long block_excl(unsigned long long v, unsigned long long *s_w,
                                                         unsigned long long *total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long x = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o)
            incl += x;
    }
    if (lane == 31)
        s_w[warp] = incl;
    __syncthreads();
    unsigned long long before = 0, tot = 0;
#pragma unroll
    for (int w = 0; w < kCatThreads / 32; ++w) {
        const unsigned long long x = s_w[w];
        before += w < warp ? x : 0ull;
        tot += x;
    }
    __syncthreads();
    *total = tot;
    return before + incl - v;
}

// ntiles_dev: the launch's tile count on the device (windowed launches), else null
__global__ void __launch_bounds__(kCatThreads) mdrq_concat_count_kernel(const unsigned long long *rec, uint64_t ntiles,
                                                                        const unsigned long long *ntiles_dev,
                                                                        unsigned long long *seg_sum)
{
    __shared__ unsigned long long s_w[kCatThreads / 32];
    if (ntiles_dev)
        ntiles = umin64(ntiles, *ntiles_dev);
    const uint64_t s0 = (uint64_t)blockIdx.x * kCatSeg;
    unsigned long long c = 0;
#pragma unroll
    for (int k = 0; k < kCatPerThread; ++k) {
        const uint64_t t = s0 + (uint64_t)k * kCatThreads + threadIdx.x;
        if (t < ntiles)
            c += rec[t] & kRecCountMask;
    }
    const unsigned long long tot = block_sum(c, s_w);
    if (threadIdx.x == 0)
        seg_sum[blockIdx.x] = tot;
}

// seg[0 .. nseg) <- exclusive prefix of seg[0 .. nseg), seg[nseg] <- the total (one block)
__global__ void __launch_bounds__(kCatThreads) mdrq_concat_scan_kernel(unsigned long long *seg, uint64_t nseg)
{
    __shared__ unsigned long long s_w[kCatThreads / 32];
    unsigned long long carry = 0;
    for (uint64_t i0 = 0; i0 < nseg; i0 += kCatThreads) {
        const uint64_t i = i0 + threadIdx.x;
        const unsigned long long v = i < nseg ? seg[i] : 0ull;
        unsigned long long tot;
        const unsigned long long ex = block_excl(v, s_w, &tot);
        if (i < nseg)
            seg[i] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0)
        seg[nseg] = carry;
}

struct ConcatParams {
    const unsigned long long *rec;       // per tile: staging position << 13 | id count
    uint64_t ntiles;                     // tiles (windowed: an upper bound)
    const unsigned long long *ntiles_dev;  // windowed: the tile count (device), else null
    const uint32_t *tile_map;            // windowed: the window of every tile, else null
    const DevWindow *windows;            // windowed: the launch's windows
    const unsigned long long *seg_base;  // exclusive prefix of the segments' id counts
    uint32_t tiles_per_query;
    uint32_t tile_rows;
    uint64_t n;                          // table rows
    const DevQuery *queries;             // the launch's queries
    const DevPred *preds;
    const unsigned long long *base_in;   // where the launch's output starts in ids (or null)
    unsigned long long *offsets;         // offsets[orig + 1] <- CSR end of query orig
    const uint32_t *stage;               // staging buffer, stage_cap ids (runs past it unwritten)
    uint64_t stage_cap;
    uint32_t *ids;                       // the answer, capacity ids
    uint64_t capacity;
};

// lo <= x <= hi in the column's type (the scan's comparison, Sec. 2.1)
__device__ __forceinline__ bool pred_holds(uint32_t x, const DevPred &pr)
{
    if (pr.type == kTypeF32) {
        const float v = __uint_as_float(x);
        return __uint_as_float(pr.lo) <= v && v <= __uint_as_float(pr.hi);
    }
    const int v = (int)x;
    return (int)pr.lo <= v && v <= (int)pr.hi;
}

// Where tile t lies: its query (an index into cp.queries), whether it is the query's
// last tile, and the rows [*r0, *r1) it covers.
struct TileSpot {
    uint64_t q;
    bool last;
    uint64_t r0, r1;
};

__device__ __forceinline__ TileSpot tile_spot(const ConcatParams &cp, uint64_t t)
{
    TileSpot ts;
    if (cp.tile_map) {
        const DevWindow w = cp.windows[cp.tile_map[t]];
        const uint64_t rt = t - w.tile_start;
        const uint64_t a = w.row_begin + rt * cp.tile_rows;
        ts.q = w.query;
        ts.last = w.last && rt == w.tiles - 1;
        ts.r0 = umax64(a, w.row_first);
        ts.r1 = umin64(a + cp.tile_rows, w.row_end);
    } else {
        ts.q = t / cp.tiles_per_query;
        const uint64_t rt = t - ts.q * cp.tiles_per_query;
        ts.last = rt == cp.tiles_per_query - 1;
        ts.r0 = rt * cp.tile_rows;
        ts.r1 = umin64(ts.r0 + cp.tile_rows, cp.n);
    }
    return ts;
}

// One warp writes the ids of one tile from dst on, recomputing them: 32 rows per step,
// each row tested against every predicate of the tile's query.
__device__ void rescan_tile(const ConcatParams &cp, const TileSpot &ts, unsigned long long dst, int lane)
{
    const DevQuery dq = cp.queries[ts.q];
    const uint64_t row_end = ts.r1;
    for (uint64_t r0 = ts.r0; r0 < row_end; r0 += 32) {
        const uint64_t row = r0 + lane;
        bool ok = row < row_end;
        for (uint32_t i = 0; i < dq.npred && __any_sync(0xffffffffu, ok); ++i) {
            const DevPred pr = cp.preds[dq.first + i];
            if (ok)
                ok = pred_holds(ld_stream_u32((const uint32_t *)pr.col + row), pr);
        }
        const uint32_t b = __ballot_sync(0xffffffffu, ok);
        const unsigned long long at = dst + __popc(b & ((1u << lane) - 1u));
        if (ok && at < cp.capacity)
            cp.ids[at] = (uint32_t)row;
        dst += __popc(b);
    }
}

// One block per segment of kCatSeg tiles: positions, CSR ends and the copy into place.
__global__ void __launch_bounds__(kCatThreads) mdrq_concat_kernel(const __grid_constant__ ConcatParams cp)
{
    const unsigned long long *__restrict__ rec = cp.rec;
    const uint64_t ntiles = cp.ntiles_dev ? umin64(cp.ntiles, *cp.ntiles_dev) : cp.ntiles;
    const uint32_t tiles_per_query = cp.tiles_per_query;
    if ((uint64_t)blockIdx.x * kCatSeg >= ntiles)
        return;  // (windowed launches: the grid covers the upper bound)
    const uint32_t *__restrict__ stage = cp.stage;
    const uint64_t stage_cap = cp.stage_cap;
    uint32_t *__restrict__ ids = cp.ids;
    const uint64_t capacity = cp.capacity;
    __shared__ unsigned long long s_rec[kCatSeg];
    __shared__ uint32_t s_rel[kCatSeg];  // a tile's first id relative to the segment's (< 2^32)
    __shared__ unsigned long long s_w[kCatThreads / 32];
    const uint64_t s0 = (uint64_t)blockIdx.x * kCatSeg;
    const uint64_t left = ntiles - s0;
    const uint32_t nt = left < (uint64_t)kCatSeg ? (uint32_t)left : (uint32_t)kCatSeg;
    for (uint32_t i = threadIdx.x; i < (uint32_t)kCatSeg; i += kCatThreads)
        s_rec[i] = i < nt ? rec[s0 + i] : 0ull;
    __syncthreads();

    // this thread's tiles j0 .. j0 + kCatPerThread - 1 (consecutive)
    const uint32_t j0 = threadIdx.x * kCatPerThread;
    uint32_t c[kCatPerThread];
    uint32_t mine = 0;
#pragma unroll
    for (int k = 0; k < kCatPerThread; ++k) {
        c[k] = (uint32_t)(s_rec[j0 + k] & kRecCountMask);
        mine += c[k];
    }
    unsigned long long seg_total;
    uint32_t r = (uint32_t)block_excl(mine, s_w, &seg_total);
    const unsigned long long base = (cp.base_in ? *cp.base_in : 0ull) + cp.seg_base[blockIdx.x];
    if (j0 < nt && !cp.tile_map) {
        const uint64_t t0 = s0 + j0;
        uint64_t q = t0 / tiles_per_query;
        uint32_t rt = (uint32_t)(t0 - q * tiles_per_query);
#pragma unroll
        for (int k = 0; k < kCatPerThread; ++k) {
            s_rel[j0 + k] = r;
            if (j0 + k < nt && rt == tiles_per_query - 1)
                cp.offsets[cp.queries[q].orig + 1] = base + r + c[k];  // query q ends with this tile
            r += c[k];
            if (++rt == tiles_per_query) {
                rt = 0;
                ++q;
            }
        }
    } else if (j0 < nt) {
#pragma unroll
        for (int k = 0; k < kCatPerThread; ++k) {
            s_rel[j0 + k] = r;
            if (j0 + k < nt) {
                const TileSpot ts = tile_spot(cp, s0 + j0 + k);
                if (ts.last)
                    cp.offsets[cp.queries[ts.q].orig + 1] = base + r + c[k];
            }
            r += c[k];
        }
    }
    __syncthreads();

    // copy: warp w takes groups of 32 tiles, lane i tile 32g + i; short runs are copied
    // by their own lane, longer ones by the whole warp, one after another
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (uint32_t g = warp; g * 32 < nt; g += kCatThreads / 32) {
        const uint32_t j = g * 32 + lane;
        const unsigned long long rc = j < nt ? s_rec[j] : 0ull;
        const uint32_t cnt = (uint32_t)(rc & kRecCountMask);
        const uint64_t pos = rc >> kRecCountBits;
        const unsigned long long dst = base + s_rel[j];
        // runs start on 16-byte boundaries and take a multiple of 4 ids; one that did not
        // fit the staging buffer whole is recomputed (rare)
        const bool staged = pos + ((cnt + 3u) & ~3u) <= stage_cap;
        const bool lost = cnt > 0 && !staged && dst < capacity;
        uint32_t lost_mask = __ballot_sync(0xffffffffu, lost);
        while (lost_mask) {
            const int l = __ffs(lost_mask) - 1;
            lost_mask &= lost_mask - 1;
            rescan_tile(cp, tile_spot(cp, s0 + g * 32 + l), __shfl_sync(0xffffffffu, dst, l), lane);
        }
        if (cnt > 0 && cnt <= kSmallRun && staged) {
            // one or two 16-byte loads
            const uint4 a = ld_stream_v4(stage + pos);
            const uint4 b = cnt > 4 ? ld_stream_v4(stage + pos + 4) : make_uint4(0, 0, 0, 0);
            const uint32_t v[kSmallRun] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
#pragma unroll
            for (uint32_t i = 0; i < kSmallRun; ++i)
                if (i < cnt && dst + i < capacity)
                    ids[dst + i] = v[i];
        }
        uint32_t big = __ballot_sync(0xffffffffu, cnt > kSmallRun && staged);
        while (big) {
            const int l = __ffs(big) - 1;
            big &= big - 1;
            const uint32_t bc = __shfl_sync(0xffffffffu, cnt, l);
            const uint64_t bp = __shfl_sync(0xffffffffu, pos, l);
            const unsigned long long bd = __shfl_sync(0xffffffffu, dst, l);
            // lane l: ids l, l + 32, ... of every 512: each load and each store instruction
            // covers 128 contiguous bytes (stores that cross the CPU-GPU link to a pinned
            // host buffer stay whole), 16 loads in flight per lane
            for (uint32_t i = lane; i < bc; i += 512) {
                uint32_t v[16];
#pragma unroll
                for (uint32_t u = 0; u < 16; ++u)
                    if (i + 32 * u < bc)
                        v[u] = ld_stream_u32(stage + bp + i + 32 * u);
#pragma unroll
                for (uint32_t u = 0; u < 16; ++u)
                    if (i + 32 * u < bc && bd + i + 32 * u < capacity)
                        ids[bd + i + 32 * u] = v[u];
            }
        }
    }
}

int concat_staged(mdrq_table *t, uint64_t ntiles, const unsigned long long *ntiles_dev, uint32_t tiles_per_query,
                  uint32_t tile_rows, const DevQuery *queries, const uint32_t *tile_map, const DevWindow *windows,
                  const unsigned long long *base_in, uint32_t *ids, uint64_t capacity, cudaStream_t s)
{
    const uint64_t nseg = (ntiles + kCatSeg - 1) / kCatSeg;
    if (nseg == 0)
        return MDRQ_OK;
    const int st = grow_device(reinterpret_cast<void **>(&t->cat_seg), &t->cat_seg_cap, (nseg + 1) * 8);
    if (st != MDRQ_OK)
        return st;
    mdrq_concat_count_kernel<<<(unsigned)nseg, kCatThreads, 0, s>>>(t->cat_rec, ntiles, ntiles_dev, t->cat_seg);
    mdrq_concat_scan_kernel<<<1, kCatThreads, 0, s>>>(t->cat_seg, nseg);
    ConcatParams cp;
    cp.rec = t->cat_rec;
    cp.ntiles = ntiles;
    cp.ntiles_dev = ntiles_dev;
    cp.tile_map = tile_map;
    cp.windows = windows;
    cp.seg_base = t->cat_seg;
    cp.tiles_per_query = tiles_per_query;
    cp.tile_rows = tile_rows;
    cp.n = t->n;
    cp.queries = queries;
    cp.preds = t->dp_dev;
    cp.base_in = base_in;
    cp.offsets = t->offsets_dev;
    cp.stage = t->cat_ids;
    cp.stage_cap = t->cat_ids_cap / 4;
    cp.ids = ids;
    cp.capacity = capacity;
    mdrq_concat_kernel<<<(unsigned)nseg, kCatThreads, 0, s>>>(cp);
    MDRQ_TRY_STATUS(cudaGetLastError());
    return MDRQ_OK;
}

void concat_free(mdrq_table *t)
{
    cudaFree(t->cat_ids);
    cudaFree(t->cat_rec);
    cudaFree(t->cat_seg);
    t->cat_ids = nullptr;
    t->cat_rec = nullptr;
    t->cat_seg = nullptr;
    t->cat_ids_cap = t->cat_rec_cap = t->cat_seg_cap = 0;
}

}  // namespace mdrq
