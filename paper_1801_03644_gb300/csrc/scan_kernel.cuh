// Fused filter + ordered compaction scan for one multidimensional range query.
//
// Method (arXiv 1801.03644): an object qualifies iff lo_j <= x_j <= hi_j on every
// constrained dimension (Sec. 2.1); the scan visits every object (Sec. 2.2.4), over a
// column-wise layout so that only constrained columns are read (Sec. 3.2, Sec. 5.5);
// per-dimension results are ANDed into a bitmask (Sec. 3.2) and the ids of matching
// objects are produced in index order, which the paper gets by concatenating the
// partial results of its partitions (Sec. 3.1).
//
// GB300 design:
//  * A persistent grid claims row tiles in increasing order from a global ticket.
//    Each warp owns U*128 consecutive rows of a tile; lane l reads rows
//    4l..4l+3 of every 128-row group with one 128-bit load per column
//    (512 contiguous bytes per warp instruction).
//  * The per-row mask of U*4 bits lives in a register. Predicates are applied one
//    column at a time; a lane whose rows have all failed issues no load for the
//    remaining columns, so the memory system never fetches a 32-byte sector whose
//    8 rows are already rejected (the early break of Sec. 2.2.4 at sector
//    granularity), and a warp whose rows have all failed stops reading columns.
//  * Matches are ranked with a packed warp scan and staged in shared memory in row
//    order; the tile's offset in the answer comes from a single-pass decoupled
//    look-back over per-tile states (aggregate / inclusive prefix), so the answer is
//    written once, coalesced and ascending, without a second pass over the columns.
//  * The look-back and the write-out run in a separate output warp that drains
//    double-buffered stages, so the eight filter warps never stall on other tiles.
//  * Every wait (on another tile's state or on a stage) is bounded; on expiry the
//    kernel records an error bit and finishes, never traps.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace mdrq {

constexpr int kBlock = 256;
constexpr int kWarps = kBlock / 32;
constexpr int kMaxPreds = 128;

constexpr uint32_t kTypeF32 = 0;
constexpr uint32_t kTypeI32 = 1;

// tile state word: [63:34] epoch, [33:32] flag, [31:0] value
constexpr uint32_t kFlagAggregate = 1;
constexpr uint32_t kFlagPrefix = 2;
constexpr uint32_t kEpochLimit = (1u << 30) - 1;

constexpr int kErrLookbackTimeout = 1;
constexpr uint32_t kMaxPolls = 1u << 20;  // x <= 1 us backoff: bounded by about 1 s

struct ScanPred {
    const void *col;  // device column (16-byte aligned)
    uint32_t type;    // kTypeF32 / kTypeI32
    uint32_t lo;      // bound bits, read as the column's type
    uint32_t hi;
    uint32_t pad;
};

struct ScanParams {
    ScanPred pred[kMaxPreds];
    uint32_t npred;
    uint32_t n_tiles;
    uint64_t n;
    unsigned long long *tile_state;  // n_tiles words
    unsigned long long *ticket;      // monotone claim counter
    unsigned long long ticket_base;  // counter value when this launch starts
    uint32_t epoch;                  // tag of this launch in tile_state
    uint32_t pad0;
    uint32_t *ids;                   // answer buffer
    uint64_t capacity;               // slots in ids
    const unsigned long long *base_in;  // offset of this answer in ids (NULL: 0)
    unsigned long long *count_out;   // receives base + answer length
    int *error;                      // error bits (kErr*)
};

__device__ __forceinline__ uint4 ld_stream_v4(const void *p)
{
    uint4 v;
    asm("ld.global.nc.L1::no_allocate.v4.u32 {%0, %1, %2, %3}, [%4];"
        : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
        : "l"(p));
    return v;
}

__device__ __forceinline__ uint32_t ld_stream_u32(const void *p)
{
    uint32_t v;
    asm("ld.global.nc.L1::no_allocate.u32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_relaxed_u64(unsigned long long *p, unsigned long long v)
{
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ unsigned long long pack_state(uint32_t epoch, uint32_t flag, uint32_t v)
{
    return ((unsigned long long)epoch << 34) | ((unsigned long long)flag << 32) | v;
}

// 4-bit mask of the rows of one 16-byte chunk that lie in [lo, hi]
__device__ __forceinline__ uint32_t in_range4(uint4 v, uint32_t type, uint32_t lo, uint32_t hi)
{
    uint32_t r;
    if (type == kTypeF32) {
        const float l = __uint_as_float(lo), h = __uint_as_float(hi);
        const float a = __uint_as_float(v.x), b = __uint_as_float(v.y);
        const float c = __uint_as_float(v.z), d = __uint_as_float(v.w);
        r = (uint32_t)((l <= a) & (a <= h)) | ((uint32_t)((l <= b) & (b <= h)) << 1) |
            ((uint32_t)((l <= c) & (c <= h)) << 2) | ((uint32_t)((l <= d) & (d <= h)) << 3);
    } else {
        const int l = (int)lo, h = (int)hi;
        const int a = (int)v.x, b = (int)v.y, c = (int)v.z, d = (int)v.w;
        r = (uint32_t)((l <= a) & (a <= h)) | ((uint32_t)((l <= b) & (b <= h)) << 1) |
            ((uint32_t)((l <= c) & (c <= h)) << 2) | ((uint32_t)((l <= d) & (d <= h)) << 3);
    }
    return r;
}

// ---------------------------------------------------------------- mbarrier helpers

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(unsigned long long *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(unsigned long long *bar)
{
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

constexpr unsigned long long kStageWaitNs = 4000000000ull;  // 4 s: longer than a look-back

// Wait for the phase of parity `parity` of `bar` to complete; false after kStageWaitNs.
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, uint32_t parity)
{
    if (mbar_try_wait(bar, parity))
        return true;
    const unsigned long long t0 = global_ns();
    while (!mbar_try_wait(bar, parity))
        if (global_ns() - t0 > kStageWaitNs)
            return false;
    return true;
}

__device__ __forceinline__ void named_bar_sync(uint32_t id, uint32_t count)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// Exclusive prefix of all tiles before `tile` (decoupled look-back), run by one full
// warp once the tile's own aggregate is published; publishes the inclusive prefix.
__device__ __forceinline__ uint32_t tile_lookback(const ScanParams &p, unsigned long long tile,
                                                  uint32_t total, int lane)
{
    unsigned long long *st = p.tile_state;
    unsigned long long excl = 0;
    long long idx = (long long)tile - 1;  // nearest predecessor
    uint32_t polls = 0, backoff = 32;
    for (;;) {
        const long long my = idx - lane;
        uint32_t flag = kFlagPrefix, val = 0;  // before tile 0: an inclusive prefix of 0
        if (my >= 0) {
            const unsigned long long w = ld_relaxed_u64(&st[my]);
            flag = (uint32_t)(w >> 34) == p.epoch ? (uint32_t)(w >> 32) & 3u : 0u;
            val = (uint32_t)w;
        }
        uint32_t pmask = __ballot_sync(0xffffffffu, flag == kFlagPrefix);
        int stop = pmask ? __ffs(pmask) - 1 : 31;  // nearest lane holding a prefix
        // only the states up to the nearest inclusive prefix are needed
        if (__any_sync(0xffffffffu, lane <= stop && flag == 0)) {
            if (++polls < kMaxPolls) {
                __nanosleep(backoff);
                backoff = backoff < 1024 ? backoff * 2 : 1024;
                continue;
            }
            // gave up: record it and treat the missing states as empty prefixes
            if (lane == 0)
                atomicOr(p.error, kErrLookbackTimeout);
            if (flag == 0) {
                flag = kFlagPrefix;
                val = 0;
            }
            pmask = __ballot_sync(0xffffffffu, flag == kFlagPrefix);
            stop = __ffs(pmask) - 1;
        }
        unsigned long long v = lane <= stop ? val : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
            v += __shfl_xor_sync(0xffffffffu, v, o);
        excl += v;
        if (pmask)
            break;
        idx -= 32;
    }
    if (lane == 0)
        st_relaxed_u64(&st[tile], pack_state(p.epoch, kFlagPrefix, (uint32_t)(excl + total)));
    return (uint32_t)excl;
}

constexpr int kStages = 2;                       // staged tiles per CTA
constexpr int kScanThreads = kBlock + 32;        // 8 filter warps + 1 output warp
constexpr unsigned long long kStopTile = ~0ull;  // "no more tiles" marker for the output warp
constexpr uint32_t kBarFilter = 1;               // named barrier of the 8 filter warps

// Warp-specialised scan. Warps 0-7 ("filter warps") claim tiles, evaluate the
// predicates, rank the matches and stage their row offsets in one of kStages shared
// buffers, publish the tile's aggregate, and move on. Warp 8 (the "output warp")
// takes staged tiles in order, resolves each tile's offset by look-back, publishes the
// inclusive prefix and writes the ids out, so no filter warp ever waits on another
// tile. Hand-off uses mbarriers: full[b] (256 filter-thread arrivals) and empty[b]
// (32 output-lane arrivals); every wait is bounded.
template <int U>
__device__ __forceinline__ void scan_cta(const ScanParams &p)
{
    static_assert(U >= 1 && U <= 4, "8-bit packed counts hold at most 4 groups");
    constexpr int kWarpRows = U * 128;
    constexpr int kTileRows = kWarps * kWarpRows;
    constexpr uint32_t kFullMask = (1u << (U * 4)) - 1u;
    static_assert(kTileRows <= 65536, "row offsets are staged as 16-bit values");

    __shared__ uint16_t s_stage[kStages][kTileRows];
    __shared__ uint32_t s_warp_total[kStages][kWarps];
    __shared__ unsigned long long s_tile[kStages];
    __shared__ uint32_t s_total[kStages];
    __shared__ unsigned long long s_ticket[2];
    __shared__ unsigned long long s_full[kStages], s_empty[kStages];
    __shared__ int s_abort;

    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;

    if (threadIdx.x == 0) {
        for (int b = 0; b < kStages; ++b) {
            mbar_init(&s_full[b], kBlock);
            mbar_init(&s_empty[b], 32);
        }
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    if (warp == kWarps) {
        // ------------------------------------------------------------ output warp
        const unsigned long long base = p.base_in ? *p.base_in : 0ull;
        uint32_t full_phase = 0;  // bit b: parity to wait for on s_full[b]
        for (uint32_t it = 0;; ++it) {
            const int b = it % kStages;
            // every lane waits; the warp leaves together if any lane gave up
            if (!__all_sync(0xffffffffu, mbar_wait(&s_full[b], (full_phase >> b) & 1u))) {
                if (lane == 0)
                    atomicOr(p.error, kErrLookbackTimeout);
                break;
            }
            full_phase ^= 1u << b;
            const unsigned long long tile = s_tile[b];
            if (tile == kStopTile)
                break;
            const uint32_t total = s_total[b];
            const uint32_t prefix = tile == 0 ? 0u : tile_lookback(p, tile, total, lane);
            if (lane == 0 && tile == p.n_tiles - 1)
                *p.count_out = base + prefix + total;
            const unsigned long long out0 = base + prefix;
            const uint32_t row0 = (uint32_t)(tile * (unsigned long long)kTileRows);
            for (uint32_t r = lane; r < total; r += 32) {
                const unsigned long long pos = out0 + r;
                if (pos < p.capacity)
                    p.ids[pos] = row0 + s_stage[b][r];
            }
            __syncwarp();
            mbar_arrive(&s_empty[b]);
        }
        return;
    }

    // ---------------------------------------------------------------- filter warps
    uint32_t empty_phase = (1u << kStages) - 1u;  // bit b: parity for s_empty[b]; buffers start empty
    if (threadIdx.x == 0)
        s_ticket[0] = atomicAdd(p.ticket, 1ull) - p.ticket_base;
    named_bar_sync(kBarFilter, kBlock);
    unsigned long long tile = s_ticket[0];
    int slot = 0;
    uint32_t it = 0;

    while (tile < p.n_tiles) {
        const int b = it % kStages;
        if (threadIdx.x == 0) {
            if (!mbar_wait(&s_empty[b], (empty_phase >> b) & 1u)) {
                atomicOr(p.error, kErrLookbackTimeout);
                s_abort = 1;
            }
            // claim the next tile now so the round trip overlaps this tile's loads
            s_ticket[slot ^ 1] = atomicAdd(p.ticket, 1ull) - p.ticket_base;
        }
        named_bar_sync(kBarFilter, kBlock);
        if (s_abort)
            break;
        empty_phase ^= 1u << b;

        const uint64_t row0 = tile * (uint64_t)kTileRows + (uint64_t)warp * kWarpRows;
        const bool full = row0 + kWarpRows <= p.n;

        // bit 4u+e of m: row row0 + 128u + 4*lane + e still qualifies
        uint32_t m = 0;
        if (full) {
            m = kFullMask;
        } else {
#pragma unroll
            for (int u = 0; u < U; ++u)
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if (row0 + 128u * u + 4u * lane + e < p.n)
                        m |= 1u << (4 * u + e);
        }

        for (uint32_t i = 0; i < p.npred; ++i) {
            if (!__any_sync(0xffffffffu, m))
                break;  // every row of this warp's chunk failed: read no more columns
            const ScanPred &pr = p.pred[i];
            const uint32_t *col = (const uint32_t *)pr.col + row0 + 4 * lane;
            uint4 v[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                v[u] = make_uint4(0, 0, 0, 0);
                const uint32_t mu = (m >> (4 * u)) & 0xfu;
                if (mu) {
                    if (full || mu == 0xfu) {
                        v[u] = ld_stream_v4(col + 128 * u);
                    } else {
                        // ragged end of the table: only rows < n may be read
                        if (mu & 1u) v[u].x = ld_stream_u32(col + 128 * u + 0);
                        if (mu & 2u) v[u].y = ld_stream_u32(col + 128 * u + 1);
                        if (mu & 4u) v[u].z = ld_stream_u32(col + 128 * u + 2);
                        if (mu & 8u) v[u].w = ld_stream_u32(col + 128 * u + 3);
                    }
                }
            }
            uint32_t keep = 0;
#pragma unroll
            for (int u = 0; u < U; ++u)
                keep |= in_range4(v[u], pr.type, pr.lo, pr.hi) << (4 * u);
            m &= keep;
        }

        // rank the matches of this warp: row order is (u, lane, e)
        uint32_t packed = 0;  // 8-bit count per u
#pragma unroll
        for (int u = 0; u < U; ++u)
            packed |= (uint32_t)__popc((m >> (4 * u)) & 0xfu) << (8 * u);
        uint32_t incl = packed;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o)
                incl += t;
        }
        const uint32_t excl_lane = incl - packed;
        const uint32_t warp_packed = __shfl_sync(0xffffffffu, incl, 31);
        uint32_t warp_total = 0;
#pragma unroll
        for (int u = 0; u < U; ++u)
            warp_total += (warp_packed >> (8 * u)) & 0xffu;
        if (lane == 0)
            s_warp_total[b][warp] = warp_total;
        named_bar_sync(kBarFilter, kBlock);

        uint32_t tile_total = 0, warp_off = 0;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) {
            const uint32_t t = s_warp_total[b][w];
            warp_off += w < warp ? t : 0u;
            tile_total += t;
        }

        // stage the row offsets (within the tile) of this warp's matches in row order
        uint32_t ubase = warp_off;
        const uint32_t off0 = (uint32_t)warp * kWarpRows + 4u * lane;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            uint32_t mu = (m >> (4 * u)) & 0xfu;
            uint32_t r = ubase + ((excl_lane >> (8 * u)) & 0xffu);
            while (mu) {
                const int e = __ffs(mu) - 1;
                s_stage[b][r++] = (uint16_t)(off0 + 128u * u + e);
                mu &= mu - 1;
            }
            ubase += (warp_packed >> (8 * u)) & 0xffu;
        }

        if (threadIdx.x == 0) {
            s_tile[b] = tile;
            s_total[b] = tile_total;
            // publish the aggregate at once (tile 0: its inclusive prefix)
            st_relaxed_u64(&p.tile_state[tile],
                           pack_state(p.epoch, tile == 0 ? kFlagPrefix : kFlagAggregate, tile_total));
        }
        mbar_arrive(&s_full[b]);
        tile = s_ticket[slot ^ 1];
        slot ^= 1;
        ++it;
    }

    // tell the output warp that no tile follows
    const int b = it % kStages;
    if (threadIdx.x == 0) {
        if (!s_abort)
            mbar_wait(&s_empty[b], (empty_phase >> b) & 1u);
        s_tile[b] = kStopTile;
    }
    mbar_arrive(&s_full[b]);
}

template <int U>
__global__ void __launch_bounds__(kScanThreads, 7) mdrq_scan_kernel(const __grid_constant__ ScanParams p)
{
    scan_cta<U>(p);
}

}  // namespace mdrq
