// Fused filter + ordered compaction scan: a batch of multidimensional range queries
// over one column-wise table, in a single persistent launch.
//
// Method (arXiv 1801.03644): an object qualifies iff lo_j <= x_j <= hi_j on every
// constrained dimension (Sec. 2.1); the scan visits every object (Sec. 2.2.4), over a
// column-wise layout so that only constrained columns are read (Sec. 3.2, Sec. 5.5);
// per-dimension results are ANDed into a bitmask (Sec. 3.2) and the ids of matching
// objects are produced in index order, which the paper gets by concatenating the
// partial results of its partitions (Sec. 3.1).
//
// GB300 design:
//  * Work unit: a row tile of one query. The tiles of all queries of a launch form one
//    sequence (query-major); a persistent grid claims them in increasing order from a
//    global ticket. Each query is still scanned on its own (no column load is shared
//    between queries): one launch merely removes the per-query launch ramp and tail.
//  * Each filter warp owns U*128 consecutive rows of a tile; lane l reads rows
//    4l..4l+3 of every 128-row group with one 128-bit load per column (512 contiguous
//    bytes per warp instruction).
//  * The per-row mask of U*4 bits lives in a register. Predicates are applied one
//    column at a time; a lane whose rows have all failed issues no load for the
//    remaining columns, so the memory system never fetches a 32-byte sector whose 8
//    rows are already rejected (the early break of Sec. 2.2.4 at sector granularity),
//    and a warp whose rows have all failed stops reading columns.
//  * Matches are ranked with a packed warp scan and staged (16-bit row offsets) in
//    shared memory, each warp in its own segment. The offset of a tile in the launch's
//    output comes from a single-pass decoupled look-back over per-tile states
//    (aggregate / inclusive prefix) kept in a ring; because the sequence runs over all
//    queries, the inclusive prefix at a query's last tile is that query's end offset in
//    the CSR answer, so the whole batch is written once, coalesced, ascending per query.
//  * Warp roles: eight filter warps per CTA claim tiles (one tile ahead), evaluate them
//    into kStages shared stages and publish each tile's aggregate (the last warp to
//    finish does it); one output warp drains the stages in order, resolves each tile's
//    offset by look-back and writes the ids. The filter warps never wait on another
//    tile or on each other.
//  * Staged output (STAGED, large launches): instead of the look-back, each tile
//    takes the next free run of a staging buffer with one atomic add and records where
//    its ids went and how many there are; a concatenation pass afterwards (concat.cu)
//    turns the tile counts into positions and copies every tile's ids into place. That
//    is the paper's concatenation of partition results (Sec. 3.1) with tiles as the
//    partitions: no tile waits on another, at the price of writing the ids twice.
//  * Every wait (on another tile's state or on a stage) is bounded; on expiry the
//    kernel records an error bit and finishes, never traps.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace mdrq {

constexpr int kBlock = 256;     // filter threads per CTA
constexpr int kWarps = kBlock / 32;
constexpr int kMaxPreds = 128;  // distinct constrained dimensions per query

constexpr uint32_t kTypeF32 = 0;
constexpr uint32_t kTypeI32 = 1;

// tile state word: [63:62] flag, [61:40] tag, [39:0] value (ids, relative to the launch)
constexpr uint32_t kFlagAggregate = 1;
constexpr uint32_t kFlagPrefix = 2;
constexpr uint32_t kTagLimit = (1u << 22) - 1;
constexpr unsigned long long kValueMask = (1ull << 40) - 1;  // a launch outputs < 2^40 ids

constexpr int kErrLookbackTimeout = 1;
constexpr int kErrStageTimeout = 2;
constexpr uint32_t kMaxPolls = 1u << 20;  // x <= 1 us backoff: bounded by about 1 s

constexpr uint32_t kZoneTileRows = 4096;  // zone maps: one (min, max) pair per 4096 rows

// One predicate of one query, as the kernel reads it.
struct DevPred {
    const void *col;    // device column (16-byte aligned)
    const uint2 *zone;  // the column's zone map (device), or null: entry i holds the
                        // bits of the minimum and maximum of rows [4096i, 4096i + 4096)
    uint32_t type;      // kTypeF32 / kTypeI32
    uint32_t lo;        // bound bits, read as the column's type
    uint32_t hi;
    uint32_t pad;
};

// One query of a launch: predicates preds[first .. first + npred), answer slot `orig`.
struct DevQuery {
    uint32_t first;
    uint32_t npred;
    uint32_t orig;
    uint32_t pad;
};

// Windowed launches: a run of rows [row_begin, row_end) (row_begin a multiple of 128) that
// query `query` of the launch scans, and its tiles [tile_start, tile_start + tiles). A
// query may have several windows, in ascending row order; the one flagged `last` has at
// least one tile (its last tile writes the query's CSR end), the others may have none.
struct DevWindow {
    unsigned long long row_begin;  // first row, rounded down to a multiple of 128
    unsigned long long row_first;  // first row (rows before it belong to no window here)
    unsigned long long row_end;
    unsigned long long tile_start;
    unsigned long long tiles;
    uint32_t query;
    uint32_t last;
};

struct ScanParams {
    const DevQuery *queries;         // nq queries (device)
    const DevPred *preds;            // their predicates (device)
    uint32_t nq;
    uint32_t tiles_per_query;        // row tiles of the table
    uint64_t n;                      // rows
    uint64_t total_tiles;            // nq * tiles_per_query
    unsigned long long *tile_state;  // ring of look-back states
    uint32_t ring_bits;              // ring size = 2^ring_bits
    uint32_t tag0;                   // tag of this launch's first ring lap
    unsigned long long *ticket;      // monotone claim counter
    unsigned long long ticket_base;  // counter value when this launch starts
    uint32_t *ids;                   // answer buffer (CSR over the queries)
    uint64_t capacity;               // slots in ids
    const unsigned long long *base_in;  // where this launch's output starts in ids
    unsigned long long *offsets;     // offsets[orig + 1] <- end of query orig's answer
    int *error;                      // error bits (kErr*)
    const DevWindow *windows;        // windowed launches: row runs and their tiles (device)
    const unsigned long long *nwindows_dev;  // windowed launches: number of windows (device)
    const unsigned long long *total_tiles_dev;  // windowed launches: tile count (device)
    const uint32_t *tile_map;        // windowed launches: the window of every tile (device)
    unsigned long long *bump;        // staged output: ids staged so far by this launch (device)
    unsigned long long *tile_rec;    // staged output: per tile, staging position << 13 | id count
};

constexpr int kRecCountBits = 13;  // a tile record's count field (a tile holds <= 4096 rows)

// Where tile t of a launch lies: its query, its first row, the end of the rows it may
// read, and whether it is the query's last tile.
struct TilePlace {
    uint32_t q;
    bool last;
    unsigned long long row0;
    unsigned long long row_first;  // rows in [row_first, row_end) belong to the tile's query
    unsigned long long row_end;
};

// WINDOWED = false: the query of tile t; true: the window of tile t (from the tile map
// the launch builds before the scan).
template <bool WINDOWED>
__device__ __forceinline__ uint32_t query_of_tile(const ScanParams &p, unsigned long long t)
{
    if (!WINDOWED)
        return (uint32_t)(t / p.tiles_per_query);
    return p.tile_map[t];
}

template <bool WINDOWED>
__device__ __forceinline__ TilePlace place_tile(const ScanParams &p, unsigned long long t, uint32_t q,
                                                uint32_t tile_rows)
{
    TilePlace tp;
    tp.q = q;
    if (WINDOWED) {
        const DevWindow w = p.windows[q];  // q is the window here
        const unsigned long long rt = t - w.tile_start;
        tp.q = w.query;
        tp.row0 = w.row_begin + rt * tile_rows;
        tp.row_first = w.row_first;
        tp.row_end = w.row_end;
        tp.last = w.last && rt == w.tiles - 1;
    } else {
        const unsigned long long rt = t - (unsigned long long)q * p.tiles_per_query;
        tp.row0 = rt * tile_rows;
        tp.row_first = 0;
        tp.row_end = p.n;
        tp.last = rt == p.tiles_per_query - 1;
    }
    return tp;
}

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

// ring slot and tag of tile t of the launch
__device__ __forceinline__ unsigned long long *state_slot(const ScanParams &p, unsigned long long t)
{
    return p.tile_state + (t & ((1ull << p.ring_bits) - 1));
}

__device__ __forceinline__ uint32_t state_tag(const ScanParams &p, unsigned long long t)
{
    return (p.tag0 + (uint32_t)(t >> p.ring_bits)) & kTagLimit;
}

__device__ __forceinline__ unsigned long long pack_state(uint32_t tag, uint32_t flag, unsigned long long v)
{
    return ((unsigned long long)flag << 62) | ((unsigned long long)tag << 40) | (v & kValueMask);
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

// lo <= x <= hi for one value read as the column's type (ordered compares): all ones if
// it holds, else zero, so that a single AND with a constant places the row's bit
template <bool F32>
__device__ __forceinline__ uint32_t in_range_ones(uint32_t x, uint32_t lo, uint32_t hi)
{
    uint32_t d;
    if (F32)
        asm("{\n\t.reg .pred p;\n\tsetp.ge.f32 p, %1, %2;\n\tset.le.and.u32.f32 %0, %1, %3, p;\n\t}"
            : "=r"(d)
            : "f"(__uint_as_float(x)), "f"(__uint_as_float(lo)), "f"(__uint_as_float(hi)));
    else
        asm("{\n\t.reg .pred p;\n\tsetp.ge.s32 p, %1, %2;\n\tset.le.and.u32.s32 %0, %1, %3, p;\n\t}"
            : "=r"(d)
            : "r"(x), "r"(lo), "r"(hi));
    return d;
}

// One predicate over a lane's U groups of 4 rows when every row of the warp lies in the
// table: a group whose rows have all failed issues no load. Returns the surviving mask.
template <int U, bool F32>
__device__ __forceinline__ uint32_t filter_full(const uint32_t *col, uint32_t m, uint32_t lo, uint32_t hi)
{
    uint4 v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
        v[u] = make_uint4(0, 0, 0, 0);
        if ((m >> (4 * u)) & 0xfu)
            v[u] = ld_stream_v4(col + 128 * u);
    }
    uint32_t keep = 0;
#pragma unroll
    for (int u = 0; u < U; ++u) {
        keep |= in_range_ones<F32>(v[u].x, lo, hi) & (1u << (4 * u));
        keep |= in_range_ones<F32>(v[u].y, lo, hi) & (2u << (4 * u));
        keep |= in_range_ones<F32>(v[u].z, lo, hi) & (4u << (4 * u));
        keep |= in_range_ones<F32>(v[u].w, lo, hi) & (8u << (4 * u));
    }
    return m & keep;
}

// The same at the ragged end of the table or of a window: only rows whose bit is set
// in m are read (they all lie inside the table).
template <int U>
__device__ __forceinline__ uint32_t filter_ragged(const uint32_t *col, uint32_t m, uint32_t type, uint32_t lo,
                                                  uint32_t hi)
{
    uint4 v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
        v[u] = make_uint4(0, 0, 0, 0);
        const uint32_t mu = (m >> (4 * u)) & 0xfu;
        if (mu == 0xfu) {
            v[u] = ld_stream_v4(col + 128 * u);
        } else if (mu) {
            if (mu & 1u) v[u].x = ld_stream_u32(col + 128 * u + 0);
            if (mu & 2u) v[u].y = ld_stream_u32(col + 128 * u + 1);
            if (mu & 4u) v[u].z = ld_stream_u32(col + 128 * u + 2);
            if (mu & 8u) v[u].w = ld_stream_u32(col + 128 * u + 3);
        }
    }
    uint32_t keep = 0;
#pragma unroll
    for (int u = 0; u < U; ++u)
        keep |= in_range4(v[u], type, lo, hi) << (4 * u);
    return m & keep;
}

// What a zone (the value range [min, max] of a row tile) says about [lo, hi]: 0 no row
// of it can qualify, 2 every row qualifies, 1 its rows must be read
__device__ __forceinline__ uint32_t zone_verdict(uint2 z, uint32_t type, uint32_t lo, uint32_t hi)
{
    bool none, all;
    if (type == kTypeF32) {
        const float l = __uint_as_float(lo), h = __uint_as_float(hi);
        const float a = __uint_as_float(z.x), b = __uint_as_float(z.y);
        none = b < l || a > h;
        all = l <= a && b <= h;
    } else {
        const int l = (int)lo, h = (int)hi, a = (int)z.x, b = (int)z.y;
        none = b < l || a > h;
        all = l <= a && b <= h;
    }
    return none ? 0u : (all ? 2u : 1u);
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

// Exclusive prefix of all tiles before tile `t` of the launch (decoupled look-back),
// run by one full warp once t's aggregate is published; publishes t's inclusive prefix.
__device__ __forceinline__ unsigned long long tile_lookback(const ScanParams &p, unsigned long long t,
                                                            uint32_t total, int lane)
{
    unsigned long long excl = 0;
    long long idx = (long long)t - 1;  // nearest predecessor
    uint32_t polls = 0, backoff = 32;
    for (;;) {
        const long long my = idx - lane;
        uint32_t flag = kFlagPrefix;  // before tile 0: an inclusive prefix of 0
        unsigned long long val = 0;
        if (my >= 0) {
            const unsigned long long w = ld_relaxed_u64(state_slot(p, (unsigned long long)my));
            const bool mine = (uint32_t)((w >> 40) & kTagLimit) == state_tag(p, (unsigned long long)my);
            flag = mine ? (uint32_t)(w >> 62) : 0u;
            val = w & kValueMask;
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
        st_relaxed_u64(state_slot(p, t), pack_state(state_tag(p, t), kFlagPrefix, excl + total));
    return excl;
}

constexpr int kStages = 3;                       // staged tiles per CTA
constexpr int kClaimSlots = kStages + 1;         // claimed-tile queue (see scan_cta)
constexpr int kScanThreads = kBlock + 32;        // 8 filter warps + 1 output warp
constexpr unsigned long long kStopTile = ~0ull;  // "no more tiles" marker

// The filter warps of a CTA run iterations 0, 1, 2, ... in lock-free step: iteration i
// fills stage i % kStages with the tile held in claim slot i % kClaimSlots. The first
// filter warp to start iteration i claims the tile of iteration i + 1, so a tile is
// claimed about one tile before it is processed and tiles are finished close to claim
// order, which keeps look-back waits short. Slot reuse is safe with kStages + 1 slots:
// a warp can run at most kStages iterations ahead of the output warp.
template <int U, bool WINDOWED = false, bool STAGED = false>
__device__ __forceinline__ void scan_cta(const ScanParams &p)
{
    static_assert(U >= 1 && U <= 4, "8-bit packed counts hold at most 4 groups");
    constexpr int kWarpRows = U * 128;
    constexpr int kTileRows = kWarps * kWarpRows;
    constexpr uint32_t kFullMask = (1u << (U * 4)) - 1u;
    static_assert(kTileRows <= 65536, "row offsets are staged as 16-bit values");
    static_assert(kTileRows < (1 << kRecCountBits), "a tile's id count fits its record");

    __shared__ uint16_t s_stage[kStages][kTileRows];  // warp w: [w*kWarpRows, ...)
    __shared__ uint32_t s_warp_total[kStages][kWarps];
    __shared__ unsigned long long s_stage_tile[kStages];  // tile held by the stage
    __shared__ uint32_t s_done[kStages];                  // filter warps finished with it
    __shared__ uint32_t s_first[kStages];                 // filter warps that started it
    __shared__ unsigned long long s_claim[kClaimSlots];   // claimed tile of an iteration
    __shared__ uint32_t s_claim_q[kClaimSlots];           // ... and its query
    __shared__ uint32_t s_stage_q[kStages];               // query of the stage's tile
    __shared__ unsigned long long s_ready[kStages], s_full[kStages], s_claimed[kClaimSlots];

    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;

    const unsigned long long total_tiles = WINDOWED ? *p.total_tiles_dev : p.total_tiles;
    auto claim = [&](int slot) {
        const unsigned long long t = atomicAdd(p.ticket, 1ull) - p.ticket_base;
        const bool real = t < total_tiles;
        s_claim[slot] = real ? t : kStopTile;
        s_claim_q[slot] = real ? query_of_tile<WINDOWED>(p, t) : 0u;
    };

    if (threadIdx.x == 0) {
        for (int b = 0; b < kStages; ++b) {
            mbar_init(&s_ready[b], 1);
            mbar_init(&s_full[b], kWarps);
            s_done[b] = 0;
            s_first[b] = 0;
        }
        for (int c = 0; c < kClaimSlots; ++c)
            mbar_init(&s_claimed[c], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        claim(0);  // the tile of iteration 0
        mbar_arrive(&s_claimed[0]);
    }
    __syncthreads();

    if (warp == kWarps) {
        // ------------------------------------------------------------ output warp
        const unsigned long long base = p.base_in ? *p.base_in : 0ull;
        uint32_t full_phase = 0;  // bit b: parity to wait for on s_full[b]
        for (uint32_t it = 0;; ++it) {
            const int b = it % kStages;
            if (!__all_sync(0xffffffffu, mbar_wait(&s_full[b], (full_phase >> b) & 1u))) {
                if (lane == 0)
                    atomicOr(p.error, kErrStageTimeout);
                break;
            }
            full_phase ^= 1u << b;
            const unsigned long long t = s_stage_tile[b];
            if (t == kStopTile)
                break;
            const TilePlace tp = place_tile<WINDOWED>(p, t, s_stage_q[b], kTileRows);
            // per-warp counts of the stage and their inclusive prefix
            const uint32_t wt = lane < kWarps ? s_warp_total[b][lane] : 0u;
            uint32_t wincl = wt;
#pragma unroll
            for (int o = 1; o < kWarps; o <<= 1) {
                const uint32_t x = __shfl_up_sync(0xffffffffu, wincl, o);
                if (lane >= o)
                    wincl += x;
            }
            const uint32_t total = __shfl_sync(0xffffffffu, wincl, kWarps - 1);
            unsigned long long excl;
            if (STAGED) {
                // the next free run of the staging buffer; the tile's place in the
                // answer is set afterwards from the counts of all tiles
                unsigned long long pos = 0;
                if (lane == 0) {
                    // runs start on 16-byte boundaries, for the ordering pass's loads
                    pos = atomicAdd(p.bump, (unsigned long long)((total + 3u) & ~3u));
                    p.tile_rec[t] = (pos << kRecCountBits) | total;
                }
                excl = __shfl_sync(0xffffffffu, pos, 0);
            } else {
                excl = t == 0 ? 0ull : tile_lookback(p, t, total, lane);
                if (lane == 0 && tp.last)
                    p.offsets[p.queries[tp.q].orig + 1] = base + excl + total;
            }
            const uint32_t row0 = (uint32_t)tp.row0;
#pragma unroll 1
            for (int w = 0; w < kWarps; ++w) {
                const uint32_t cnt = __shfl_sync(0xffffffffu, wt, w);
                const unsigned long long out0 = (STAGED ? 0ull : base) + excl + __shfl_sync(0xffffffffu, wincl - wt, w);
                const uint16_t *seg = &s_stage[b][w * kWarpRows];
                for (uint32_t r = lane; r < cnt; r += 32) {
                    const unsigned long long pos = out0 + r;
                    if (pos < p.capacity)
                        p.ids[pos] = row0 + seg[r];
                }
            }
            __syncwarp();
            if (lane == 0)
                mbar_arrive(&s_ready[b]);
        }
        return;
    }

    // ---------------------------------------------------------------- filter warps
    uint32_t ready_phase = (1u << kStages) - 1u;  // bit b: parity for s_ready[b]; stages start free
    for (uint32_t it = 0;; ++it) {
        const int b = it % kStages;
        const int c = it % kClaimSlots;
        const bool ok = mbar_wait(&s_ready[b], (ready_phase >> b) & 1u) &&
                        mbar_wait(&s_claimed[c], (it / kClaimSlots) & 1u);
        if (!__all_sync(0xffffffffu, ok)) {
            if (lane == 0)
                atomicOr(p.error, kErrStageTimeout);
            break;
        }
        ready_phase ^= 1u << b;
        const unsigned long long t = s_claim[c];
        if (lane == 0 && t != kStopTile && atomicAdd(&s_first[b], 1u) == 0) {
            // first warp into this iteration: claim the next iteration's tile
            const int c1 = (it + 1) % kClaimSlots;
            claim(c1);
            mbar_arrive(&s_claimed[c1]);
        }

        uint32_t m = 0, ubase = 0;
        if (t != kStopTile) {
            const TilePlace tp = place_tile<WINDOWED>(p, t, s_claim_q[c], kTileRows);
            const DevQuery dq = p.queries[tp.q];
            const uint64_t row0 = tp.row0 + (uint64_t)warp * kWarpRows;
            const bool full = row0 + kWarpRows <= tp.row_end && (!WINDOWED || row0 >= tp.row_first);

            // bit 4u+e of m: row row0 + 128u + 4*lane + e still qualifies
            if (full) {
                m = kFullMask;
            } else {
#pragma unroll
                for (int u = 0; u < U; ++u)
#pragma unroll
                    for (int e = 0; e < 4; ++e)
                        if (row0 + 128u * u + 4u * lane + e < tp.row_end &&
                            (!WINDOWED || row0 + 128u * u + 4u * lane + e >= tp.row_first))
                            m |= 1u << (4 * u + e);
            }

            for (uint32_t i = 0; i < dq.npred; ++i) {
                if (!__any_sync(0xffffffffu, m))
                    break;  // every row of this warp's chunk failed: read no more columns
                const DevPred pr = p.preds[dq.first + i];
                const uint32_t *col = (const uint32_t *)pr.col + row0 + 4 * lane;
                // the branches on the warp's extent and the column type are warp-uniform
                if (!full)
                    m = filter_ragged<U>(col, m, pr.type, pr.lo, pr.hi);
                else if (pr.type == kTypeF32)
                    m = filter_full<U, true>(col, m, pr.lo, pr.hi);
                else
                    m = filter_full<U, false>(col, m, pr.lo, pr.hi);
            }

            // rank the matches of this warp: row order is (u, lane, e)
            uint32_t packed = 0;  // 8-bit count per u
#pragma unroll
            for (int u = 0; u < U; ++u)
                packed |= (uint32_t)__popc((m >> (4 * u)) & 0xfu) << (8 * u);
            uint32_t incl = packed;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t x = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o)
                    incl += x;
            }
            const uint32_t excl_lane = incl - packed;
            const uint32_t warp_packed = __shfl_sync(0xffffffffu, incl, 31);

            // stage the row offsets (within the tile) of this warp's matches in row order
            uint16_t *seg = &s_stage[b][warp * kWarpRows];
            const uint32_t off0 = (uint32_t)warp * kWarpRows + 4u * lane;
#pragma unroll
            for (int u = 0; u < U; ++u) {
                uint32_t mu = (m >> (4 * u)) & 0xfu;
                uint32_t r = ubase + ((excl_lane >> (8 * u)) & 0xffu);
                while (mu) {
                    const int e = __ffs(mu) - 1;
                    seg[r++] = (uint16_t)(off0 + 128u * u + e);
                    mu &= mu - 1;
                }
                ubase += (warp_packed >> (8 * u)) & 0xffu;
            }
        }
        __syncwarp();
        if (lane == 0) {
            s_warp_total[b][warp] = ubase;
            __threadfence_block();
            // the last filter warp to finish the iteration hands the stage over and, for
            // a tile, publishes its aggregate at once (the launch's first tile: its prefix)
            if (atomicAdd(&s_done[b], 1u) == kWarps - 1) {
                __threadfence_block();
                if (!STAGED && t != kStopTile) {
                    uint32_t total = 0;
#pragma unroll
                    for (int w = 0; w < kWarps; ++w)
                        total += *(volatile uint32_t *)&s_warp_total[b][w];
                    st_relaxed_u64(state_slot(p, t),
                                   pack_state(state_tag(p, t), t == 0 ? kFlagPrefix : kFlagAggregate, total));
                }
                s_stage_tile[b] = t;
                s_stage_q[b] = s_claim_q[c];
                s_done[b] = 0;
                s_first[b] = 0;
            }
            mbar_arrive(&s_full[b]);
        }
        if (t == kStopTile)
            break;
    }
}

template <int U>
__global__ void __launch_bounds__(kScanThreads, 7) mdrq_scan_kernel(const __grid_constant__ ScanParams p)
{
    scan_cta<U, false>(p);
}

// The same with staged output (tile records and a staging buffer; concat.cu orders it).
template <int U>
__global__ void __launch_bounds__(kScanThreads, 7) mdrq_scan_staged_kernel(const __grid_constant__ ScanParams p)
{
    scan_cta<U, false, true>(p);
}


}  // namespace mdrq
