// Batched shared scan: many multidimensional range queries evaluated together.
//
// The paper answers one query at a time (Sec. 7.1.2). For a batch, this scan reads each
// constrained column once per group ("chunk") of up to 32*G queries and decides, for
// every row, the exact set of queries of the chunk it satisfies (the conjunction of
// Sec. 2.1) without one comparison per predicate:
//
//  * Per chunk and per column j some query of the chunk constrains, the end points of
//    the chunk's intervals on j cut the value line into "elementary intervals". The
//    cut points are each lower bound lo and the successor of each upper bound hi
//    (the next float32 above hi, or hi + 1 for int32), sorted and deduplicated; an
//    end point that every value of the column already satisfies (lo <= min, hi >= max)
//    is left out. A value x lies in elementary interval e(x) = #{cut points <= x}.
//  * Within one elementary interval every query's predicate on j is either true for
//    all values or false for all values (x >= lo iff the cut lo is counted, x <= hi
//    iff the cut succ(hi) is not). So a table T_j[e] of G 32-bit words holds the bit
//    of every query of the chunk whose predicate on j contains elementary interval e
//    (and of every query that does not constrain j).
//  * A row's matching queries are then the AND over the chunk's columns of
//    T_j[e_j(x_j)]: one binary search (exact compares in the column's type) and G
//    word loads from shared memory per row and column, independent of how many
//    predicates the chunk has.
//
// Coded columns: when the batch fits, each constrained column is first encoded once for
// the whole batch into 16-bit codes, code(x) = #{cut points of the batch <= x} over the
// union of all chunks' cut points of that column (one binary search per row and
// column instead of one per row, column and chunk). A chunk's elementary interval is
// then a function of the code, held as a lookup table in its image: e = L[code]. The
// passes read 2-byte codes instead of 4-byte values and look up instead of searching.
//
// Output is CSR over the batch, ascending per query, in two passes over the table:
// pass 1 counts each query's matches per warp unit of consecutive rows, an exclusive
// scan per query (and over the queries) turns the counts into write offsets, and
// pass 2 recomputes the masks and writes the ids, ranking rows inside a 32-row step
// with warp ballots. Work items are (chunk, 8 units) pairs in chunk-major order over
// a persistent grid; a CTA copies a chunk's cut points and tables into shared memory
// when it moves to that chunk.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <utility>
#include <vector>

#include "mdrq.h"
#include "scan_kernel.cuh"
#include "table.h"

namespace mdrq {

constexpr int kSharedWarps = 8;
constexpr int kSharedThreads = kSharedWarps * 32;
constexpr uint64_t kMaxUnitRows = 8192;          // rows per warp unit, large tables
constexpr uint64_t kMinUnitRows = 256;           // rows per warp unit, small tables
constexpr int kSharedG = 4;                      // 32-bit mask words per chunk: 128 queries
constexpr uint32_t kChunkImageWords = 14 * 1024; // default shared-memory budget of one chunk (56 KiB)
constexpr uint32_t kMaxImageWords = 52 * 1024;   // largest budget a table may set (208 KiB)
constexpr uint32_t kColWords = 8;                // words of one ChunkCol in an image
constexpr uint32_t kHintBuckets = 1024;          // value buckets of a column's search hint
constexpr uint32_t kMaxHintSteps = 15;           // most cut points one bucket may hold
constexpr int kCountPlanes = 4;                  // bit planes of the pass-1 lane counters
constexpr unsigned long long kSkipQuery = ~0ull;  // qbase of a query pass 2 must not write
constexpr int kPrefetchCols = 8;                 // column values per row kept in flight
constexpr uint64_t kMaskBudgetBytes = 32ull << 30;  // default largest row-bit store between the passes
constexpr uint32_t kBlockSteps = 16;     // cached write pass: 32-row steps per id block
constexpr uint32_t kBlockStride = kBlockSteps + 1;  // words per query in the block buffer (padded)
constexpr uint32_t kLanesPerWord = 32 / kBlockSteps;  // lanes sharing one step's word in a flush
constexpr uint32_t kLaneBits = kBlockSteps == 32 ? 0xffffffffu : (1u << kBlockSteps) - 1u;
constexpr uint32_t kLaneRun = 16;  // cached write pass: a query's block ids its own lane writes
constexpr size_t kBlockBufferBytes = (size_t)kSharedWarps * kSharedG * 32 * kBlockStride * 4;
constexpr uint32_t kCodedMaxCuts = 16383;        // coded columns: most cut points of one column
constexpr int kBallotQueries = 2;                // write pass: up to this many matching queries
                                                 // per step are ranked by ballots, more by a
                                                 // bit-matrix transpose

// One column of a chunk's shared-memory image (kColWords words). The first 16 bytes are
// what the passes read for every row (one 128-bit shared-memory load):
//   w0: image word of the cut points (bits 0-15), their number m (bits 16-24), the
//       search hint's walk length (bits 25-28), type (bit 31: 1 = int32); for a coded
//       column, bits 0-15 locate the code lookup table L, of bytes when bit 30 is set
//       (the chunk has at most 255 cut points on the column) or else of 16-bit entries;
//   w1: image word of the tables (bits 0-15) and of the hint (bits 16-31);
//   w2, w3: the hint's bucket base and scale (float; scale 0: no hint).
// col: the device column, or for a coded column its 16-bit codes.
struct ChunkCol {
    uint32_t w0, w1;
    float base;           // search hint: bucket trunc((x - base) * scale), clamped
    float scale;
    const uint32_t *col;  // device column
    uint32_t pad[2];
};
static_assert(sizeof(ChunkCol) == kColWords * 4, "ChunkCol layout");

// One chunk of the batch.
struct ChunkHdr {
    uint32_t ncols;       // columns constrained by some query of the chunk
    uint32_t nq;          // queries of the chunk (<= 32 * G)
    uint32_t q0;          // index of its first query among the batch's live queries
    uint32_t img_words;   // words of its shared-memory image
    uint64_t img_off;     // plan word of the image
    uint64_t iv_off;      // plan word of its intervals: ncols x nq words (elo | ehi << 16)
};

struct SharedParams {
    const uint32_t *plan;           // chunk images and interval lists (device)
    uint32_t *plan_rw;              // same buffer, writable (table build)
    const ChunkHdr *chunks;
    uint32_t nchunks;
    uint32_t nlive;
    uint64_t n;
    uint64_t n_units;
    uint64_t unit_rows;             // rows per warp unit (a multiple of 32)
    uint64_t items;                 // nchunks * ceil(n_units / kSharedWarps)
    uint32_t *counts;               // [live query][unit]: matches, then exclusive prefix
    unsigned long long *totals;     // [live query]
    unsigned long long *qbase;      // [live query]: CSR start
    const uint32_t *live_orig;      // [live query]: index in the caller's batch
    unsigned long long *offsets;    // offsets[orig + 1] <- CSR end of that query
    uint32_t *ids;
    uint64_t capacity;
    uint4 *masks;                   // [chunk][32-row step][lane]: the step's rows of queries
                                    // 32g + lane, g = 0..3 (CACHED passes; rows padded to 32)
};

// e(x) = number of cut points <= x, by a fixed-step binary search (uniform across lanes)
__device__ __forceinline__ uint32_t elementary_interval(const uint32_t *cut, uint32_t m, uint32_t xbits,
                                                        uint32_t type)
{
    uint32_t pos = 0;
    uint32_t step = m ? 1u << (31 - __clz(m)) : 0u;
    if (type == kTypeF32) {
        const float x = __uint_as_float(xbits);
        for (; step; step >>= 1)
            if (pos + step <= m && __uint_as_float(cut[pos + step - 1]) <= x)
                pos += step;
    } else {
        const int x = (int)xbits;
        for (; step; step >>= 1)
            if (pos + step <= m && (int)cut[pos + step - 1] <= x)
                pos += step;
    }
    return pos;
}

// e(x) from the column's hint. The bucket function trunc((x - base) * scale) is
// monotone in x, and the hint holds, per bucket, the number of cut points in lower
// buckets; the cut points in x's own bucket (at most `steps`, computed on the host
// with the same float arithmetic) are then compared in order until one exceeds x.
__device__ __forceinline__ uint32_t interval_of(const uint32_t *img, uint4 hot, uint32_t xbits)
{
    const uint32_t *cut = img + (hot.x & 0xffffu);
    const uint32_t m = (hot.x >> 16) & 0x1ffu;
    const bool f32 = (hot.x >> 31) == 0u;
    const float scale = __uint_as_float(hot.w);
    if (scale == 0.0f)
        return elementary_interval(cut, m, xbits, f32 ? kTypeF32 : kTypeI32);
    const uint32_t steps = (hot.x >> 25) & 0xfu;
    const float xf = f32 ? __uint_as_float(xbits) : (float)(int)xbits;
    int b = __float2int_rz((xf - __uint_as_float(hot.z)) * scale);
    b = b < 0 ? 0 : (b >= (int)kHintBuckets ? (int)kHintBuckets - 1 : b);
    const uint32_t h = img[(hot.y >> 16) + (b >> 1)];
    uint32_t pos = (b & 1) ? (h >> 16) : (h & 0xffffu);
    const uint32_t end = pos + steps < m ? pos + steps : m;  // the bucket's cuts lie below end
    if (f32) {
        const float x = __uint_as_float(xbits);
        while (pos < end && __uint_as_float(cut[pos]) <= x)
            ++pos;
    } else {
        const int x = (int)xbits;
        while (pos < end && (int)cut[pos] <= x)
            ++pos;
    }
    return pos;
}

// A coded column's elementary interval: the chunk's lookup table entry of the code
__device__ __forceinline__ uint32_t coded_interval(const uint32_t *img, uint4 hot, uint32_t code)
{
    const uint32_t *lut = img + (hot.x & 0xffffu);
    if (hot.x & (1u << 30))
        return reinterpret_cast<const unsigned char *>(lut)[code];
    return reinterpret_cast<const unsigned short *>(lut)[code];
}

// Row r's value of a chunk column (its 16-bit code when CODED), read through the
// read-only path
template <bool CODED>
__device__ __forceinline__ uint32_t column_value(const uint32_t *desc, uint64_t r)
{
    const uint32_t *col = reinterpret_cast<const ChunkCol *>(desc)->col;
    if (CODED)
        return __ldg(reinterpret_cast<const unsigned short *>(col) + r);
    return __ldg(col + r);
}

// The batch's codes of one column: code(x) = #{cut points <= x} over the sorted cut
// points cut[0 .. m) of every chunk (m <= kCodedMaxCuts). With a hint (scale != 0) the
// value's bucket trunc((x - base) * scale), clamped to [0, kEncodeBuckets), gives the
// number of cut points in lower buckets (16-bit entries in the plan after the cut
// points), and at most `steps` compares walk the cut points of its own bucket: the
// bucket function is monotone in x and the host computed the entries with the same
// float arithmetic, so this is exact. Without a hint, the fixed-step search.
constexpr uint32_t kEncodeBuckets = 4096;

struct EncodeCol {
    const uint32_t *col;      // device column
    unsigned short *codes;    // n codes
    uint64_t cut_off;         // plan word of its cut points (then the hint, if any)
    uint32_t m;
    uint32_t type;
    uint32_t steps;           // most cut points in one bucket (hint only)
    float base, scale;        // bucket function (scale 0: no hint)
    uint32_t pad;
};

__global__ void __launch_bounds__(256) mdrq_shared_encode_kernel(const EncodeCol *ec, const uint32_t *plan,
                                                                 uint64_t n)
{
    extern __shared__ uint32_t s_cut[];
    const EncodeCol c = ec[blockIdx.y];
    const bool hinted = c.scale != 0.0f;
    const uint32_t words = c.m + (hinted ? kEncodeBuckets / 2 : 0u);
    for (uint32_t i = threadIdx.x; i < words; i += blockDim.x)
        s_cut[i] = plan[c.cut_off + i];
    __syncthreads();
    const unsigned short *hint = reinterpret_cast<const unsigned short *>(s_cut + c.m);
    const bool f32 = c.type == kTypeF32;
    auto code_of = [&](uint32_t x) -> uint32_t {
        uint32_t pos;
        if (hinted) {
            const float xf = f32 ? __uint_as_float(x) : (float)(int)x;
            int b = __float2int_rz((xf - c.base) * c.scale);
            b = b < 0 ? 0 : (b >= (int)kEncodeBuckets ? (int)kEncodeBuckets - 1 : b);
            pos = hint[b];
            const uint32_t end = pos + c.steps < c.m ? pos + c.steps : c.m;
            if (f32) {
                const float xv = __uint_as_float(x);
                while (pos < end && __uint_as_float(s_cut[pos]) <= xv)
                    ++pos;
            } else {
                while (pos < end && (int)s_cut[pos] <= (int)x)
                    ++pos;
            }
        } else {
            pos = elementary_interval(s_cut, c.m, x, c.type);
        }
        return pos;
    };
    // four rows per thread: one 16-byte load (the column is 16-byte aligned) and one
    // 8-byte store (each code column starts on a multiple of 8 codes); the last n % 4
    // rows one by one
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t n4 = n / 4;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) {
        const uint4 v = __ldg(reinterpret_cast<const uint4 *>(c.col) + i);
        const uint32_t a = code_of(v.x), b = code_of(v.y), d = code_of(v.z), e = code_of(v.w);
        reinterpret_cast<uint2 *>(c.codes)[i] = make_uint2(a | (b << 16), d | (e << 16));
    }
    for (uint64_t r = 4 * n4 + (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += stride)
        c.codes[r] = (unsigned short)code_of(__ldg(c.col + r));
}

// T[e][g] for every elementary interval of every (chunk, column): bit i of word g is
// set when query 32g + i of the chunk accepts that interval. Block (chunk, column).
__global__ void __launch_bounds__(256) mdrq_shared_tables_kernel(SharedParams p, uint32_t max_cols)
{
    const uint32_t c = blockIdx.x / max_cols, a = blockIdx.x % max_cols;
    if (c >= p.nchunks)
        return;
    const ChunkHdr h = p.chunks[c];
    if (a >= h.ncols)
        return;
    uint32_t *img = p.plan_rw + h.img_off;
    const ChunkCol cc = *reinterpret_cast<const ChunkCol *>(img + a * kColWords);
    const uint32_t *iv = p.plan + h.iv_off + (uint64_t)a * h.nq;
    const uint32_t m = (cc.w0 >> 16) & 0x1ffu, tab_off = cc.w1 & 0xffffu;
    const uint32_t words = (m + 1) * kSharedG;
    for (uint32_t w = threadIdx.x; w < words; w += blockDim.x) {
        const uint32_t e = w / kSharedG, g = w % kSharedG;
        uint32_t bits = 0;
        for (uint32_t i = 0; i < 32; ++i) {
            const uint32_t q = g * 32 + i;
            if (q < h.nq) {
                const uint32_t r = iv[q];
                if ((r & 0xffffu) <= e && e <= (r >> 16))
                    bits |= 1u << i;
            }
        }
        img[tab_off + w] = bits;
    }
}

// 32 x 32 bit transpose across a warp: on return, bit k of lane l's word is bit l of
// lane k's word on entry. Five exchange stages, each swapping the off-diagonal blocks.
__device__ __forceinline__ uint32_t warp_transpose32(uint32_t x, int lane)
{
    const uint32_t lo_mask[5] = {0x0000ffffu, 0x00ff00ffu, 0x0f0f0f0fu, 0x33333333u, 0x55555555u};
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        const int sft = 16 >> k;
        const uint32_t m = lo_mask[k];
        const uint32_t y = __shfl_xor_sync(0xffffffffu, x, sft);
        x = (lane & sft) ? ((y & ~m) >> sft) | (x & ~m) : (x & m) | ((y & m) << sft);
    }
    return x;
}

// Add the bit-sliced counters into cnt (lane l: query 32g + l) and clear them.
__device__ __forceinline__ void flush_counts(uint32_t (&plane)[kSharedG][kCountPlanes], uint32_t (&cnt)[kSharedG],
                                             int lane)
{
#pragma unroll
    for (int g = 0; g < kSharedG; ++g) {
#pragma unroll
        for (int j = 0; j < kCountPlanes; ++j) {
            cnt[g] += (uint32_t)__popc(warp_transpose32(plane[g][j], lane)) << j;
            plane[g][j] = 0u;
        }
    }
}

// Pass 1 (WRITE = false): per live query and unit, the number of matching rows.
// Pass 2 (WRITE = true): the ids, at qbase[q] + counts[q][unit] (exclusive prefix).
// CACHED: pass 1 also stores the chunk's row bits (16 bytes per row and chunk), transposed
// per 32-row step so that lane l holds the step's rows of queries l, 32 + l, 64 + l and
// 96 + l; it counts them with popcounts, and pass 2 reads them instead of evaluating the
// columns again and without transposing them.
// CODED: the chunk columns are the batch's 16-bit codes (mdrq_shared_encode_kernel),
// each chunk's elementary interval a table lookup.
template <bool WRITE, bool CACHED, bool CODED>
// (64 registers, so that four blocks fit an SM: measured faster than 80 and three)
__global__ void __launch_bounds__(kSharedThreads, 4) mdrq_shared_pass_kernel(SharedParams p)
{
    constexpr bool kLoadMasks = WRITE && CACHED;
    const uint64_t n_pad = (p.n + 31) & ~31ull;  // rows of the stored row bits
    // columns whose next-step values are loaded ahead: fewer for 2-byte codes, whose
    // lookups are short, than for values, whose searches are long (measured)
    constexpr int kPre = CODED ? 4 : kPrefetchCols;
    extern __shared__ __align__(16) uint32_t s_img[];
    __shared__ uint32_t s_chunk;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const uint64_t groups = (p.n_units + kSharedWarps - 1) / kSharedWarps;
    uint32_t cur = 0xffffffffu;
    ChunkHdr h;

    for (uint64_t item = blockIdx.x; item < p.items; item += gridDim.x) {
        const uint32_t c = (uint32_t)(item / groups);
        if (c != cur) {
            // move to chunk c: copy its image into shared memory
            __syncthreads();
            h = p.chunks[c];
            const uint4 *src = reinterpret_cast<const uint4 *>(p.plan + h.img_off);
            uint4 *dst = reinterpret_cast<uint4 *>(s_img);
            for (uint32_t i = threadIdx.x; !kLoadMasks && i < h.img_words / 4; i += blockDim.x)
                dst[i] = src[i];
            if (threadIdx.x == 0)
                s_chunk = c;
            __syncthreads();
            cur = c;
        }
        const uint64_t unit = (item % groups) * kSharedWarps + warp;
        if (unit >= p.n_units)
            continue;
        const uint64_t r_begin = unit * p.unit_rows;
        const uint64_t r_end = r_begin + p.unit_rows < p.n ? r_begin + p.unit_rows : p.n;

        // lane i keeps the figures of query 32g + i of the chunk
        uint32_t cnt[kSharedG];
        unsigned long long off[kSharedG];
#pragma unroll
        for (int g = 0; g < kSharedG; ++g) {
            cnt[g] = 0;
            off[g] = 0;
            const uint32_t qi = g * 32 + lane;
            if (WRITE && qi < h.nq) {
                const uint64_t lq = h.q0 + qi;
                const unsigned long long qb = p.qbase[lq];
                off[g] = qb == kSkipQuery ? kSkipQuery : qb + p.counts[lq * p.n_units + unit];
            }
        }
        uint32_t plane[kSharedG][kCountPlanes];  // pass 1: bit-sliced per-lane counters
        uint32_t since_flush = 0;
#pragma unroll
        for (int g = 0; g < kSharedG; ++g)
#pragma unroll
            for (int j = 0; j < kCountPlanes; ++j)
                plane[g][j] = 0u;
        uint32_t valid_words[kSharedG];  // bits of the chunk's real queries
#pragma unroll
        for (int g = 0; g < kSharedG; ++g) {
            const int left = (int)h.nq - g * 32;
            valid_words[g] = left >= 32 ? 0xffffffffu : left > 0 ? (1u << left) - 1u : 0u;
        }

        // values of the first kPre columns for the next 32-row step are loaded
        // while the current step is evaluated (software pipelining of the column reads)
        const uint32_t npre = kLoadMasks ? 0u : (h.ncols < kPre ? h.ncols : kPre);
        uint32_t xn[kPre];
#pragma unroll
        for (int i = 0; i < kPre; ++i) {
            const uint64_t r = r_begin + lane;
            xn[i] = 0u;
            if (i < (int)npre && r < r_end)
                xn[i] = column_value<CODED>(s_img + i * kColWords, r);
        }
        // cached write pass: this warp's block buffer of transposed step matrices
        uint32_t *tb = s_img + (size_t)warp * kSharedG * 32 * kBlockStride;
        uint32_t seen[kSharedG] = {0u, 0u, 0u, 0u};  // per lane: rows seen for its queries
        uint32_t sb = 0;                             // steps in the block buffer
        uint64_t block_row0 = r_begin;
        for (uint64_t r0 = r_begin; r0 < r_end; r0 += 32) {
            const uint64_t r = r0 + lane;
            const bool valid = r < r_end;
            uint32_t mask[kSharedG];
            if (kLoadMasks) {
                // stored transposed by pass 1: lane l gets the step's rows of query 32g + l
                const uint4 m4 = __ldcs(p.masks + (uint64_t)c * n_pad + r0 + lane);
                mask[0] = m4.x;
                mask[1] = m4.y;
                mask[2] = m4.z;
                mask[3] = m4.w;
            } else {
                uint32_t x[kPre];
#pragma unroll
                for (int i = 0; i < kPre; ++i) {
                    x[i] = xn[i];
                    const uint64_t rn = r + 32;
                    xn[i] = 0u;
                    if (i < (int)npre && rn < r_end)
                        xn[i] = column_value<CODED>(s_img + i * kColWords, rn);
                }
#pragma unroll
                for (int g = 0; g < kSharedG; ++g)
                    mask[g] = valid ? valid_words[g] : 0u;
#pragma unroll
                for (int i = 0; i < kPre; ++i) {
                    if (i < (int)npre) {
                        const uint4 hot = *reinterpret_cast<const uint4 *>(s_img + i * kColWords);
                        const uint32_t e = CODED ? coded_interval(s_img, hot, x[i]) : interval_of(s_img, hot, x[i]);
                        const uint4 t = *reinterpret_cast<const uint4 *>(s_img + (hot.y & 0xffffu) + e * kSharedG);
                        mask[0] &= t.x;
                        mask[1] &= t.y;
                        mask[2] &= t.z;
                        mask[3] &= t.w;
                    }
                }
                // columns beyond the prefetched ones: loaded together, then evaluated
                for (uint32_t a0 = npre; a0 < h.ncols; a0 += kPre) {
                    uint32_t y[kPre];
#pragma unroll
                    for (int i = 0; i < kPre; ++i) {
                        y[i] = 0u;
                        if (a0 + i < h.ncols && valid)
                            y[i] = column_value<CODED>(s_img + (a0 + i) * kColWords, r);
                    }
#pragma unroll
                    for (int i = 0; i < kPre; ++i) {
                        if (a0 + i < h.ncols) {
                            const uint4 hot = *reinterpret_cast<const uint4 *>(s_img + (a0 + i) * kColWords);
                            const uint32_t e = CODED ? coded_interval(s_img, hot, y[i])
                                                     : interval_of(s_img, hot, y[i]);
                            const uint4 t = *reinterpret_cast<const uint4 *>(s_img + (hot.y & 0xffffu) + e * kSharedG);
                            mask[0] &= t.x;
                            mask[1] &= t.y;
                            mask[2] &= t.z;
                            mask[3] &= t.w;
                        }
                    }
                }
                if (CACHED) {
                    // stored transposed (lane l: the step's rows of query 32g + l), so that
                    // pass 2 needs no transpose; pass 1 counts them with a popcount
#pragma unroll
                    for (int g = 0; g < kSharedG; ++g)
                        mask[g] = __any_sync(0xffffffffu, mask[g]) ? warp_transpose32(mask[g], lane) : 0u;
                    __stcs(p.masks + (uint64_t)c * n_pad + r0 + lane, make_uint4(mask[0], mask[1], mask[2], mask[3]));
                }
            }
            if (kLoadMasks) {
                // the step's (row, query) bit matrix, transposed (lane l: the rows of
                // query 32g + l), goes to the warp's block buffer; every kBlockSteps steps
                // the block's ids are written query by query by the whole warp
#pragma unroll
                for (int g = 0; g < kSharedG; ++g) {
                    const uint32_t tr = mask[g];  // transposed already (pass 1)
                    tb[(g * 32 + lane) * kBlockStride + sb] = tr;
                    seen[g] |= tr;
                }
                if (++sb == kBlockSteps || r0 + 32 >= r_end) {
                    __syncwarp();
#pragma unroll
                    for (int g = 0; g < kSharedG; ++g) {
                        // lane l's own query 32g + l: its ids in the block
                        const uint32_t *wq = tb + (g * 32 + lane) * kBlockStride;
                        uint32_t mine = 0;
                        if (seen[g])
                            for (uint32_t w = 0; w < sb; ++w)
                                mine += __popc(wq[w]);
                        seen[g] = 0u;
                        const unsigned long long qb = off[g];
                        // a query with few ids in the block: its own lane writes them, the
                        // warp's 32 queries at once
                        if (mine != 0u && mine <= kLaneRun && qb != kSkipQuery) {
                            unsigned long long pos = qb;
                            for (uint32_t w = 0; w < sb; ++w) {
                                uint32_t x = wq[w];
                                while (x) {
                                    const int e = __ffs(x) - 1;
                                    x &= x - 1;
                                    if (pos < p.capacity)
                                        p.ids[pos] = (uint32_t)(block_row0 + 32 * w + e);
                                    ++pos;
                                }
                            }
                        }
                        if (qb != kSkipQuery)
                            off[g] = qb + mine;
                        // more ids: the whole warp, one query at a time; lane i takes rows
                        // [Bi, Bi + B) of the block (B = kBlockSteps): bits B (i % (32 / B))
                        // .. of step i / (32 / B)
                        uint32_t qs = __ballot_sync(0xffffffffu, mine > kLaneRun);
                        while (qs) {
                            const int q = __ffs(qs) - 1;
                            qs &= qs - 1;
                            const uint32_t word = (uint32_t)lane / kLanesPerWord;
                            const uint32_t w = word < sb ? tb[(g * 32 + q) * kBlockStride + word] : 0u;
                            uint32_t bits = (w >> (kBlockSteps * ((uint32_t)lane % kLanesPerWord))) & kLaneBits;
                            const uint32_t c8 = __popc(bits);
                            uint32_t incl = c8;
#pragma unroll
                            for (int o = 1; o < 32; o <<= 1) {
                                const uint32_t x = __shfl_up_sync(0xffffffffu, incl, o);
                                if (lane >= o)
                                    incl += x;
                            }
                            const unsigned long long base = __shfl_sync(0xffffffffu, qb, q);
                            if (base != kSkipQuery) {
                                unsigned long long pos = base + incl - c8;
                                while (bits) {
                                    const int e = __ffs(bits) - 1;
                                    bits &= bits - 1;
                                    if (pos < p.capacity)
                                        p.ids[pos] = (uint32_t)(block_row0 + kBlockSteps * lane + e);
                                    ++pos;
                                }
                            }
                        }
                    }
                    __syncwarp();
                    sb = 0;
                    block_row0 = r0 + 32;
                }
            } else if (WRITE) {
                // the ids of this step's matches, query by query in row order. With few
                // queries matching, each is ranked by a warp ballot; with more, the
                // 32 x 32 (row, query) bit matrix is transposed so that lane l holds the
                // rows of query 32g + l and writes them itself, one per iteration.
                const uint32_t lt = (1u << lane) - 1u;
#pragma unroll
                for (int g = 0; g < kSharedG; ++g) {
                    uint32_t any = __reduce_or_sync(0xffffffffu, mask[g]);
                    if (__popc(any) > kBallotQueries) {
                        uint32_t rows = warp_transpose32(mask[g], lane);
                        if (rows && off[g] != kSkipQuery) {
                            unsigned long long o = off[g];
                            do {
                                const int e = __ffs(rows) - 1;
                                rows &= rows - 1;
                                if (o < p.capacity)
                                    p.ids[o] = (uint32_t)(r0 + e);
                                ++o;
                            } while (rows);
                            off[g] = o;
                        }
                        continue;
                    }
                    while (any) {
                        const int q = __ffs(any) - 1;
                        any &= any - 1;
                        const bool bit = (mask[g] >> q) & 1u;
                        const uint32_t b = __ballot_sync(0xffffffffu, bit);
                        const unsigned long long o = __shfl_sync(0xffffffffu, off[g], q);
                        if (bit && o != kSkipQuery) {
                            const unsigned long long pos = o + __popc(b & lt);
                            if (pos < p.capacity)
                                p.ids[pos] = (uint32_t)r;
                        }
                        if (lane == q && o != kSkipQuery)
                            off[g] += __popc(b);
                    }
                }
            } else if (CACHED) {
                // count the stored, transposed bits: lane l counts query 32g + l
#pragma unroll
                for (int g = 0; g < kSharedG; ++g)
                    cnt[g] += (uint32_t)__popc(mask[g]);
            } else {
                // count: add this lane's bits into per-lane bit-sliced counters (plane j
                // holds bit j of 32 counters); flush them before they can overflow
#pragma unroll
                for (int g = 0; g < kSharedG; ++g) {
                    uint32_t carry = mask[g];
#pragma unroll
                    for (int j = 0; j < kCountPlanes; ++j) {
                        const uint32_t t = plane[g][j] & carry;
                        plane[g][j] ^= carry;
                        carry = t;
                    }
                }
                if (++since_flush == (1u << kCountPlanes) - 1u) {
                    flush_counts(plane, cnt, lane);
                    since_flush = 0;
                }
            }
        }
        if (!WRITE) {
            if (!CACHED)
                flush_counts(plane, cnt, lane);
#pragma unroll
            for (int g = 0; g < kSharedG; ++g) {
                const uint32_t qi = g * 32 + lane;
                if (qi < h.nq)
                    p.counts[(uint64_t)(h.q0 + qi) * p.n_units + unit] = cnt[g];
            }
        }
    }
}

// Exclusive scan of one live query's unit counts, in place; totals[q] = the sum.
// Persistent blocks of 1024 threads loop over the queries.
__global__ void __launch_bounds__(1024) mdrq_shared_scan_kernel(SharedParams p)
{
    __shared__ unsigned long long s_warp[32];
    __shared__ unsigned long long s_carry;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (uint32_t q = blockIdx.x; q < p.nlive; q += gridDim.x) {
        uint32_t *c = p.counts + (uint64_t)q * p.n_units;
        if (threadIdx.x == 0)
            s_carry = 0;
        __syncthreads();
        for (uint64_t base = 0; base < p.n_units; base += blockDim.x) {
            const uint64_t i = base + threadIdx.x;
            const unsigned long long v = i < p.n_units ? c[i] : 0ull;
            unsigned long long x = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o)
                    x += y;
            }
            if (lane == 31)
                s_warp[warp] = x;
            __syncthreads();
            if (warp == 0) {
                unsigned long long w = s_warp[lane];
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const unsigned long long y = __shfl_up_sync(0xffffffffu, w, o);
                    if (lane >= o)
                        w += y;
                }
                s_warp[lane] = w;  // inclusive over warps
            }
            __syncthreads();
            const unsigned long long carry = s_carry;
            const unsigned long long excl = carry + (warp ? s_warp[warp - 1] : 0ull) + x - v;
            if (i < p.n_units)
                c[i] = (uint32_t)excl;  // < n < 2^32 per query
            __syncthreads();
            if (threadIdx.x == blockDim.x - 1)
                s_carry = carry + s_warp[31];
            __syncthreads();
        }
        if (threadIdx.x == 0)
            p.totals[q] = s_carry;
        __syncthreads();
    }
}

// qbase = exclusive scan of totals over the live queries (CSR starts); offsets[orig+1]
// = CSR end of each live query. One block.
__global__ void __launch_bounds__(1024) mdrq_shared_qbase_kernel(SharedParams p)
{
    __shared__ unsigned long long s_warp[32];
    __shared__ unsigned long long s_carry;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0)
        s_carry = 0;
    __syncthreads();
    for (uint32_t base = 0; base < p.nlive; base += blockDim.x) {
        const uint32_t i = base + threadIdx.x;
        const unsigned long long v = i < p.nlive ? p.totals[i] : 0ull;
        unsigned long long x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o)
                x += y;
        }
        if (lane == 31)
            s_warp[warp] = x;
        __syncthreads();
        if (warp == 0) {
            unsigned long long w = s_warp[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned long long y = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o)
                    w += y;
            }
            s_warp[lane] = w;
        }
        __syncthreads();
        const unsigned long long carry = s_carry;
        const unsigned long long incl = carry + (warp ? s_warp[warp - 1] : 0ull) + x;
        if (i < p.nlive) {
            p.qbase[i] = incl - v;
            p.offsets[p.live_orig[i] + 1] = incl;
        }
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1)
            s_carry = carry + s_warp[31];
        __syncthreads();
    }
}

// Device buffers of the shared scan, kept with the table and grown on demand.
struct SharedScanState {
    uint32_t *plan = nullptr;
    size_t plan_cap = 0;
    ChunkHdr *chunks = nullptr;
    size_t chunks_cap = 0;
    uint32_t *live_orig = nullptr;
    size_t live_cap = 0;
    uint32_t *counts = nullptr;
    size_t counts_cap = 0;
    unsigned long long *totals = nullptr;
    size_t totals_cap = 0;
    unsigned long long *qbase = nullptr;
    size_t qbase_cap = 0;
    unsigned char *stage = nullptr;  // pinned: chunk headers, plan, live_orig
    size_t stage_cap = 0;
    int grid_scan = 0;
    bool smem_attr = false;            // pass kernels opted in to kMaxImageWords
    uint4 *masks = nullptr;            // row masks between the passes
    size_t masks_cap = 0;
    unsigned short *codes = nullptr;   // coded columns: 16-bit codes, one column after another
    size_t codes_cap = 0;
    EncodeCol *ecols = nullptr;        // coded columns to encode
    size_t ecols_cap = 0;
    bool coded = false;                // the prepared batch uses coded columns
    // (image words | cached << 31, (count-pass grid, write-pass grid))
    std::vector<std::pair<uint32_t, std::pair<int, int>>> grid_for_words;
    // the batch prepared by shared_scan_count, for shared_scan_write
    SharedParams params;
    uint32_t grid = 0;
    size_t smem = 0;
    bool ready = false;
};

namespace {

// one column's cut points and each query's elementary-interval range on it
struct ColPlan {
    uint32_t dim;
    std::vector<double> cuts;  // sorted, distinct (exact values of the column type)
};

double successor(double v, int32_t type)
{
    if (type == MDRQ_F32)
        return (double)std::nextafter((float)v, INFINITY);
    return v + 1.0;
}

uint32_t to_bits(double v, int32_t type)
{
    if (type == MDRQ_F32) {
        const float f = (float)v;
        uint32_t b;
        std::memcpy(&b, &f, 4);
        return b;
    }
    return (uint32_t)(int32_t)v;
}

}  // namespace

namespace {

using PassKernel = void (*)(SharedParams);

// pass 1 of a batch (stores row masks when cached; reads codes when coded)
PassKernel count_kernel(bool cached, bool coded)
{
    if (coded)
        return cached ? mdrq_shared_pass_kernel<false, true, true> : mdrq_shared_pass_kernel<false, false, true>;
    return cached ? mdrq_shared_pass_kernel<false, true, false> : mdrq_shared_pass_kernel<false, false, false>;
}

// pass 2: from the stored row masks when cached, else evaluating the columns again
PassKernel write_kernel(bool cached, bool coded)
{
    if (cached)
        return mdrq_shared_pass_kernel<true, true, false>;
    return coded ? mdrq_shared_pass_kernel<true, false, true> : mdrq_shared_pass_kernel<true, false, false>;
}

}  // namespace

SharedScanState *shared_state_new() { return new (std::nothrow) SharedScanState(); }

void shared_state_free(SharedScanState *S)
{
    if (!S)
        return;
    cudaFree(S->plan);
    cudaFree(S->chunks);
    cudaFree(S->live_orig);
    cudaFree(S->counts);
    cudaFree(S->totals);
    cudaFree(S->qbase);
    cudaFree(S->masks);
    cudaFree(S->codes);
    cudaFree(S->ecols);
    cudaFreeHost(S->stage);
    delete S;
}

unsigned long long *shared_state_qbase(SharedScanState *S) { return S->qbase; }
unsigned long long *shared_state_totals(SharedScanState *S) { return S->totals; }

int shared_scan_count(mdrq_table *t, SharedScanState &S, const std::vector<EncodedQuery> &enc,
                      const std::vector<uint32_t> &live, cudaStream_t s)
{
    S.ready = false;
    const uint32_t nlive = (uint32_t)live.size();
    if (nlive == 0 || t->n == 0)
        return MDRQ_OK;

    // ---- chunks: consecutive live queries, at most 32 * G each, image within budget
    struct Chunk {
        uint32_t q0, nq;
    };
    std::vector<Chunk> chunks;
    const uint32_t budget = t->shared_image_words ? t->shared_image_words : kChunkImageWords;
    {
        uint32_t q = 0;
        while (q < nlive) {
            Chunk ch{q, 0};
            std::vector<uint32_t> per_dim(t->d, 0);
            uint32_t ncols = 0, pairs = 0;
            while (q < nlive && ch.nq < 32u * kSharedG) {
                const EncodedQuery &e = enc[live[q]];
                uint32_t add_cols = 0;
                for (uint32_t j : e.dims)
                    add_cols += per_dim[j] == 0;
                // upper bound of the image: columns + 2 cuts per pair + (cuts + 1) * G table words
                const uint32_t nc = ncols + add_cols, np = pairs + (uint32_t)e.dims.size();
                const uint64_t words = (uint64_t)nc * kColWords + 2ull * np + 4 +
                                       (2ull * np + nc) * kSharedG + 4ull * nc;
                if (ch.nq > 0 && words > budget)
                    break;
                if (ch.nq == 0 && words > budget)
                    return MDRQ_E_INVAL;  // one query alone does not fit (more than ~900 dimensions)
                for (uint32_t j : e.dims)
                    per_dim[j] += 1;
                ncols = nc;
                pairs = np;
                ++ch.nq;
                ++q;
            }
            chunks.push_back(ch);
        }
    }

    // ---- per chunk: columns and cut points
    std::vector<std::vector<ColPlan>> chunk_cols(chunks.size());
    std::vector<std::vector<int>> chunk_slot(chunks.size());
    for (size_t ci = 0; ci < chunks.size(); ++ci) {
        const Chunk &ch = chunks[ci];
        // columns in first-use order, with their cut points
        std::vector<int> &slot = chunk_slot[ci];
        slot.assign(t->d, -1);
        std::vector<ColPlan> &cols = chunk_cols[ci];
        for (uint32_t k = 0; k < ch.nq; ++k) {
            const EncodedQuery &e = enc[live[ch.q0 + k]];
            for (size_t i = 0; i < e.dims.size(); ++i) {
                const uint32_t j = e.dims[i];
                if (slot[j] < 0) {
                    slot[j] = (int)cols.size();
                    cols.push_back(ColPlan{j, {}});
                }
                const ColumnInfo &c = t->cols[j];
                const double lo = bound_value(e.preds[i].lo, c.type), hi = bound_value(e.preds[i].hi, c.type);
                const double mn = bound_value(c.min_bits, c.type), mx = bound_value(c.max_bits, c.type);
                if (lo > mn)
                    cols[slot[j]].cuts.push_back(lo);
                if (hi < mx)
                    cols[slot[j]].cuts.push_back(successor(hi, c.type));
            }
        }
        for (ColPlan &cp : cols) {
            std::sort(cp.cuts.begin(), cp.cuts.end());
            cp.cuts.erase(std::unique(cp.cuts.begin(), cp.cuts.end()), cp.cuts.end());
        }
    }

    // ---- coded columns: the union of every chunk's cut points per column; used when
    // each union stays within kCodedMaxCuts, every chunk's coded image fits the largest
    // image budget and the codes (2 bytes per row and column) fit the device
    std::vector<std::vector<double>> gcuts(t->d);
    std::vector<int> gslot(t->d, -1);
    std::vector<uint32_t> gdims;
    for (const auto &cols : chunk_cols)
        for (const ColPlan &cp : cols) {
            if (gslot[cp.dim] < 0) {
                gslot[cp.dim] = (int)gdims.size();
                gdims.push_back(cp.dim);
            }
            gcuts[cp.dim].insert(gcuts[cp.dim].end(), cp.cuts.begin(), cp.cuts.end());
        }
    bool coded = t->shared_coded && !gdims.empty();
    for (uint32_t j : gdims) {
        std::vector<double> &g = gcuts[j];
        std::sort(g.begin(), g.end());
        g.erase(std::unique(g.begin(), g.end()), g.end());
        coded = coded && g.size() <= kCodedMaxCuts;
    }
    // a column's lookup table: bytes when the chunk has at most 255 cut points on it
    auto lut_words = [&](const ColPlan &cp) -> uint64_t {
        const uint64_t entries = gcuts[cp.dim].size() + 1;
        return cp.cuts.size() <= 255 ? (entries + 3) / 4 : (entries + 1) / 2;
    };
    auto coded_image_words = [&](const std::vector<ColPlan> &cols) {
        uint64_t w = (uint64_t)cols.size() * kColWords;
        for (const ColPlan &cp : cols)
            w += lut_words(cp);
        w = (w + 3) & ~3ull;
        for (const ColPlan &cp : cols)
            w += (uint64_t)(cp.cuts.size() + 1) * kSharedG;
        return (w + 3) & ~3ull;
    };
    for (const auto &cols : chunk_cols)
        coded = coded && coded_image_words(cols) <= std::min<uint64_t>(kMaxImageWords, 0xffff);
    const uint64_t code_stride = (t->n + 7) & ~7ull;  // codes per column, a multiple of 8
    if (coded) {
        const uint64_t code_bytes = (uint64_t)gdims.size() * code_stride * 2;
        size_t free_b = 0, total_b = 0;
        coded = code_bytes <= kMaskBudgetBytes &&
                (S.codes_cap >= code_bytes ||
                 (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess && code_bytes <= free_b / 4 &&
                  grow_device((void **)&S.codes, &S.codes_cap, (size_t)code_bytes) == MDRQ_OK));
        (void)cudaGetLastError();
    }

    // ---- per chunk: images and intervals, laid out as plan words
    std::vector<ChunkHdr> hdrs(chunks.size());
    std::vector<uint32_t> plan;
    plan.reserve(1 << 16);
    uint32_t max_cols = 1;
    uint32_t max_img = 4;  // words of the largest chunk image: the launches' shared memory
    for (size_t ci = 0; ci < chunks.size(); ++ci) {
        const Chunk &ch = chunks[ci];
        const std::vector<int> &slot = chunk_slot[ci];
        const std::vector<ColPlan> &cols = chunk_cols[ci];
        const uint32_t ncols = (uint32_t)cols.size();
        max_cols = std::max(max_cols, ncols);
        uint64_t img_off;
        uint32_t img_words;
        if (coded) {
            // image: ChunkCol[ncols], lookup tables (code -> this chunk's elementary
            // interval, bytes or 16-bit entries), (pad to 4), tables
            while (plan.size() % 4)
                plan.push_back(0);
            img_off = plan.size();
            img_words = (uint32_t)coded_image_words(cols);
            plan.resize(img_off + img_words, 0);
            uint32_t w = ncols * kColWords;
            std::vector<uint32_t> lut_off(ncols), tab_off(ncols);
            for (uint32_t a = 0; a < ncols; ++a) {
                lut_off[a] = w;
                w += (uint32_t)lut_words(cols[a]);
            }
            w = (w + 3) & ~3u;
            for (uint32_t a = 0; a < ncols; ++a) {
                tab_off[a] = w;
                w += (uint32_t)(cols[a].cuts.size() + 1) * kSharedG;
            }
            for (uint32_t a = 0; a < ncols; ++a) {
                const uint32_t j = cols[a].dim;
                const std::vector<double> &g = gcuts[j], &cut = cols[a].cuts;
                ChunkCol cc;
                std::memset(&cc, 0, sizeof(cc));
                const bool bytes = cut.size() <= 255;
                cc.w0 = lut_off[a] | ((uint32_t)cut.size() << 16) | ((bytes ? 1u : 0u) << 30) |
                        ((t->cols[j].type == MDRQ_I32 ? 1u : 0u) << 31);
                cc.w1 = tab_off[a];
                cc.col = reinterpret_cast<const uint32_t *>(S.codes + (size_t)gslot[j] * code_stride);
                std::memcpy(&plan[img_off + a * kColWords], &cc, sizeof(ChunkCol));
                // code k: the values in [g[k-1], g[k]); the chunk's cut points at or
                // below them are its cut points among g[0 .. k)
                uint32_t e = 0;
                size_t ci2 = 0;
                for (size_t k = 0; k <= g.size(); ++k) {
                    if (k > 0) {
                        while (ci2 < cut.size() && cut[ci2] <= g[k - 1])
                            ++ci2;
                        e = (uint32_t)ci2;
                    }
                    if (bytes)
                        plan[img_off + lut_off[a] + k / 4] |= e << (8 * (k & 3));
                    else
                        plan[img_off + lut_off[a] + k / 2] |= e << (16 * (k & 1));
                }
            }
            max_img = std::max(max_img, img_words);
        } else {
            // image: ChunkCol[ncols], hints, cut points, (pad to 4), tables ((m + 1) * G words each)
            while (plan.size() % 4)
                plan.push_back(0);
            img_off = plan.size();
            uint32_t w = ncols * kColWords;
            struct ColLayout {
                uint32_t type = 0, m = 0, cut_off = 0, tab_off = 0, hint_off = 0, steps = 0;
                float base = 0.0f, scale = 0.0f;
                const uint32_t *col = nullptr;
            };
            std::vector<ColLayout> cl(ncols);
            std::vector<std::vector<uint32_t>> hint(ncols);
            for (uint32_t a = 0; a < ncols; ++a) {
                const ColumnInfo &ci_ = t->cols[cols[a].dim];
                cl[a].col = static_cast<const uint32_t *>(ci_.ptr);
                cl[a].type = (uint32_t)ci_.type;
                cl[a].m = (uint32_t)cols[a].cuts.size();
                // search hint over [min, max] in kHintBuckets equal value buckets, with the
                // bucket function the device evaluates (float: trunc((x - base) * scale),
                // clamped): bucket b starts at the number of cuts in lower buckets, and the
                // walk covers the most cuts one bucket holds; used when that stays short
                const std::vector<double> &cut = cols[a].cuts;
                const double mn = bound_value(ci_.min_bits, ci_.type), mx = bound_value(ci_.max_bits, ci_.type);
                const double range = mx - mn;
                const float base = (float)mn, scale = (float)(kHintBuckets / range);
                if (std::isfinite(range) && range > 0 && cl[a].m > 8 && std::isfinite(base) && std::isfinite(scale) &&
                    scale > 0.0f) {
                    auto bucket = [&](double v) {
                        const float xf = cl[a].type == MDRQ_F32 ? (float)v : (float)(int32_t)v;
                        const float tq = (xf - base) * scale;
                        if (!(tq >= 1.0f))
                            return 0u;  // negative, below one, or NaN
                        if (tq >= (float)(kHintBuckets - 1))
                            return kHintBuckets - 1;
                        return (uint32_t)tq;  // truncation, as __float2int_rz
                    };
                    std::vector<uint32_t> in_bucket(kHintBuckets, 0);
                    for (double c : cut)
                        ++in_bucket[bucket(c)];
                    uint32_t steps = 0;
                    for (uint32_t b = 0; b < kHintBuckets; ++b)
                        steps = std::max(steps, in_bucket[b]);
                    if (steps <= kMaxHintSteps) {
                        cl[a].base = base;
                        cl[a].scale = scale;
                        cl[a].steps = steps;
                        hint[a].assign(kHintBuckets / 2, 0);
                        uint32_t below = 0;
                        for (uint32_t b = 0; b < kHintBuckets; ++b) {
                            hint[a][b >> 1] |= below << ((b & 1) * 16);
                            below += in_bucket[b];
                        }
                    }
                }
            }
            // hints where the image budget leaves room for them (the rest search by bisection)
            {
                uint64_t base_words = (uint64_t)ncols * kColWords + 8;
                for (uint32_t a = 0; a < ncols; ++a)
                    base_words += cl[a].m + (uint64_t)(cl[a].m + 1) * kSharedG;
                for (uint32_t a = 0; a < ncols; ++a) {
                    if (hint[a].empty())
                        continue;
                    if (base_words + kHintBuckets / 2 > budget) {
                        hint[a].clear();
                        cl[a].base = cl[a].scale = 0.0f;
                        cl[a].steps = 0;
                        continue;
                    }
                    base_words += kHintBuckets / 2;
                    cl[a].hint_off = w;
                    w += kHintBuckets / 2;
                }
            }
            for (uint32_t a = 0; a < ncols; ++a) {
                cl[a].cut_off = w;
                w += cl[a].m;
            }
            w = (w + 3) & ~3u;
            for (uint32_t a = 0; a < ncols; ++a) {
                cl[a].tab_off = w;
                w += (cl[a].m + 1) * kSharedG;
            }
            img_words = (w + 3) & ~3u;
            if (img_words > budget || img_words > 0xffffu)
                return MDRQ_E_INVAL;  // cannot happen: the chunking bounded it
            max_img = std::max(max_img, img_words);
            plan.resize(img_off + img_words, 0);
            for (uint32_t a = 0; a < ncols; ++a) {
                ChunkCol cc;
                std::memset(&cc, 0, sizeof(cc));
                cc.w0 = cl[a].cut_off | (cl[a].m << 16) | (cl[a].steps << 25) | ((cl[a].type == MDRQ_I32 ? 1u : 0u) << 31);
                cc.w1 = cl[a].tab_off | (cl[a].hint_off << 16);
                cc.base = cl[a].base;
                cc.scale = cl[a].scale;
                cc.col = cl[a].col;
                std::memcpy(&plan[img_off + a * kColWords], &cc, sizeof(ChunkCol));
                for (size_t i = 0; i < hint[a].size(); ++i)
                    plan[img_off + cl[a].hint_off + i] = hint[a][i];
                for (uint32_t i = 0; i < cl[a].m; ++i)
                    plan[img_off + cl[a].cut_off + i] = to_bits(cols[a].cuts[i], (int32_t)cl[a].type);
            }
        }
        // intervals: word [a][k] = elo | ehi << 16, the elementary intervals query k accepts on column a
        const uint64_t iv_off = plan.size();
        plan.resize(iv_off + (uint64_t)ncols * ch.nq, 0);
        for (uint32_t a = 0; a < ncols; ++a)
            for (uint32_t k = 0; k < ch.nq; ++k)
                plan[iv_off + (uint64_t)a * ch.nq + k] = 0xffffu << 16;  // not constrained: all
        for (uint32_t k = 0; k < ch.nq; ++k) {
            const EncodedQuery &e = enc[live[ch.q0 + k]];
            for (size_t i = 0; i < e.dims.size(); ++i) {
                const uint32_t a = (uint32_t)slot[e.dims[i]];
                const ColumnInfo &c = t->cols[e.dims[i]];
                const std::vector<double> &cut = cols[a].cuts;
                const double lo = bound_value(e.preds[i].lo, c.type), hi = bound_value(e.preds[i].hi, c.type);
                const double mn = bound_value(c.min_bits, c.type), mx = bound_value(c.max_bits, c.type);
                // x >= lo iff e(x) > rank(lo); x <= hi iff e(x) <= rank(succ(hi))
                uint32_t elo = 0, ehi = (uint32_t)cut.size();
                if (lo > mn)
                    elo = (uint32_t)(std::lower_bound(cut.begin(), cut.end(), lo) - cut.begin()) + 1;
                if (hi < mx)
                    ehi = (uint32_t)(std::lower_bound(cut.begin(), cut.end(), successor(hi, c.type)) - cut.begin());
                plan[iv_off + (uint64_t)a * ch.nq + k] = elo | (ehi << 16);
            }
        }
        ChunkHdr &h = hdrs[ci];
        h.ncols = ncols;
        h.nq = ch.nq;
        h.q0 = ch.q0;
        h.img_words = img_words;
        h.img_off = img_off;
        h.iv_off = iv_off;
    }
    // coded columns: each column's sorted cut points, for the encode kernel
    std::vector<EncodeCol> ecols;
    uint32_t max_gcuts = 0;
    if (coded) {
        for (size_t gi = 0; gi < gdims.size(); ++gi) {
            const uint32_t j = gdims[gi];
            EncodeCol ec;
            ec.col = static_cast<const uint32_t *>(t->cols[j].ptr);
            ec.codes = S.codes + gi * code_stride;
            ec.cut_off = plan.size();
            ec.m = (uint32_t)gcuts[j].size();
            ec.type = (uint32_t)t->cols[j].type;
            ec.steps = 0;
            ec.base = ec.scale = 0.0f;
            ec.pad = 0;
            for (double v : gcuts[j])
                plan.push_back(to_bits(v, t->cols[j].type));
            // the bucket hint: cut points below each of kEncodeBuckets value buckets over
            // [min, max], with the kernel's float bucket function; kept when no bucket
            // holds more than kMaxHintSteps cut points
            const ColumnInfo &ci_ = t->cols[j];
            const double mn = bound_value(ci_.min_bits, ci_.type), mx = bound_value(ci_.max_bits, ci_.type);
            const double range = mx - mn;
            const float base = (float)mn, scale = (float)(kEncodeBuckets / range);
            if (std::isfinite(range) && range > 0 && ec.m > 8 && std::isfinite(base) && std::isfinite(scale) &&
                scale > 0.0f) {
                auto bucket = [&](double v) {
                    const float xf = ec.type == MDRQ_F32 ? (float)v : (float)(int32_t)v;
                    const float tq = (xf - base) * scale;
                    if (!(tq >= 1.0f))
                        return 0u;  // negative, below one, or NaN
                    if (tq >= (float)(kEncodeBuckets - 1))
                        return kEncodeBuckets - 1;
                    return (uint32_t)tq;  // truncation, as __float2int_rz
                };
                std::vector<uint32_t> in_bucket(kEncodeBuckets, 0);
                for (double c : gcuts[j])
                    ++in_bucket[bucket(c)];
                uint32_t steps = 0;
                for (uint32_t b = 0; b < kEncodeBuckets; ++b)
                    steps = std::max(steps, in_bucket[b]);
                if (steps <= kMaxHintSteps) {
                    ec.steps = steps;
                    ec.base = base;
                    ec.scale = scale;
                    const size_t h0 = plan.size();
                    plan.resize(h0 + kEncodeBuckets / 2, 0);
                    uint32_t below = 0;
                    for (uint32_t b = 0; b < kEncodeBuckets; ++b) {
                        plan[h0 + (b >> 1)] |= below << ((b & 1) * 16);
                        below += in_bucket[b];
                    }
                }
            }
            max_gcuts = std::max(max_gcuts, ec.m + (ec.scale != 0.0f ? kEncodeBuckets / 2 : 0u));
            ecols.push_back(ec);
        }
    }
    S.coded = coded;

    // ---- grid shape: the persistent grid at the occupancy of the largest image; enough
    // warp units to fill it (small tables get smaller units), at most kMaxUnitRows rows
    // each, unless the table sets the unit size (mdrq_set_shared_config)
    if (!S.smem_attr) {
        const int most = (int)kMaxImageWords * 4;
        const PassKernel all[] = {count_kernel(false, false), count_kernel(true, false), count_kernel(false, true),
                                  count_kernel(true, true),   write_kernel(true, false), write_kernel(false, false),
                                  write_kernel(false, true)};
        for (PassKernel k : all)
            if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, most) != cudaSuccess)
                return cuda_status(cudaGetLastError());
        if (cudaFuncSetAttribute(mdrq_shared_encode_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(kCodedMaxCuts + kEncodeBuckets / 2) * 4) != cudaSuccess)
            return cuda_status(cudaGetLastError());
        S.smem_attr = true;
        S.grid_scan = t->sm_count * 2;
    }
    // row masks kept between the passes when they fit: 16 bytes per row (rows padded to
    // a multiple of 32) and chunk
    const uint64_t mask_bytes = (uint64_t)chunks.size() * ((t->n + 31) & ~31ull) * sizeof(uint4);
    const uint64_t budget_bytes = t->shared_bits_budget == ~0ull ? kMaskBudgetBytes : t->shared_bits_budget;
    bool cached = mask_bytes <= budget_bytes && S.masks_cap >= mask_bytes;
    if (!cached && mask_bytes <= budget_bytes) {
        size_t free_b = 0, total_b = 0;
        if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess && mask_bytes <= free_b / 4)
            cached = grow_device((void **)&S.masks, &S.masks_cap, (size_t)mask_bytes) == MDRQ_OK;
        (void)cudaGetLastError();
    }
    max_img = (max_img + 1023) & ~1023u;  // whole 4 KiB steps: few distinct launch shapes
    const size_t smem = (size_t)max_img * 4;
    // the cached write pass holds no chunk image but the warps' id block buffers
    const size_t smem_write = cached ? kBlockBufferBytes : smem;
    // persistent grids of the two passes (their register budgets differ)
    int grid_pass = 0, grid_write = 0;
    const uint32_t key = max_img | (cached ? 0x80000000u : 0u) | (coded ? 0x40000000u : 0u);
    for (const auto &g : S.grid_for_words)
        if (g.first == key) {
            grid_pass = g.second.first;
            grid_write = g.second.second;
        }
    if (grid_pass == 0) {
        int bps = 0, bpw = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, count_kernel(cached, coded), kSharedThreads, smem) !=
                cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bpw, write_kernel(cached, coded), kSharedThreads,
                                                          smem_write) != cudaSuccess)
            return cuda_status(cudaGetLastError());
        grid_pass = t->sm_count * std::max(1, bps);
        grid_write = t->sm_count * std::max(1, bpw);
        S.grid_for_words.emplace_back(key, std::make_pair(grid_pass, grid_write));
    }
    uint64_t unit_rows;
    if (t->shared_unit_rows) {
        unit_rows = std::max<uint64_t>(32, ((uint64_t)t->shared_unit_rows + 31) & ~31ull);
    } else {
        const uint64_t want_units = (uint64_t)grid_pass * kSharedWarps * 4 / std::max<size_t>(1, chunks.size());
        unit_rows = (t->n + want_units - 1) / std::max<uint64_t>(1, want_units);
        unit_rows = std::min<uint64_t>(kMaxUnitRows, std::max<uint64_t>(kMinUnitRows, (unit_rows + 31) & ~31ull));
    }

    // ---- device buffers
    const uint64_t n_units = (t->n + unit_rows - 1) / unit_rows;
    const size_t hdr_bytes = hdrs.size() * sizeof(ChunkHdr);
    const size_t plan_bytes = plan.size() * 4;
    const size_t live_bytes = (size_t)nlive * 4;
    const size_t ecol_bytes = ecols.size() * sizeof(EncodeCol);
    int st = grow_device((void **)&S.plan, &S.plan_cap, std::max<size_t>(16, plan_bytes));
    if (st == MDRQ_OK && ecol_bytes)
        st = grow_device((void **)&S.ecols, &S.ecols_cap, ecol_bytes);
    if (st == MDRQ_OK)
        st = grow_device((void **)&S.chunks, &S.chunks_cap, hdr_bytes);
    if (st == MDRQ_OK)
        st = grow_device((void **)&S.live_orig, &S.live_cap, live_bytes);
    if (st == MDRQ_OK)
        st = grow_device((void **)&S.counts, &S.counts_cap, (size_t)nlive * n_units * 4);
    if (st == MDRQ_OK)
        st = grow_device((void **)&S.totals, &S.totals_cap, (size_t)nlive * 8);
    if (st == MDRQ_OK)
        st = grow_device((void **)&S.qbase, &S.qbase_cap, (size_t)nlive * 8);
    if (st == MDRQ_OK)
        st = grow_pinned((void **)&S.stage, &S.stage_cap, hdr_bytes + plan_bytes + live_bytes + 16 + ecol_bytes);
    if (st != MDRQ_OK)
        return st;
    std::memcpy(S.stage, hdrs.data(), hdr_bytes);
    std::memcpy(S.stage + hdr_bytes, plan.data(), plan_bytes);
    for (uint32_t i = 0; i < nlive; ++i)
        reinterpret_cast<uint32_t *>(S.stage + hdr_bytes + plan_bytes)[i] = live[i];
    MDRQ_TRY_STATUS(cudaMemcpyAsync(S.chunks, S.stage, hdr_bytes, cudaMemcpyHostToDevice, s));
    MDRQ_TRY_STATUS(cudaMemcpyAsync(S.plan, S.stage + hdr_bytes, plan_bytes, cudaMemcpyHostToDevice, s));
    MDRQ_TRY_STATUS(cudaMemcpyAsync(S.live_orig, S.stage + hdr_bytes + plan_bytes, live_bytes,
                                    cudaMemcpyHostToDevice, s));
    if (ecol_bytes) {
        unsigned char *es = S.stage + ((hdr_bytes + plan_bytes + live_bytes + 15) & ~(size_t)15);
        std::memcpy(es, ecols.data(), ecol_bytes);
        MDRQ_TRY_STATUS(cudaMemcpyAsync(S.ecols, es, ecol_bytes, cudaMemcpyHostToDevice, s));
    }

    SharedParams p;
    std::memset(&p, 0, sizeof(p));
    p.plan = S.plan;
    p.plan_rw = S.plan;
    p.chunks = S.chunks;
    p.nchunks = (uint32_t)hdrs.size();
    p.nlive = nlive;
    p.n = t->n;
    p.n_units = n_units;
    p.unit_rows = unit_rows;
    p.items = (uint64_t)hdrs.size() * ((n_units + kSharedWarps - 1) / kSharedWarps);
    p.counts = S.counts;
    p.totals = S.totals;
    p.qbase = S.qbase;
    p.live_orig = S.live_orig;
    p.offsets = t->offsets_dev;

    const uint32_t grid = (uint32_t)std::min<uint64_t>((uint64_t)grid_pass, p.items);
    mdrq_shared_tables_kernel<<<(uint32_t)hdrs.size() * max_cols, 256, 0, s>>>(p, max_cols);
    if (coded) {
        const uint32_t bx = std::max<uint32_t>(1, (uint32_t)t->sm_count * 8 / (uint32_t)ecols.size());
        mdrq_shared_encode_kernel<<<dim3(bx, (uint32_t)ecols.size()), 256, (size_t)max_gcuts * 4, s>>>(S.ecols, S.plan,
                                                                                                       t->n);
    }
    p.masks = cached ? S.masks : nullptr;
    count_kernel(cached, coded)<<<grid, kSharedThreads, smem, s>>>(p);
    mdrq_shared_scan_kernel<<<std::min<uint32_t>(nlive, (uint32_t)S.grid_scan), 1024, 0, s>>>(p);
    MDRQ_TRY_STATUS(cudaGetLastError());
    S.params = p;
    S.grid = (uint32_t)std::min<uint64_t>((uint64_t)grid_write, p.items);
    S.smem = smem_write;
    S.ready = true;
    t->last_launches += coded ? 4 : 3;
    if (t->timing)
        t->acc_kernels += coded ? 4 : 3;
    return MDRQ_OK;
}

// Pass 2 of the batch prepared by shared_scan_count. csr: place the answers as one CSR
// array (query bases from the counts, offsets_dev filled); otherwise S.qbase already
// holds every live query's base in ids (kSkipQuery: not written).
int shared_scan_write(mdrq_table *t, SharedScanState &S, uint32_t *ids, uint64_t capacity, bool csr, cudaStream_t s)
{
    if (!S.ready)
        return MDRQ_OK;
    SharedParams p = S.params;
    p.ids = ids;
    p.capacity = capacity;
    if (csr)
        mdrq_shared_qbase_kernel<<<1, 1024, 0, s>>>(p);
    write_kernel(p.masks != nullptr, S.coded)<<<S.grid, kSharedThreads, S.smem, s>>>(p);
    MDRQ_TRY_STATUS(cudaGetLastError());
    t->last_launches += csr ? 2 : 1;
    if (t->timing)
        t->acc_kernels += csr ? 2 : 1;
    return MDRQ_OK;
}

int shared_scan_batch(mdrq_table *t, const std::vector<EncodedQuery> &enc, const std::vector<uint32_t> &live,
                      uint32_t *ids, uint64_t capacity, cudaStream_t s)
{
    if (live.empty() || t->n == 0)
        return MDRQ_OK;
    if (!t->shared) {
        t->shared = shared_state_new();
        if (!t->shared)
            return MDRQ_E_NOMEM;
    }
    const int st = shared_scan_count(t, *t->shared, enc, live, s);
    if (st != MDRQ_OK)
        return st;
    return shared_scan_write(t, *t->shared, ids, capacity, true, s);
}

void shared_scan_free(mdrq_table *t)
{
    if (!t || !t->shared)
        return;
    shared_state_free(t->shared);
    t->shared = nullptr;
}

}  // namespace mdrq
