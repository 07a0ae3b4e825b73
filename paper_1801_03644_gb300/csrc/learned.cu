// Learned range narrower: a CDF model over a Z-order sort key limits each query's scan
// to a window of rows, which the windowed scan then checks exactly.
//
// The paper's scans visit every object (Sec. 2.2.4) and its index structures prune by
// space partitioning (Sec. 2.2.1-2.2.3). Here the table is stored sorted by a 32-bit
// Morton (Z-order) key over up to four float32 dimensions (8 bits each: the cell
// clamp(floor(x * 256), 0, 255)). The key is monotone in every one of those dimensions,
// so every object inside a query box has a key between the keys of the box's low and
// high corners, Z(lo) <= key <= Z(hi), and therefore lies in the run of rows between
// lower_bound(Z(lo)) and upper_bound(Z(hi)) of the sorted key column.
//
// A model predicts those two positions from the keys:
//  * PLA: a piecewise-linear function through every (n / S)-th (key, position) pair of
//    the sorted key column, S = 4096 segments, evaluated in FP32 (segment base exact).
//  * MLP: position / n ~ f(key / 2^32), f a 1-32-32-1 ReLU network in FP32, trained on
//    the device with Adam on an evenly spaced sample of (key, position) pairs.
// Its largest error over all n keys, eps, is measured exhaustively on the device. The
// window [pred(Z(lo)) - eps - 1, pred(Z(hi)) + eps + 2) is then checked against the key
// column and widened (doubling steps) until the key before it is < Z(lo) and the key
// after it is > Z(hi), which proves that no qualifying row lies outside it, whatever
// the model; a binary search inside it then finds lower_bound and upper_bound exactly.
// The windowed scan evaluates every predicate of the query on those rows only.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <thread>
#include <vector>

#include "mdrq.h"
#include "scan_kernel.cuh"
#include "table.h"

namespace mdrq {

constexpr uint32_t kPlaSegments = 4096;
constexpr int kMlpHidden = 32;
constexpr int kMlpParams = kMlpHidden + kMlpHidden + kMlpHidden * kMlpHidden + kMlpHidden + kMlpHidden + 1;
constexpr uint32_t kMlpSample = 1u << 20;   // training pairs
constexpr uint32_t kMlpBatch = 8192;        // pairs per step
constexpr uint32_t kMlpSteps = 3000;

// parameter layout of the MLP
constexpr int kW1 = 0, kB1 = kW1 + kMlpHidden, kW2 = kB1 + kMlpHidden, kB2 = kW2 + kMlpHidden * kMlpHidden,
              kW3 = kB2 + kMlpHidden, kB3 = kW3 + kMlpHidden;

struct LearnedModel {
    int kind = 0;                   // MDRQ_MODEL_PLA / MDRQ_MODEL_MLP
    uint32_t ndims = 0;
    uint32_t dims[4] = {0, 0, 0, 0};
    uint32_t *keys = nullptr;       // sorted key column (device)
    // PLA: segment i covers keys [knot_key[i], knot_key[i+1]) from position knot_pos[i]
    uint32_t segments = 0;
    unsigned long long *knot_key = nullptr;  // segments + 1 (last = max key + 1)
    unsigned long long *knot_pos = nullptr;  // segments + 1
    float *slope = nullptr;                  // segments
    float *mlp = nullptr;                    // kMlpParams
    unsigned long long max_error = 0;
    double train_ms = 0;
    // per-batch buffers
    DevWindow *windows = nullptr;
    size_t windows_cap = 0;
    unsigned long long *qkeys = nullptr;     // 2 per query: Z(lo), Z(hi)
    size_t qkeys_cap = 0;
    unsigned long long *total_tiles = nullptr;
    unsigned long long *scratch = nullptr;   // error / check words
    size_t last_nq = 0;                      // queries of the last chunk's windows
};

// ---------------------------------------------------------------- keys

__device__ __forceinline__ uint32_t zcell(float x)
{
    const float c = floorf(x * 256.0f);
    return c < 0.0f ? 0u : (c > 255.0f ? 255u : (uint32_t)c);
}

struct KeyCols {
    const float *col[4];
    uint32_t ndims;
};

__global__ void mdrq_zkey_kernel(KeyCols kc, uint64_t n, uint32_t *keys)
{
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t k = 0;
        for (uint32_t j = 0; j < kc.ndims; ++j) {
            const uint32_t c = zcell(kc.col[j][i]);
            for (int b = 0; b < 8; ++b)
                k |= ((c >> b) & 1u) << (4 * b + j);
        }
        keys[i] = k;
    }
}

// out[0] += rows i with keys[i - 1] > keys[i]
__global__ void mdrq_unsorted_kernel(const uint32_t *keys, uint64_t n, unsigned long long *out)
{
    unsigned long long bad = 0;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x + 1; i < n;
         i += (uint64_t)gridDim.x * blockDim.x)
        bad += keys[i - 1] > keys[i];
    for (int o = 16; o > 0; o >>= 1)
        bad += __shfl_xor_sync(0xffffffffu, bad, o);
    if ((threadIdx.x & 31) == 0 && bad)
        atomicAdd(out, bad);
}

// ---------------------------------------------------------------- PLA

// knots: position i * n / S and its key, plus the end knot (n, max key + 1)
__global__ void mdrq_pla_fit_kernel(const uint32_t *keys, uint64_t n, uint32_t S, unsigned long long *knot_key,
                                    unsigned long long *knot_pos, float *slope)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i > S)
        return;
    const unsigned long long pos = i < S ? (unsigned long long)i * n / S : n;
    const unsigned long long key = i < S ? keys[pos] : (unsigned long long)keys[n - 1] + 1;
    knot_key[i] = key;
    knot_pos[i] = pos;
    if (i < S) {
        const unsigned long long pos1 = (unsigned long long)(i + 1) * n / S;
        const unsigned long long key1 = i + 1 < S ? keys[pos1] : (unsigned long long)keys[n - 1] + 1;
        slope[i] = key1 > key ? (float)(pos1 - pos) / (float)(key1 - key) : 0.0f;
    }
}

__device__ __forceinline__ double pla_predict(const unsigned long long *knot_key, const unsigned long long *knot_pos,
                                              const float *slope, uint32_t S, unsigned long long k)
{
    // the last segment whose first key is <= k (segment 0 for keys below the first)
    uint32_t lo = 0, hi = S;
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (knot_key[mid] <= k)
            lo = mid;
        else
            hi = mid;
    }
    const unsigned long long k0 = knot_key[lo];
    const float dk = k >= k0 ? (float)(k - k0) : -(float)(k0 - k);
    return (double)knot_pos[lo] + (double)(dk * slope[lo]);
}

// ---------------------------------------------------------------- MLP

__device__ __forceinline__ float mlp_forward(const float *w, float u, float *h1, float *h2)
{
#pragma unroll
    for (int i = 0; i < kMlpHidden; ++i)
        h1[i] = fmaxf(0.0f, fmaf(w[kW1 + i], u, w[kB1 + i]));
#pragma unroll 4
    for (int o = 0; o < kMlpHidden; ++o) {
        float a = w[kB2 + o];
#pragma unroll
        for (int i = 0; i < kMlpHidden; ++i)
            a = fmaf(w[kW2 + o * kMlpHidden + i], h1[i], a);
        h2[o] = fmaxf(0.0f, a);
    }
    float y = w[kB3];
#pragma unroll
    for (int i = 0; i < kMlpHidden; ++i)
        y = fmaf(w[kW3 + i], h2[i], y);
    return y;
}

// deterministic initial weights: a counter-based hash (splitmix64) of the parameter index
__global__ void mdrq_mlp_init_kernel(float *w, float *adam)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kMlpParams)
        return;
    unsigned long long z = 0x9e3779b97f4a7c15ull * (unsigned long long)(i + 1);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    z ^= z >> 31;
    const float r = (float)(z >> 40) / (float)(1ull << 24) * 2.0f - 1.0f;  // U[-1, 1)
    float v;
    if (i < kB1)
        v = r * 2.0f;                                    // W1: fan-in 1
    else if (i < kW2)
        v = (float)(i - kB1) / kMlpHidden - 0.5f * r;    // b1: spread the kinks over [0, 1)
    else if (i < kB2)
        v = r * 0.3f;                                    // W2
    else if (i < kW3)
        v = 0.01f;                                       // b2
    else if (i < kB3)
        v = r * 0.3f;                                    // W3
    else
        v = 0.0f;                                        // b3
    w[i] = v;
    adam[2 * i] = 0.0f;
    adam[2 * i + 1] = 0.0f;
}

// Gradients of the mean squared error for one step: block b takes kMlpBlockPairs pairs,
// one thread each (forward and the backward pass to the hidden activations), stages the
// activations in shared memory, then sums every parameter's gradient over its pairs and
// writes the block's partial sums (summed in a fixed order by the update kernel).
constexpr int kMlpBlockPairs = 64;
constexpr int kMlpGradBlocks = kMlpBatch / kMlpBlockPairs;
constexpr int kPad = kMlpHidden + 1;

__global__ void __launch_bounds__(kMlpBlockPairs) mdrq_mlp_grad_kernel(const float *w, const uint32_t *keys,
                                                                        uint64_t n, uint32_t step, float *partial)
{
    __shared__ float s_w[kMlpParams];
    __shared__ float s_h1[kMlpBlockPairs][kPad], s_h2[kMlpBlockPairs][kPad];
    __shared__ float s_dh1[kMlpBlockPairs][kPad], s_dh2[kMlpBlockPairs][kPad];
    __shared__ float s_u[kMlpBlockPairs], s_dy[kMlpBlockPairs];
    for (int i = threadIdx.x; i < kMlpParams; i += blockDim.x)
        s_w[i] = w[i];
    __syncthreads();
    // pair j of this step: a multiplicative walk over the evenly spaced sample
    const uint32_t j = blockIdx.x * kMlpBlockPairs + threadIdx.x;
    const uint32_t sidx = (uint32_t)(((unsigned long long)step * kMlpBatch + j) * 2654435761ull % kMlpSample);
    const unsigned long long pos = (unsigned long long)sidx * n / kMlpSample;
    const float u = (float)keys[pos] * (1.0f / 4294967296.0f);
    const float target = (float)((double)pos / (double)n);
    float h1[kMlpHidden], h2[kMlpHidden];
    const float y = mlp_forward(s_w, u, h1, h2);
    const float dy = 2.0f * (y - target) / kMlpBatch;
    const int t = threadIdx.x;
    s_u[t] = u;
    s_dy[t] = dy;
#pragma unroll
    for (int i = 0; i < kMlpHidden; ++i) {
        s_h1[t][i] = h1[i];
        s_h2[t][i] = h2[i];
        s_dh2[t][i] = h2[i] > 0.0f ? dy * s_w[kW3 + i] : 0.0f;
    }
#pragma unroll 4
    for (int i = 0; i < kMlpHidden; ++i) {
        float a = 0.0f;
#pragma unroll
        for (int o = 0; o < kMlpHidden; ++o)
            a = fmaf(s_dh2[t][o], s_w[kW2 + o * kMlpHidden + i], a);
        s_dh1[t][i] = h1[i] > 0.0f ? a : 0.0f;
    }
    __syncthreads();
    float *out = partial + (size_t)blockIdx.x * kMlpParams;
    for (int prm = threadIdx.x; prm < kMlpParams; prm += blockDim.x) {
        float g = 0.0f;
        if (prm < kB1) {
            for (int s = 0; s < kMlpBlockPairs; ++s)
                g = fmaf(s_dh1[s][prm - kW1], s_u[s], g);
        } else if (prm < kW2) {
            for (int s = 0; s < kMlpBlockPairs; ++s)
                g += s_dh1[s][prm - kB1];
        } else if (prm < kB2) {
            const int o = (prm - kW2) / kMlpHidden, i = (prm - kW2) % kMlpHidden;
            for (int s = 0; s < kMlpBlockPairs; ++s)
                g = fmaf(s_dh2[s][o], s_h1[s][i], g);
        } else if (prm < kW3) {
            for (int s = 0; s < kMlpBlockPairs; ++s)
                g += s_dh2[s][prm - kB2];
        } else if (prm < kB3) {
            for (int s = 0; s < kMlpBlockPairs; ++s)
                g = fmaf(s_dy[s], s_h2[s][prm - kW3], g);
        } else {
            for (int s = 0; s < kMlpBlockPairs; ++s)
                g += s_dy[s];
        }
        out[prm] = g;
    }
}

// Adam step (beta1 0.9, beta2 0.999) with a cosine-decayed learning rate
__global__ void mdrq_mlp_adam_kernel(float *w, const float *partial, float *adam, uint32_t step)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kMlpParams)
        return;
    float g = 0.0f;
    for (int b = 0; b < kMlpGradBlocks; ++b)
        g += partial[(size_t)b * kMlpParams + i];
    const float lr = 1e-4f + 0.5f * (3e-3f - 1e-4f) * (1.0f + cospif((float)step / kMlpSteps));
    const float m = 0.9f * adam[2 * i] + 0.1f * g;
    const float v = 0.999f * adam[2 * i + 1] + 0.001f * g * g;
    adam[2 * i] = m;
    adam[2 * i + 1] = v;
    const float mh = m / (1.0f - powf(0.9f, (float)(step + 1)));
    const float vh = v / (1.0f - powf(0.999f, (float)(step + 1)));
    w[i] -= lr * mh / (sqrtf(vh) + 1e-8f);
}

__device__ __forceinline__ double mlp_predict(const float *w, uint64_t n, unsigned long long k)
{
    float h1[kMlpHidden], h2[kMlpHidden];
    const float u = (float)k * (1.0f / 4294967296.0f);
    return (double)mlp_forward(w, u, h1, h2) * (double)n;
}

// ---------------------------------------------------------------- error and windows

struct ModelView {
    int kind;
    uint32_t segments;
    const unsigned long long *knot_key;
    const unsigned long long *knot_pos;
    const float *slope;
    const float *mlp;
    uint64_t n;
};

__device__ __forceinline__ double model_predict(const ModelView &mv, const float *w_shared, unsigned long long k)
{
    if (mv.kind == MDRQ_MODEL_PLA)
        return pla_predict(mv.knot_key, mv.knot_pos, mv.slope, mv.segments, k);
    return mlp_predict(w_shared, mv.n, k);
}

// out[0] = max over rows i of ceil(|pred(keys[i]) - i|)
__global__ void __launch_bounds__(256) mdrq_model_error_kernel(ModelView mv, const uint32_t *keys,
                                                               unsigned long long *out)
{
    __shared__ float s_w[kMlpParams];
    if (mv.kind == MDRQ_MODEL_MLP)
        for (int i = threadIdx.x; i < kMlpParams; i += blockDim.x)
            s_w[i] = mv.mlp[i];
    __syncthreads();
    unsigned long long worst = 0;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < mv.n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const double e = fabs(model_predict(mv, s_w, keys[i]) - (double)i);
        const unsigned long long ce = e < 1.8e19 ? (unsigned long long)ceil(e) : ~0ull;
        worst = ce > worst ? ce : worst;
    }
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long x = __shfl_xor_sync(0xffffffffu, worst, o);
        worst = x > worst ? x : worst;
    }
    if ((threadIdx.x & 31) == 0)
        atomicMax(out, worst);
}

// first position in [lo, hi) whose key is > k (keys[lo..hi) sorted); keys[hi] unread
__device__ __forceinline__ unsigned long long upper_in(const uint32_t *keys, unsigned long long lo,
                                                       unsigned long long hi, unsigned long long k)
{
    while (lo < hi) {
        const unsigned long long mid = lo + ((hi - lo) >> 1);
        if ((unsigned long long)keys[mid] <= k)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

// first position in [lo, hi) whose key is >= k
__device__ __forceinline__ unsigned long long lower_in(const uint32_t *keys, unsigned long long lo,
                                                       unsigned long long hi, unsigned long long k)
{
    while (lo < hi) {
        const unsigned long long mid = lo + ((hi - lo) >> 1);
        if ((unsigned long long)keys[mid] < k)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

// Per query: the exact row run [lower_bound(Z(lo)), upper_bound(Z(hi))) of its key
// range, found from the model's window after the window has been proven to contain
// it; stored with its start rounded down to a multiple of 4 (128-bit loads).
__global__ void __launch_bounds__(128) mdrq_window_kernel(ModelView mv, const uint32_t *keys, unsigned long long eps,
                                                          const unsigned long long *qkeys, uint32_t nw,
                                                          DevWindow *windows, unsigned long long *probe_count)
{
    __shared__ float s_w[kMlpParams];
    if (mv.kind == MDRQ_MODEL_MLP)
        for (int i = threadIdx.x; i < kMlpParams; i += blockDim.x)
            s_w[i] = mv.mlp[i];
    __syncthreads();
    const uint32_t q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nw)
        return;
    const unsigned long long zlo = qkeys[2 * q], zhi = qkeys[2 * q + 1];
    const long long n = (long long)mv.n;
    const double plo = model_predict(mv, s_w, zlo), phi = model_predict(mv, s_w, zhi);
    long long w0 = (long long)floor(fmin(fmax(plo, -1.0), (double)n)) - (long long)eps - 1;
    long long w1 = (long long)ceil(fmin(fmax(phi, -1.0), (double)n)) + (long long)eps + 2;
    w0 = w0 < 0 ? 0 : (w0 > n ? n : w0);
    w1 = w1 < w0 ? w0 : (w1 > n ? n : w1);
    unsigned long long probes = 0;
    // prove: every row before w0 has key < Z(lo), every row from w1 on has key > Z(hi)
    for (long long step = 1; w0 > 0 && (unsigned long long)keys[w0 - 1] >= zlo; step *= 2) {
        w0 = w0 > step ? w0 - step : 0;
        ++probes;
    }
    for (long long step = 1; w1 < n && (unsigned long long)keys[w1] <= zhi; step *= 2) {
        w1 = w1 + step < n ? w1 + step : n;
        ++probes;
    }
    // the exact run inside the proven window
    const unsigned long long lb = lower_in(keys, (unsigned long long)w0, (unsigned long long)w1, zlo);
    const unsigned long long ub = upper_in(keys, lb, (unsigned long long)w1, zhi);
    DevWindow w = windows[q];  // query and last were set by the host
    w.row_begin = lb & ~3ull;
    w.row_first = lb;
    w.row_end = ub;
    w.tile_start = 0;
    w.tiles = 0;
    windows[q] = w;
    if (probes)
        atomicAdd(probe_count, probes);
}

// tiles per window (at least 1 for a query's last window) and their exclusive prefix;
// total into *total. One block.
__global__ void __launch_bounds__(1024) mdrq_window_tiles_kernel(DevWindow *windows, uint32_t nq, uint32_t tile_rows,
                                                                 unsigned long long *total)
{
    __shared__ unsigned long long s_warp[32];
    __shared__ unsigned long long s_carry;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0)
        s_carry = 0;
    __syncthreads();
    for (uint32_t base = 0; base < nq; base += blockDim.x) {
        const uint32_t i = base + threadIdx.x;
        unsigned long long v = 0;
        if (i < nq) {
            // rows from the aligned start; none when the window holds no row
            const unsigned long long rows =
                windows[i].row_end > windows[i].row_first ? windows[i].row_end - windows[i].row_begin : 0;
            v = rows ? (rows + tile_rows - 1) / tile_rows : (windows[i].last ? 1 : 0);
        }
        unsigned long long x = v;
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
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned long long y = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o)
                    w += y;
            }
            s_warp[lane] = w;
        }
        __syncthreads();
        const unsigned long long carry = s_carry;
        if (i < nq) {
            windows[i].tile_start = carry + (warp ? s_warp[warp - 1] : 0ull) + x - v;
            windows[i].tiles = v;
        }
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1)
            s_carry = carry + s_warp[31];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        *total = s_carry;
}

// ---------------------------------------------------------------- host

namespace {

ModelView view_of(const LearnedModel &m, uint64_t n)
{
    ModelView v;
    v.kind = m.kind;
    v.segments = m.segments;
    v.knot_key = m.knot_key;
    v.knot_pos = m.knot_pos;
    v.slope = m.slope;
    v.mlp = m.mlp;
    v.n = n;
    return v;
}

uint32_t host_cell(float x)
{
    const float c = std::floor(x * 256.0f);
    return c < 0.0f ? 0u : (c > 255.0f ? 255u : (uint32_t)c);
}

uint32_t host_key(const uint32_t *cells, uint32_t ndims)
{
    uint32_t k = 0;
    for (uint32_t j = 0; j < ndims; ++j)
        for (int b = 0; b < 8; ++b)
            k |= ((cells[j] >> b) & 1u) << (4 * b + j);
    return k;
}

constexpr uint32_t kRangesPerQuery = 1024;  // budget of the box decomposition

// The key ranges of a query box (cells clo..chi per key dimension). A node is a run of
// keys sharing their top `len` bits (len 0: all keys); its points' cells are fixed in
// the bits that prefix covers, so its cell extent per dimension is an interval. Nodes
// crossing the box's border are split in two by their next key bit, the shortest
// prefixes (largest runs) first; halves inside the box become ranges, halves outside it
// are dropped. When the budget is reached the crossing nodes left are kept whole (they
// cover keys outside the box, which the scan rejects). Ranges are returned sorted,
// adjacent ones merged.
void box_ranges(const uint32_t *clo, const uint32_t *chi, uint32_t nd, std::vector<std::pair<uint64_t, uint64_t>> &out)
{
    const uint32_t bits = 8 * nd;  // key bits in use: bit 4b + j for j < nd
    // key bit position of the i-th most significant bit in use
    auto bit_at = [&](uint32_t i) {
        const uint32_t b = 7 - i / nd, j = (nd - 1) - i % nd;
        return 4 * b + j;
    };
    struct Node {
        uint32_t len;      // bits fixed
        uint32_t lo[4];    // cell extent of the node per dimension
        uint32_t hi[4];
        uint32_t key;      // the fixed bits (others 0)
    };
    // 0: outside, 1: crossing, 2: inside
    auto classify = [&](const Node &x) {
        bool inside = true;
        for (uint32_t j = 0; j < nd; ++j) {
            if (x.hi[j] < clo[j] || x.lo[j] > chi[j])
                return 0;
            inside = inside && x.lo[j] >= clo[j] && x.hi[j] <= chi[j];
        }
        return inside ? 2 : 1;
    };
    // the node's key run: its fixed bits, then all zeros / all ones in the free used bits
    auto emit = [&](const Node &x) {
        uint64_t hi = x.key;
        for (uint32_t i = x.len; i < bits; ++i)
            hi |= 1ull << bit_at(i);
        out.emplace_back((uint64_t)x.key, hi);
    };
    out.clear();
    thread_local std::vector<Node> pending[33];  // reused: no allocation after warm-up
    for (auto &v : pending)
        v.clear();
    size_t npending = 0;
    Node root;
    root.len = 0;
    root.key = 0;
    for (uint32_t j = 0; j < 4; ++j) {
        root.lo[j] = 0;
        root.hi[j] = 255;
    }
    if (classify(root) == 2) {
        emit(root);
    } else {
        pending[0].push_back(root);
        npending = 1;
    }
    for (uint32_t len = 0; len < bits; ++len) {
        while (!pending[len].empty() && out.size() + npending + 1 <= kRangesPerQuery) {
            const Node f = pending[len].back();
            pending[len].pop_back();
            --npending;
            const uint32_t pos = bit_at(len);
            const uint32_t j = pos % 4, b = pos / 4;  // the split halves dimension j's cell range
            for (uint32_t half = 0; half < 2; ++half) {
                Node ch = f;
                ch.len = len + 1;
                ch.key = f.key | (half << pos);
                const uint32_t mid = f.lo[j] + (1u << b);  // first cell of the upper half
                if (half)
                    ch.lo[j] = mid;
                else
                    ch.hi[j] = mid - 1;
                const int cls = classify(ch);
                if (cls == 2)
                    emit(ch);
                else if (cls == 1) {
                    pending[len + 1].push_back(ch);
                    ++npending;
                }
            }
        }
        if (!pending[len].empty())
            break;  // budget reached
    }
    for (uint32_t len = 0; len <= bits; ++len)
        for (const Node &f : pending[len])
            emit(f);
    std::sort(out.begin(), out.end());
    size_t k = 0;
    for (size_t i = 0; i < out.size(); ++i) {
        if (k > 0 && out[i].first <= out[k - 1].second + 1)
            out[k - 1].second = std::max(out[k - 1].second, out[i].second);
        else
            out[k++] = out[i];
    }
    out.resize(k);
}

}  // namespace

void learned_free(mdrq_table *t)
{
    if (!t || !t->learned)
        return;
    LearnedModel &m = *t->learned;
    cudaFree(m.keys);
    cudaFree(m.knot_key);
    cudaFree(m.knot_pos);
    cudaFree(m.slope);
    cudaFree(m.mlp);
    cudaFree(m.windows);
    cudaFree(m.qkeys);
    cudaFree(m.total_tiles);
    cudaFree(m.scratch);
    delete t->learned;
    t->learned = nullptr;
}

int learn(mdrq_table *t, const uint32_t *dims, uint32_t ndims, int kind, cudaStream_t s)
{
    if (!t || !dims || ndims == 0 || ndims > 4 || (kind != MDRQ_MODEL_PLA && kind != MDRQ_MODEL_MLP) || t->n == 0)
        return MDRQ_E_INVAL;
    for (uint32_t j = 0; j < ndims; ++j)
        if (dims[j] >= t->d || t->cols[dims[j]].type != MDRQ_F32)
            return MDRQ_E_INVAL;
    learned_free(t);
    LearnedModel *m = new (std::nothrow) LearnedModel();
    if (!m)
        return MDRQ_E_NOMEM;
    t->learned = m;
    m->kind = kind;
    m->ndims = ndims;
    for (uint32_t j = 0; j < ndims; ++j)
        m->dims[j] = dims[j];
    const auto t0 = std::chrono::steady_clock::now();
    const uint64_t n = t->n;
    int st = MDRQ_OK;
    do {
        if ((st = cuda_status(cudaMalloc(&m->keys, n * 4))) ||
            (st = cuda_status(cudaMalloc(&m->scratch, 4 * 8))) ||
            (st = cuda_status(cudaMalloc(&m->total_tiles, 8))))
            break;
        KeyCols kc;
        for (int j = 0; j < 4; ++j)
            kc.col[j] = j < (int)ndims ? static_cast<const float *>(t->cols[dims[j]].ptr) : nullptr;
        kc.ndims = ndims;
        const uint32_t grid = (uint32_t)std::min<uint64_t>((n + 255) / 256, (uint64_t)t->sm_count * 16);
        mdrq_zkey_kernel<<<grid, 256, 0, s>>>(kc, n, m->keys);
        if ((st = cuda_status(cudaMemsetAsync(m->scratch, 0, 4 * 8, s))))
            break;
        mdrq_unsorted_kernel<<<grid, 256, 0, s>>>(m->keys, n, m->scratch);
        unsigned long long bad = 0;
        if ((st = cuda_status(cudaMemcpyAsync(&bad, m->scratch, 8, cudaMemcpyDeviceToHost, s))) ||
            (st = cuda_status(cudaStreamSynchronize(s))))
            break;
        if (bad) {
            st = MDRQ_E_INVAL;  // the rows are not in key order
            break;
        }
        if (kind == MDRQ_MODEL_PLA) {
            m->segments = (uint32_t)std::min<uint64_t>(kPlaSegments, n);
            if ((st = cuda_status(cudaMalloc(&m->knot_key, (m->segments + 1) * 8ull))) ||
                (st = cuda_status(cudaMalloc(&m->knot_pos, (m->segments + 1) * 8ull))) ||
                (st = cuda_status(cudaMalloc(&m->slope, m->segments * 4ull))))
                break;
            mdrq_pla_fit_kernel<<<(m->segments + 256) / 256, 256, 0, s>>>(m->keys, n, m->segments, m->knot_key,
                                                                         m->knot_pos, m->slope);
        } else {
            float *grad = nullptr, *adam = nullptr;
            if ((st = cuda_status(cudaMalloc(&m->mlp, kMlpParams * 4))) ||
                (st = cuda_status(cudaMalloc(&grad, (size_t)kMlpGradBlocks * kMlpParams * 4))) ||
                (st = cuda_status(cudaMalloc(&adam, kMlpParams * 8)))) {
                cudaFree(grad);
                cudaFree(adam);
                break;
            }
            const uint32_t pb = (kMlpParams + 255) / 256;
            mdrq_mlp_init_kernel<<<pb, 256, 0, s>>>(m->mlp, adam);
            for (uint32_t step = 0; step < kMlpSteps; ++step) {
                mdrq_mlp_grad_kernel<<<kMlpGradBlocks, kMlpBlockPairs, 0, s>>>(m->mlp, m->keys, n, step, grad);
                mdrq_mlp_adam_kernel<<<pb, 256, 0, s>>>(m->mlp, grad, adam, step);
            }
            st = cuda_status(cudaStreamSynchronize(s));
            cudaFree(grad);
            cudaFree(adam);
            if (st)
                break;
        }
        if ((st = cuda_status(cudaGetLastError())))
            break;
        // eps: the largest error over every key of the table
        if ((st = cuda_status(cudaMemsetAsync(m->scratch, 0, 8, s))))
            break;
        const ModelView mv = view_of(*m, n);
        mdrq_model_error_kernel<<<(uint32_t)t->sm_count * 8, 256, 0, s>>>(mv, m->keys, m->scratch);
        if ((st = cuda_status(cudaMemcpyAsync(&m->max_error, m->scratch, 8, cudaMemcpyDeviceToHost, s))) ||
            (st = cuda_status(cudaStreamSynchronize(s))))
            break;
    } while (0);
    if (st != MDRQ_OK) {
        learned_free(t);
        return st;
    }
    m->train_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return MDRQ_OK;
}

// Windows for the live queries (device), then one windowed scan launch.
int learned_batch(mdrq_table *t, const std::vector<EncodedQuery> &enc, const std::vector<uint32_t> &live,
                  uint32_t q0, uint32_t nlive, uint32_t *ids, uint64_t capacity, const unsigned long long *base_in,
                  cudaStream_t s)
{
    LearnedModel *m = t->learned;
    if (!m)
        return MDRQ_E_INVAL;
    if (nlive == 0)
        return MDRQ_OK;
    // Z(lo), Z(hi) of each key range of each query's box: cells of its bounds on the key
    // dimensions (the whole cell range where a key dimension is unconstrained)
    // the decompositions of the queries run on the host threads, then are concatenated
    // in query order
    std::vector<std::vector<std::pair<uint64_t, uint64_t>>> per_query(nlive);
    auto decompose = [&](uint32_t i) {
        const EncodedQuery &e = enc[live[q0 + i]];
        uint32_t clo[4] = {0, 0, 0, 0}, chi[4] = {0, 0, 0, 0};
        for (uint32_t j = 0; j < m->ndims; ++j) {
            clo[j] = 0;
            chi[j] = 255;
            for (size_t p = 0; p < e.dims.size(); ++p) {
                if (e.dims[p] == m->dims[j]) {
                    float lo, hi;
                    std::memcpy(&lo, &e.preds[p].lo, 4);
                    std::memcpy(&hi, &e.preds[p].hi, 4);
                    clo[j] = host_cell(lo);
                    chi[j] = host_cell(hi);
                }
            }
        }
        box_ranges(clo, chi, m->ndims, per_query[i]);
        if (per_query[i].empty())
            per_query[i].emplace_back(1, 0);  // no key can match: an empty window
    };
    const uint32_t nthreads =
        std::max(1u, std::min<uint32_t>(std::thread::hardware_concurrency(), (nlive + 63) / 64));
    if (nthreads <= 1) {
        for (uint32_t i = 0; i < nlive; ++i)
            decompose(i);
    } else {
        std::vector<std::thread> pool;
        for (uint32_t w = 0; w < nthreads; ++w)
            pool.emplace_back([&, w]() {
                for (uint32_t i = w; i < nlive; i += nthreads)
                    decompose(i);
            });
        for (std::thread &th : pool)
            th.join();
    }
    std::vector<unsigned long long> qk;
    std::vector<DevWindow> win;
    for (uint32_t i = 0; i < nlive; ++i) {
        const std::vector<std::pair<uint64_t, uint64_t>> &ranges = per_query[i];
        for (size_t r = 0; r < ranges.size(); ++r) {
            qk.push_back(ranges[r].first);
            qk.push_back(ranges[r].second);
            DevWindow w;
            std::memset(&w, 0, sizeof(w));
            w.query = i;
            w.last = r + 1 == ranges.size();
            win.push_back(w);
        }
    }
    const uint32_t nw = (uint32_t)win.size();
    int st = grow_device((void **)&m->windows, &m->windows_cap, (size_t)nw * sizeof(DevWindow));
    if (st == MDRQ_OK)
        st = grow_device((void **)&m->qkeys, &m->qkeys_cap, (size_t)nw * 16);
    if (st != MDRQ_OK)
        return st;
    MDRQ_TRY_STATUS(cudaMemcpyAsync(m->qkeys, qk.data(), qk.size() * 8, cudaMemcpyHostToDevice, s));
    MDRQ_TRY_STATUS(cudaMemcpyAsync(m->windows, win.data(), win.size() * sizeof(DevWindow), cudaMemcpyHostToDevice, s));
    MDRQ_TRY_STATUS(cudaMemsetAsync(m->scratch + 1, 0, 8, s));
    m->last_nq = nw;
    const ModelView mv = view_of(*m, t->n);
    mdrq_window_kernel<<<(nw + 127) / 128, 128, 0, s>>>(mv, m->keys, m->max_error, m->qkeys, nw, m->windows,
                                                        m->scratch + 1);
    constexpr uint32_t kTile = (uint32_t)kWarps * 4 * 128;
    mdrq_window_tiles_kernel<<<1, 1024, 0, s>>>(m->windows, nw, kTile, m->total_tiles);
    MDRQ_TRY_STATUS(cudaGetLastError());
    return launch_window_scan(t, q0, nlive, nw, ids, capacity, base_in, m->windows, m->total_tiles, s);
}

int learned_window_rows(mdrq_table *t, uint64_t *rows, uint64_t *probes)
{
    if (!t || !t->learned)
        return MDRQ_E_INVAL;
    LearnedModel &m = *t->learned;
    const size_t nq = m.last_nq;
    std::vector<DevWindow> w(nq);
    unsigned long long pr = 0;
    if (nq)
        MDRQ_TRY_STATUS(cudaMemcpy(w.data(), m.windows, nq * sizeof(DevWindow), cudaMemcpyDeviceToHost));
    MDRQ_TRY_STATUS(cudaMemcpy(&pr, m.scratch + 1, 8, cudaMemcpyDeviceToHost));
    uint64_t sum = 0;
    for (const DevWindow &x : w)
        sum += x.row_end - x.row_first;
    if (rows)
        *rows = sum;
    if (probes)
        *probes = pr;
    return MDRQ_OK;
}

int learned_info(const mdrq_table *t, uint64_t *max_error, uint32_t *segments, double *train_ms)
{
    if (!t || !t->learned)
        return MDRQ_E_INVAL;
    if (max_error)
        *max_error = t->learned->max_error;
    if (segments)
        *segments = t->learned->kind == MDRQ_MODEL_PLA ? t->learned->segments : 0;
    if (train_ms)
        *train_ms = t->learned->train_ms;
    return MDRQ_OK;
}

}  // namespace mdrq
