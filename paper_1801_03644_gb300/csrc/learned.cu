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
//  * MLP: a two-stage model whose first stage is a 1-32-32-1 ReLU network in FP32,
//    f(u) ~ position / n with u = (key - min key) / (max key - min key), trained on the
//    device with Adam on an evenly spaced sample of (key, position) pairs; it routes a
//    key to one of L = 2^18 leaves, leaf floor(f(u) * L), and the leaf's linear model
//    (through the first and the last (key, position) pair routed to it) predicts the
//    position. On its own the network cannot follow the staircase-shaped CDF of Z-order
//    keys over skewed columns (its error stays near a fifth of n); the leaves correct it
//    locally.
//  * NONE: no model; the window is the whole key column (the ablation that shows what
//    a model saves: only search probes, since the scanned runs are exact either way).
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
#include <vector>

#include "mdrq.h"
#include "scan_kernel.cuh"
#include "table.h"

namespace mdrq {

constexpr uint32_t kPlaSegments = 4096;
constexpr uint32_t kKeyCellBounds = 255;   // bounds of 256 cells per key dimension
constexpr uint32_t kMlpLeaves = 1u << 18;  // second stage of the MLP-rooted model
constexpr int kMlpHidden = 32;
constexpr int kMlpParams = kMlpHidden + kMlpHidden + kMlpHidden * kMlpHidden + kMlpHidden + kMlpHidden + 1;
constexpr uint32_t kMlpSample = 1u << 20;   // training pairs
constexpr uint32_t kMlpBatch = 8192;        // pairs per step
constexpr uint32_t kMlpSteps = 3000;

// parameter layout of the MLP
constexpr int kW1 = 0, kB1 = kW1 + kMlpHidden, kW2 = kB1 + kMlpHidden, kB2 = kW2 + kMlpHidden * kMlpHidden,
              kW3 = kB2 + kMlpHidden, kB3 = kW3 + kMlpHidden;

struct LearnedModel {
    int kind = 0;                   // MDRQ_MODEL_PLA / MDRQ_MODEL_MLP / MDRQ_MODEL_NONE
    uint32_t ndims = 0;
    uint32_t dims[4] = {0, 0, 0, 0};
    uint32_t *keys = nullptr;       // sorted key column (device)
    // PLA: segment i covers keys [knot_key[i], knot_key[i+1]) from position knot_pos[i];
    // MLP: leaf i predicts knot_pos[i] + (key - knot_key[i]) * slope[i]
    uint32_t segments = 0;
    unsigned long long key_min = 0;          // MLP input: (key - key_min) * key_inv
    float key_inv = 0.0f;
    std::vector<float> cells[4];             // each key dimension's cell bounds (empty: equal width)
    float *cells_dev = nullptr;              // the same, kKeyCellBounds per dimension (device)
    unsigned long long *knot_key = nullptr;  // segments + 1 (last = max key + 1)
    unsigned long long *knot_pos = nullptr;  // segments + 1
    float *slope = nullptr;                  // segments
    float *mlp = nullptr;                    // kMlpParams
    unsigned long long max_error = 0;
    double train_ms = 0;
    // per-batch buffers
    DevWindow *slots = nullptr;              // kRangesPerQuery windows per query, uncompacted
    size_t slots_cap = 0;
    DevWindow *windows = nullptr;            // the windows of all queries, compacted
    size_t windows_cap = 0;
    unsigned char *qaux = nullptr;           // per query: cells, counts, tiles, bases (device)
    size_t qaux_cap = 0;
    std::vector<uint32_t> qcells;            // per query: lo cells, hi cells (host staging)
    unsigned long long *totals = nullptr;    // [0] tiles, [1] windows of the last chunk
    unsigned long long *scratch = nullptr;   // error / check words
    bool have_windows = false;
};

// ---------------------------------------------------------------- keys

// Cell of a value on one key dimension: with bounds (255 ascending values), the number
// of bounds at or below x; without, clamp(floor(x * 256), 0, 255) in float32. Either is
// monotone in x, which is all the key's ordering argument needs.
__host__ __device__ __forceinline__ uint32_t zcell(float x, const float *bounds)
{
    if (bounds) {
        uint32_t c = 0;
        for (uint32_t step = 128; step; step >>= 1)
            if (c + step <= kKeyCellBounds && bounds[c + step - 1] <= x)
                c += step;
        return c;
    }
    const float c = floorf(x * 256.0f);
    return c < 0.0f ? 0u : (c > 255.0f ? 255u : (uint32_t)c);
}

struct KeyCols {
    const float *col[4];
    const float *bounds[4];  // device cell bounds of each key dimension, or null
    uint32_t ndims;
};

__global__ void mdrq_zkey_kernel(KeyCols kc, uint64_t n, uint32_t *keys)
{
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t k = 0;
        for (uint32_t j = 0; j < kc.ndims; ++j) {
            const uint32_t c = zcell(kc.col[j][i], kc.bounds[j]);
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
                                                                        uint64_t n, uint32_t step,
                                                                        unsigned long long key_min, float key_inv,
                                                                        float *partial)
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
    const float u = (float)((unsigned long long)keys[pos] - key_min) * key_inv;
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

// ---------------------------------------------------------------- error and windows

struct ModelView {
    int kind;
    uint32_t segments;                   // PLA segments or MLP leaves
    const unsigned long long *knot_key;  // PLA knots or leaf first keys
    const unsigned long long *knot_pos;
    const float *slope;
    const float *mlp;
    unsigned long long key_min;
    float key_inv;
    uint64_t n;
};

// the leaf the MLP-rooted model sends key k to (first stage, weights in shared memory)
__device__ __forceinline__ uint32_t mlp_leaf(const ModelView &mv, const float *w, unsigned long long k)
{
    float h1[kMlpHidden], h2[kMlpHidden];
    const float d = k >= mv.key_min ? (float)(k - mv.key_min) : -(float)(mv.key_min - k);
    const float y = mlp_forward(w, d * mv.key_inv, h1, h2) * (float)mv.segments;
    if (!(y > 0.0f))  // also NaN
        return 0;
    return y >= (float)(mv.segments - 1) ? mv.segments - 1 : (uint32_t)y;
}

__device__ __forceinline__ double model_predict(const ModelView &mv, const float *w_shared, unsigned long long k)
{
    if (mv.kind == MDRQ_MODEL_PLA)
        return pla_predict(mv.knot_key, mv.knot_pos, mv.slope, mv.segments, k);
    const uint32_t l = mlp_leaf(mv, w_shared, k);
    const unsigned long long k0 = mv.knot_key[l];
    const float dk = k >= k0 ? (float)(k - k0) : -(float)(k0 - k);
    return (double)mv.knot_pos[l] + (double)(dk * mv.slope[l]);
}

// MLP-rooted model, second stage: the first and the last row each leaf receives. One
// row per thread, a warp's rows consecutive: the lanes sent to one leaf form groups
// whose lowest lane holds the group's first row and highest lane its last.
__global__ void __launch_bounds__(256) mdrq_leaf_span_kernel(ModelView mv, const uint32_t *keys, uint32_t *first,
                                                             uint32_t *last)
{
    __shared__ float s_w[kMlpParams];
    for (int i = threadIdx.x; i < kMlpParams; i += blockDim.x)
        s_w[i] = mv.mlp[i];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    for (uint64_t base = (uint64_t)blockIdx.x * blockDim.x; base < mv.n; base += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t i = base + threadIdx.x;
        const bool live = i < mv.n;
        const uint32_t leaf = live ? mlp_leaf(mv, s_w, keys[i]) : 0xffffffffu;
        const uint32_t group = __match_any_sync(0xffffffffu, leaf);
        if (live && lane == __ffs(group) - 1)
            atomicMin(&first[leaf], (uint32_t)i);
        if (live && lane == 31 - __clz(group))
            atomicMax(&last[leaf], (uint32_t)i);
    }
}

// a leaf's line through its first and last (key, row) pair; an empty leaf is marked
// with first = 0xffffffff and filled in on the host
__global__ void mdrq_leaf_fit_kernel(const uint32_t *keys, const uint32_t *first, const uint32_t *last, uint32_t L,
                                     unsigned long long *leaf_key, unsigned long long *leaf_pos, float *slope)
{
    const uint32_t l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= L)
        return;
    const uint32_t p0 = first[l], p1 = last[l];
    if (p0 == 0xffffffffu) {
        leaf_key[l] = ~0ull;
        leaf_pos[l] = 0;
        slope[l] = 0.0f;
        return;
    }
    const unsigned long long k0 = keys[p0], k1 = keys[p1];
    leaf_key[l] = k0;
    leaf_pos[l] = p0;
    slope[l] = k1 > k0 ? (float)(p1 - p0) / (float)(k1 - k0) : 0.0f;
}

// out[0] = max over rows i of ceil(|pred(keys[i]) - i|)
__global__ void __launch_bounds__(256) mdrq_model_error_kernel(ModelView mv, const uint32_t *keys,
                                                               unsigned long long *out)
{
    if (mv.kind == MDRQ_MODEL_NONE) {
        if (blockIdx.x == 0 && threadIdx.x == 0)
            *out = mv.n;  // the window is the whole column
        return;
    }
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

// first position in [lo, hi) whose key is > k (keys[lo..hi) sorted); keys[hi] unread;
// *probes counts the keys read
__device__ __forceinline__ unsigned long long upper_in(const uint32_t *keys, unsigned long long lo,
                                                       unsigned long long hi, unsigned long long k,
                                                       unsigned long long *probes)
{
    while (lo < hi) {
        ++*probes;
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
                                                       unsigned long long hi, unsigned long long k,
                                                       unsigned long long *probes)
{
    while (lo < hi) {
        ++*probes;
        const unsigned long long mid = lo + ((hi - lo) >> 1);
        if ((unsigned long long)keys[mid] < k)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

// The exact row run [lower_bound(Z(lo)), upper_bound(Z(hi))) of one key range, found
// from the model's window after the window has been proven to contain it: every row
// before its start must have a key below Z(lo) and every row from its end on a key
// above Z(hi), else the window is widened by doubling steps (counted in *widenings).
// *probes counts every key read: the two checks, the widening steps and the searches.
__device__ __forceinline__ void prove_run(const ModelView &mv, const float *s_w, const uint32_t *keys,
                                          unsigned long long eps, unsigned long long zlo, unsigned long long zhi,
                                          unsigned long long *lb_out, unsigned long long *ub_out,
                                          unsigned long long *widenings, unsigned long long *probes)
{
    const long long n = (long long)mv.n;
    long long w0 = 0, w1 = n;
    if (mv.kind != MDRQ_MODEL_NONE) {
        const double plo = model_predict(mv, s_w, zlo), phi = model_predict(mv, s_w, zhi);
        w0 = (long long)floor(fmin(fmax(plo, -1.0), (double)n)) - (long long)eps - 1;
        w1 = (long long)ceil(fmin(fmax(phi, -1.0), (double)n)) + (long long)eps + 2;
        w0 = w0 < 0 ? 0 : (w0 > n ? n : w0);
        w1 = w1 < w0 ? w0 : (w1 > n ? n : w1);
    }
    for (long long step = 1; w0 > 0 && (++*probes, (unsigned long long)keys[w0 - 1] >= zlo); step *= 2) {
        w0 = w0 > step ? w0 - step : 0;
        ++*widenings;
    }
    for (long long step = 1; w1 < n && (++*probes, (unsigned long long)keys[w1] <= zhi); step *= 2) {
        w1 = w1 + step < n ? w1 + step : n;
        ++*widenings;
    }
    const unsigned long long lb = lower_in(keys, (unsigned long long)w0, (unsigned long long)w1, zlo, probes);
    *lb_out = lb;
    *ub_out = upper_in(keys, lb, (unsigned long long)w1, zhi, probes);
}

// ---------------------------------------------------------------- box decomposition

constexpr uint32_t kRangesPerQuery = 1024;  // budget of the box decomposition
constexpr int kBoxThreads = 256;
constexpr int kBoxPer = kRangesPerQuery / kBoxThreads;  // nodes (ranges) per thread
constexpr size_t kBoxSmem = 3 * (size_t)kRangesPerQuery * 16;

// inclusive scan of one value per thread over the block (kBoxThreads threads); ends
// with a barrier, so s_warp may be reused at once
__device__ __forceinline__ uint32_t block_incl_scan(uint32_t v, uint32_t *s_warp)
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
        uint32_t w = lane < kBoxThreads / 32 ? s_warp[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t x = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o)
                w += x;
        }
        if (lane < kBoxThreads / 32)
            s_warp[lane] = w;
    }
    __syncthreads();
    const uint32_t r = v + (warp ? s_warp[warp - 1] : 0u);
    __syncthreads();
    return r;
}

// A node of the key-bit tree: a run of keys sharing their top `len` used bits (`key`
// holds them, the other bits 0). Its points' cells are fixed in the bits the prefix
// covers, so per dimension j its cell extent is an interval: byte j of lo .. byte j of hi.
struct BoxNode {
    uint32_t key, lo, hi, len;
};

// key bit position of the i-th most significant used bit (bit 4b + j holds bit b of
// dimension j's cell)
__device__ __forceinline__ uint32_t used_bit(uint32_t i, uint32_t nd)
{
    return 4 * (7 - i / nd) + ((nd - 1) - i % nd);
}

// 0: outside the box, 1: crossing its border, 2: inside
__device__ __forceinline__ uint32_t classify_node(const BoxNode &x, uint32_t clo, uint32_t chi, uint32_t nd)
{
    bool inside = true;
    for (uint32_t j = 0; j < nd; ++j) {
        const uint32_t a = (x.lo >> (8 * j)) & 0xffu, b = (x.hi >> (8 * j)) & 0xffu;
        const uint32_t l = (clo >> (8 * j)) & 0xffu, h = (chi >> (8 * j)) & 0xffu;
        if (b < l || a > h)
            return 0;
        inside = inside && a >= l && b <= h;
    }
    return inside ? 2u : 1u;
}

// the lower (half 0) or upper (half 1) child: the node's next used bit fixed, which
// halves the cell extent of that bit's dimension
__device__ __forceinline__ BoxNode child_of(const BoxNode &f, uint32_t half, uint32_t nd)
{
    const uint32_t pos = used_bit(f.len, nd);
    const uint32_t j = pos % 4, b = pos / 4;
    BoxNode c = f;
    c.len = f.len + 1;
    c.key = f.key | (half << pos);
    const uint32_t mid = ((f.lo >> (8 * j)) & 0xffu) + (1u << b);  // first cell of the upper half
    if (half)
        c.lo = (f.lo & ~(0xffu << (8 * j))) | (mid << (8 * j));
    else
        c.hi = (f.hi & ~(0xffu << (8 * j))) | ((mid - 1) << (8 * j));
    return c;
}

// the node's key run: its fixed bits, then all zeros / all ones in the free used bits
__device__ __forceinline__ ulonglong2 run_of_node(const BoxNode &x, uint32_t nd)
{
    unsigned long long hi = x.key;
    for (uint32_t i = x.len; i < 8 * nd; ++i)
        hi |= 1ull << used_bit(i, nd);
    return make_ulonglong2(x.key, hi);
}

// One block per query (cells clo / chi: byte j = cell of the bound on key dimension j).
// (1) Its box as at most kRangesPerQuery key ranges: level by level, the nodes crossing
//     the border are split in key order while the range count stays within the budget
//     (inside halves become ranges, outside halves are dropped); once a split would pass
//     it, the crossing nodes left are kept whole, covering keys outside the box that the
//     scan rejects. Ranges are sorted and adjacent ones merged.
// (2) Per range, its exact row run through the model (prove_run) and its tiles of
//     tile_rows rows from the run's 128-aligned start; the query's last range gets one
//     tile even when empty, so that its answer is closed.
// Writes the query's windows to slots[q * kRangesPerQuery + i] with tile_start local to
// the query, the range count to counts[q] and the tile total to qtiles[q].
__global__ void __launch_bounds__(kBoxThreads) mdrq_box_windows_kernel(
    ModelView mv, const uint32_t *keys, unsigned long long eps, const uint32_t *qcells, uint32_t nd,
    uint32_t tile_rows, DevWindow *slots, uint32_t *counts, uint32_t *qtiles, unsigned long long *counters)
{
    extern __shared__ __align__(16) unsigned char s_raw[];
    BoxNode *cur = reinterpret_cast<BoxNode *>(s_raw);
    BoxNode *nxt = cur + kRangesPerQuery;
    ulonglong2 *out = reinterpret_cast<ulonglong2 *>(nxt + kRangesPerQuery);
    __shared__ uint32_t s_warp[kBoxThreads / 32];
    __shared__ uint32_t s_ncur, s_nout, s_split, s_ins, s_cross;

    const uint32_t q = blockIdx.x;
    const uint32_t clo = qcells[2 * q], chi = qcells[2 * q + 1];
    const uint32_t B = kRangesPerQuery, bits = 8 * nd;
    if (threadIdx.x == 0) {
        BoxNode root;
        root.key = 0;
        root.len = 0;
        root.lo = 0;
        root.hi = nd >= 4 ? 0xffffffffu : ((1u << (8 * nd)) - 1u);
        s_nout = 0;
        s_ncur = 0;
        const uint32_t c = classify_node(root, clo, chi, nd);
        if (c == 2)
            out[s_nout++] = run_of_node(root, nd);
        else if (c == 1)
            cur[s_ncur++] = root;
    }
    __syncthreads();
    // invariant: s_nout + s_ncur <= B
    for (uint32_t len = 0; len < bits && s_ncur > 0; ++len) {
        const uint32_t ncur = s_ncur, nout = s_nout;
        // per node: inside children (low 16 bits) and crossing children (high 16 bits)
        uint32_t packed[kBoxPer], cls[kBoxPer];
        uint32_t mine = 0;
#pragma unroll
        for (int k = 0; k < kBoxPer; ++k) {
            const uint32_t i = threadIdx.x * kBoxPer + k;
            packed[k] = 0;
            cls[k] = 0;
            if (i < ncur) {
                const uint32_t c0 = classify_node(child_of(cur[i], 0, nd), clo, chi, nd);
                const uint32_t c1 = classify_node(child_of(cur[i], 1, nd), clo, chi, nd);
                cls[k] = c0 | (c1 << 2);
                packed[k] = (c0 == 2) + (c1 == 2) + (((c0 == 1) + (c1 == 1)) << 16);
            }
            mine += packed[k];
        }
        if (threadIdx.x == 0)
            s_split = ncur;
        const uint32_t incl = block_incl_scan(mine, s_warp);
        // ranges if nodes 0..i are split: nout + (children of 0..i) + (ncur - i - 1);
        // nodes are split up to the first i at which that passes the budget
        uint32_t run = incl - mine;
#pragma unroll
        for (int k = 0; k < kBoxPer; ++k) {
            const uint32_t i = threadIdx.x * kBoxPer + k;
            run += packed[k];
            if (i < ncur && nout + ncur + (run & 0xffffu) + (run >> 16) - (i + 1) > B) {
                atomicMin(&s_split, i);
                break;
            }
        }
        __syncthreads();
        const uint32_t split = s_split;
        // children of the split nodes: inside ones appended to out, crossing ones to nxt,
        // both in key order; the totals are the scan value at node split - 1
        uint32_t pin = (incl - mine) & 0xffffu, pcr = (incl - mine) >> 16;
        run = incl - mine;
        if (split == 0 && threadIdx.x == 0) {
            s_ins = 0;
            s_cross = 0;
        }
#pragma unroll
        for (int k = 0; k < kBoxPer; ++k) {
            const uint32_t i = threadIdx.x * kBoxPer + k;
            run += packed[k];
            if (i < split) {
                const BoxNode f = cur[i];
                for (uint32_t h = 0; h < 2; ++h) {
                    const uint32_t c = (cls[k] >> (2 * h)) & 3u;
                    if (c == 2)
                        out[nout + pin++] = run_of_node(child_of(f, h, nd), nd);
                    else if (c == 1)
                        nxt[pcr++] = child_of(f, h, nd);
                }
                if (i + 1 == split) {
                    s_ins = run & 0xffffu;
                    s_cross = run >> 16;
                }
            }
        }
        __syncthreads();
        const uint32_t n_in = s_ins, n_cr = s_cross;
        if (split < ncur) {
            // budget reached: the unsplit nodes and the new crossing nodes are kept whole
            for (uint32_t i = split + threadIdx.x; i < ncur; i += blockDim.x)
                out[nout + n_in + (i - split)] = run_of_node(cur[i], nd);
            for (uint32_t i = threadIdx.x; i < n_cr; i += blockDim.x)
                out[nout + n_in + (ncur - split) + i] = run_of_node(nxt[i], nd);
            __syncthreads();
            if (threadIdx.x == 0) {
                s_nout = nout + n_in + (ncur - split) + n_cr;
                s_ncur = 0;
            }
        } else {
            for (uint32_t i = threadIdx.x; i < n_cr; i += blockDim.x)
                cur[i] = nxt[i];
            __syncthreads();
            if (threadIdx.x == 0) {
                s_nout = nout + n_in;
                s_ncur = n_cr;
            }
        }
        __syncthreads();
    }
    // (at full depth a node is one cell: inside or outside, so nothing is left in cur)
    const uint32_t nout = s_nout;
    // bitonic sort of out by first key (the runs are disjoint), padded with sentinels
    uint32_t n2 = 1;
    while (n2 < nout)
        n2 <<= 1;
    for (uint32_t i = nout + threadIdx.x; i < n2; i += blockDim.x)
        out[i] = make_ulonglong2(~0ull, ~0ull);
    __syncthreads();
    for (uint32_t k = 2; k <= n2; k <<= 1) {
        for (uint32_t jj = k >> 1; jj > 0; jj >>= 1) {
            for (uint32_t i = threadIdx.x; i < n2; i += blockDim.x) {
                const uint32_t l = i ^ jj;
                if (l > i) {
                    const ulonglong2 a = out[i], b = out[l];
                    if ((a.x > b.x) == ((i & k) == 0)) {
                        out[i] = b;
                        out[l] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
    // merge adjacent runs: a merged range starts where a run does not begin right after
    // the previous one's last key
    uint32_t starts = 0, flag[kBoxPer];
#pragma unroll
    for (int k = 0; k < kBoxPer; ++k) {
        const uint32_t i = threadIdx.x * kBoxPer + k;
        flag[k] = i < nout && (i == 0 || out[i].x != out[i - 1].y + 1);
        starts += flag[k];
    }
    const uint32_t nstart = block_incl_scan(starts, s_warp);
    // merged ranges go to cur (reinterpreted as key pairs: 16 bytes each, same size)
    ulonglong2 *rng = reinterpret_cast<ulonglong2 *>(cur);
    {
        uint32_t pos = nstart - starts;
#pragma unroll
        for (int k = 0; k < kBoxPer; ++k) {
            const uint32_t i = threadIdx.x * kBoxPer + k;
            if (i < nout) {
                if (flag[k])
                    rng[pos++].x = out[i].x;
                if (i + 1 == nout || out[i + 1].x != out[i].y + 1)
                    rng[pos - 1].y = out[i].y;
            }
        }
    }
    if (threadIdx.x == blockDim.x - 1)
        s_nout = nstart;
    __syncthreads();
    uint32_t nr = s_nout;
    const bool none = nr == 0;  // the box holds no cell: one empty window closes the query
    if (none)
        nr = 1;
    // the model's weights (MLP) go to out, which is free now
    float *s_w = reinterpret_cast<float *>(out);
    if (mv.kind == MDRQ_MODEL_MLP)
        for (int i = threadIdx.x; i < kMlpParams; i += blockDim.x)
            s_w[i] = mv.mlp[i];
    __syncthreads();
    // (2) row runs and tiles of the ranges, thread t taking ranges t*kBoxPer.. in key order
    unsigned long long lbs[kBoxPer], ubs[kBoxPer];
    uint32_t tl[kBoxPer], mytiles = 0;
    unsigned long long widenings = 0, probes = 0, ranges = 0;
#pragma unroll
    for (int k = 0; k < kBoxPer; ++k) {
        const uint32_t i = threadIdx.x * kBoxPer + k;
        lbs[k] = ubs[k] = 0;
        tl[k] = 0;
        if (i < nr) {
            if (!none) {
                prove_run(mv, s_w, keys, eps, rng[i].x, rng[i].y, &lbs[k], &ubs[k], &widenings, &probes);
                ++ranges;
            }
            const unsigned long long rows = ubs[k] > lbs[k] ? ubs[k] - (lbs[k] & ~127ull) : 0;
            tl[k] = rows ? (uint32_t)((rows + tile_rows - 1) / tile_rows) : (i + 1 == nr ? 1u : 0u);
        }
        mytiles += tl[k];
    }
    const uint32_t tincl = block_incl_scan(mytiles, s_warp);
    uint32_t tpos = tincl - mytiles;
    DevWindow *dst = slots + (size_t)q * kRangesPerQuery;
#pragma unroll
    for (int k = 0; k < kBoxPer; ++k) {
        const uint32_t i = threadIdx.x * kBoxPer + k;
        if (i < nr) {
            DevWindow w;
            w.row_begin = lbs[k] & ~127ull;  // whole 128-row groups (aligned 512-byte loads)
            w.row_first = lbs[k];
            w.row_end = ubs[k];
            w.tile_start = tpos;
            w.tiles = tl[k];
            w.query = q;
            w.last = i + 1 == nr;
            dst[i] = w;
        }
        tpos += tl[k];
    }
    if (threadIdx.x == blockDim.x - 1) {
        counts[q] = nr;
        qtiles[q] = tincl;
    }
    for (int o = 16; o > 0; o >>= 1) {
        widenings += __shfl_xor_sync(0xffffffffu, widenings, o);
        probes += __shfl_xor_sync(0xffffffffu, probes, o);
        ranges += __shfl_xor_sync(0xffffffffu, ranges, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (widenings)
            atomicAdd(&counters[0], widenings);
        if (probes)
            atomicAdd(&counters[1], probes);
        if (ranges)
            atomicAdd(&counters[2], ranges);
    }
}

// Exclusive scans of the per-query window counts and tile totals (one block):
// wbase[q], tbase[q]; totals[0] = all tiles, totals[1] = all windows.
__global__ void __launch_bounds__(1024) mdrq_window_base_kernel(const uint32_t *counts, const uint32_t *qtiles,
                                                                uint32_t nq, unsigned long long *wbase,
                                                                unsigned long long *tbase,
                                                                unsigned long long *totals)
{
    __shared__ unsigned long long s_warp[2][32];
    __shared__ unsigned long long s_carry[2];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x < 2)
        s_carry[threadIdx.x] = 0;
    __syncthreads();
    for (uint32_t b0 = 0; b0 < nq; b0 += blockDim.x) {
        const uint32_t i = b0 + threadIdx.x;
        const unsigned long long v0 = i < nq ? counts[i] : 0ull, v1 = i < nq ? qtiles[i] : 0ull;
        unsigned long long x0 = v0, x1 = v1;
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y0 = __shfl_up_sync(0xffffffffu, x0, o);
            const unsigned long long y1 = __shfl_up_sync(0xffffffffu, x1, o);
            if (lane >= o) {
                x0 += y0;
                x1 += y1;
            }
        }
        if (lane == 31) {
            s_warp[0][warp] = x0;
            s_warp[1][warp] = x1;
        }
        __syncthreads();
        if (warp < 2) {
            unsigned long long w = lane < (int)(blockDim.x / 32) ? s_warp[warp][lane] : 0ull;
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned long long y = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o)
                    w += y;
            }
            s_warp[warp][lane] = w;
        }
        __syncthreads();
        const unsigned long long c0 = s_carry[0], c1 = s_carry[1];
        if (i < nq) {
            wbase[i] = c0 + (warp ? s_warp[0][warp - 1] : 0ull) + x0 - v0;
            tbase[i] = c1 + (warp ? s_warp[1][warp - 1] : 0ull) + x1 - v1;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            s_carry[0] = c0 + s_warp[0][31];
            s_carry[1] = c1 + s_warp[1][31];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        totals[0] = s_carry[1];
        totals[1] = s_carry[0];
    }
}

// compaction: query q's windows from its slots to windows[wbase[q] ..], tile starts
// made global (one block per query)
__global__ void __launch_bounds__(256) mdrq_window_fill_kernel(const DevWindow *slots, uint32_t per_query,
                                                               const uint32_t *counts,
                                                               const unsigned long long *wbase,
                                                               const unsigned long long *tbase, DevWindow *windows)
{
    const uint32_t q = blockIdx.x;
    const uint32_t cnt = counts[q];
    const unsigned long long wb = wbase[q], tb = tbase[q];
    const DevWindow *src = slots + (size_t)q * per_query;
    for (uint32_t i = threadIdx.x; i < cnt; i += blockDim.x) {
        DevWindow w = src[i];
        w.tile_start += tb;
        windows[wb + i] = w;
    }
}

int window_list(uint32_t nq, uint32_t per_query, const uint32_t *counts, const uint32_t *qtiles,
                unsigned long long *wbase, unsigned long long *tbase, const DevWindow *slots, DevWindow *windows,
                unsigned long long *totals, cudaStream_t s)
{
    mdrq_window_base_kernel<<<1, 1024, 0, s>>>(counts, qtiles, nq, wbase, tbase, totals);
    mdrq_window_fill_kernel<<<nq, 256, 0, s>>>(slots, per_query, counts, wbase, tbase, windows);
    return cuda_status(cudaGetLastError());
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
    v.key_min = m.key_min;
    v.key_inv = m.key_inv;
    v.n = n;
    return v;
}

uint32_t host_cell(float x, const std::vector<float> &bounds)
{
    return zcell(x, bounds.empty() ? nullptr : bounds.data());
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
    cudaFree(m.cells_dev);
    cudaFree(m.slots);
    cudaFree(m.windows);
    cudaFree(m.qaux);
    cudaFree(m.totals);
    cudaFree(m.scratch);
    delete t->learned;
    t->learned = nullptr;
}

int learn(mdrq_table *t, const uint32_t *dims, uint32_t ndims, int kind, cudaStream_t s)
{
    if (!t || !dims || ndims == 0 || ndims > 4 ||
        (kind != MDRQ_MODEL_PLA && kind != MDRQ_MODEL_MLP && kind != MDRQ_MODEL_NONE) || t->n == 0)
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
            (st = cuda_status(cudaMalloc(&m->totals, 16))))
            break;
        KeyCols kc;
        bool any_cells = false;
        for (uint32_t j = 0; j < ndims; ++j) {
            m->cells[j] = t->cols[dims[j]].key_cells;
            any_cells = any_cells || !m->cells[j].empty();
        }
        if (any_cells) {
            if ((st = cuda_status(cudaMalloc(&m->cells_dev, 4ull * kKeyCellBounds * 4))))
                break;
            for (uint32_t j = 0; j < ndims; ++j)
                if (!m->cells[j].empty() &&
                    (st = cuda_status(cudaMemcpyAsync(m->cells_dev + j * kKeyCellBounds, m->cells[j].data(),
                                                      kKeyCellBounds * 4, cudaMemcpyHostToDevice, s))))
                    break;
            if (st)
                break;
        }
        for (int j = 0; j < 4; ++j) {
            kc.col[j] = j < (int)ndims ? static_cast<const float *>(t->cols[dims[j]].ptr) : nullptr;
            kc.bounds[j] = j < (int)ndims && !m->cells[j].empty() ? m->cells_dev + j * kKeyCellBounds : nullptr;
        }
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
        } else if (kind == MDRQ_MODEL_MLP) {
            // the network's input: the key normalised over the column's key range
            unsigned long long ends[2] = {0, 0};
            {
                uint32_t k0 = 0, k1 = 0;
                if ((st = cuda_status(cudaMemcpyAsync(&k0, m->keys, 4, cudaMemcpyDeviceToHost, s))) ||
                    (st = cuda_status(cudaMemcpyAsync(&k1, m->keys + n - 1, 4, cudaMemcpyDeviceToHost, s))) ||
                    (st = cuda_status(cudaStreamSynchronize(s))))
                    break;
                ends[0] = k0;
                ends[1] = k1;
            }
            m->key_min = ends[0];
            m->key_inv = ends[1] > ends[0] ? (float)(1.0 / (double)(ends[1] - ends[0])) : 0.0f;
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
                mdrq_mlp_grad_kernel<<<kMlpGradBlocks, kMlpBlockPairs, 0, s>>>(m->mlp, m->keys, n, step, m->key_min,
                                                                               m->key_inv, grad);
                mdrq_mlp_adam_kernel<<<pb, 256, 0, s>>>(m->mlp, grad, adam, step);
            }
            st = cuda_status(cudaStreamSynchronize(s));
            cudaFree(grad);
            cudaFree(adam);
            if (st)
                break;
            // second stage: each leaf's line through its first and last row
            const uint32_t L = kMlpLeaves;
            m->segments = L;
            uint32_t *span = nullptr;
            if ((st = cuda_status(cudaMalloc(&m->knot_key, L * 8ull))) ||
                (st = cuda_status(cudaMalloc(&m->knot_pos, L * 8ull))) ||
                (st = cuda_status(cudaMalloc(&m->slope, L * 4ull))) ||
                (st = cuda_status(cudaMalloc(&span, L * 8ull))))
                break;
            uint32_t *first = span, *last = span + L;
            if ((st = cuda_status(cudaMemsetAsync(first, 0xff, L * 4ull, s))) ||
                (st = cuda_status(cudaMemsetAsync(last, 0, L * 4ull, s)))) {
                cudaFree(span);
                break;
            }
            const ModelView mv0 = view_of(*m, n);
            mdrq_leaf_span_kernel<<<(uint32_t)t->sm_count * 8, 256, 0, s>>>(mv0, m->keys, first, last);
            mdrq_leaf_fit_kernel<<<(L + 255) / 256, 256, 0, s>>>(m->keys, first, last, L, m->knot_key, m->knot_pos,
                                                                  m->slope);
            // an empty leaf (reached by no key of the table, only by query keys) predicts
            // the row after the last row of the nearest non-empty leaf before it
            std::vector<uint32_t> hlast(L), hfirst(L);
            std::vector<unsigned long long> hkey(L), hpos(L);
            std::vector<float> hslope(L);
            if ((st = cuda_status(cudaMemcpyAsync(hfirst.data(), first, L * 4ull, cudaMemcpyDeviceToHost, s))) ||
                (st = cuda_status(cudaMemcpyAsync(hlast.data(), last, L * 4ull, cudaMemcpyDeviceToHost, s))) ||
                (st = cuda_status(cudaMemcpyAsync(hkey.data(), m->knot_key, L * 8ull, cudaMemcpyDeviceToHost, s))) ||
                (st = cuda_status(cudaMemcpyAsync(hpos.data(), m->knot_pos, L * 8ull, cudaMemcpyDeviceToHost, s))) ||
                (st = cuda_status(cudaMemcpyAsync(hslope.data(), m->slope, L * 4ull, cudaMemcpyDeviceToHost, s))) ||
                (st = cuda_status(cudaStreamSynchronize(s)))) {
                cudaFree(span);
                break;
            }
            cudaFree(span);
            unsigned long long after = 0;  // the row after the last non-empty leaf so far
            for (uint32_t l = 0; l < L; ++l) {
                if (hfirst[l] == 0xffffffffu) {
                    hkey[l] = 0;
                    hpos[l] = after;
                    hslope[l] = 0.0f;
                } else {
                    after = std::min<unsigned long long>((unsigned long long)hlast[l] + 1, n);
                }
            }
            if ((st = cuda_status(cudaMemcpyAsync(m->knot_key, hkey.data(), L * 8ull, cudaMemcpyHostToDevice, s))) ||
                (st = cuda_status(cudaMemcpyAsync(m->knot_pos, hpos.data(), L * 8ull, cudaMemcpyHostToDevice, s))) ||
                (st = cuda_status(cudaMemcpyAsync(m->slope, hslope.data(), L * 4ull, cudaMemcpyHostToDevice, s))) ||
                (st = cuda_status(cudaStreamSynchronize(s))))
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

// Windows for the live queries, built on the device, then one windowed scan launch.
int learned_batch(mdrq_table *t, const std::vector<EncodedQuery> &enc, const std::vector<uint32_t> &live,
                  uint32_t q0, uint32_t nlive, uint32_t *ids, uint64_t capacity, const unsigned long long *base_in,
                  cudaStream_t s)
{
    LearnedModel *m = t->learned;
    if (!m)
        return MDRQ_E_INVAL;
    if (nlive == 0)
        return MDRQ_OK;
    // cells of each query's bounds on the key dimensions (the whole cell range where a
    // key dimension is unconstrained), one byte per dimension
    m->qcells.resize(2 * (size_t)nlive);
    for (uint32_t i = 0; i < nlive; ++i) {
        const EncodedQuery &e = enc[live[q0 + i]];
        uint32_t clo = 0, chi = 0;
        for (uint32_t j = 0; j < m->ndims; ++j) {
            uint32_t cl = 0, ch = 255;
            for (size_t p = 0; p < e.dims.size(); ++p) {
                if (e.dims[p] == m->dims[j]) {
                    float lo, hi;
                    std::memcpy(&lo, &e.preds[p].lo, 4);
                    std::memcpy(&hi, &e.preds[p].hi, 4);
                    cl = host_cell(lo, m->cells[j]);
                    ch = host_cell(hi, m->cells[j]);
                }
            }
            clo |= cl << (8 * j);
            chi |= ch << (8 * j);
        }
        m->qcells[2 * i] = clo;
        m->qcells[2 * i + 1] = chi;
    }
    const size_t max_windows = (size_t)nlive * kRangesPerQuery;
    int st = grow_device((void **)&m->slots, &m->slots_cap, max_windows * sizeof(DevWindow));
    if (st == MDRQ_OK)
        st = grow_device((void **)&m->windows, &m->windows_cap, max_windows * sizeof(DevWindow));
    if (st == MDRQ_OK)
        st = grow_device((void **)&m->qaux, &m->qaux_cap, (size_t)nlive * 32);
    if (st != MDRQ_OK)
        return st;
    uint32_t *qcells = reinterpret_cast<uint32_t *>(m->qaux);
    uint32_t *counts = qcells + 2 * (size_t)nlive;
    uint32_t *qtiles = counts + nlive;
    unsigned long long *wbase = reinterpret_cast<unsigned long long *>(qtiles + nlive);
    unsigned long long *tbase = wbase + nlive;
    MDRQ_TRY_STATUS(cudaMemcpyAsync(qcells, m->qcells.data(), (size_t)nlive * 8, cudaMemcpyHostToDevice, s));
    MDRQ_TRY_STATUS(cudaMemsetAsync(m->scratch + 1, 0, 3 * 8, s));
    MDRQ_TRY_STATUS(cudaFuncSetAttribute(mdrq_box_windows_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kBoxSmem));
    const ModelView mv = view_of(*m, t->n);
    constexpr uint32_t kTile = (uint32_t)kWarps * 4 * 128;
    mdrq_box_windows_kernel<<<nlive, kBoxThreads, kBoxSmem, s>>>(mv, m->keys, m->max_error, qcells, m->ndims, kTile,
                                                                 m->slots, counts, qtiles, m->scratch + 1);
    st = window_list(nlive, kRangesPerQuery, counts, qtiles, wbase, tbase, m->slots, m->windows, m->totals, s);
    if (st != MDRQ_OK)
        return st;
    m->have_windows = true;
    return launch_window_scan(t, q0, nlive, max_windows, m->totals + 1, 0, 3, ids, capacity, base_in, m->windows,
                              m->totals, s);
}

int learned_window_rows(mdrq_table *t, uint64_t *rows, uint64_t *widenings)
{
    if (!t || !t->learned)
        return MDRQ_E_INVAL;
    LearnedModel &m = *t->learned;
    unsigned long long nw = 0, pr = 0;
    if (m.have_windows)
        MDRQ_TRY_STATUS(cudaMemcpy(&nw, m.totals + 1, 8, cudaMemcpyDeviceToHost));
    std::vector<DevWindow> w(nw);
    if (nw)
        MDRQ_TRY_STATUS(cudaMemcpy(w.data(), m.windows, nw * sizeof(DevWindow), cudaMemcpyDeviceToHost));
    MDRQ_TRY_STATUS(cudaMemcpy(&pr, m.scratch + 1, 8, cudaMemcpyDeviceToHost));
    uint64_t sum = 0;
    for (const DevWindow &x : w)
        sum += x.row_end > x.row_first ? x.row_end - x.row_first : 0;
    if (rows)
        *rows = sum;
    if (widenings)
        *widenings = pr;
    return MDRQ_OK;
}

int learned_search_info(mdrq_table *t, uint64_t *ranges, uint64_t *probes)
{
    if (!t || !t->learned)
        return MDRQ_E_INVAL;
    unsigned long long c[2] = {0, 0};  // probes, ranges
    MDRQ_TRY_STATUS(cudaMemcpy(c, t->learned->scratch + 2, 16, cudaMemcpyDeviceToHost));
    if (probes)
        *probes = c[0];
    if (ranges)
        *ranges = c[1];
    return MDRQ_OK;
}

int learned_export(const mdrq_table *t, mdrq_model_desc *desc, uint64_t *knot_key, uint64_t *knot_pos, float *slope,
                   float *mlp, uint32_t capacity)
{
    if (!t || !t->learned || !desc)
        return MDRQ_E_INVAL;
    const LearnedModel &m = *t->learned;
    std::memset(desc, 0, sizeof(*desc));
    desc->kind = m.kind;
    desc->segments = m.kind == MDRQ_MODEL_NONE ? 0 : m.segments;
    desc->mlp_params = m.kind == MDRQ_MODEL_MLP ? (uint32_t)kMlpParams : 0;
    desc->key_min = m.key_min;
    desc->key_inv = m.key_inv;
    desc->max_error = m.max_error;
    // PLA knots: segments + 1 (the end knot); MLP leaves: segments
    const uint32_t entries = m.kind == MDRQ_MODEL_PLA ? m.segments + 1 : (m.kind == MDRQ_MODEL_MLP ? m.segments : 0);
    if (entries && (knot_key || knot_pos || slope)) {
        if (capacity < entries)
            return MDRQ_E_CAPACITY;
        if (knot_key)
            MDRQ_TRY_STATUS(cudaMemcpy(knot_key, m.knot_key, entries * 8ull, cudaMemcpyDeviceToHost));
        if (knot_pos)
            MDRQ_TRY_STATUS(cudaMemcpy(knot_pos, m.knot_pos, entries * 8ull, cudaMemcpyDeviceToHost));
        if (slope)
            MDRQ_TRY_STATUS(cudaMemcpy(slope, m.slope, m.segments * 4ull, cudaMemcpyDeviceToHost));
    }
    if (mlp && m.kind == MDRQ_MODEL_MLP)
        MDRQ_TRY_STATUS(cudaMemcpy(mlp, m.mlp, kMlpParams * 4ull, cudaMemcpyDeviceToHost));
    return MDRQ_OK;
}

int set_key_cells(mdrq_table *t, uint32_t dim, const float *bounds, uint32_t nbounds)
{
    if (!t || dim >= t->d || (nbounds != 0 && (nbounds != kKeyCellBounds || !bounds)))
        return MDRQ_E_INVAL;
    if (nbounds == 0) {
        t->cols[dim].key_cells.clear();
        return MDRQ_OK;
    }
    for (uint32_t i = 0; i < nbounds; ++i)
        if (std::isnan(bounds[i]) || (i > 0 && !(bounds[i - 1] <= bounds[i])))
            return MDRQ_E_INVAL;
    t->cols[dim].key_cells.assign(bounds, bounds + nbounds);
    return MDRQ_OK;
}

int learned_info(const mdrq_table *t, uint64_t *max_error, uint32_t *segments, double *train_ms)
{
    if (!t || !t->learned)
        return MDRQ_E_INVAL;
    if (max_error)
        *max_error = t->learned->max_error;
    if (segments)
        *segments = t->learned->segments;
    if (train_ms)
        *train_ms = t->learned->train_ms;
    return MDRQ_OK;
}

}  // namespace mdrq
