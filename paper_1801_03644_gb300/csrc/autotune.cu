// Autotuner of the shared scan's shape (rows per warp unit, shared-memory budget per
// chunk) and of the AUTO mode's choice between the plain and the shared scan, by
// timing the caller's batch. Candidates are measured with CUDA events around the whole
// batch (host planning, copies and kernels), best of two runs each.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <vector>

#include "mdrq.h"
#include "table.h"

namespace mdrq {
namespace {

constexpr uint32_t kImageKibMin = 16, kImageKibMax = 208;

struct Timer {
    cudaEvent_t a = nullptr, b = nullptr;
    ~Timer()
    {
        if (a)
            cudaEventDestroy(a);
        if (b)
            cudaEventDestroy(b);
    }
};

// one timed run of the batch in the table's current mode and configuration
int timed_run(mdrq_table *t, const std::vector<EncodedQuery> &enc, const std::vector<uint32_t> &live, uint32_t nq,
              size_t npreds, uint32_t *ids, uint64_t capacity, std::vector<uint64_t> &offsets, Timer &tm,
              cudaStream_t s, double *ms)
{
    MDRQ_TRY_STATUS(cudaEventRecord(tm.a, s));
    int st = enqueue_batch(t, enc, live, nq, npreds, ids, capacity, s);
    if (st != MDRQ_OK)
        return st;
    MDRQ_TRY_STATUS(cudaEventRecord(tm.b, s));
    st = finish_batch(t, live, nq, offsets.data(), s);
    if (st != MDRQ_OK)
        return st;
    float f = 0;
    MDRQ_TRY_STATUS(cudaEventElapsedTime(&f, tm.a, tm.b));
    *ms = f;
    return offsets[nq] > capacity ? MDRQ_E_CAPACITY : MDRQ_OK;
}

int best_of_two(mdrq_table *t, const std::vector<EncodedQuery> &enc, const std::vector<uint32_t> &live, uint32_t nq,
                size_t npreds, uint32_t *ids, uint64_t capacity, std::vector<uint64_t> &offsets, Timer &tm,
                cudaStream_t s, double *ms)
{
    double a = 0, b = 0;
    int st = timed_run(t, enc, live, nq, npreds, ids, capacity, offsets, tm, s, &a);
    if (st == MDRQ_OK)
        st = timed_run(t, enc, live, nq, npreds, ids, capacity, offsets, tm, s, &b);
    *ms = std::min(a, b);
    return st;
}

int autotune(mdrq_table *t, const mdrq_qdesc *qs, uint32_t nq, cudaStream_t s, mdrq_tuning *out)
{
    std::vector<EncodedQuery> enc;
    std::vector<uint32_t> live;
    size_t npreds = 0;
    int st = encode_batch(t, qs, nq, enc, live, npreds);
    if (st != MDRQ_OK)
        return st;
    *out = mdrq_tuning{};
    out->mode = t->auto_mode >= 0 ? t->auto_mode : MDRQ_BATCH_PLAIN;
    if (live.empty())
        return MDRQ_OK;
    MDRQ_TRY_STATUS(cudaSetDevice(t->device));
    const int mode0 = t->batch_mode;
    const uint32_t unit0 = t->shared_unit_rows, img0 = t->shared_image_words;
    std::vector<uint64_t> offsets((size_t)nq + 1);
    Timer tm;
    MDRQ_TRY_STATUS(cudaEventCreate(&tm.a));
    MDRQ_TRY_STATUS(cudaEventCreate(&tm.b));
    uint32_t *ids = nullptr;
    auto restore = [&]() {
        t->batch_mode = mode0;
        t->shared_unit_rows = unit0;
        t->shared_image_words = img0;
        cudaFree(ids);
    };

    // the answer's size, from a shared-scan run with no room (it writes nothing)
    t->batch_mode = MDRQ_BATCH_SHARED;
    t->shared_unit_rows = 0;
    t->shared_image_words = 0;
    st = enqueue_batch(t, enc, live, nq, npreds, nullptr, 0, s);
    if (st == MDRQ_OK)
        st = finish_batch(t, live, nq, offsets.data(), s);
    if (st != MDRQ_OK) {
        restore();
        return st;
    }
    const uint64_t capacity = offsets[nq];
    if (capacity > 0 && cudaMalloc(&ids, (size_t)capacity * 4) != cudaSuccess) {
        (void)cudaGetLastError();
        restore();
        return MDRQ_E_NOMEM;
    }

    double plain = 0, shared_default = 0;
    t->batch_mode = MDRQ_BATCH_PLAIN;
    st = best_of_two(t, enc, live, nq, npreds, ids, capacity, offsets, tm, s, &plain);
    t->batch_mode = MDRQ_BATCH_SHARED;
    if (st == MDRQ_OK)
        st = best_of_two(t, enc, live, nq, npreds, ids, capacity, offsets, tm, s, &shared_default);
    if (st != MDRQ_OK) {
        restore();
        return st;
    }
    uint32_t best_unit = 0, best_img = 0, tried = 0;
    double best = shared_default;
    // unit sizes under the default budget, then budgets under the best unit size
    const uint32_t units[] = {512, 1024, 2048, 4096, 8192, 16384, 32768};
    for (uint32_t u : units) {
        if ((uint64_t)u * 64 > t->n && u != units[0])
            break;  // fewer than 64 units: the grid cannot fill
        t->shared_unit_rows = u;
        t->shared_image_words = 0;
        double ms = 0;
        st = best_of_two(t, enc, live, nq, npreds, ids, capacity, offsets, tm, s, &ms);
        if (st != MDRQ_OK) {
            restore();
            return st;
        }
        ++tried;
        if (ms < best) {
            best = ms;
            best_unit = u;
        }
    }
    const uint32_t budgets_kib[] = {24, 40, 96, 160};
    for (uint32_t kib : budgets_kib) {
        t->shared_unit_rows = best_unit;
        t->shared_image_words = kib * 256;
        double ms = 0;
        st = best_of_two(t, enc, live, nq, npreds, ids, capacity, offsets, tm, s, &ms);
        if (st != MDRQ_OK) {
            restore();
            return st;
        }
        ++tried;
        if (ms < best) {
            best = ms;
            best_img = kib * 256;
        }
    }
    restore();
    t->shared_unit_rows = best_unit;
    t->shared_image_words = best_img;
    t->auto_mode = best < plain ? MDRQ_BATCH_SHARED : MDRQ_BATCH_PLAIN;
    out->mode = t->auto_mode;
    out->unit_rows = best_unit;
    out->image_kib = best_img / 256;
    out->candidates = tried;
    out->plain_ms = plain;
    out->shared_default_ms = shared_default;
    out->shared_ms = best;
    return MDRQ_OK;
}

}  // namespace
}  // namespace mdrq

extern "C" {

int mdrq_set_shared_config(mdrq_table *t, uint32_t unit_rows, uint32_t image_kib)
{
    if (!t || (image_kib != 0 && (image_kib < mdrq::kImageKibMin || image_kib > mdrq::kImageKibMax)))
        return MDRQ_E_INVAL;
    t->shared_unit_rows = unit_rows == 0 ? 0 : std::max<uint32_t>(32, (unit_rows + 31) & ~31u);
    t->shared_image_words = image_kib * 256;
    return MDRQ_OK;
}

int mdrq_set_shared_bits_budget(mdrq_table *t, uint64_t max_bytes)
{
    if (!t)
        return MDRQ_E_INVAL;
    t->shared_bits_budget = max_bytes;
    return MDRQ_OK;
}

int mdrq_set_shared_codes(mdrq_table *t, int enable)
{
    if (!t)
        return MDRQ_E_INVAL;
    t->shared_coded = enable != 0;
    return MDRQ_OK;
}

int mdrq_autotune(mdrq_table *t, const mdrq_qdesc *qs, uint32_t nq, void *stream, mdrq_tuning *out)
{
    if (!t || !out || (nq > 0 && !qs))
        return MDRQ_E_INVAL;
    return mdrq::autotune(t, qs, nq, static_cast<cudaStream_t>(stream), out);
}

}  // extern "C"
