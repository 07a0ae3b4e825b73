// Serving loop: continuous batching of queries that arrive over time.
//
// The paper measures throughput over a fixed workload of queries (Sec. 7.1.2); a
// server answers queries as they come. Callers submit queries from any thread
// (mdrq_server_submit); a scheduler thread forms a batch from whatever has arrived,
// runs the shared scan's count phase, admits the batch's queries in arrival order
// while their exact answer sizes fit in the free part of a fixed device arena (the
// result-buffer budget), and runs the write phase straight into the admitted queries'
// arena slots. Queries that do not fit wait for the next batch, ahead of later arrivals.
// Two batches can be on the GPU at once, each with its own stream and scan state, so
// the next batch's count phase overlaps the current batch's write phase while new
// queries keep arriving. A completion thread waits on each batch's event, marks its
// queries answered (their latency ends there) and wakes waiters. Answers stay in the
// arena, as device memory, until the caller releases them.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdint>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "mdrq.h"
#include "table.h"

namespace mdrq {
namespace {

using Clock = std::chrono::steady_clock;

// Batches of at most this many queries are answered by the plain scan, whose cost
// follows the columns the queries read; the shared scan's two passes over every row of
// the table only pay for larger batches. The scratch answer buffer of a stream holds
// (that many) * n ids within kPlainServeScratchBytes, which lowers the limit on large
// tables (no plain path when not even one answer fits).
constexpr uint32_t kPlainServeMax = 12;
constexpr uint64_t kPlainServeScratchBytes = 1ull << 30;

struct Request {
    EncodedQuery enc;
    int status = 1;           // 1 waiting, 0 answered, < 0 failed
    uint64_t count = 0;       // answer length
    uint64_t slot = 0;        // arena word of the answer
    uint64_t words = 0;       // arena words held
    Clock::time_point t_submit, t_done;
};

// First-fit allocator of arena words, with coalescing of free neighbours.
class Arena {
public:
    void reset(uint64_t words)
    {
        free_.clear();
        if (words)
            free_[0] = words;
        used_ = 0;
    }
    bool alloc(uint64_t words, uint64_t &at)
    {
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= words) {
                at = it->first;
                const uint64_t rest = it->second - words;
                const uint64_t after = it->first + words;
                free_.erase(it);
                if (rest)
                    free_[after] = rest;
                used_ += words;
                return true;
            }
        }
        return false;
    }
    void release(uint64_t at, uint64_t words)
    {
        if (!words)
            return;
        used_ -= words;
        auto it = free_.emplace(at, words).first;
        auto next = std::next(it);
        if (next != free_.end() && it->first + it->second == next->first) {
            it->second += next->second;
            free_.erase(next);
        }
        if (it != free_.begin()) {
            auto prev = std::prev(it);
            if (prev->first + prev->second == it->first) {
                prev->second += it->second;
                free_.erase(it);
            }
        }
    }
    uint64_t used() const { return used_; }

private:
    std::map<uint64_t, uint64_t> free_;
    uint64_t used_ = 0;
};

struct InFlight {
    std::vector<uint64_t> tickets;
    int slot;
};

}  // namespace
}  // namespace mdrq

using namespace mdrq;

struct mdrq_server {
    mdrq_table *t = nullptr;
    uint32_t *arena_dev = nullptr;
    uint64_t arena_words = 0;
    uint32_t max_batch = 0;

    cudaStream_t stream[2] = {nullptr, nullptr};
    cudaEvent_t done_ev[2] = {nullptr, nullptr};
    SharedScanState *state[2] = {nullptr, nullptr};
    // small batches: a plain scan on a private table per stream into a scratch answer
    // buffer of kPlainServeMax * n ids, then copies into the admitted queries' slots
    mdrq_table *plain[2] = {nullptr, nullptr};
    uint32_t *scratch_ids[2] = {nullptr, nullptr};
    uint64_t scratch_cap = 0;
    uint32_t plain_max = 0;  // batches up to this size take the plain scan
    unsigned long long *host_buf[2] = {nullptr, nullptr};  // pinned: totals, then bases
    size_t host_cap[2] = {0, 0};
    bool busy[2] = {false, false};

    std::mutex mu;
    std::condition_variable cv_sched, cv_done, cv_flight;
    std::deque<uint64_t> pending;
    std::unordered_map<uint64_t, Request> reqs;
    std::deque<InFlight> inflight;
    Arena arena;
    uint64_t next_ticket = 1;
    bool stopping = false;
    bool scheduler_done = false;
    int fatal = MDRQ_OK;

    uint64_t batches = 0, deferred = 0, completed = 0;
    std::vector<double> latencies_us;

    std::thread scheduler, completer;
};

namespace {

void finish(mdrq_server *S, uint64_t ticket, int status, Clock::time_point now)
{
    Request &r = S->reqs[ticket];
    r.status = status;
    r.t_done = now;
    if (status == MDRQ_OK) {
        ++S->completed;
        S->latencies_us.push_back(std::chrono::duration<double, std::micro>(now - r.t_submit).count());
    }
}

void scheduler_main(mdrq_server *S)
{
    cudaSetDevice(S->t->device);
    std::vector<uint64_t> batch;
    std::vector<EncodedQuery> enc;
    std::vector<uint32_t> live;
    for (;;) {
        int k = -1;
        {
            std::unique_lock<std::mutex> lock(S->mu);
            S->cv_sched.wait(lock, [&] {
                return (S->stopping && S->pending.empty()) || S->fatal != MDRQ_OK ||
                       (!S->pending.empty() && (!S->busy[0] || !S->busy[1]));
            });
            if (S->fatal != MDRQ_OK) {
                // the GPU failed (here or in the completer): no further batch runs, and
                // the queries still waiting end with the failure's status instead of
                // leaving their waiters blocked; submit refuses new queries from now on
                const Clock::time_point now = Clock::now();
                while (!S->pending.empty()) {
                    finish(S, S->pending.front(), S->fatal, now);
                    S->pending.pop_front();
                }
                S->cv_done.notify_all();
                return;
            }
            if (S->pending.empty())
                return;  // stopping, nothing left
            k = S->busy[0] ? 1 : 0;
            batch.clear();
            while (!S->pending.empty() && batch.size() < S->max_batch) {
                batch.push_back(S->pending.front());
                S->pending.pop_front();
            }
            enc.clear();
            for (uint64_t tk : batch)
                enc.push_back(S->reqs[tk].enc);
            S->busy[k] = true;
        }
        live.resize(batch.size());
        for (size_t i = 0; i < live.size(); ++i)
            live[i] = (uint32_t)i;
        const size_t nb = batch.size();
        cudaStream_t st = S->stream[k];
        const bool plain = S->plain[k] && nb <= S->plain_max;

        // exact answer sizes of the batch: the shared scan's count phase, or for a small
        // batch the whole plain scan into the scratch buffer
        int rc = grow_pinned((void **)&S->host_buf[k], &S->host_cap[k], nb * 8 * 3 + 8);
        // host-side failure injection (mdrq_inject_fault): this batch's scratch
        // allocation fails before any of its GPU work is enqueued
        if (rc == MDRQ_OK && __atomic_exchange_n(&S->t->inject_nomem, 0, __ATOMIC_ACQ_REL))
            rc = MDRQ_E_NOMEM;
        unsigned long long *totals = S->host_buf[k], *bases = S->host_buf[k] + nb;
        uint64_t *offs = reinterpret_cast<uint64_t *>(S->host_buf[k] + 2 * nb);
        if (plain) {
            size_t npreds = 0;
            for (const EncodedQuery &e : enc)
                npreds += e.preds.size();
            if (rc == MDRQ_OK)
                rc = enqueue_batch(S->plain[k], enc, live, (uint32_t)nb, npreds, S->scratch_ids[k], S->scratch_cap,
                                   st);
            if (rc == MDRQ_OK)
                rc = finish_batch(S->plain[k], live, (uint32_t)nb, offs, st);
            for (size_t i = 0; rc == MDRQ_OK && i < nb; ++i)
                totals[i] = offs[i + 1] - offs[i];
        } else {
            if (rc == MDRQ_OK)
                rc = shared_scan_count(S->t, *S->state[k], enc, live, st);
            if (rc == MDRQ_OK)
                rc = cuda_status(
                    cudaMemcpyAsync(totals, shared_state_totals(S->state[k]), nb * 8, cudaMemcpyDeviceToHost, st));
            if (rc == MDRQ_OK)
                rc = cuda_status(cudaStreamSynchronize(st));
        }

        std::vector<uint64_t> admitted;
        bool wait_for_release = false;
        {
            std::lock_guard<std::mutex> lock(S->mu);
            ++S->batches;
            if (rc != MDRQ_OK) {
                S->fatal = rc;
                const Clock::time_point now = Clock::now();
                for (uint64_t tk : batch)
                    finish(S, tk, rc, now);
                S->busy[k] = false;
                S->cv_done.notify_all();
                continue;
            }
            // admission in arrival order by answer size; the rest waits, in order
            const Clock::time_point now = Clock::now();
            size_t i = 0;
            for (; i < nb; ++i) {
                Request &r = S->reqs[batch[i]];
                r.count = totals[i];
                if (r.count == 0) {
                    bases[i] = ~0ull;
                    finish(S, batch[i], MDRQ_OK, now);
                    continue;
                }
                uint64_t at = 0;
                if (!S->arena.alloc(r.count, at)) {
                    if (r.count > S->arena_words) {
                        bases[i] = ~0ull;
                        finish(S, batch[i], MDRQ_E_CAPACITY, now);  // can never fit
                        continue;
                    }
                    break;
                }
                r.slot = at;
                r.words = r.count;
                bases[i] = at;
                admitted.push_back(batch[i]);
            }
            for (size_t j = nb; j > i; --j) {
                S->pending.push_front(batch[j - 1]);
                ++S->deferred;
            }
            for (size_t j = i; j < nb; ++j)
                bases[j] = ~0ull;
            if (admitted.empty()) {
                S->busy[k] = false;
                if (i < nb && S->inflight.empty() && S->stopping) {
                    // stopping with answers that cannot fit until their holders release
                    // memory: those queries fail rather than wait forever
                    while (!S->pending.empty()) {
                        finish(S, S->pending.front(), MDRQ_E_CAPACITY, now);
                        S->pending.pop_front();
                    }
                }
                // nothing fitted: wait until answers are released. Counting the same
                // queries again before then would only repeat the count phase (its
                // sizes cannot change) and take HBM from the batch in flight.
                wait_for_release = i < nb;
            }
            S->cv_done.notify_all();
        }
        if (admitted.empty()) {
            if (wait_for_release) {
                std::unique_lock<std::mutex> lock(S->mu);
                const uint64_t used = S->arena.used();
                S->cv_sched.wait_for(lock, std::chrono::milliseconds(50), [&] {
                    return S->stopping || S->fatal != MDRQ_OK || S->arena.used() < used;
                });
            }
            continue;
        }
        // write phase straight into the arena slots (small batches: copies of the
        // admitted answers from the scratch buffer)
        if (plain) {
            rc = MDRQ_OK;
            for (size_t i = 0; i < nb && rc == MDRQ_OK; ++i)
                if (bases[i] != ~0ull)
                    rc = cuda_status(cudaMemcpyAsync(S->arena_dev + bases[i], S->scratch_ids[k] + offs[i],
                                                     (size_t)totals[i] * 4, cudaMemcpyDeviceToDevice, st));
        } else {
            rc = cuda_status(
                cudaMemcpyAsync(shared_state_qbase(S->state[k]), bases, nb * 8, cudaMemcpyHostToDevice, st));
            if (rc == MDRQ_OK)
                rc = shared_scan_write(S->t, *S->state[k], S->arena_dev, S->arena_words, false, st);
        }
        if (rc == MDRQ_OK)
            rc = cuda_status(cudaEventRecord(S->done_ev[k], st));
        std::lock_guard<std::mutex> lock(S->mu);
        if (rc != MDRQ_OK) {
            S->fatal = rc;
            const Clock::time_point now = Clock::now();
            for (uint64_t tk : admitted)
                finish(S, tk, rc, now);
            S->busy[k] = false;
            S->cv_done.notify_all();
            continue;
        }
        S->inflight.push_back(InFlight{admitted, k});
        S->cv_flight.notify_all();
    }
}

void completer_main(mdrq_server *S)
{
    cudaSetDevice(S->t->device);
    for (;;) {
        InFlight f;
        {
            std::unique_lock<std::mutex> lock(S->mu);
            S->cv_flight.wait(lock, [&] { return !S->inflight.empty() || S->scheduler_done; });
            if (S->inflight.empty())
                return;
            f = S->inflight.front();
        }
        const int rc = cuda_status(cudaEventSynchronize(S->done_ev[f.slot]));
        std::lock_guard<std::mutex> lock(S->mu);
        const Clock::time_point now = Clock::now();
        for (uint64_t tk : f.tickets)
            finish(S, tk, rc, now);
        if (rc != MDRQ_OK)
            S->fatal = rc;
        S->inflight.pop_front();
        S->busy[f.slot] = false;
        S->cv_done.notify_all();
        S->cv_sched.notify_all();
    }
}

void server_destroy(mdrq_server *S)
{
    for (int k = 0; k < 2; ++k) {
        if (S->state[k])
            shared_state_free(S->state[k]);
        free_shadow(S->plain[k]);
        cudaFree(S->scratch_ids[k]);
        if (S->stream[k])
            cudaStreamDestroy(S->stream[k]);
        if (S->done_ev[k])
            cudaEventDestroy(S->done_ev[k]);
        cudaFreeHost(S->host_buf[k]);
    }
    cudaFree(S->arena_dev);
    (void)cudaGetLastError();
    delete S;
}

}  // namespace

extern "C" {

int mdrq_server_start(mdrq_table *t, uint64_t result_bytes, uint32_t max_batch, mdrq_server **out)
{
    if (!t || !out || result_bytes < 4 || max_batch == 0)
        return MDRQ_E_INVAL;
    *out = nullptr;
    mdrq_server *S = new (std::nothrow) mdrq_server();
    if (!S)
        return MDRQ_E_NOMEM;
    S->t = t;
    S->max_batch = max_batch;
    S->arena_words = result_bytes / 4;
    int rc = cuda_status(cudaSetDevice(t->device));
    if (rc == MDRQ_OK)
        rc = cuda_status(cudaMalloc(&S->arena_dev, S->arena_words * 4));
    for (int k = 0; k < 2 && rc == MDRQ_OK; ++k) {
        rc = cuda_status(cudaStreamCreateWithFlags(&S->stream[k], cudaStreamNonBlocking));
        if (rc == MDRQ_OK)
            rc = cuda_status(cudaEventCreateWithFlags(&S->done_ev[k], cudaEventDisableTiming));
        if (rc == MDRQ_OK) {
            S->state[k] = shared_state_new();
            if (!S->state[k])
                rc = MDRQ_E_NOMEM;
        }
        S->plain_max = t->n > 0 ? (uint32_t)std::min<uint64_t>(kPlainServeMax, kPlainServeScratchBytes / (t->n * 4)) : 0;
        if (rc == MDRQ_OK && S->plain_max > 0) {
            S->scratch_cap = (uint64_t)S->plain_max * t->n;
            rc = make_shadow(t, S->stream[k], &S->plain[k]);
            if (rc == MDRQ_OK) {
                S->plain[k]->batch_mode = MDRQ_BATCH_PLAIN;
                // small latency-bound batches: ordered in the scan, no staging memory
                S->plain[k]->output_order = MDRQ_ORDER_LOOKBACK;
                rc = cuda_status(cudaMalloc(&S->scratch_ids[k], S->scratch_cap * 4));
            }
        }
    }
    if (rc == MDRQ_OK)
        rc = cuda_status(cudaDeviceSynchronize());  // the private tables' scratch is cleared
    if (rc != MDRQ_OK) {
        server_destroy(S);
        return rc;
    }
    S->arena.reset(S->arena_words);
    S->scheduler = std::thread(scheduler_main, S);
    S->completer = std::thread(completer_main, S);
    *out = S;
    return MDRQ_OK;
}

int mdrq_server_submit(mdrq_server *S, const mdrq_pred *preds, uint32_t npreds, uint64_t *ticket)
{
    if (!S || !ticket)
        return MDRQ_E_INVAL;
    EncodedQuery e;
    const int rc = encode_query(S->t, preds, npreds, e);
    if (rc != MDRQ_OK)
        return rc;
    std::lock_guard<std::mutex> lock(S->mu);
    if (S->stopping)
        return MDRQ_E_INVAL;
    if (S->fatal != MDRQ_OK)
        return S->fatal;
    const uint64_t tk = S->next_ticket++;
    Request &r = S->reqs[tk];
    r.t_submit = Clock::now();
    if (e.empty || S->t->n == 0) {
        finish(S, tk, MDRQ_OK, r.t_submit);  // proven empty on the host
    } else {
        r.enc = std::move(e);
        S->pending.push_back(tk);
        S->cv_sched.notify_one();
    }
    *ticket = tk;
    return MDRQ_OK;
}

int mdrq_server_wait(mdrq_server *S, uint64_t ticket, int64_t timeout_us, const uint32_t **ids, uint64_t *count,
                     double *latency_us)
{
    if (!S)
        return MDRQ_E_INVAL;
    std::unique_lock<std::mutex> lock(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end())
        return MDRQ_E_INVAL;
    auto ready = [&] {
        auto f = S->reqs.find(ticket);
        return f == S->reqs.end() || f->second.status != 1;
    };
    if (timeout_us < 0)
        S->cv_done.wait(lock, ready);
    else if (!S->cv_done.wait_for(lock, std::chrono::microseconds(timeout_us), ready))
        return MDRQ_E_TIMEOUT;
    it = S->reqs.find(ticket);
    if (it == S->reqs.end())
        return MDRQ_E_INVAL;  // released meanwhile by another thread
    const Request &r = it->second;
    if (ids)
        *ids = r.count && r.status == MDRQ_OK ? S->arena_dev + r.slot : nullptr;
    if (count)
        *count = r.count;
    if (latency_us)
        *latency_us = std::chrono::duration<double, std::micro>(r.t_done - r.t_submit).count();
    return r.status;
}

int mdrq_server_submit_batch(mdrq_server *S, const mdrq_qdesc *qs, uint32_t nq, uint64_t *tickets)
{
    if (!S || (nq > 0 && (!qs || !tickets)))
        return MDRQ_E_INVAL;
    std::vector<EncodedQuery> enc(nq);
    for (uint32_t i = 0; i < nq; ++i) {
        if (qs[i].reserved != 0)
            return MDRQ_E_INVAL;
        const int rc = encode_query(S->t, qs[i].preds, qs[i].npreds, enc[i]);
        if (rc != MDRQ_OK)
            return rc;
    }
    std::lock_guard<std::mutex> lock(S->mu);
    if (S->stopping)
        return MDRQ_E_INVAL;
    if (S->fatal != MDRQ_OK)
        return S->fatal;
    const Clock::time_point now = Clock::now();
    for (uint32_t i = 0; i < nq; ++i) {
        const uint64_t tk = S->next_ticket++;
        Request &r = S->reqs[tk];
        r.t_submit = now;
        if (enc[i].empty || S->t->n == 0) {
            finish(S, tk, MDRQ_OK, now);
        } else {
            r.enc = std::move(enc[i]);
            S->pending.push_back(tk);
        }
        tickets[i] = tk;
    }
    S->cv_sched.notify_one();
    return MDRQ_OK;
}

int mdrq_server_wait_many(mdrq_server *S, const uint64_t *tickets, uint32_t n, int64_t timeout_us, int *status,
                          uint64_t *counts, double *latency_us, int release)
{
    if (!S || (n > 0 && !tickets))
        return MDRQ_E_INVAL;
    std::unique_lock<std::mutex> lock(S->mu);
    for (uint32_t i = 0; i < n; ++i)
        if (S->reqs.find(tickets[i]) == S->reqs.end())
            return MDRQ_E_INVAL;
    auto all_done = [&] {
        for (uint32_t i = 0; i < n; ++i) {
            auto f = S->reqs.find(tickets[i]);
            if (f != S->reqs.end() && f->second.status == 1)
                return false;
        }
        return true;
    };
    if (timeout_us < 0)
        S->cv_done.wait(lock, all_done);
    else if (!S->cv_done.wait_for(lock, std::chrono::microseconds(timeout_us), all_done))
        return MDRQ_E_TIMEOUT;
    bool freed = false;
    for (uint32_t i = 0; i < n; ++i) {
        auto it = S->reqs.find(tickets[i]);
        if (it == S->reqs.end()) {
            if (status)
                status[i] = MDRQ_E_INVAL;  // released meanwhile by another thread
            continue;
        }
        const Request &r = it->second;
        if (status)
            status[i] = r.status;
        if (counts)
            counts[i] = r.count;
        if (latency_us)
            latency_us[i] = std::chrono::duration<double, std::micro>(r.t_done - r.t_submit).count();
        if (release) {
            S->arena.release(r.slot, r.words);
            S->reqs.erase(it);
            freed = true;
        }
    }
    if (freed)
        S->cv_sched.notify_all();
    return MDRQ_OK;
}

int mdrq_server_release(mdrq_server *S, uint64_t ticket)
{
    if (!S)
        return MDRQ_E_INVAL;
    std::lock_guard<std::mutex> lock(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end() || it->second.status == 1)
        return MDRQ_E_INVAL;
    S->arena.release(it->second.slot, it->second.words);
    S->reqs.erase(it);
    S->cv_sched.notify_all();
    return MDRQ_OK;
}

int mdrq_server_stats(mdrq_server *S, uint64_t *completed, uint64_t *batches, uint64_t *deferred, double *p50_us,
                      double *p99_us)
{
    if (!S)
        return MDRQ_E_INVAL;
    std::lock_guard<std::mutex> lock(S->mu);
    std::vector<double> l = S->latencies_us;
    std::sort(l.begin(), l.end());
    auto pct = [&](double p) { return l.empty() ? 0.0 : l[std::min(l.size() - 1, (size_t)(p * (l.size() - 1) + 0.5))]; };
    if (completed)
        *completed = S->completed;
    if (batches)
        *batches = S->batches;
    if (deferred)
        *deferred = S->deferred;
    if (p50_us)
        *p50_us = pct(0.50);
    if (p99_us)
        *p99_us = pct(0.99);
    return MDRQ_OK;
}

int mdrq_server_stop(mdrq_server *S)
{
    if (!S)
        return MDRQ_OK;
    {
        std::lock_guard<std::mutex> lock(S->mu);
        S->stopping = true;
        S->cv_sched.notify_all();
    }
    S->scheduler.join();
    {
        std::lock_guard<std::mutex> lock(S->mu);
        S->scheduler_done = true;
        S->cv_flight.notify_all();
    }
    S->completer.join();
    const int rc = S->fatal;
    cudaDeviceSynchronize();
    server_destroy(S);
    return rc;
}

}  // extern "C"
