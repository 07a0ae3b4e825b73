// Prepared batches: a fixed query batch recorded once as a CUDA graph and replayed.
//
// The batch runs on a private table that borrows the parent's columns and column
// statistics but has its own scratch (claim counter, look-back ring, error word),
// query tables, offsets and shared-scan state, so replays never race with calls on
// the parent. A first, ordinary run sizes every buffer; the second run is captured,
// so the captured work allocates nothing. The plain scan's look-back tags repeat at
// every replay, so on the private table each scan launch clears its ring first.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <new>
#include <vector>

#include "mdrq.h"
#include "table.h"

struct mdrq_prepared {
    mdrq_table *shadow = nullptr;
    uint32_t nq = 0;
    std::vector<uint32_t> live;
    uint64_t capacity = 0;
    uint64_t kernels = 0;
    cudaStream_t capture = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace {

void release(mdrq_prepared *p)
{
    if (!p)
        return;
    if (p->shadow)
        cudaSetDevice(p->shadow->device);
    cudaDeviceSynchronize();
    if (p->exec)
        cudaGraphExecDestroy(p->exec);
    if (p->graph)
        cudaGraphDestroy(p->graph);
    if (p->capture)
        cudaStreamDestroy(p->capture);
    mdrq::free_shadow(p->shadow);
    (void)cudaGetLastError();
    delete p;
}

cudaStream_t as_stream(void *s) { return static_cast<cudaStream_t>(s); }

int prepare(mdrq_table *t, const mdrq_qdesc *qs, uint32_t nq, uint32_t *ids, uint64_t capacity, uint64_t *offsets,
            cudaStream_t s, mdrq_prepared *p)
{
    using namespace mdrq;
    MDRQ_TRY_STATUS(cudaSetDevice(t->device));
    mdrq_table *sh = nullptr;
    int st = make_shadow(t, s, &sh);
    if (st != MDRQ_OK)
        return st;
    p->shadow = sh;
    std::vector<EncodedQuery> enc;
    size_t npreds = 0;
    st = encode_batch(sh, qs, nq, enc, p->live, npreds);
    if (st != MDRQ_OK)
        return st;
    p->nq = nq;
    p->capacity = capacity;
    // first run: sizes every buffer of the private table and gives the offsets
    st = enqueue_batch(sh, enc, p->live, nq, npreds, ids, capacity, s);
    if (st == MDRQ_OK)
        st = finish_batch(sh, p->live, nq, offsets, s);
    if (st != MDRQ_OK)
        return st;
    if (offsets[nq] > capacity)
        return MDRQ_E_CAPACITY;
    // second run, captured on a private stream (after the first run, which s finished)
    MDRQ_TRY_STATUS(cudaStreamCreateWithFlags(&p->capture, cudaStreamNonBlocking));
    sh->graph_capture = true;
    MDRQ_TRY_STATUS(cudaStreamBeginCapture(p->capture, cudaStreamCaptureModeThreadLocal));
    st = enqueue_batch(sh, enc, p->live, nq, npreds, ids, capacity, p->capture);
    const cudaError_t ce = cudaStreamEndCapture(p->capture, &p->graph);
    if (st != MDRQ_OK)
        return st;
    MDRQ_TRY_STATUS(ce);
    MDRQ_TRY_STATUS(cudaGraphInstantiate(&p->exec, p->graph, 0));
    size_t nodes = 0;
    MDRQ_TRY_STATUS(cudaGraphGetNodes(p->graph, nullptr, &nodes));
    std::vector<cudaGraphNode_t> list(nodes);
    if (nodes)
        MDRQ_TRY_STATUS(cudaGraphGetNodes(p->graph, list.data(), &nodes));
    for (cudaGraphNode_t n : list) {
        cudaGraphNodeType type;
        MDRQ_TRY_STATUS(cudaGraphNodeGetType(n, &type));
        p->kernels += type == cudaGraphNodeTypeKernel;
    }
    return MDRQ_OK;
}

}  // namespace

extern "C" {

int mdrq_prepare_batch(mdrq_table *t, const mdrq_qdesc *qs, uint32_t nq, uint32_t *ids, uint64_t capacity,
                       uint64_t *offsets, void *stream, mdrq_prepared **out)
{
    if (!out)
        return MDRQ_E_INVAL;
    *out = nullptr;
    if (!t || !offsets || (nq > 0 && !qs) || (capacity > 0 && !ids) || t->batch_mode == MDRQ_BATCH_LEARNED)
        return MDRQ_E_INVAL;
    mdrq_prepared *p = new (std::nothrow) mdrq_prepared();
    if (!p)
        return MDRQ_E_NOMEM;
    const int st = prepare(t, qs, nq, ids, capacity, offsets, as_stream(stream), p);
    if (st != MDRQ_OK) {
        release(p);
        return st;
    }
    *out = p;
    return MDRQ_OK;
}

int mdrq_prepared_launch(mdrq_prepared *p, void *stream)
{
    if (!p || !p->exec)
        return MDRQ_E_INVAL;
    MDRQ_TRY_STATUS(cudaSetDevice(p->shadow->device));
    MDRQ_TRY_STATUS(cudaGraphLaunch(p->exec, as_stream(stream)));
    return MDRQ_OK;
}

int mdrq_prepared_wait(mdrq_prepared *p, uint64_t *offsets, void *stream)
{
    if (!p || !offsets)
        return MDRQ_E_INVAL;
    MDRQ_TRY_STATUS(cudaSetDevice(p->shadow->device));
    const int st = mdrq::finish_batch(p->shadow, p->live, p->nq, offsets, as_stream(stream));
    if (st != MDRQ_OK)
        return st;
    return offsets[p->nq] > p->capacity ? MDRQ_E_CAPACITY : MDRQ_OK;
}

int mdrq_prepared_kernels(const mdrq_prepared *p, uint64_t *kernels)
{
    if (!p || !kernels)
        return MDRQ_E_INVAL;
    *kernels = p->kernels;
    return MDRQ_OK;
}

void mdrq_prepared_free(mdrq_prepared *p) { release(p); }

}  // extern "C"
