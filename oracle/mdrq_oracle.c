/*
 * Plain CPU oracle for the multidimensional range query (MDRQ).
 *
 * TEST INFRASTRUCTURE. Only the test suite, the smoke check and the benchmark's
 * CPU-baseline / reference leg may load this code. The GPU library shares nothing
 * with it: no header, no helper, no constant.
 *
 * What it computes (Sec. 2.1, "Problem Definition"): a data object t_i of a dataset
 * of n objects qualifies for a range query iff lb_j <= t_i[j] <= ub_j holds for every
 * dimension j the query constrains; dimensions the query leaves out behave as
 * [-inf, +inf] (partial-match queries, Sec. 2.1). The answer is the set of the
 * qualifying objects' identifiers, where the identifier of an object is its array
 * index i (Sec. 2.2.4). This file returns that set as an ascending uint32 list.
 *
 * How: two plain evaluations of that rule, which must agree.
 *  - oracle_mdrq, object at a time: every object in index order is tested against
 *    the rule of Sec. 2.1 ("for every constrained dimension" is decided false at the
 *    first dimension the object fails) and its index is appended when it qualifies.
 *    This is the sequential scan of Sec. 2.2.4.
 *  - oracle_mdrq_columnwise, dimension at a time: each constrained dimension is
 *    evaluated over its whole column into one flag per object, the flags of all
 *    constrained dimensions are ANDed, and the indices whose flag survives are
 *    listed in index order. This is the vertically partitioned evaluation of
 *    Sec. 3.2 (one array per dimension, per-dimension results combined by AND).
 * The data is held column-wise (one array per dimension, Sec. 3.2) for both; the
 * layout changes only where a value is read from, not which objects qualify.
 *
 * Comparisons are made in double precision: every float32 and every int32 value
 * is exactly representable as a double, so `lo <= x && x <= hi` in double decides
 * exactly what the same comparison decides in the column's own type (IEEE ordered
 * compare for float32, so -0.0 == +0.0; signed compare for int32). A NaN value
 * never satisfies a closed interval written this way.
 *
 * The parallel variant partitions the rows horizontally (Sec. 3.1) into p
 * contiguous ranges, scans each range on its own POSIX thread with the same loop,
 * and concatenates the partial results in partition order (Sec. 3.1, Sec. 5.4).
 * Contiguous ranges (instead of the paper's random assignment) keep the
 * concatenation ascending; the set of identifiers is the same either way.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_F32 0
#define ORACLE_I32 1

#define ORACLE_E_INVAL (-1)
#define ORACLE_E_NOMEM (-2)

typedef struct {
    const void *const *cols; /* cols[j]: column j, n values */
    const int32_t *types;    /* types[j]: ORACLE_F32 or ORACLE_I32 */
    const uint32_t *dims;    /* dims[p]: dimension of predicate p */
    const double *lo;        /* lo[p]: lower bound lb of predicate p */
    const double *hi;        /* hi[p]: upper bound ub of predicate p */
    uint32_t k;              /* number of predicates */
} oracle_query_t;

/* value of object i in dimension j, exactly, as a double */
static double value_at(const oracle_query_t *q, uint32_t j, uint64_t i)
{
    if (q->types[j] == ORACLE_F32)
        return (double)((const float *)q->cols[j])[i];
    return (double)((const int32_t *)q->cols[j])[i];
}

typedef struct {
    uint32_t *ids;
    uint64_t len;
    uint64_t cap;
    int failed;
} id_vector_t;

static void push_back(id_vector_t *v, uint32_t id)
{
    if (v->failed)
        return;
    if (v->len == v->cap) {
        uint64_t ncap = v->cap ? 2 * v->cap : 1024;
        uint32_t *nid = (uint32_t *)realloc(v->ids, ncap * sizeof(uint32_t));
        if (!nid) {
            v->failed = 1;
            return;
        }
        v->ids = nid;
        v->cap = ncap;
    }
    v->ids[v->len++] = id;
}

/* Sec. 2.1: object i qualifies iff lb_j <= t_i[j] <= ub_j holds for every
 * constrained dimension j; "for every" is false as soon as one predicate fails. */
static int qualifies(const oracle_query_t *q, uint64_t i)
{
    for (uint32_t p = 0; p < q->k; ++p) {
        double x = value_at(q, q->dims[p], i);
        if (!(q->lo[p] <= x && x <= q->hi[p]))
            return 0;
    }
    return 1;
}

/* Object at a time (Sec. 2.2.4): objects [begin, end) in index order, each
 * appended when it qualifies. */
static void scan_objects(const oracle_query_t *q, uint64_t begin, uint64_t end, id_vector_t *out)
{
    for (uint64_t i = begin; i < end; ++i)
        if (qualifies(q, i))
            push_back(out, (uint32_t)i);
}

/* 1 iff lb <= v <= ub (closed interval, Sec. 2.1), without a branch */
static unsigned char in_interval(double lb, double v, double ub)
{
    return (unsigned char)((lb <= v) & (v <= ub));
}

/* Dimension at a time (Sec. 3.2): one flag per object of [begin, end), ANDed with
 * each constrained dimension's result over its column; the objects whose flag
 * survives, in index order. Its flag loops are independent per object, so the
 * compiler may vectorise them (asked for here only; the object-at-a-time scan above
 * is compiled as the rest of the file). */
__attribute__((optimize("O3"))) static void scan_dimensions(const oracle_query_t *q, uint64_t begin, uint64_t end, id_vector_t *out)
{
    const uint64_t m = end - begin;
    unsigned char *flag = (unsigned char *)malloc(m > 0 ? m : 1);
    if (!flag) {
        out->failed = 1;
        return;
    }
    memset(flag, 1, m);
    for (uint32_t c = 0; c < q->k; ++c) {
        const uint32_t dim = q->dims[c];
        const double lb = q->lo[c], ub = q->hi[c];
        if (q->types[dim] == ORACLE_F32) {
            const float *fcol = (const float *)q->cols[dim] + begin;
            for (uint64_t r = 0; r < m; ++r)
                flag[r] &= in_interval(lb, (double)fcol[r], ub);
        } else {
            const int32_t *icol = (const int32_t *)q->cols[dim] + begin;
            for (uint64_t r = 0; r < m; ++r)
                flag[r] &= in_interval(lb, (double)icol[r], ub);
        }
    }
    for (uint64_t r = 0; r < m; ++r)
        if (flag[r])
            push_back(out, (uint32_t)(begin + r));
    free(flag);
}

typedef void (*scan_fn)(const oracle_query_t *, uint64_t, uint64_t, id_vector_t *);

typedef struct {
    const oracle_query_t *q;
    scan_fn scan;
    uint64_t begin, end;
    id_vector_t part;
} worker_t;

static void *worker_main(void *arg)
{
    worker_t *w = (worker_t *)arg;
    w->scan(w->q, w->begin, w->end, &w->part);
    return NULL;
}

/*
 * Answer one MDRQ with the given evaluation. On success returns the number of
 * qualifying objects and stores a malloc'd ascending id list in *ids_out (NULL when
 * the answer is empty); release it with oracle_free. nthreads <= 1 scans on the
 * calling thread; otherwise the rows are split into nthreads contiguous partitions
 * (Sec. 3.1). Returns ORACLE_E_INVAL for a bad argument (n >= 2^32, a dimension >= d,
 * a type other than the two above) and ORACLE_E_NOMEM if memory runs out.
 */
static int64_t answer(const void *const *cols, const int32_t *types, uint32_t d, uint64_t n,
                      const uint32_t *dims, const double *lo, const double *hi, uint32_t k,
                      int nthreads, uint32_t **ids_out, scan_fn scan)
{
    *ids_out = NULL;
    if (n > 0xFFFFFFFFull || (k > 0 && (!dims || !lo || !hi)))
        return ORACLE_E_INVAL;
    for (uint32_t j = 0; j < d; ++j)
        if (types[j] != ORACLE_F32 && types[j] != ORACLE_I32)
            return ORACLE_E_INVAL;
    for (uint32_t p = 0; p < k; ++p)
        if (dims[p] >= d || (n > 0 && !cols[dims[p]]))
            return ORACLE_E_INVAL;

    oracle_query_t q = {cols, types, dims, lo, hi, k};
    if (nthreads < 1)
        nthreads = 1;
    if ((uint64_t)nthreads > n)
        nthreads = n > 0 ? (int)n : 1;

    worker_t *w = (worker_t *)calloc((size_t)nthreads, sizeof(worker_t));
    pthread_t *tid = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    if (!w || !tid) {
        free(w);
        free(tid);
        return ORACLE_E_NOMEM;
    }
    for (int t = 0; t < nthreads; ++t) {
        w[t].q = &q;
        w[t].scan = scan;
        w[t].begin = n * (uint64_t)t / (uint64_t)nthreads;
        w[t].end = n * (uint64_t)(t + 1) / (uint64_t)nthreads;
    }
    if (nthreads == 1) {
        worker_main(&w[0]);
    } else {
        int started = 0;
        for (; started < nthreads; ++started)
            if (pthread_create(&tid[started], NULL, worker_main, &w[started]) != 0)
                break;
        /* a thread that could not be started is scanned here instead */
        for (int t = started; t < nthreads; ++t)
            worker_main(&w[t]);
        for (int t = 0; t < started; ++t)
            pthread_join(tid[t], NULL);
    }

    /* Sec. 3.1: concatenate the partial results in partition order */
    uint64_t total = 0;
    int failed = 0;
    for (int t = 0; t < nthreads; ++t) {
        total += w[t].part.len;
        failed |= w[t].part.failed;
    }
    uint32_t *ids = NULL;
    if (!failed && total > 0) {
        ids = (uint32_t *)malloc(total * sizeof(uint32_t));
        if (!ids)
            failed = 1;
        else {
            uint64_t at = 0;
            for (int t = 0; t < nthreads; ++t) {
                if (w[t].part.len)
                    memcpy(ids + at, w[t].part.ids, w[t].part.len * sizeof(uint32_t));
                at += w[t].part.len;
            }
        }
    }
    for (int t = 0; t < nthreads; ++t)
        free(w[t].part.ids);
    free(w);
    free(tid);
    if (failed)
        return ORACLE_E_NOMEM;
    *ids_out = ids;
    return (int64_t)total;
}

/* Object at a time (Sec. 2.1 rule per object, Sec. 2.2.4 scan). Arguments as above. */
int64_t oracle_mdrq(const void *const *cols, const int32_t *types, uint32_t d, uint64_t n,
                    const uint32_t *dims, const double *lo, const double *hi, uint32_t k,
                    int nthreads, uint32_t **ids_out)
{
    return answer(cols, types, d, n, dims, lo, hi, k, nthreads, ids_out, scan_objects);
}

/* Dimension at a time (Sec. 3.2 flags ANDed over the constrained columns). Same
 * arguments and result as oracle_mdrq. */
int64_t oracle_mdrq_columnwise(const void *const *cols, const int32_t *types, uint32_t d, uint64_t n,
                               const uint32_t *dims, const double *lo, const double *hi, uint32_t k,
                               int nthreads, uint32_t **ids_out)
{
    return answer(cols, types, d, n, dims, lo, hi, k, nthreads, ids_out, scan_dimensions);
}

void oracle_free(uint32_t *ids) { free(ids); }
