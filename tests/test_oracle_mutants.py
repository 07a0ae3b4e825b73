"""Planted mistakes in a copy of the oracle must each fail at least one pin.

Each mutant is a textual edit of ``oracle/mdrq_oracle.c`` (a dropped term, a wrong
sign or index, a transposed operand, an off-by-one), compiled on the CPU into a
temporary directory. The real oracle is never modified. ``MUTANTS`` plant mistakes in
the object-at-a-time evaluation and the shared partition driver and are checked
through ``oracle_mdrq``; ``COLUMNWISE_MUTANTS`` plant them in the dimension-at-a-time
evaluation and are checked through ``oracle_mdrq_columnwise``.
"""
import os

import pytest

import oracle
import pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "mdrq_oracle.c")

MUTANTS = {
    "open_lower_bound": ("q->lo[p] <= x", "q->lo[p] < x"),
    "open_upper_bound": ("x <= q->hi[p]", "x < q->hi[p]"),
    "dropped_upper_term": ("!(q->lo[p] <= x && x <= q->hi[p])", "!(q->lo[p] <= x)"),
    "dropped_lower_term": ("!(q->lo[p] <= x && x <= q->hi[p])", "!(x <= q->hi[p])"),
    "transposed_operands": ("q->lo[p] <= x && x <= q->hi[p]", "x <= q->lo[p] && q->hi[p] <= x"),
    "wrong_dimension_index": ("value_at(q, q->dims[p], i)", "value_at(q, p, i)"),
    "wrong_id": ("push_back(out, (uint32_t)i)", "push_back(out, (uint32_t)(i + 1))"),
    "negated_match": ("if (qualifies(q, i))", "if (!qualifies(q, i))"),
    "skips_first_row": ("for (uint64_t i = begin; i < end; ++i)",
                        "for (uint64_t i = begin + 1; i < end; ++i)"),
    "dropped_last_predicate": ("for (uint32_t p = 0; p < q->k; ++p) {\n        double",
                               "for (uint32_t p = 0; p + 1 < q->k; ++p) {\n        double"),
    "float_sign_flipped": ("return (double)((const float *)q->cols[j])[i];",
                           "return -(double)((const float *)q->cols[j])[i];"),
    "int_read_unsigned": ("return (double)((const int32_t *)q->cols[j])[i];",
                          "return (double)((const uint32_t *)q->cols[j])[i];"),
    "partition_gap": ("w[t].end = n * (uint64_t)(t + 1) / (uint64_t)nthreads;",
                      "w[t].end = n * (uint64_t)(t + 1) / (uint64_t)nthreads"
                      " - (uint64_t)(t + 1 < nthreads && n > (uint64_t)nthreads);"),
    "partitions_concatenated_backwards": (
        "for (int t = 0; t < nthreads; ++t) {\n                if (w[t].part.len)",
        "for (int t = nthreads - 1; t >= 0; --t) {\n                if (w[t].part.len)"),
    "float_read_as_int": ("return (double)((const float *)q->cols[j])[i];",
                          "return (double)((const int32_t *)q->cols[j])[i];"),
    "type_dispatch_inverted": ("if (q->types[j] == ORACLE_F32)\n        return",
                               "if (q->types[j] != ORACLE_F32)\n        return"),
    "skips_last_row": ("for (uint64_t i = begin; i < end; ++i)",
                       "for (uint64_t i = begin; i + 1 < end; ++i)"),
    "partitions_overwrite": ("                at += w[t].part.len;\n", ""),
    "last_partition_short": ("w[t].end = n * (uint64_t)(t + 1) / (uint64_t)nthreads;",
                             "w[t].end = n * (uint64_t)(t + 1) / (uint64_t)nthreads"
                             " - (uint64_t)(t + 1 == nthreads && n > 1);"),
    "first_predicate_lower_bound_for_all": ("q->lo[p] <= x", "q->lo[0] <= x"),
}


COLUMNWISE_MUTANTS = {
    "open_lower_bound": ("(lb <= v) & (v <= ub)", "(lb < v) & (v <= ub)"),
    "open_upper_bound": ("(lb <= v) & (v <= ub)", "(lb <= v) & (v < ub)"),
    "dropped_upper_term": ("(lb <= v) & (v <= ub)", "(lb <= v)"),
    "or_instead_of_and": ("(lb <= v) & (v <= ub)", "(lb <= v) | (v <= ub)"),
    "flags_overwritten_not_anded": ("flag[r] &= in_interval(lb, (double)fcol[r], ub);",
                                    "flag[r] = in_interval(lb, (double)fcol[r], ub);"),
    "int_flags_overwritten": ("flag[r] &= in_interval(lb, (double)icol[r], ub);",
                              "flag[r] = in_interval(lb, (double)icol[r], ub);"),
    "flags_start_clear": ("memset(flag, 1, m);", "memset(flag, 0, m);"),
    "wrong_dimension": ("const uint32_t dim = q->dims[c];", "const uint32_t dim = c;"),
    "bounds_of_first_predicate": ("const double lb = q->lo[c], ub = q->hi[c];",
                                  "const double lb = q->lo[0], ub = q->hi[c];"),
    "partition_offset_dropped": ("(const float *)q->cols[dim] + begin;", "(const float *)q->cols[dim];"),
    "int_partition_offset_dropped": ("(const int32_t *)q->cols[dim] + begin;", "(const int32_t *)q->cols[dim];"),
    "ids_local_to_partition": ("push_back(out, (uint32_t)(begin + r));", "push_back(out, (uint32_t)r);"),
    "type_dispatch_inverted": ("if (q->types[dim] == ORACLE_F32) {", "if (q->types[dim] != ORACLE_F32) {"),
    "dropped_last_dimension": ("for (uint32_t c = 0; c < q->k; ++c) {", "for (uint32_t c = 0; c + 1 < q->k; ++c) {"),
    "skips_last_object": ("for (uint64_t r = 0; r < m; ++r)\n        if (flag[r])",
                          "for (uint64_t r = 0; r + 1 < m; ++r)\n        if (flag[r])"),
    "int_read_unsigned": ("const int32_t *icol = (const int32_t *)", "const uint32_t *icol = (const uint32_t *)"),
}


def _caught(text: str, old: str, new: str, entry: str, tmp_path) -> list:
    assert text.count(old) == 1, "mutation site not found exactly once: %r" % old
    src = tmp_path / "mutant.c"
    src.write_text(text.replace(old, new))
    lib = oracle.compile_library(str(src), str(tmp_path / "libmutant.so"))
    f = getattr(oracle.Oracle(lib), entry)
    caught = []
    for pin in pins.ALL_PINS:
        try:
            pin(f)
        except AssertionError:
            caught.append(pin.__name__)
            break
    return caught


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(name, tmp_path):
    old, new = MUTANTS[name]
    assert _caught(open(SRC).read(), old, new, "mdrq", tmp_path), "no pin failed for mutant %s" % name


@pytest.mark.parametrize("name", sorted(COLUMNWISE_MUTANTS))
def test_planted_columnwise_mistake_is_caught(name, tmp_path):
    old, new = COLUMNWISE_MUTANTS[name]
    assert _caught(open(SRC).read(), old, new, "mdrq_columnwise", tmp_path), \
        "no pin failed for mutant %s" % name
