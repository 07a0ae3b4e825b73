"""Planted mistakes in a copy of the oracle must each fail at least one pin.

Each mutant is a textual edit of ``oracle/mdrq_oracle.c`` (a dropped term, a wrong
sign or index, a transposed operand, an off-by-one), compiled on the CPU into a
temporary directory. The real oracle is never modified.
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
    "negated_match": ("if (match)\n", "if (!match)\n"),
    "skips_first_row": ("for (uint64_t i = begin; i < end; ++i)",
                        "for (uint64_t i = begin + 1; i < end; ++i)"),
    "dropped_last_predicate": ("for (uint32_t p = 0; p < q->k; ++p) {\n            double",
                               "for (uint32_t p = 0; p + 1 < q->k; ++p) {\n            double"),
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


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(name, tmp_path):
    old, new = MUTANTS[name]
    text = open(SRC).read()
    assert text.count(old) == 1, "mutation site not found exactly once: %r" % old
    src = tmp_path / "mutant.c"
    src.write_text(text.replace(old, new))
    lib = oracle.compile_library(str(src), str(tmp_path / "libmutant.so"))
    mutant = oracle.Oracle(lib)
    caught = []
    for pin in pins.ALL_PINS:
        try:
            pin(mutant.mdrq)
        except AssertionError:
            caught.append(pin.__name__)
            break
    assert caught, "no pin failed for mutant %s" % name
