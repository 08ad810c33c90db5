"""Plant plausible mistakes in copies of the oracle and check that the pins catch each.

Each mutant is the oracle's C source with one textual edit (a flipped
comparison, a dropped term, a wrong sign, a transposed index, a wrong
exponent bias, a broken tie rule), compiled into a temporary library. The
real oracle is never modified. A mutant that no pin rejects would mean the
pins leave that part of the oracle unchecked.
"""
import os

import pytest

import oracle
import oracle_pins as P
from oracle import Oracle

SRC = os.path.join(os.path.dirname(oracle.__file__), "oracle.c")

MUTANTS = {
    "max_becomes_min_in_gather": ("else if (s > w->best[d]) w->best[d] = s;",
                                  "else if (s < w->best[d]) w->best[d] = s;"),
    "residual_term_dropped": ("double v = cterm + rho_at(ix, t) * rterm;", "double v = cterm;"),
    "residual_sign_flipped": ("double v = cterm + rho_at(ix, t) * rterm;",
                              "double v = cterm - rho_at(ix, t) * rterm;"),
    "norm_ignored": ("double v = cterm + rho_at(ix, t) * rterm;", "double v = cterm + rterm;"),
    "subspace_index_transposed": ("int m = k / ix->ds, r = k % ix->ds;",
                                  "int m = k % ix->M, r = k / ix->M;"),
    "fp16_bias_off_by_one": ("else v = ldexp((double)(m + 1024), e - 25);",
                             "else v = ldexp((double)(m + 1024), e - 24);"),
    "tie_break_id_desc": ("return (x->id > y->id) - (x->id < y->id);",
                          "return (x->id < y->id) - (x->id > y->id);"),
    "last_query_token_dropped_in_gather": (
        "  for (int i = 0; i < ntok; i++) {\n    const float *qi = q + (int64_t)i * ix->dim;\n    int64_t nti = 0;",
        "  for (int i = 0; i < ntok - 1; i++) {\n    const float *qi = q + (int64_t)i * ix->dim;\n    int64_t nti = 0;"),
    "refine_max_becomes_min": ("if (v > m) m = v;", "if (m == -INFINITY || v < m) m = v;"),
    "bf16_widening_wrong_shift": ("uint32_t u = ((uint32_t)h) << 16;", "uint32_t u = ((uint32_t)h) << 15;"),
    "query_centroid_transposed": ("s += (double)q[k] * cent_at(ix, j, k);",
                                  "s += (double)q[k] * cent_at(ix, k % ix->C, (int)(j % ix->dim));"),
    "doc_without_hit_counted": ("if (!w->hit[d]) { w->hit[d] = 1; w->acc[d] = 0.0;",
                                "if (!w->hit[d]) { w->hit[d] = 1; w->acc[d] = 0.5;"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site for {name} not unique"
    msrc = tmp_path / "oracle_mutant.c"
    msrc.write_text(src.replace(old, new))
    lib = oracle.build(force=True, src=str(msrc), out=str(tmp_path / "liboracle_mutant.so"))

    def make(ix, dim):
        return Oracle(ix, dim=dim, lib=lib)

    caught = []
    for pin in P.ALL_PINS:
        try:
            pin(make)
        except AssertionError:
            caught.append(pin.__name__)
        except ValueError:
            caught.append(pin.__name__)
    assert caught, f"no pin rejects mutant {name}"
