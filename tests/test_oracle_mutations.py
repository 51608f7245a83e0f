"""The pins must catch plausible mistakes: each mutant build of oracle.c fails at least one pin.

Mutations are applied to a temporary copy of the source; oracle.c itself is untouched.
"""
import os

import pytest

import oracle
import pins

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(os.path.dirname(HERE), "oracle", "oracle.c")

MUTANTS = {
    "under_dose_sign": ("d -= 2.0 * c[2 * s] * e;", "d += 2.0 * c[2 * s] * e;"),
    "over_term_coefficient": ("F += c[2 * s + 1] * e * e;", "F += c[2 * s] * e * e;"),
    "no_normalisation": ("c[2 * s + k] = present ? w / (double)count : 0.0;",
                         "c[2 * s + k] = present ? w : 0.0;"),
    "transposed_index": ("trow[q] = j;", "trow[q] = P->col[k] % P->m;"),
    "no_projection": ("xt[i] = y > 0.0 ? y : 0.0;", "xt[i] = y;"),
    "no_sufficient_decrease": ("if (Gt < G - (q->eps / lam) * d2) break;", "if (Gt < G) break;"),
    "lambda_not_reset": ("double lam = lambda0; /* step 2 */",
                         "static double keep = 0.0; double lam = keep > 0.0 ? keep : lambda0; keep = lam;"),
    "dose_wrong_operand": ("s += (double)P->val[k] * x[P->col[k]];", "s += (double)P->val[k] * x[j % P->n];"),
    "gradient_drops_value": ("s += (double)tval[k] * r[trow[k]];", "s += r[trow[k]];"),
    "backtrack_wrong_direction": ("lam = lam / q->alpha; /* step 4 */", "lam = lam * q->alpha; /* step 4 */"),
    "voxel_target_under_sign": ("d -= 2.0 * vcu * e;", "d += 2.0 * vcu * e;"),
    "voxel_target_no_normalise": ("*co = P->m > 0 ? P->vt_wo / (P->vt_normalise ? (double)P->m : 1.0) : 0.0;",
                                  "*co = P->m > 0 ? P->vt_wo : 0.0;"),
    "kkt_zero": ("return worst / (g1_inf > 1.0 ? g1_inf : 1.0);", "return 0.0 * worst * g1_inf;"),
    "kkt_no_projection": ("double e = fabs(x[i] - p);", "double e = fabs(g[i]);"),
    "rel_denominator": ("rel = Gt > 0.0 ? fabs(Gt - G) / Gt : 0.0;", "rel = G > 0.0 ? fabs(Gt - G) / G : 0.0;"),
    "rel_absolute": ("rel = Gt > 0.0 ? fabs(Gt - G) / Gt : 0.0;", "rel = fabs(Gt - G);"),
}


def _run_pins(orc, tiny_case):
    failures = []
    for name in pins.ALL_PINS:
        try:
            getattr(pins, name)(orc)
        except AssertionError as e:
            failures.append(name)
    for fn in (lambda: pins.pin_gradient_fd(orc, tiny_case, n_coords=12),
               lambda: pins.pin_invariants(orc, tiny_case, max_iter=8),
               lambda: pins.pin_initial_point(orc, tiny_case)):
        try:
            fn()
        except AssertionError:
            failures.append("phantom")
    return failures


def test_unmutated_source_passes(orc, tiny_case):
    assert _run_pins(orc, tiny_case) == []


@pytest.mark.parametrize("mutant", sorted(MUTANTS))
def test_mutant_is_caught(tmp_path, tiny_case, mutant):
    old, new = MUTANTS[mutant]
    src = open(SRC).read()
    assert src.count(old) == 1, mutant
    path = tmp_path / "oracle_mutant.c"
    path.write_text(src.replace(old, new))
    lib = oracle.build(force=True, src=str(path), out=str(tmp_path / "liboracle_mutant.so"))
    failures = _run_pins(oracle.Oracle(lib), tiny_case)
    assert failures, f"mutation {mutant} was not caught by any pin"
