"""Planted mistakes: each mutant is a copy of the oracle's C source with one
plausible error (a dropped term, a wrong sign or index, a transposed
operand, a wrong schedule). It is compiled on the CPU and the cheap pins of
test_oracle_pins.py are run against it; at least one must fail. This shows
the pins constrain every part of the oracle, not that the oracle is right.
"""

import os

import pytest

import oracle as oracle_mod

from . import test_oracle_pins as pins

# (name, original text, mutated text) -- each original must occur exactly once
MUTANTS = [
    ("philox_no_key_schedule", "k0 += weyl0;", "k0 += 0u;"),
    ("philox_wrong_multiplier", "mul1 = 0xCD9E8D57u", "mul1 = 0xCD9E8D55u"),
    ("box_muller_variance", "sqrt(-2.0 * log(u1))", "sqrt(-1.0 * log(u1))"),
    ("house_dropped_term", "for (int64_t i = 1; i < len; ++i) {\n        const double e",
     "for (int64_t i = 2; i < len; ++i) {\n        const double e"),
    ("house_tau_sign", "const double tau = (beta - alpha) / beta;",
     "const double tau = (alpha - beta) / beta;"),
    ("qr_no_sign_fix", "    fix_signs(m, l, q, r);\n", "\n"),
    ("qrcp_downdated_rows", "for (int64_t i = j; i < l; ++i) s += w[i * l + c] * w[i * l + c];",
     "for (int64_t i = 0; i < l; ++i) s += w[i * l + c] * w[i * l + c];"),
    ("qrcp_no_swap_of_perm", "perm[j] = perm[piv];\n            perm[piv] = tp;",
     "(void)tp;"),
    ("power_loop_one_short", "for (int64_t it = 0; it <= q; ++it) {\n            mm_ax(m, n, l, a, lda, x, c1);      /* eq. 4 */\n            if",
     "for (int64_t it = 0; it <= q - 1; ++it) {\n            mm_ax(m, n, l, a, lda, x, c1);      /* eq. 4 */\n            if"),
    ("d_transposed", "mm_xty(m, l, l, q1, w, d);", "mm_xty(m, l, l, w, q1, d);"),
    ("v_without_permutation", "v[i * l + j] = q2[i * l + perm[j]];", "v[i * l + j] = q2[i * l + j];"),
    ("aty_wrong_operand", "mm_aty(m, n, l, a, lda, q1, c2);    /* eq. 5 with C1 -> Q1 */",
     "mm_aty(m, n, l, a, lda, x, c2);    /* eq. 5 with C1 -> Q1 */"),
    ("shrink_wrong_sign", "const double mag = fabs(x[i]) - delta;", "const double mag = fabs(x[i]) + delta;"),
    ("mu_schedule_max", "mu = fmin(rho * mu, mu_bar);", "mu = fmax(rho * mu, mu_bar);"),
    ("sparse_step_scaled_dual", "const double xv = mat[i * ldm + c] - l_out[i * n + c] + y[i * n + c] * inv_mu;",
     "const double xv = mat[i * ldm + c] - l_out[i * n + c] + y[i * n + c] * mu;"),
    ("rank_threshold_mu", "if (t[i * l + i] > inv_mu) ++rj;", "if (t[i * l + i] > mu) ++rj;"),
]

# the cheap pins (all but the n >= 1000 Table 1 runs)
CHEAP = [
    (pins.test_philox_known_answers, ()),
    (pins.test_products_match_blas, ()),
    (pins.test_gaussian_is_standard_normal, ()),
    (pins.test_qr_matches_lapack, (50, 12, 1.0)),
    (pins.test_qr_matches_lapack, (200, 60, 1e6)),
    (pins.test_qr_rank_deficient_still_orthonormal, ()),
    (pins.test_qrcp_matches_lapack_dgeqp3, (15, 1)),
    (pins.test_qrcp_pivots_brute_force, (4, 0)),
    (pins.test_qrcp_pivots_brute_force, (6, 1)),
    (pins.test_qrcp_rank_revealing_inequalities, ()),
    (pins.test_qrcp_ties_take_lowest_index, ()),
    (pins.test_exact_rank_is_reproduced, (300, 200, 10, 10, 5, 0)),
    (pins.test_exact_rank_is_reproduced, (200, 300, 8, 8, 4, 1)),
    (pins.test_closed_form_projection, (0,)),
    (pins.test_closed_form_projection, (2,)),
    (pins.test_d_equals_r2_transpose, ()),
    (pins.test_error_versus_truncated_svd, (2,)),
    (pins.test_literal_and_reorthonormalised_forms_agree, ()),
    (pins.test_shrink_operator, ()),
    (pins.test_norm2_matches_lapack, ()),
    (pins.test_rpca_mu_schedule_and_histories, ()),
    (pins.test_rpca_c4_shape_small, ()),
]


def test_unmutated_source_passes_cheap_pins(oracle_lib, tmp_path):
    path = oracle_mod.compile_variant(oracle_mod.source_text(), str(tmp_path / "liboracle_ref.so"))
    with oracle_mod.use_library(path):
        for fn, args in CHEAP:
            fn(oracle_mod, *args)


@pytest.mark.parametrize("name,orig,mut", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_is_caught(oracle_lib, tmp_path, name, orig, mut):
    src = oracle_mod.source_text()
    assert src.count(orig) == 1, f"mutation anchor for {name} not unique"
    path = oracle_mod.compile_variant(src.replace(orig, mut), str(tmp_path / f"liboracle_{name}.so"))
    caught = []
    with oracle_mod.use_library(path):
        for fn, args in CHEAP:
            try:
                fn(oracle_mod, *args)
            except Exception as exc:  # AssertionError, OracleError, LinAlgError
                caught.append(f"{fn.__name__}{args}: {type(exc).__name__}")
                break
    assert caught, f"no pin detects the planted mistake {name}"
    os.remove(path)


# Planted mistakes in the lower-triangular-T variant (a Python composition of
# the C oracle): each returns what a plausible slip in corutv_lower would, and
# the lower-variant pins must reject it.
def _lower_mutants(orc):
    import numpy as np

    def base(a, k, p, q, psi=None, seed=0, stream=0):
        return orc.corutv(np.ascontiguousarray(a.T), k, p, q, psi=psi, seed=seed, stream=stream)

    def t_not_transposed(*args, **kw):
        o = base(*args, **kw)
        return {"U": o["V"], "T": o["T"], "V": o["U"], "perm": o["perm"]}

    def factors_not_swapped(*args, **kw):
        o = base(*args, **kw)
        return {"U": o["U"], "T": np.ascontiguousarray(o["T"].T), "V": o["V"], "perm": o["perm"]}

    def u_without_permutation(*args, **kw):
        o = base(*args, **kw)
        return {"U": o["Q2"], "T": np.ascontiguousarray(o["T"].T), "V": o["U"], "perm": o["perm"]}

    def run_on_a_not_at(a, k, p, q, psi=None, seed=0, stream=0):
        o = orc.corutv(a, k, p, q, psi=None, seed=seed, stream=stream)
        return {"U": o["U"], "T": np.ascontiguousarray(o["T"].T), "V": o["V"], "perm": o["perm"]}

    return {"t_not_transposed": t_not_transposed, "factors_not_swapped": factors_not_swapped,
            "u_without_permutation": u_without_permutation, "run_on_a_not_at": run_on_a_not_at}


@pytest.mark.parametrize("name", ["t_not_transposed", "factors_not_swapped", "u_without_permutation",
                                  "run_on_a_not_at"])
def test_planted_mistake_in_lower_variant_is_caught(oracle_lib, name):
    import types
    fake = types.SimpleNamespace(**{k: getattr(oracle_lib, k) for k in dir(oracle_lib) if not k.startswith("__")})
    fake.corutv_lower = _lower_mutants(oracle_lib)[name]
    failed = 0
    checks = [lambda: pins.test_lower_variant_reproduces_exact_rank(fake, 200, 300, 8, 8, 4, 1),
              lambda: pins.test_lower_variant_reproduces_exact_rank(fake, 120, 400, 5, 10, 10, 2),
              lambda: pins.test_lower_variant_error_versus_truncated_svd(fake, 2)]
    for check in checks:
        try:
            check()
        except (AssertionError, ValueError):
            failed += 1
    assert failed > 0, name
