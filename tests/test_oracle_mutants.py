"""The pins have teeth: plausible mistakes planted in copies of the oracle
source (dropped terms, wrong signs or indices, transposed operands, a
missing conjugate) are each caught by at least one pin.

Each mutant is a textual substitution applied to a temporary copy of the
oracle; the oracle in the repository is never modified.
"""
from __future__ import annotations

import os
import shutil

import pytest

import oracle
from oracle import build as obuild
from tests import test_oracle_pins as P

BODY = "mlb_oracle_body.h"
MAIN = "mlb_oracle.c"

# (name, file, original text, planted mistake)
MUTANTS = [
    ("beta_tilde_sign", BODY, "S bt = -e / c[i];", "S bt = e / c[i];"),
    ("q_sweep_wrong_c", BODY,
     "bt = -SFX(dot)(N, Q + (int64_t)s * N, wi, ops) / c[s];",
     "bt = -SFX(dot)(N, Q + (int64_t)s * N, wi, ops) / c[s - 1];"),
    ("omega_mul_not_div", BODY, "g[i] = z[i] - g[i] / omega;",
     "g[i] = z[i] - g[i] * omega;"),
    ("f_sweep_uses_q", BODY,
     "S beta = -SFX(dot)(N, F + (int64_t)s * N, gi, ops) / c[s];",
     "S beta = -SFX(dot)(N, Q + (int64_t)s * N, gi, ops) / c[s];"),
    ("ahq_not_transposed", BODY, "f[ci[k]] += CONJ(av[k]) * q[r];",
     "f[r] += CONJ(av[k]) * q[ci[k]];"),
    ("dot_without_conj", BODY, "s += CONJ(u[i]) * v[i];", "s += u[i] * v[i];"),
    ("dropped_g_term", BODY,
     "SFX(axpy)(N, bt, G + (int64_t)s * N, gi, ops);\n                }",
     "\n                }"),
    ("block_end_wrong_c", BODY, "alpha = e / c[n - 1];", "alpha = e / c[0];"),
    ("e_wrong_shadow", BODY, "e = SFX(dot)(N, Q + (int64_t)i * N, r, ops);",
     "e = SFX(dot)(N, Q + (int64_t)(i - 1) * N, r, ops);"),
    ("omega_inverted", BODY, "omega = zu / zz;", "omega = zz / zu;"),
    ("kappa_inverted", BODY, "omega = omega * kappa / arho;",
     "omega = omega * arho / kappa;"),
    ("q_sweep_short", BODY, "for (int32_t s = i + 1; s <= n - 1; ++s) {",
     "for (int32_t s = i + 1; s < n - 1; ++s) {"),
    ("r_update_sign", BODY,
     "SFX(axpy)(N, -alpha, W + (int64_t)(i - 1) * N, r, ops);",
     "SFX(axpy)(N, alpha, W + (int64_t)(i - 1) * N, r, ops);"),
    ("gn_truncates", MAIN, "q -= 1;", "q -= 0;"),
    ("j0_branch_wrong_g", BODY, "SFX(xpay)(N, r, beta, G, gi, ops);",
     "SFX(xpay)(N, r, beta, gi, gi, ops);"),
    # preconditioned path (Algorithm 7.1, M != I)
    ("precond_x_along_g", BODY,
     "SFX(axpy)(N, alpha, Gh + (int64_t)(i - 1) * N, x, ops);",
     "SFX(axpy)(N, alpha, G + (int64_t)(i - 1) * N, x, ops);"),
    ("precond_w_from_g", BODY,
     "SFX(matvec)(N, rp, ci, av, Gh + (int64_t)i * N, wi, ops);",
     "SFX(matvec)(N, rp, ci, av, gi, wi, ops);"),
    ("precond_F_unscaled", BODY,
     "v[t] = v[t] / CONJ(mdiag[t]);", "v[t] = v[t];"),
    ("precond_omega_step_u", BODY, "SFX(axpy)(N, omega, uh, x, ops);",
     "SFX(axpy)(N, omega, r, x, ops);"),
    ("precond_minv_multiplies", BODY, "dst[t] = src[t] / mdiag[t];",
     "dst[t] = src[t] * mdiag[t];"),
    # ILU(0) factors and their application
    ("ilu_no_update", BODY, "lu[ij] = lu[ij] - lu[ik] * lu[kj];", "lu[ij] = lu[ij];"),
    ("ilu_no_divide", BODY, "lu[ik] = lu[ik] / ukk;", "lu[ik] = lu[ik];"),
    ("ilu_update_sign", BODY, "lu[ij] = lu[ij] - lu[ik] * lu[kj];", "lu[ij] = lu[ij] + lu[ik] * lu[kj];"),
    ("ilu_backward_no_div", BODY, "dst[i] = s / lu[dp[i]];", "dst[i] = s;"),
    ("ilu_forward_drops_last_term", BODY,
     "for (int64_t k = rp[i]; k < dp[i]; ++k)\n            s -= lu[k] * dst[ci[k]];",
     "for (int64_t k = rp[i]; k + 1 < dp[i]; ++k)\n            s -= lu[k] * dst[ci[k]];"),
    ("ilu_minv_h_no_conj", BODY,
     "for (int64_t k = dp[i] + 1; k < rp[i + 1]; ++k)\n            v[ci[k]] -= CONJ(lu[k]) * v[i];",
     "for (int64_t k = dp[i] + 1; k < rp[i + 1]; ++k)\n            v[ci[k]] -= lu[k] * v[i];"),
    ("ilu_minv_h_skips_L", BODY,
     "for (int64_t k = rp[i]; k < dp[i]; ++k)\n            v[ci[k]] -= CONJ(lu[k]) * v[i];",
     "for (int64_t k = rp[i]; k < rp[i]; ++k)\n            v[ci[k]] -= CONJ(lu[k]) * v[i];"),
]

# fast pins, in the order they are tried
PINS = [
    lambda o: P.test_table_2_1_bit_exact(o),
    lambda o: P.test_index_identity_eq_2_1(o, 3),
    lambda o: P.test_spmv_and_ahq_match_dense_products(o),
    lambda o: P.test_finite_termination_within_N_steps(o, 8, 8, False),
    lambda o: P.test_finite_termination_within_N_steps(o, 6, 9, True),
    lambda o: P.test_finite_termination_within_N_steps(o, 8, 3, False),
    lambda o: P.test_finite_termination_within_N_steps(o, 10, 2, True),
    lambda o: P.test_n1_matches_textbook_bicgstab(o, 300, "random"),
    lambda o: P.test_n1_matches_textbook_bicgstab_complex(o),
    lambda o: P.test_kappa_guard_matches_safeguarded_bicgstab(o),
    lambda o: P.test_block0_biorthogonality(o, True),
    lambda o: P.test_table_4_3_operation_counts_per_block(o, 4),
    lambda o: P.test_cd2d_agrees_with_dense_lu(o, 4),
    lambda o: P.test_precond_equals_method_on_right_scaled_system(o, False),
    lambda o: P.test_precond_finite_termination(o, 8, 3),
    lambda o: P.test_ilu0_reproduces_A_on_its_pattern(o, True, 0.2),
    lambda o: P.test_ilu_minv_and_minv_h_match_dense_solves(o, True),
    lambda o: P.test_ilu_precond_equals_method_on_right_preconditioned_system(o, False),
]


def _caught(bound) -> bool:
    for pin in PINS:
        try:
            pin(bound)
        except (AssertionError, FloatingPointError, ValueError,
                ZeroDivisionError, OverflowError):
            return True
    return False


def test_unmutated_copy_passes_every_pin(tmp_path):
    src = tmp_path / "src"
    shutil.copytree(os.path.dirname(oracle.__file__), src,
                    ignore=shutil.ignore_patterns("_build", "__pycache__"))
    so = obuild.compile_oracle(str(src / MAIN), str(tmp_path / "orc.so"),
                               include_dir=str(src))
    assert not _caught(oracle.Bound(oracle.load(so)))


@pytest.mark.parametrize("name,fname,orig,mut", MUTANTS,
                         ids=[m[0] for m in MUTANTS])
def test_planted_mistake_is_caught(tmp_path, name, fname, orig, mut):
    src = tmp_path / "src"
    shutil.copytree(os.path.dirname(oracle.__file__), src,
                    ignore=shutil.ignore_patterns("_build", "__pycache__"))
    text = (src / fname).read_text()
    assert text.count(orig) >= 1, f"mutation site for {name} not found"
    (src / fname).write_text(text.replace(orig, mut, 1))
    so = obuild.compile_oracle(str(src / MAIN), str(tmp_path / "orc.so"),
                               include_dir=str(src))
    assert _caught(oracle.Bound(oracle.load(so))), name
