"""The multi-core build of the oracle (OpenMP, fixed-block reductions).

Pinned to the sequential oracle, which the other oracle tests pin to the
paper: it runs the same steps and differs only in the order of the
additions inside inner products and norms (fixed 1024-entry blocks), so
  * its results are bit-identical for every thread count;
  * its first iterates agree with the sequential oracle's to rounding
    (the method amplifies rounding on ill-conditioned systems after some
    iterations, so the comparison stops early there);
  * on a well-conditioned system its converged solution agrees with the
    sequential one to well below the solve tolerance;
  * on a system of a single block (N <= 1024) it is bit-identical to the
    sequential build (same summation order).
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle as O
from paper_1106_3678_gb300 import workloads as W

pytestmark = pytest.mark.filterwarnings("ignore")


@pytest.fixture(scope="module")
def par():
    lib = O.load_par()
    yield lib
    O.par_threads(1)


def test_results_do_not_depend_on_the_thread_count(par):
    A = W.cd3d_lognormal(20)
    b = W.uniform_rhs(A.n_rows, seed=2)
    Q = O.q_gauss(0, A.n_rows, 4)
    runs = []
    for t in (1, 2, 3, 5):
        O.par_threads(t)
        r = O.mlbicgstabt(A, b, np.zeros(A.n_rows), Q, 150, 0.0, err_hist=True, lib=par)
        runs.append(r)
    for r in runs[1:]:
        assert np.array_equal(r.x, runs[0].x)
        assert np.array_equal(r.err_hist, runs[0].err_hist)
        assert r.ops == runs[0].ops


def test_first_iterates_agree_with_the_sequential_oracle(par):
    O.par_threads(3)
    A = W.cd3d_lognormal(24)
    b = W.uniform_rhs(A.n_rows, seed=2)
    Q = O.q_gauss(0, A.n_rows, 4)
    for k in (1, 3, 5):
        r0 = O.mlbicgstabt(A, b, np.zeros(A.n_rows), Q, k, 0.0)
        r1 = O.mlbicgstabt(A, b, np.zeros(A.n_rows), Q, k, 0.0, lib=par)
        assert r0.ops == r1.ops
        assert np.linalg.norm(r1.x - r0.x) <= 1e-11 * np.linalg.norm(r0.x), k
        assert abs(r1.err - r0.err) <= 1e-11 * r0.err


@pytest.mark.parametrize("complex_", [False, True])
def test_converged_solution_agrees_with_the_sequential_oracle(par, complex_):
    O.par_threads(4)
    if complex_:
        A = W.helmholtz3d_c(16, 16, 8, k=3.0)
        b = W.row_sums(A)
    else:
        A = W.cd2d(64)
        b = W.row_sums(A)
    Q = O.q_gauss(0, A.n_rows, 4, complex_=complex_)
    r0 = O.solve(A, b, np.zeros_like(b), Q, 5000, 1e-10)
    r1 = O.solve(A, b, np.zeros_like(b), Q, 5000, 1e-10, lib=par)
    assert r0.flag == 0 and r1.flag == 0
    assert r0.true_relres < 1e-10 and r1.true_relres < 1e-10
    assert np.linalg.norm(r1.x - r0.x) <= 1e-9 * np.linalg.norm(r0.x)
    assert abs(r1.iter - r0.iter) <= max(2, r0.iter // 50)


def test_single_block_is_bit_identical_to_the_sequential_build(par):
    O.par_threads(2)
    A = W.cd2d(32)                      # N = 1024: one block
    b = W.row_sums(A)
    Q = O.q_gauss(0, A.n_rows, 4)
    r0 = O.mlbicgstabt(A, b, np.zeros(A.n_rows), Q, 2000, 1e-10, err_hist=True)
    r1 = O.mlbicgstabt(A, b, np.zeros(A.n_rows), Q, 2000, 1e-10, err_hist=True, lib=par)
    assert np.array_equal(r0.x, r1.x) and np.array_equal(r0.err_hist, r1.err_hist)
    assert r0.iter == r1.iter
