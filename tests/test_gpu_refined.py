"""FP32-inner / FP64-refined solves against the plain FP64 CPU oracle.

The refined path runs ML(n)BiCGStabt in FP32 (matrix values, vectors,
per-thread accumulation; FP64 coefficients) inside an FP64 iterative
refinement.  Its iterates differ from the FP64 method by design, so parity
is on what is unique: the solution.  Bars: flag 0, true relative residual
||b - A x||/||b|| < tol = 1e-10 (computed in FP64 by the library and
re-checked here with the oracle's product), and ||x - x_oracle|| within
1e-8 relative of the FP64 oracle's solution.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle as O
from paper_1106_3678_gb300 import mlbicgstab as M
from paper_1106_3678_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1106_3678_gb300 import build
    build.build()
    M.load()


def _refined_vs_oracle(A, b, n, maxit=20000, tol=1e-10, inner_tol=1e-5, grid=0):
    cplx = np.iscomplexobj(A.val)
    h = M.mlbicgstab_create(A, n=n, q_seed=0, precision=M.MLB_PREC_FP32_REFINED,
                            inner_tol=inner_tol, max_outer=20, grid=grid)
    x = np.zeros(A.n_rows, dtype=b.dtype)
    res, hist = M.mlbicgstab_solve(h, b, x, tol, maxit, hist_cap=32)
    ref = O.solve(A, b, np.zeros_like(b), O.q_gauss(0, A.n_rows, n, complex_=cplx), maxit, tol)
    assert ref.flag == 0 and ref.true_relres < tol
    assert res.status == 0 and res.flag == 0, res.as_dict()
    assert res.true_relres < tol
    assert O.true_relres(A, b, x) < tol
    rel = np.linalg.norm(x - ref.x) / np.linalg.norm(ref.x)
    assert rel <= 1e-8, rel
    # outer true residuals are recorded and decrease to below tol
    h_ = hist[:res.outer + 1]
    assert np.all(np.isfinite(h_)) and h_[-1] < tol and res.outer >= 1
    return res, ref


@pytest.mark.parametrize("n", [1, 4, 8])
def test_refined_cd2d(n):
    A = W.cd2d(32)
    _refined_vs_oracle(A, W.row_sums(A), n)


@pytest.mark.parametrize("grid", [1, 3])
def test_refined_cd2d_grid_variants(grid):
    A = W.cd2d(32)
    _refined_vs_oracle(A, W.row_sums(A), 4, grid=grid)


@pytest.mark.parametrize("m,n", [(16, 4), (23, 8)])
def test_refined_cd3d(m, n):
    A = W.cd3d_lognormal(m)
    _refined_vs_oracle(A, W.uniform_rhs(A.n_rows, seed=2), n)


def test_refined_complex():
    A = W.helmholtz3d_c(8, 8, 4, k=3.0)
    _refined_vs_oracle(A, W.row_sums(A), 4, maxit=3000)


def test_refined_reports_fp32_and_fp64_work():
    A = W.cd2d(32)
    b = W.row_sums(A)
    h = M.mlbicgstab_create(A, n=4, precision=M.MLB_PREC_FP32_REFINED)
    x = np.zeros(A.n_rows)
    res, _ = M.mlbicgstab_solve(h, b, x, 1e-10, 2000)
    # every outer step: one FP64 residual product; every inner iteration
    # 1 + 1/n FP32 products on average
    assert res.spmv >= res.outer + 1 + res.iter
    assert res.bytes > 0 and res.kernel_ms > 0
