"""FP32-inner / FP64-refined solves against the plain FP64 CPU oracle.

The refined path runs ML(n)BiCGStabt in FP32 (matrix values, vectors,
preconditioner factors, per-thread accumulation; FP64 coefficients) inside
an FP64 iterative refinement with reliable updates (the FP32 iterate moved
into the FP64 solution and the FP32 residual replaced by the FP64 true
residual whenever it has fallen by the factor inner_tol).  Its iterates
differ from the FP64 method by design, so parity is on what is unique: the
solution.  Bars: flag 0, true relative residual ||b - A x||/||b|| < tol =
1e-10 (computed in FP64 by the library and re-checked here with the
oracle's product), and ||x - x_oracle|| within 1e-8 relative of the FP64
oracle's solution.
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


def _oracle_pc(A, precond):
    if precond == M.MLB_PRECOND_ILU0:
        return dict(ilu=O.ilu0(A))
    if precond == M.MLB_PRECOND_JACOBI:
        return dict(mdiag=O.jacobi_diag(A))
    return {}


def _refined_vs_oracle(A, b, n, maxit=20000, tol=1e-10, inner_tol=None, grid=0,
                       precond=M.MLB_PRECOND_NONE, AH=None, weight=None):
    cplx = np.iscomplexobj(A.val)
    h = M.mlbicgstab_create(A, AH=AH, n=n, q_seed=0, precision=M.MLB_PREC_FP32_REFINED,
                            inner_tol=inner_tol, max_outer=20, grid=grid, precond=precond)
    x = np.zeros(A.n_rows, dtype=b.dtype)
    res, hist = M.mlbicgstab_solve(h, b, x, tol, maxit, hist_cap=32)
    ref = O.solve(A, b, np.zeros_like(b), O.q_gauss(0, A.n_rows, n, complex_=cplx), maxit, tol,
                  **_oracle_pc(A, precond))
    assert ref.flag == 0 and ref.true_relres < tol
    assert res.status == 0 and res.flag == 0, res.as_dict()
    assert res.true_relres < tol
    assert O.true_relres(A, b, x) < tol
    w = 1.0 if weight is None else weight
    rel = np.linalg.norm(w * (x - ref.x)) / np.linalg.norm(w * ref.x)
    assert rel <= 1e-8, rel
    # true residuals at the start of every inner call, then the final one
    h_ = hist[:res.outer + 1]
    assert np.all(np.isfinite(h_)) and h_[-1] < tol and res.outer >= 1
    h.destroy()
    return res, ref


@pytest.mark.parametrize("n", [1, 4, 8])
def test_refined_cd2d(n):
    A = W.cd2d(32)
    _refined_vs_oracle(A, W.row_sums(A), n)


@pytest.mark.parametrize("grid", [1, 3])
def test_refined_cd2d_grid_variants(grid):
    A = W.cd2d(32)
    _refined_vs_oracle(A, W.row_sums(A), 4, grid=grid)


@pytest.mark.parametrize("inner_tol", [1e-1, 1e-3, 1e-5])
def test_refined_reliable_update_factor(inner_tol):
    A = W.cd2d(32)
    _refined_vs_oracle(A, W.row_sums(A), 4, inner_tol=inner_tol)


@pytest.mark.parametrize("m,n", [(16, 4), (23, 8)])
def test_refined_cd3d(m, n):
    A = W.cd3d_lognormal(m)
    _refined_vs_oracle(A, W.uniform_rhs(A.n_rows, seed=2), n)


def test_refined_complex():
    A = W.helmholtz3d_c(8, 8, 4, k=3.0)
    _refined_vs_oracle(A, W.row_sums(A), 4, maxit=3000)


@pytest.mark.parametrize("m,n", [(32, 4), (48, 4), (32, 8)])
def test_refined_ilu0_cd3d(m, n):
    """FP32 ILU(0) factors inside the FP32 inner solve; x against the FP64
    oracle preconditioned by the same (FP64) ILU(0)."""
    A = W.cd3d_lognormal(m)
    _refined_vs_oracle(A, W.uniform_rhs(A.n_rows, seed=2), n, precond=M.MLB_PRECOND_ILU0)


def test_refined_ilu0_reservoir_reduced():
    A = W.bsr3_to_csr(W.reservoir_bsr3(16, 16, 8))
    _refined_vs_oracle(A, W.row_sums(A), 8, precond=M.MLB_PRECOND_ILU0)


def test_refined_ilu0_complex():
    A = W.helmholtz3d_c(16, 16, 8, k=6.0)
    _refined_vs_oracle(A, W.row_sums(A), 4, maxit=4000, precond=M.MLB_PRECOND_ILU0,
                       AH=W.conj_transpose(A))


def test_refined_jacobi_column_scaled():
    """Columns scaled by 10^U[-3,3]: x itself spans six orders of magnitude
    and is determined only to cond(A) times the residual, so the two
    solutions are compared in the variable the iteration works on, y = M x
    (M = diag(A)), whose system A M^{-1} is the well-conditioned one."""
    A = W.cd2d(32)
    rng = np.random.default_rng(7)
    s = 10.0 ** rng.uniform(-3, 3, A.n_rows)
    A.val = A.val * s[A.col]
    _refined_vs_oracle(A, W.row_sums(A), 4, precond=M.MLB_PRECOND_JACOBI, weight=np.abs(O.jacobi_diag(A)))


def test_refined_never_returns_a_worse_x_than_it_started_from():
    """Systems on which FP32 cannot resolve the inner problem (strong
    log-normal contrast, no preconditioner) and a small iteration budget:
    whatever the flag, the returned x has a true residual no larger than
    the start's (x_0 = 0: relative residual 1), and flag 0 only with the
    residual below tol."""
    for sigma, m in ((4.0, 12), (5.0, 10)):
        A = W.cd3d_lognormal(m, sigma=sigma)
        b = W.uniform_rhs(A.n_rows, seed=2)
        h = M.mlbicgstab_create(A, n=4, precision=M.MLB_PREC_FP32_REFINED, max_outer=6)
        x = np.zeros(A.n_rows)
        res, hist = M.mlbicgstab_solve(h, b, x, 1e-12, 3000, hist_cap=8)
        rr = O.true_relres(A, b, x)
        assert res.status == 0 and res.flag in (0, 1), res.as_dict()
        assert rr <= 1.0 + 1e-12, (sigma, m, rr, res.as_dict())
        assert abs(rr - res.true_relres) <= 1e-6 * max(rr, 1e-300) + 1e-15
        if res.flag == 0:
            assert rr < 1e-12
        h.destroy()


def test_refined_reports_fp32_and_fp64_work():
    A = W.cd2d(32)
    b = W.row_sums(A)
    h = M.mlbicgstab_create(A, n=4, precision=M.MLB_PREC_FP32_REFINED)
    x = np.zeros(A.n_rows)
    res, _ = M.mlbicgstab_solve(h, b, x, 1e-10, 2000)
    # every inner iteration 1 + 1/n FP32 products on average, plus at least
    # the first FP64 residual product
    assert res.spmv >= 1 + res.iter
    assert res.bytes > 0 and res.kernel_ms > 0
    h.destroy()


def test_refined_batch_with_ilu0_matches_single_solves():
    """Refined batch (one CTA per system) mixing ILU(0) and unpreconditioned
    handles: every system converges to tol and agrees with the FP64 oracle
    to 1e-8."""
    sys_ = [W.cd2d(20), W.cd3d_lognormal(10), W.cd2d(28)]
    pcs = [M.MLB_PRECOND_ILU0, M.MLB_PRECOND_NONE, M.MLB_PRECOND_ILU0]
    hs, bs, xs = [], [], []
    for A, pc in zip(sys_, pcs):
        hs.append(M.mlbicgstab_create(A, n=4, precision=M.MLB_PREC_FP32_REFINED, precond=pc))
        bs.append(W.row_sums(A))
        xs.append(np.zeros(A.n_rows))
    res = M.mlbicgstab_solve_batch(hs, bs, xs, [1e-10] * 3, [5000] * 3)
    for A, pc, b, x, r in zip(sys_, pcs, bs, xs, res):
        assert r.status == 0 and r.flag == 0, r.as_dict()
        assert O.true_relres(A, b, x) < 1e-10
        ref = O.solve(A, b, np.zeros_like(b), O.q_gauss(0, A.n_rows, 4), 5000, 1e-10, **_oracle_pc(A, pc))
        assert np.linalg.norm(x - ref.x) / np.linalg.norm(ref.x) <= 1e-8
    for h in hs:
        h.destroy()
