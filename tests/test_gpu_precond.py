"""Jacobi preconditioning (Algorithm 7.1 with M = diag(A)) through the C ABI.

The library stores A M^{-1} and iterates on y = M x; the oracle applies M
literally, step by step (g^ = M^{-1} g, x along g^, u^ = M^{-1} u).  The two
agree to rounding: early residual histories within the sequential-sum bound
used for the unpreconditioned solves; converged solutions within 1e-8, or,
for the badly column-scaled batch systems, within the forward-error bound
cond(A) * 2 tol of two solutions whose residuals both meet tol.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle as O
from paper_1106_3678_gb300 import mlbicgstab as M
from paper_1106_3678_gb300 import workloads as W

pytestmark = pytest.mark.gpu
EPS = np.finfo(np.float64).eps


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1106_3678_gb300 import build
    build.build()
    M.load()


def _col_scaled(A, s):
    return W.CSR(row_ptr=A.row_ptr.copy(), col=A.col.copy(), val=A.val * s[A.col], n_rows=A.n_rows)


def _cond(A):
    D = np.zeros((A.n_rows, A.n_rows), dtype=A.val.dtype)
    for r in range(A.n_rows):
        D[r, A.col[A.row_ptr[r]:A.row_ptr[r + 1]]] += A.val[A.row_ptr[r]:A.row_ptr[r + 1]]
    return np.linalg.cond(D)


def _early_tol(N):
    return max(1e-10, 4 * N * EPS)


@pytest.mark.parametrize("n", [1, 4, 8])
def test_jacobi_matches_oracle(n):
    A = _col_scaled(W.cd2d(32), 10.0 ** np.random.default_rng(7).uniform(-1, 1, 1024))
    b = W.row_sums(A)
    N = A.n_rows
    d = O.jacobi_diag(A)
    h = M.mlbicgstab_create(A, n=n, q_seed=0, precond=M.MLB_PRECOND_JACOBI)
    assert M.mlbicgstab_info(h)["precond"] == M.MLB_PRECOND_JACOBI
    x = np.zeros(N)
    K = 12
    res, eh = M.mlbicgstab_solve(h, b, x, 0.0, K, hist_cap=K + 1)
    ref = O.mlbicgstabt(A, b, np.zeros(N), O.q_gauss(0, N, n), K, 0.0, err_hist=True, mdiag=d)
    assert (res.iter, res.j, res.i) == (ref.iter, ref.j, ref.i)
    np.testing.assert_allclose(eh[:K + 1], ref.err_hist[:K + 1], rtol=_early_tol(N))
    np.testing.assert_allclose(x, ref.x, rtol=0, atol=1e-9 * np.max(np.abs(ref.x)))
    # full solve
    x = np.zeros(N)
    res, _ = M.mlbicgstab_solve(h, b, x, 1e-10, 3000)
    ref = O.solve(A, b, np.zeros(N), O.q_gauss(0, N, n), 3000, 1e-10, mdiag=d)
    assert res.flag == 0 and ref.flag == 0
    assert res.true_relres < 1e-10
    assert np.linalg.norm(x - ref.x) <= 1e-8 * np.linalg.norm(ref.x)


def test_jacobi_complex_matches_oracle():
    A, _, b = W.random_dense_system(200, seed=9, complex_=True)
    N = A.n_rows
    s = np.random.default_rng(3).uniform(0.2, 5.0, N) * np.exp(1j * np.random.default_rng(4).uniform(-0.3, 0.3, N))
    A = _col_scaled(A, s)
    d = O.jacobi_diag(A)
    for AH in (None, W.conj_transpose(A)):
        h = M.mlbicgstab_create(A, AH=AH, n=4, q_seed=0, precond=M.MLB_PRECOND_JACOBI)
        x = np.zeros(N, dtype=complex)
        res, _ = M.mlbicgstab_solve(h, b, x, 1e-12, 400)
        ref = O.solve(A, b, np.zeros(N, dtype=complex), O.q_gauss(0, N, 4, complex_=True), 400, 1e-12, mdiag=d)
        assert res.flag == 0 and ref.flag == 0
        assert abs(res.iter - ref.iter) <= 2
        assert np.linalg.norm(x - ref.x) <= 1e-9 * np.linalg.norm(ref.x)


def test_jacobi_undoes_column_scaling_on_gpu():
    """M = diag(A) right preconditioning is invariant to A -> A S: the
    scaled system takes the iterations of the unscaled one (to rounding),
    and without the preconditioner it takes many more."""
    A = W.cd2d(32)
    b = W.row_sums(A)
    N = A.n_rows
    s = 10.0 ** np.random.default_rng(11).uniform(-3, 3, N)
    AS = _col_scaled(A, s)
    its = {}
    for name, mat, pc in (("A", A, 1), ("AS", AS, 1), ("AS_plain", AS, 0)):
        h = M.mlbicgstab_create(mat, n=4, q_seed=0, precond=pc)
        x = np.zeros(N)
        r, _ = M.mlbicgstab_solve(h, b, x, 1e-10, 20000)
        its[name] = (r.iter, r.flag, r.true_relres, x)
    assert its["A"][1] == 0 and its["AS"][1] == 0
    assert abs(its["A"][0] - its["AS"][0]) <= 3
    np.testing.assert_allclose(its["AS"][3] * s, its["A"][3], rtol=1e-6, atol=1e-8)
    assert its["AS_plain"][1] != 0 or its["AS_plain"][0] > 2 * its["AS"][0]


@pytest.mark.parametrize("precision", [M.MLB_PREC_FP64, M.MLB_PREC_FP32_REFINED])
def test_jacobi_batch_equals_single_cta(precision):
    systems = []
    rng = np.random.default_rng(12)
    for A, _ in W.batch_cd(12, seed=13, n_min=300, n_max=3000):
        systems.append(_col_scaled(A, 10.0 ** rng.uniform(-1, 1, A.n_rows)))
    hs = [M.mlbicgstab_create(A, n=4, q_seed=0, precond=1, precision=precision) for A in systems]
    bs = [W.row_sums(A) for A in systems]
    xs = [np.zeros(A.n_rows) for A in systems]
    res = M.mlbicgstab_solve_batch(hs, bs, xs, [1e-10] * len(hs), [4000] * len(hs))
    for A, b, r, x in zip(systems, bs, res, xs):
        assert r.flag == 0 and r.true_relres < 1e-10
        h1 = M.mlbicgstab_create(A, n=4, q_seed=0, precond=1, precision=precision, grid=1)
        x1 = np.zeros(A.n_rows)
        r1, _ = M.mlbicgstab_solve(h1, b, x1, 1e-10, 4000)
        assert (r.iter, r.flag) == (r1.iter, r1.flag)
        np.testing.assert_array_equal(x, x1)
        ref = O.solve(A, b, np.zeros(A.n_rows), O.q_gauss(0, A.n_rows, 4), 4000, 1e-10, mdiag=O.jacobi_diag(A))
        assert ref.flag == 0 and ref.true_relres < 1e-10
        # two solutions whose residuals are below tol differ by at most
        # cond(A) * 2 tol relative (forward error of a backward-stable stop);
        # the column scaling makes these systems worse conditioned than the
        # unscaled ones, so the bound is computed, not assumed
        rel = np.linalg.norm(x - ref.x) / np.linalg.norm(ref.x)
        assert rel <= 1e-8 or rel <= 2.0 * _cond(A) * 1e-10


def test_jacobi_edge_cases():
    import torch
    A = W.cd2d(8)
    # a zero diagonal entry has no Jacobi preconditioner
    Z = W.CSR(row_ptr=A.row_ptr.copy(), col=A.col.copy(), val=A.val.copy(), n_rows=A.n_rows)
    Z.val[(Z.col == 0) & (np.arange(Z.nnz) < Z.row_ptr[1])] = 0.0
    with pytest.raises(M.MlbError) as e:
        M.mlbicgstab_create(Z, n=2, precond=M.MLB_PRECOND_JACOBI)
    assert e.value.code == M.MLB_ERR_ARG
    # the fused product of a preconditioned handle is not A x
    h = M.mlbicgstab_create(A, n=2, precond=M.MLB_PRECOND_JACOBI)
    x = torch.ones(A.n_rows, dtype=torch.float64, device="cuda")
    y = torch.empty_like(x)
    with pytest.raises(M.MlbError) as e:
        M.mlbicgstab_spmv_qdot(h, x, y)
    assert e.value.code == M.MLB_ERR_UNSUPPORTED
    # b = 0 gives x = 0 at iteration 0; a nonzero x_0 is mapped through M
    b = np.zeros(A.n_rows)
    x0 = np.zeros(A.n_rows)
    r, _ = M.mlbicgstab_solve(h, b, x0, 1e-10, 100)
    assert r.iter == 0 and r.flag == 0 and not x0.any()
    bb = W.row_sums(A)
    xs = np.ones(A.n_rows)            # the exact solution as x_0
    r, _ = M.mlbicgstab_solve(h, bb, xs, 1e-10, 100)
    assert r.iter == 0 and r.flag == 0
    np.testing.assert_allclose(xs, 1.0, rtol=1e-14)
