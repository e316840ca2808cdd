"""ILU(0) preconditioning (Algorithm 7.1 with M = L U, the preconditioner of
the paper's experiments, §5) through the C ABI.

The library factors A on the host and, in every product of the iteration,
applies M^{-1} by level-scheduled triangular solves inside the persistent
kernel; it iterates on y = M x.  The oracle applies M literally (g^ =
M^{-1} g beside g, x along g^).  They agree to rounding: early residual
histories within the sequential-sum bound used for the other paths,
converged solutions within 1e-8 (or the forward-error bound cond(A) 2 tol
of two solutions whose residuals meet tol).
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle as O
from paper_1106_3678_gb300 import mlbicgstab as M
from paper_1106_3678_gb300 import workloads as W

pytestmark = pytest.mark.gpu
EPS = np.finfo(np.float64).eps
ILU = M.MLB_PRECOND_ILU0


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1106_3678_gb300 import build
    build.build()
    M.load()


def _early_tol(N):
    return max(1e-10, 4 * N * EPS)


def _hist_close(got, want, N):
    """Residual histories ||r_k||/||b|| agree to the rounding of forming r:
    a relative part, and an absolute part of about N eps in these units,
    which does not shrink as ||r_k|| falls (ILU(0) lowers the residual by
    orders of magnitude within the first few steps)."""
    np.testing.assert_allclose(got, want, rtol=_early_tol(N), atol=4 * N * EPS)


def _random_sparse(N, density, seed, cplx=False, shift=3.0):
    rng = np.random.default_rng(seed)
    D = np.where(rng.uniform(size=(N, N)) < density, rng.standard_normal((N, N)), 0.0)
    if cplx:
        D = D + 1j * np.where(D != 0, rng.standard_normal((N, N)), 0.0)
    D = D + shift * np.eye(N)
    return W.dense_to_csr(D), D


@pytest.mark.parametrize("n", [1, 4, 8])
@pytest.mark.parametrize("mat", ["cd2d", "cd3d"])
def test_ilu_matches_oracle(n, mat):
    A = W.cd2d(32) if mat == "cd2d" else W.cd3d_lognormal(12)
    b = W.uniform_rhs(A.n_rows, seed=5)
    N = A.n_rows
    f = O.ilu0(A)
    h = M.mlbicgstab_create(A, n=n, q_seed=0, precond=ILU)
    assert M.mlbicgstab_info(h)["precond"] == ILU
    Q = O.q_gauss(0, N, n)
    K = 10
    x = np.zeros(N)
    res, eh = M.mlbicgstab_solve(h, b, x, 0.0, K, hist_cap=K + 1)
    ref = O.mlbicgstabt(A, b, np.zeros(N), Q, K, 0.0, err_hist=True, ilu=f)
    assert (res.iter, res.j, res.i) == (ref.iter, ref.j, ref.i)
    _hist_close(eh[:K + 1], ref.err_hist[:K + 1], N)
    np.testing.assert_allclose(x, ref.x, rtol=0, atol=1e-9 * np.max(np.abs(ref.x)))
    # full solve: far fewer iterations than M = I, the oracle's count, and
    # the oracle's solution
    x = np.zeros(N)
    res, _ = M.mlbicgstab_solve(h, b, x, 1e-10, 5000)
    ref = O.solve(A, b, np.zeros(N), Q, 5000, 1e-10, ilu=f)
    assert res.flag == 0 and ref.flag == 0
    assert res.true_relres < 1e-10
    assert abs(res.iter - ref.iter) <= max(2, ref.iter // 10)
    assert np.linalg.norm(x - ref.x) <= 1e-8 * np.linalg.norm(ref.x)
    plain = O.solve(A, b, np.zeros(N), Q, 5000, 1e-10)
    assert res.iter * 2 < plain.iter


def test_ilu_complex_matches_oracle():
    A, D = _random_sparse(300, 0.02, seed=61, cplx=True)
    b = np.random.default_rng(62).standard_normal(300) + 1j * np.random.default_rng(63).standard_normal(300)
    f = O.ilu0(A)
    for AH in (None, W.conj_transpose(A)):
        h = M.mlbicgstab_create(A, AH=AH, n=4, q_seed=0, precond=ILU)
        x = np.zeros(300, dtype=complex)
        K = 8
        res, eh = M.mlbicgstab_solve(h, b, x, 0.0, K, hist_cap=K + 1)
        ref = O.mlbicgstabt(A, b, np.zeros(300, dtype=complex), O.q_gauss(0, 300, 4, complex_=True), K, 0.0,
                            err_hist=True, ilu=f)
        _hist_close(eh[:K + 1], ref.err_hist[:K + 1], 300)
        x = np.zeros(300, dtype=complex)
        res, _ = M.mlbicgstab_solve(h, b, x, 1e-12, 400)
        assert res.flag == 0 and res.true_relres < 1e-12
        xs = np.linalg.solve(D, b)
        assert np.linalg.norm(x - xs) <= 1e-10 * np.linalg.norm(xs)


def test_ilu_with_full_pattern_is_exact_and_converges_at_once():
    """A dense pattern makes ILU(0) the exact LU: A M^{-1} = I, so the first
    step solves the system."""
    A, D, b = W.random_dense_system(60, seed=64)
    h = M.mlbicgstab_create(A, n=4, q_seed=0, precond=ILU)
    x = np.zeros(60)
    res, _ = M.mlbicgstab_solve(h, b, x, 1e-12, 50)
    assert res.flag == 0 and res.iter == 1
    xs = np.linalg.solve(D, b)
    assert np.linalg.norm(x - xs) <= 1e-12 * np.linalg.norm(xs)


def test_ilu_batch_equals_single_cta():
    """Batch: one CTA per system with CTA barriers between levels; the same
    arithmetic as a single solve on a grid of one CTA, bit for bit."""
    systems = [A for A, _ in W.batch_cd(10, seed=65, n_min=300, n_max=3000)]
    hs = [M.mlbicgstab_create(A, n=4, q_seed=0, precond=ILU) for A in systems]
    bs = [W.uniform_rhs(A.n_rows, seed=66) for A in systems]
    xs = [np.zeros(A.n_rows) for A in systems]
    res = M.mlbicgstab_solve_batch(hs, bs, xs, [1e-10] * len(hs), [2000] * len(hs))
    for A, b, r, x in zip(systems, bs, res, xs):
        assert r.flag == 0 and r.true_relres < 1e-10
        h1 = M.mlbicgstab_create(A, n=4, q_seed=0, precond=ILU, grid=1)
        x1 = np.zeros(A.n_rows)
        r1, _ = M.mlbicgstab_solve(h1, b, x1, 1e-10, 2000)
        assert (r.iter, r.flag) == (r1.iter, r1.flag)
        np.testing.assert_array_equal(x, x1)
        ref = O.solve(A, b, np.zeros(A.n_rows), O.q_gauss(0, A.n_rows, 4), 2000, 1e-10, ilu=O.ilu0(A))
        assert ref.flag == 0
        assert np.linalg.norm(x - ref.x) <= 1e-8 * np.linalg.norm(ref.x)


def test_ilu_many_levels_across_the_grid():
    """32^3 log-normal system (93 + 93 levels over all CTAs, a grid barrier
    per level): converges like the oracle to the oracle's solution."""
    A = W.cd3d_lognormal(32)
    b = W.uniform_rhs(A.n_rows, seed=2)
    N = A.n_rows
    h = M.mlbicgstab_create(A, n=4, q_seed=0, precond=ILU)
    x = np.zeros(N)
    res, _ = M.mlbicgstab_solve(h, b, x, 1e-10, 4000)
    ref = O.solve(A, b, np.zeros(N), O.q_gauss(0, N, 4), 4000, 1e-10, ilu=O.ilu0(A))
    assert res.flag == 0 and ref.flag == 0 and res.true_relres < 1e-10
    assert abs(res.iter - ref.iter) <= max(3, ref.iter // 10)
    assert np.linalg.norm(x - ref.x) <= 1e-7 * np.linalg.norm(ref.x)


def test_ilu_edge_cases():
    A = W.cd2d(8)
    N = A.n_rows
    # a zero pivot has no ILU(0)
    Z = W.CSR(row_ptr=A.row_ptr.copy(), col=A.col.copy(), val=A.val.copy(), n_rows=N)
    Z.val[(Z.col == 0) & (np.arange(Z.nnz) < Z.row_ptr[1])] = 0.0
    with pytest.raises(M.MlbError) as e:
        M.mlbicgstab_create(Z, n=2, precond=ILU)
    assert e.value.code == M.MLB_ERR_ARG
    # a row without a stored diagonal
    keep = np.ones(A.nnz, dtype=bool)
    keep[np.flatnonzero((A.col == 1) & (np.arange(A.nnz) >= A.row_ptr[1]) & (np.arange(A.nnz) < A.row_ptr[2]))] = False
    rp = np.concatenate([[0], np.cumsum([keep[A.row_ptr[r]:A.row_ptr[r + 1]].sum() for r in range(N)])])
    D = W.CSR(row_ptr=rp.astype(np.int64), col=A.col[keep].copy(), val=A.val[keep].copy(), n_rows=N)
    with pytest.raises(M.MlbError) as e:
        M.mlbicgstab_create(D, n=2, precond=ILU)
    assert e.value.code == M.MLB_ERR_ARG
    # the refined mode's FP32 factors are checked the same way
    with pytest.raises(M.MlbError) as e:
        M.mlbicgstab_create(D, n=2, precond=ILU, precision=M.MLB_PREC_FP32_REFINED)
    assert e.value.code == M.MLB_ERR_ARG
    # columns given out of order (and a repeated entry) are sorted and merged
    perm = np.concatenate([np.arange(A.row_ptr[r], A.row_ptr[r + 1])[::-1] for r in range(N)])
    S = W.CSR(row_ptr=A.row_ptr.copy(), col=A.col[perm].copy(), val=A.val[perm].copy(), n_rows=N)
    b = W.row_sums(A)
    h0 = M.mlbicgstab_create(A, n=2, q_seed=0, precond=ILU)
    h1 = M.mlbicgstab_create(S, n=2, q_seed=0, precond=ILU)
    x0, x1 = np.zeros(N), np.zeros(N)
    r0, _ = M.mlbicgstab_solve(h0, b, x0, 1e-12, 500)
    r1, _ = M.mlbicgstab_solve(h1, b, x1, 1e-12, 500)
    assert r0.flag == 0 and r1.flag == 0
    np.testing.assert_allclose(x1, 1.0, rtol=1e-10)
    # b = 0 gives x = 0 at iteration 0; the exact solution as x_0 returns at
    # once (x_0 -> M x_0 -> M^{-1} M x_0 up to rounding)
    x = np.zeros(N)
    r, _ = M.mlbicgstab_solve(h0, np.zeros(N), x, 1e-10, 100)
    assert r.iter == 0 and r.flag == 0 and not x.any()
    x = np.ones(N)
    r, _ = M.mlbicgstab_solve(h0, b, x, 1e-10, 100)
    assert r.iter == 0 and r.flag == 0
    np.testing.assert_allclose(x, 1.0, rtol=1e-13)


def test_ilu_block_reservoir_matches_oracle():
    """3x3-block reservoir system (21 entries per row: most rows have more
    entries per triangle than the solve keeps in registers).  ILU(0) solves
    it in a handful of iterations where M = I needs thousands."""
    A = W.bsr3_to_csr(W.reservoir_bsr3(8, 8, 4))
    b = W.row_sums(A)
    N = A.n_rows
    f = O.ilu0(A)
    Q = O.q_gauss(0, N, 8)
    h = M.mlbicgstab_create(A, n=8, q_seed=0, precond=ILU)
    x = np.zeros(N)
    K = 6
    res, eh = M.mlbicgstab_solve(h, b, x, 0.0, K, hist_cap=K + 1)
    ref = O.mlbicgstabt(A, b, np.zeros(N), Q, K, 0.0, err_hist=True, ilu=f)
    _hist_close(eh[:K + 1], ref.err_hist[:K + 1], N)
    x = np.zeros(N)
    res, _ = M.mlbicgstab_solve(h, b, x, 1e-10, 2000)
    ref = O.solve(A, b, np.zeros(N), Q, 2000, 1e-10, ilu=f)
    assert res.flag == 0 and ref.flag == 0 and res.true_relres < 1e-10
    assert abs(res.iter - ref.iter) <= 2 and res.iter < 50
    np.testing.assert_allclose(x, 1.0, rtol=1e-8)


def test_ilu_with_kappa_set_n_and_autotuned_grid():
    """ILU(0) combined with the Eq. 5.1 guard, a handle built for n = 8 and
    set to n = 4, and a launch configuration chosen by the autotuner (the
    levels are then split over a different number of CTAs)."""
    A = W.cd3d_lognormal(16)
    b = W.uniform_rhs(A.n_rows, seed=7)
    N = A.n_rows
    f = O.ilu0(A)
    h = M.mlbicgstab_create(A, n=8, q_seed=0, precond=ILU, kappa=0.7)
    M.mlbicgstab_set_n(h, 4)
    Q4 = O.q_gauss(0, N, 8)[:, :4]
    ref = O.solve(A, b, np.zeros(N), Q4, 2000, 1e-10, kappa=0.7, ilu=f)
    assert ref.flag == 0
    x = np.zeros(N)
    res, _ = M.mlbicgstab_solve(h, b, x, 1e-10, 2000)
    assert res.flag == 0 and res.true_relres < 1e-10
    assert abs(res.iter - ref.iter) <= max(2, ref.iter // 10)
    assert np.linalg.norm(x - ref.x) <= 1e-8 * np.linalg.norm(ref.x)
    grid0 = M.mlbicgstab_info(h)["grid"]
    tune = M.mlbicgstab_autotune(h, iters=5, use_cache=False)
    assert tune["grid"] == M.mlbicgstab_info(h)["grid"]
    x2 = np.zeros(N)
    res2, _ = M.mlbicgstab_solve(h, b, x2, 1e-10, 2000)
    assert res2.flag == 0 and res2.true_relres < 1e-10
    assert np.linalg.norm(x2 - ref.x) <= 1e-8 * np.linalg.norm(ref.x)
    # one CTA (the level loop with CTA barriers only) gives the same answer
    h1 = M.mlbicgstab_create(A, n=4, q_seed=0, precond=ILU, kappa=0.7, grid=1)
    x1 = np.zeros(N)
    r1, _ = M.mlbicgstab_solve(h1, b, x1, 1e-10, 2000)
    assert r1.flag == 0 and np.linalg.norm(x1 - ref.x) <= 1e-8 * np.linalg.norm(ref.x)
    assert grid0 >= 1


def test_ilu_full_size_cd3d_first_iterations_elementwise():
    """The 128^3 ILU(0) workload at full size in the bench's launch
    geometry: 6 iterations against the oracle's, x element by element."""
    A = W.cd3d_lognormal(128)
    b = W.uniform_rhs(A.n_rows, seed=2)
    N = A.n_rows
    h = M.mlbicgstab_create(A, n=4, q_seed=0, precond=ILU)
    K = 6
    x = np.zeros(N)
    res, eh = M.mlbicgstab_solve(h, b, x, 0.0, K, hist_cap=K + 1)
    ref = O.mlbicgstabt(A, b, np.zeros(N), O.q_gauss(0, N, 4), K, 0.0, err_hist=True, ilu=O.ilu0(A))
    assert (res.iter, res.j, res.i) == (ref.iter, ref.j, ref.i)
    _hist_close(eh[:K + 1], ref.err_hist[:K + 1], N)
    assert np.max(np.abs(x - ref.x)) <= 1e-8 * np.max(np.abs(ref.x))


def test_ilu_full_size_reservoir_solve():
    """The 3x3-block reservoir workload at full size (393,216 rows), solved
    to 1e-10 with ILU(0): the oracle's iteration count and solution, and
    the true residual recomputed on the host."""
    A = W.bsr3_to_csr(W.reservoir_bsr3())
    b = W.row_sums(A)
    N = A.n_rows
    h = M.mlbicgstab_create(A, n=8, q_seed=0, precond=ILU)
    x = np.zeros(N)
    res, _ = M.mlbicgstab_solve(h, b, x, 1e-10, 200)
    ref = O.solve(A, b, np.zeros(N), O.q_gauss(0, N, 8), 200, 1e-10, ilu=O.ilu0(A))
    assert res.flag == 0 and ref.flag == 0
    assert abs(res.iter - ref.iter) <= 1
    assert O.true_relres(A, b, x) < 1e-10
    assert np.linalg.norm(x - ref.x) <= 1e-8 * np.linalg.norm(ref.x)


def test_batch_mixing_preconditioners():
    """One batch with handles of every preconditioner: the kernel with the
    ILU(0) passes runs every item by its own view, and each result equals
    the same system solved alone on one CTA, bit for bit."""
    systems = [A for A, _ in W.batch_cd(6, seed=71, n_min=300, n_max=2000)]
    pcs = [M.MLB_PRECOND_NONE, M.MLB_PRECOND_JACOBI, ILU] * 2
    hs = [M.mlbicgstab_create(A, n=4, q_seed=0, precond=pc) for A, pc in zip(systems, pcs)]
    bs = [W.uniform_rhs(A.n_rows, seed=72) for A in systems]
    xs = [np.zeros(A.n_rows) for A in systems]
    res = M.mlbicgstab_solve_batch(hs, bs, xs, [1e-10] * 6, [4000] * 6)
    for A, pc, b, r, x in zip(systems, pcs, bs, res, xs):
        assert r.flag == 0 and r.true_relres < 1e-10
        h1 = M.mlbicgstab_create(A, n=4, q_seed=0, precond=pc, grid=1)
        x1 = np.zeros(A.n_rows)
        r1, _ = M.mlbicgstab_solve(h1, b, x1, 1e-10, 4000)
        assert (r.iter, r.flag) == (r1.iter, r1.flag), pc
        np.testing.assert_array_equal(x, x1)
