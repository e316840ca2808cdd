"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Each test names the passage it rests on.  None of them re-derives the
oracle's own formulas: they compare with printed values (Table 2.1), with
independently written textbook methods (Bi-CGSTAB for n = 1), with library
routines (LAPACK via numpy.linalg.solve, SciPy/NumPy products), with exact
finite-termination properties of the Petrov–Galerkin construction
(Algorithm 3.1 and its FOM/GMRES relations), and with the operation counts
of Table 4.3.
"""
from __future__ import annotations

import os

import numpy as np
import pytest

from paper_1106_3678_gb300 import workloads as W
from tests import textbook as TB

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- §2 -------

def test_table_2_1_bit_exact(orc):
    """Table 2.1 (n = 3, k = 0..12), every entry."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "table_2_1.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 13
    for n, k, g, r in (map(int, row) for row in rows):
        assert orc.gn(n, k) == g
        assert orc.rn(n, k) == r


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 16])
def test_index_identity_eq_2_1(orc, n):
    """Eq. 2.1: k = jn + i with 1 <= i <= n gives g_n(k) = j, r_n(k) = i,
    for every integer j, negative ones included (floor toward -inf)."""
    for j in range(-7, 9):
        for i in range(1, n + 1):
            assert orc.gn(n, j * n + i) == j
            assert orc.rn(n, j * n + i) == i


# ------------------------------------------------------- products ----------

def test_spmv_and_ahq_match_dense_products(orc):
    """y = A x and F = A^H Q against dense NumPy products (real, complex)."""
    rng = np.random.default_rng(7)
    for cplx in (False, True):
        A, M, _ = W.random_dense_system(9, seed=3, complex_=cplx)
        x = rng.standard_normal(9) + (1j * rng.standard_normal(9) if cplx else 0)
        np.testing.assert_allclose(orc.spmv(A, x), M @ x, rtol=1e-14, atol=1e-14)
        Q = rng.standard_normal((9, 4))
        if cplx:
            Q = Q + 1j * rng.standard_normal((9, 4))
        F = orc.ahq(A, Q, 3)
        np.testing.assert_allclose(F, M.conj().T @ Q[:, :3], rtol=1e-13,
                                   atol=1e-13)
    A = W.cd2d(8)
    Md = TB.dense(A)
    x = rng.standard_normal(A.n_rows)
    np.testing.assert_allclose(orc.spmv(A, x), Md @ x, rtol=1e-14, atol=1e-14)


def test_shadow_generator_is_standard_normal(orc):
    """The documented generator yields N(0,1) samples, column-major, with
    complex entries built from consecutive normals."""
    from scipy import stats
    N, n = 20000, 3
    Q = orc.q_gauss(11, N, n)
    assert Q.shape == (N, n)
    flat = Q.reshape(-1, order="F")
    assert abs(flat.mean()) < 0.02 and abs(flat.var() - 1.0) < 0.03
    assert stats.kstest(flat, "norm").pvalue > 1e-3
    assert flat[5] == orc.normal_at(11, 5)
    assert Q[7, 2] == orc.normal_at(11, 2 * N + 7)
    Qc = orc.q_gauss(11, 5, 2, complex_=True)
    assert Qc[1, 1].real == orc.normal_at(11, 2 * (5 + 1))
    assert Qc[1, 1].imag == orc.normal_at(11, 2 * (5 + 1) + 1)
    assert not np.array_equal(orc.q_gauss(12, 10, 1), orc.q_gauss(11, 10, 1))


# ------------------------------------------------ n = 1 is BiCGStab --------

def _n1_max_rel_diff(orc, A, b, matvec, q, steps):
    x0 = np.zeros(A.n_rows, dtype=b.dtype)
    res = orc.mlbicgstabt(A, b, x0, q[:, None], maxit=steps, tol=0.0,
                          x_hist=steps)
    assert res.iter == steps and res.flag == 1
    xs, _ = TB.bicgstab(matvec, b, x0, q, steps)
    return [np.linalg.norm(res.x_hist[k] - xs[k]) / np.linalg.norm(xs[k])
            for k in range(steps)]


@pytest.mark.parametrize("N", [300, 1000])
@pytest.mark.parametrize("shadow", ["r0", "random"])
def test_n1_matches_textbook_bicgstab(orc, N, shadow):
    """§4.3: ML(1)BiCGStabt is BiCGStab.  One oracle iteration at n = 1 is a
    full Bi-CGSTAB step (the i-loop is empty), so x after each iteration is
    compared with the textbook iterate: relative difference <= 1e-12 over
    the first 20 iterations, on well-conditioned systems where rounding
    differences are not amplified."""
    A, M, b = W.random_dense_system(N, seed=1, shift=2.0)
    q = b.copy() if shadow == "r0" else np.random.default_rng(4).standard_normal(N)
    d = _n1_max_rel_diff(orc, A, b, lambda v: M @ v, q, 20)
    assert max(d) <= 1e-12, d


def test_n1_matches_textbook_bicgstab_cd2d(orc):
    """The same equivalence on the 32x32 convection-diffusion system.  Here
    the two rounding orders drift apart geometrically from ~1e-16 (near
    breakdowns of BiCGStab amplify them), so the 1e-12 bound is held over
    the first 12 steps, where the growth has not yet reached it."""
    A = W.cd2d(32)
    b = W.row_sums(A)
    for q in (b.copy(), np.random.default_rng(4).standard_normal(A.n_rows)):
        d = _n1_max_rel_diff(orc, A, b, TB.csr_matvec(A), q, 12)
        assert max(d) <= 1e-12, d


def test_n1_matches_textbook_bicgstab_complex(orc):
    """Same pin in complex arithmetic (conjugated inner products)."""
    A, M, b = W.random_dense_system(40, seed=8, complex_=True, shift=2.0)
    x0 = np.zeros(40, dtype=complex)
    q = np.random.default_rng(9).standard_normal(40) * (1 + 0.5j)
    res = orc.mlbicgstabt(A, b, x0, q[:, None], maxit=15, tol=0.0, x_hist=15)
    xs, _ = TB.bicgstab(lambda v: M @ v, b, x0, q, 15)
    for k in range(15):
        rel = np.linalg.norm(res.x_hist[k] - xs[k]) / np.linalg.norm(xs[k])
        assert rel <= 1e-12, (k, rel)


def test_kappa_guard_matches_safeguarded_bicgstab(orc):
    """Eq. 5.1 (kappa = 0.7, the value of the paper's sample run) at n = 1
    against Bi-CGSTAB with the Sleijpen–van der Vorst safeguard; the
    problem, I + 0.7·(skew-symmetric), makes (Au)^H u small relative to
    ||Au|| ||u|| so that the guard fires at every step, while staying well
    conditioned.  The enlarged omega makes the residual erratic, which
    amplifies the rounding differences of the two formulations
    geometrically from ~1e-16, so the 1e-12 bound is held over 6 steps."""
    N = 200
    rng = np.random.default_rng(2)
    R = rng.standard_normal((N, N)) / np.sqrt(N)
    M = np.eye(N) + 0.7 * (R - R.T)
    A = W.dense_to_csr(M)
    b = rng.standard_normal(N)
    x0 = np.zeros(N)
    q = rng.standard_normal(N)
    mv = lambda v: M @ v  # noqa: E731
    xs, guards = TB.bicgstab(mv, b, x0, q, 6, kappa=0.7)
    assert all(g < 0.7 for g in guards)  # the guard really fires
    res = orc.mlbicgstabt(A, b, x0, q[:, None], maxit=6, tol=0.0, kappa=0.7,
                          x_hist=6)
    for k in range(6):
        rel = np.linalg.norm(res.x_hist[k] - xs[k]) / np.linalg.norm(xs[k])
        assert rel <= 1e-12, (k, rel)
    # and without the guard the iterates differ: the pin has teeth
    res0 = orc.mlbicgstabt(A, b, x0, q[:, None], maxit=6, tol=0.0, x_hist=6)
    assert np.linalg.norm(res0.x_hist[-1] - xs[-1]) > 1e-6 * np.linalg.norm(xs[-1])


# ---------------------------------------- n >= N: finite termination ------

@pytest.mark.parametrize("N,n", [(6, 1), (6, 2), (8, 3), (8, 4), (10, 2),
                                 (10, 5), (5, 5), (8, 8), (12, 12), (6, 9),
                                 (10, 11)])
@pytest.mark.parametrize("cplx", [False, True])
def test_finite_termination_within_N_steps(orc, N, n, cplx):
    """Algorithm 3.1's Petrov–Galerkin conditions p_m^H r̂_k = 0 for m <= k,
    with p_m = (A^H)^{g_n(m)} q_{r_n(m)}: once N independent p_m are used,
    r̂_N = 0, and eq. 4.1 gives r_N = Omega(A) r̂_N = 0.  So in exact
    arithmetic the method stops by step N for every n; for n >= N this is
    the FOM/GMRES relation of §3 (block 0 only), for n < N it exercises
    the j >= 1 recurrences.  The solve must stop by iteration N (tol
    1e-14, far below the pre-termination residuals) and agree with LAPACK."""
    A, M, b = W.random_dense_system(N, seed=100 + N + n, complex_=cplx)
    rng = np.random.default_rng(10 * N + n)
    Q = rng.standard_normal((N, n))
    if cplx:
        Q = Q + 1j * rng.standard_normal((N, n))
    x0 = np.zeros(N, dtype=b.dtype)
    res = orc.mlbicgstabt(A, b, x0, Q, maxit=4 * N, tol=1e-14)
    assert res.flag == 0
    assert res.iter <= N
    xs = np.linalg.solve(M, b)
    assert np.linalg.norm(res.x - xs) <= 1e-10 * np.linalg.norm(xs)


@pytest.mark.parametrize("cplx", [False, True])
def test_block0_biorthogonality(orc, cplx):
    """Inside block 0 the residuals satisfy q_m^H r_k = 0 for m <= k
    (Algorithm 3.1 with p_m = q_m, r_k = r̂_k while k < n)."""
    N, n = 30, 8
    A, M, b = W.random_dense_system(N, seed=5, complex_=cplx)
    rng = np.random.default_rng(6)
    Q = rng.standard_normal((N, n)) + (1j * rng.standard_normal((N, n)) if cplx else 0)
    x0 = np.zeros(N, dtype=b.dtype)
    res = orc.mlbicgstabt(A, b, x0, Q, maxit=n - 1, tol=0.0, x_hist=n - 1)
    r0 = b - M @ x0
    for k in range(1, n):
        rk = b - M @ res.x_hist[k - 1]
        for m in range(1, k + 1):
            q = Q[:, m - 1]
            assert abs(np.vdot(q, rk)) <= 1e-10 * np.linalg.norm(q) * np.linalg.norm(r0), (k, m)


# ------------------------------------------------ dense LU agreement -------

@pytest.mark.parametrize("n", [1, 4, 8])
def test_cd2d_agrees_with_dense_lu(orc, n):
    """The 32x32 convection-diffusion system (N = 1024): the solution lands
    within 1e-10 relative of a LAPACK LU solve (tol tightened to 1e-13 so
    that cond(A)·tol stays below the bound)."""
    A = W.cd2d(32)
    b = W.row_sums(A)
    Q = orc.q_gauss(0, A.n_rows, n)
    res = orc.mlbicgstabt(A, b, np.zeros(A.n_rows), Q, maxit=4000, tol=1e-13)
    assert res.flag == 0
    xs = np.linalg.solve(TB.dense(A), b)
    assert np.linalg.norm(res.x - xs) <= 1e-10 * np.linalg.norm(xs)
    assert np.max(np.abs(res.x - 1.0)) < 1e-9   # b = A·1


@pytest.mark.parametrize("n", [2, 4])
def test_complex_helmholtz_small_agrees_with_lu(orc, n):
    A = W.helmholtz3d_c(8, 8, 4, k=3.0)
    b = W.row_sums(A)
    Q = orc.q_gauss(0, A.n_rows, n, complex_=True)
    res = orc.mlbicgstabt(A, b, np.zeros(A.n_rows, complex), Q, maxit=3000,
                          tol=1e-13)
    assert res.flag == 0
    xs = np.linalg.solve(TB.dense(A), b)
    assert np.linalg.norm(res.x - xs) <= 1e-10 * np.linalg.norm(xs)


# --------------------------------------------- Table 4.3 op counts ---------

@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 8])
def test_table_4_3_operation_counts_per_block(orc, n):
    """Table 4.3 per iteration, times n for one full block j >= 1:
    matvec n+1, dot n^2+n+2, saxpy 1.5n^2+2.5n+2, 'alpha v' n.  The norms of
    the stopping rule (not in the table) are n+1 per block.  Block 0 takes
    the f-sweep branch of Algorithm 7.1 instead of the q-sweep."""
    A = W.cd2d(16)
    b = W.row_sums(A)
    Q = orc.q_gauss(3, A.n_rows, n)
    nblocks = 4
    res = orc.mlbicgstabt(A, b, np.zeros(A.n_rows), Q, maxit=nblocks * n + 1,
                          tol=0.0, blk_ops=nblocks + 1, trace=True)
    assert res.iter == nblocks * n + 1 and res.flag == 1
    bo = res.blk_ops
    for j in range(1, nblocks):
        d = bo[j + 1] - bo[j]
        assert d[0] == n + 1
        assert d[1] == n * n + n + 2
        assert 2 * d[2] == 3 * n * n + 5 * n + 4
        assert d[3] == n
        assert d[4] == n + 1
    # block 0: per step i (1..n-1) dots i+2, saxpys i+2; the block end as
    # in later blocks (dots n+3, saxpys 2n+4, one 'alpha v', 2 matvecs)
    d0 = bo[1] - bo[0]
    assert d0[0] == (n - 1) + 2
    assert d0[1] == sum(i + 2 for i in range(1, n)) + n + 3
    assert d0[2] == sum(i + 2 for i in range(1, n)) + 2 * n + 4
    assert d0[3] == 1
    # the trace walks k = jn + i (eq. 2.1)
    for k in range(1, res.iter + 1):
        j, i = res.trace[k - 1]
        assert (j, i) == (orc.gn(n, k), orc.rn(n, k))


# ------------------------------------------------ flags and edge cases -----

def test_zero_rhs_uses_unit_denominator(orc):
    """b = 0 with x0 = 0: ||b|| is replaced by 1, r0 = 0, err = 0 < tol,
    so the call returns at once with flag 0 and iter 0 (§5 stopping rule)."""
    A = W.cd2d(8)
    Q = orc.q_gauss(0, A.n_rows, 3)
    res = orc.mlbicgstabt(A, np.zeros(A.n_rows), np.zeros(A.n_rows), Q, 100, 1e-10)
    assert (res.iter, res.flag, res.err) == (0, 0, 0.0)
    # nonzero x0 with b = 0: err = ||A x0|| / 1
    x0 = np.ones(A.n_rows)
    res = orc.mlbicgstabt(A, np.zeros(A.n_rows), x0, Q, 0, 1e-10, err_hist=True)
    assert res.err_hist[0] == pytest.approx(np.linalg.norm(TB.dense(A) @ x0), rel=1e-14)


def test_exact_initial_guess_returns_immediately(orc):
    A = W.cd2d(8)
    b = W.row_sums(A)
    Q = orc.q_gauss(0, A.n_rows, 4)
    res = orc.mlbicgstabt(A, b, np.ones(A.n_rows), Q, 100, 1e-10)
    assert res.iter == 0 and res.flag == 0


def test_iteration_limit_flag(orc):
    A = W.cd2d(16)
    b = W.row_sums(A)
    for n, maxit in [(4, 7), (4, 8), (3, 5), (1, 3)]:
        Q = orc.q_gauss(0, A.n_rows, n)
        res = orc.mlbicgstabt(A, b, np.zeros(A.n_rows), Q, maxit, 1e-14)
        assert res.flag == 1 and res.iter == maxit


def test_breakdown_c_zero(orc):
    """q_1 orthogonal to A r_0 makes c_0 = 0: breakdown (flag -1) at setup.
    With b = e_k and x_0 = 0, A r_0 is column k of A, computed exactly, and
    q_1 = (a_jk e_i - a_ik e_j) is exactly orthogonal to it."""
    A = W.cd2d(6)
    N = A.n_rows
    k = 7
    b = np.zeros(N)
    b[k] = 1.0
    colk = TB.dense(A)[:, k]
    i, j = np.nonzero(colk)[0][:2]
    q = np.zeros(N)
    q[i], q[j] = colk[j], -colk[i]
    res = orc.mlbicgstabt(A, b, np.zeros(N), q[:, None], 50, 1e-10)
    assert res.flag == -1 and res.iter == 0


def test_breakdown_zero_Au(orc):
    """A = I, n = 1, tol = 0: alpha = 1 makes u = 0 exactly, so ||A u|| = 0
    and the omega step breaks down (flag -1) after the first half step."""
    N = 10
    A = W.dense_to_csr(np.eye(N))
    b = np.arange(1.0, N + 1)
    q = np.ones(N)
    res = orc.mlbicgstabt(A, b, np.zeros(N), q[:, None], 50, 0.0)
    assert res.flag == -1


def test_restart_wrapper_reaches_true_residual(orc):
    """The restart wrapper stops on the true residual ||b - A x||/||b||."""
    A = W.cd2d(32)
    b = W.row_sums(A)
    Q = orc.q_gauss(0, A.n_rows, 4)
    res = orc.solve(A, b, np.zeros(A.n_rows), Q, 2000, 1e-10)
    assert res.flag == 0 and res.true_relres < 1e-10


# ---------------------------------------------------------------------------
# Preconditioning: Algorithm 7.1 with a diagonal M (Jacobi, M = diag(A))
# ---------------------------------------------------------------------------

def _col_scaled(A, s):
    """A diag(s) (column j of A multiplied by s_j)."""
    return W.CSR(row_ptr=A.row_ptr.copy(), col=A.col.copy(), val=A.val * s[A.col], n_rows=A.n_rows)


def test_precond_identity_is_unpreconditioned(orc):
    """M = I given explicitly is Algorithm 4.1: division by 1 is exact, so
    every iterate is the same bits as the M = I path."""
    A, _, b = W.random_dense_system(40, seed=41)
    Q = np.random.default_rng(42).standard_normal((40, 4))
    x0 = np.zeros(40)
    r0 = orc.mlbicgstabt(A, b, x0, Q, maxit=25, tol=0.0, err_hist=True, x_hist=25)
    r1 = orc.mlbicgstabt(A, b, x0, Q, maxit=25, tol=0.0, err_hist=True, x_hist=25, mdiag=np.ones(40))
    np.testing.assert_array_equal(r0.err_hist, r1.err_hist)
    np.testing.assert_array_equal(r0.x_hist, r1.x_hist)


@pytest.mark.parametrize("cplx", [False, True])
def test_precond_equals_method_on_right_scaled_system(orc, cplx):
    """Algorithm 7.1 with right preconditioner M solves A M^{-1} y = b with
    x = M^{-1} y: its residuals r = b - A x are those of the M = I method on
    A' = A M^{-1} (F = M^{-H} A^H Q = A'^H Q).  In exact arithmetic the two
    residual sequences coincide; in FP64 they agree to rounding on a
    well-conditioned system, and x_k = M^{-1} y_k."""
    N, n = 36, 4
    A, _, b = W.random_dense_system(N, seed=43, complex_=cplx)
    rng = np.random.default_rng(44)
    # a positive (or nearly real) M keeps A M^{-1} as well conditioned as A,
    # so the two FP64 sequences stay within rounding of each other
    d = rng.uniform(0.5, 2.0, N)
    if cplx:
        d = d * np.exp(1j * rng.uniform(-0.3, 0.3, N))
    Q = rng.standard_normal((N, n)) + (1j * rng.standard_normal((N, n)) if cplx else 0)
    x0 = np.zeros(N, dtype=b.dtype)
    K = 20
    rp = orc.mlbicgstabt(A, b, x0, Q, maxit=K, tol=0.0, err_hist=True, x_hist=K, mdiag=d)
    Ap = _col_scaled(A, 1.0 / d)
    ry = orc.mlbicgstabt(Ap, b, x0, Q, maxit=K, tol=0.0, err_hist=True, x_hist=K)
    np.testing.assert_allclose(rp.err_hist, ry.err_hist, rtol=1e-7)
    for k in range(K):
        xk = ry.x_hist[k] / d
        assert np.linalg.norm(rp.x_hist[k] - xk) <= 1e-7 * np.linalg.norm(xk), k


def test_jacobi_undoes_column_scaling(orc):
    """With M = diag(A), right preconditioning makes the method invariant to
    a column scaling A -> A S (S diagonal): A S (diag(A) S)^{-1} =
    A diag(A)^{-1}.  So the residual history on A S equals the one on A (to
    rounding) and the solution is S^{-1} times A's, whatever S is; without
    preconditioning the scaled system behaves differently."""
    A = W.cd2d(16)
    b = W.row_sums(A)
    N = A.n_rows
    s = 10.0 ** np.random.default_rng(45).uniform(-2, 2, N)
    AS = _col_scaled(A, s)
    Q = orc.q_gauss(0, N, 4)
    x0 = np.zeros(N)
    r1 = orc.mlbicgstabt(A, b, x0, Q, maxit=400, tol=1e-10, err_hist=True, mdiag=orc.jacobi_diag(A))
    r2 = orc.mlbicgstabt(AS, b, x0, Q, maxit=400, tol=1e-10, err_hist=True, mdiag=orc.jacobi_diag(AS))
    assert r1.flag == 0 and r2.flag == 0
    assert abs(r1.iter - r2.iter) <= 2
    k = min(r1.iter, r2.iter, 30)
    np.testing.assert_allclose(r1.err_hist[:k], r2.err_hist[:k], rtol=1e-6)
    np.testing.assert_allclose(r2.x * s, r1.x, rtol=1e-7, atol=1e-9)
    r3 = orc.mlbicgstabt(AS, b, x0, Q, maxit=30, tol=0.0, err_hist=True)
    assert np.max(np.abs(r3.err_hist[1:31] / r2.err_hist[1:31] - 1.0)) > 1e-3


@pytest.mark.parametrize("N,n", [(8, 3), (9, 9)])
def test_precond_finite_termination(orc, N, n):
    """A M^{-1} is still an N x N system, so the preconditioned method also
    stops by step N in exact arithmetic; it must converge by iteration N at
    tol 1e-14 and agree with LAPACK on A x = b."""
    A, M, b = W.random_dense_system(N, seed=200 + N + n)
    d = np.random.default_rng(N).uniform(0.5, 3.0, N)
    Q = np.random.default_rng(N + 1).standard_normal((N, n))
    res = orc.mlbicgstabt(A, b, np.zeros(N), Q, maxit=4 * N, tol=1e-14, mdiag=d)
    assert res.flag == 0 and res.iter <= N
    xs = np.linalg.solve(M, b)
    assert np.linalg.norm(res.x - xs) <= 1e-10 * np.linalg.norm(xs)


def test_jacobi_diag_definition(orc):
    """jacobi_diag sums a row's diagonal entries (duplicates included)."""
    A = W.CSR(row_ptr=np.array([0, 2, 4, 5], dtype=np.int64), col=np.array([0, 0, 0, 2, 2], dtype=np.int32),
              val=np.array([1.0, 2.0, -3.0, 5.0, 7.0]), n_rows=3)
    np.testing.assert_array_equal(orc.jacobi_diag(A), [3.0, 0.0, 7.0])


# ------------------------------------------- ILU(0) preconditioning --------
# The paper's experiments precondition with ILU(0) (§5); Algorithm 7.1 takes
# any M.  ILU(0) is pinned by its definition (Saad, Algorithm 10.4): L unit
# lower and U upper triangular, both inside A's pattern, with (L U)_ij = a_ij
# on that pattern; where elimination makes no fill outside the pattern this
# is the exact LU factorisation.

def _random_sparse(N, density, seed, cplx=False, shift=4.0):
    """Random sparse matrix with a full diagonal, diagonally shifted."""
    rng = np.random.default_rng(seed)
    M = np.where(rng.uniform(size=(N, N)) < density, rng.standard_normal((N, N)), 0.0)
    if cplx:
        M = M + 1j * np.where(M != 0, rng.standard_normal((N, N)), 0.0)
    M = M + shift * np.eye(N)
    return W.dense_to_csr(M), M


def _ilu_dense(A, f):
    """Dense L (unit diagonal) and U from the factors in A's pattern."""
    N = A.n_rows
    L = np.eye(N, dtype=f.lu.dtype)
    U = np.zeros((N, N), dtype=f.lu.dtype)
    for r in range(N):
        for k in range(A.row_ptr[r], A.row_ptr[r + 1]):
            c = A.col[k]
            if c < r:
                L[r, c] = f.lu[k]
            else:
                U[r, c] = f.lu[k]
        assert A.col[f.dpos[r]] == r
    return L, U


@pytest.mark.parametrize("cplx", [False, True])
@pytest.mark.parametrize("density", [0.05, 0.2])
def test_ilu0_reproduces_A_on_its_pattern(orc, cplx, density):
    A, M = _random_sparse(60, density, seed=300 + int(100 * density), cplx=cplx)
    f = orc.ilu0(A)
    L, U = _ilu_dense(A, f)
    P = M != 0
    LU = L @ U
    np.testing.assert_allclose(LU[P], M[P], rtol=0, atol=1e-12 * np.abs(M).max())
    # fill outside the pattern exists (this is an incomplete factorisation)
    if density == 0.2:
        assert np.abs(LU[~P]).max() > 1e-3


@pytest.mark.parametrize("kind", ["full", "tridiagonal", "lower", "upper"])
@pytest.mark.parametrize("cplx", [False, True])
def test_ilu0_without_fill_is_the_exact_lu(orc, kind, cplx):
    """Patterns whose elimination creates no fill (dense, tridiagonal,
    triangular): ILU(0) = LU, so M^{-1} b is A^{-1} b (LAPACK)."""
    N = 30
    rng = np.random.default_rng(310 + len(kind))
    M = rng.standard_normal((N, N)) + (1j * rng.standard_normal((N, N)) if cplx else 0)
    if kind == "tridiagonal":
        M = np.triu(np.tril(M, 1), -1)
    elif kind == "lower":
        M = np.tril(M)
    elif kind == "upper":
        M = np.triu(M)
    M = M + 6.0 * np.eye(N)
    A = W.dense_to_csr(M)
    f = orc.ilu0(A)
    L, U = _ilu_dense(A, f)
    np.testing.assert_allclose(L @ U, M, rtol=0, atol=1e-12 * np.abs(M).max())
    b = rng.standard_normal(N) + (1j * rng.standard_normal(N) if cplx else 0)
    np.testing.assert_allclose(orc.minv(A, b, ilu=f), np.linalg.solve(M, b), rtol=1e-11, atol=1e-13)


@pytest.mark.parametrize("cplx", [False, True])
def test_ilu_minv_and_minv_h_match_dense_solves(orc, cplx):
    """M^{-1} v and M^{-H} v (Algorithm 7.1, steps 2, 31, 37) against LAPACK
    on the dense M = L U, for an incomplete factorisation with fill."""
    A, _ = _random_sparse(50, 0.15, seed=320, cplx=cplx)
    f = orc.ilu0(A)
    L, U = _ilu_dense(A, f)
    Md = L @ U
    rng = np.random.default_rng(321)
    v = rng.standard_normal(50) + (1j * rng.standard_normal(50) if cplx else 0)
    np.testing.assert_allclose(orc.minv(A, v, ilu=f), np.linalg.solve(Md, v), rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(orc.minv_h(A, v, ilu=f), np.linalg.solve(Md.conj().T, v), rtol=1e-10, atol=1e-12)


def test_ilu_minv_of_diagonal_pattern_is_jacobi(orc):
    """A diagonal matrix: L = I, U = A, so M^{-1} is the Jacobi division
    (bit for bit) and M^{-H} the division by the conjugate."""
    d = np.random.default_rng(322).uniform(0.5, 2.0, 20) * np.exp(1j * np.linspace(0, 1, 20))
    A = W.dense_to_csr(np.diag(d))
    f = orc.ilu0(A)
    v = np.random.default_rng(323).standard_normal(20) + 0j
    np.testing.assert_array_equal(orc.minv(A, v, ilu=f), orc.minv(A, v, mdiag=d))
    np.testing.assert_array_equal(orc.minv_h(A, v, ilu=f), orc.minv_h(A, v, mdiag=d))
    # numpy's complex division may round the last bit differently from C's
    np.testing.assert_allclose(orc.minv_h(A, v, ilu=f), v / d.conj(), rtol=4e-16, atol=0)


@pytest.mark.parametrize("cplx", [False, True])
def test_ilu_precond_with_M_equal_A_converges_in_one_step(orc, cplx):
    """On a dense pattern ILU(0) is A itself, so A M^{-1} = I: the first
    step gives alpha = 1, x_1 = A^{-1} b and r_1 = 0 (up to rounding)."""
    A, M, b = W.random_dense_system(25, seed=324, complex_=cplx)
    Q = np.random.default_rng(325).standard_normal((25, 4))
    res = orc.mlbicgstabt(A, b, np.zeros(25, dtype=b.dtype), Q, maxit=5, tol=1e-12, ilu=orc.ilu0(A))
    assert res.flag == 0 and res.iter == 1
    xs = np.linalg.solve(M, b)
    assert np.linalg.norm(res.x - xs) <= 1e-12 * np.linalg.norm(xs)


@pytest.mark.parametrize("cplx", [False, True])
def test_ilu_precond_equals_method_on_right_preconditioned_system(orc, cplx):
    """Algorithm 7.1 with M = L U gives the residuals of the M = I method on
    A' = A M^{-1} (formed densely with LAPACK), and x_k = M^{-1} y_k."""
    N, n = 40, 4
    A, _ = _random_sparse(N, 0.12, seed=326, cplx=cplx, shift=3.0)
    f = orc.ilu0(A)
    L, U = _ilu_dense(A, f)
    Md = L @ U
    Ap = W.dense_to_csr(A_dense(A) @ np.linalg.inv(Md))
    rng = np.random.default_rng(327)
    b = rng.standard_normal(N) + (1j * rng.standard_normal(N) if cplx else 0)
    Q = rng.standard_normal((N, n)) + (1j * rng.standard_normal((N, n)) if cplx else 0)
    x0 = np.zeros(N, dtype=b.dtype)
    K = 15
    rp = orc.mlbicgstabt(A, b, x0, Q, maxit=K, tol=0.0, err_hist=True, x_hist=K, ilu=f)
    ry = orc.mlbicgstabt(Ap, b, x0, Q, maxit=K, tol=0.0, err_hist=True, x_hist=K)
    np.testing.assert_allclose(rp.err_hist, ry.err_hist, rtol=1e-7)
    for k in range(K):
        xk = np.linalg.solve(Md, ry.x_hist[k])
        assert np.linalg.norm(rp.x_hist[k] - xk) <= 1e-7 * np.linalg.norm(xk), k


def A_dense(A):
    D = np.zeros((A.n_rows, A.n_rows), dtype=A.val.dtype)
    for r in range(A.n_rows):
        D[r, A.col[A.row_ptr[r]:A.row_ptr[r + 1]]] += A.val[A.row_ptr[r]:A.row_ptr[r + 1]]
    return D


@pytest.mark.parametrize("N,n", [(8, 3), (9, 9)])
def test_ilu_precond_finite_termination(orc, N, n):
    """A M^{-1} is N x N: the ILU-preconditioned method stops by step N in
    exact arithmetic; at tol 1e-14 it converges by iteration N and agrees
    with LAPACK on A x = b."""
    A, M = _random_sparse(N, 0.3, seed=330 + N + n)
    b = np.random.default_rng(N).standard_normal(N)
    Q = np.random.default_rng(N + 1).standard_normal((N, n))
    res = orc.mlbicgstabt(A, b, np.zeros(N), Q, maxit=4 * N, tol=1e-14, ilu=orc.ilu0(A))
    assert res.flag == 0 and res.iter <= N
    xs = np.linalg.solve(M, b)
    assert np.linalg.norm(res.x - xs) <= 1e-10 * np.linalg.norm(xs)


def test_ilu0_rejects_inputs_without_a_factorisation(orc):
    # zero pivot: [[0, 1], [1, 0]] with the diagonal stored as zeros
    Z = W.CSR(row_ptr=np.array([0, 2, 4], dtype=np.int64), col=np.array([0, 1, 0, 1], dtype=np.int32),
              val=np.array([0.0, 1.0, 1.0, 0.0]), n_rows=2)
    with pytest.raises(orc_mod().IluError) as e:
        orc.ilu0(Z)
    assert e.value.args[0] == -3
    # a row without a stored diagonal entry
    D = W.CSR(row_ptr=np.array([0, 1, 2], dtype=np.int64), col=np.array([1, 1], dtype=np.int32),
              val=np.array([1.0, 2.0]), n_rows=2)
    with pytest.raises(orc_mod().IluError) as e:
        orc.ilu0(D)
    assert e.value.args[0] == -1
    # columns not increasing within a row
    U = W.CSR(row_ptr=np.array([0, 2, 3], dtype=np.int64), col=np.array([1, 0, 1], dtype=np.int32),
              val=np.array([1.0, 2.0, 3.0]), n_rows=2)
    with pytest.raises(orc_mod().IluError):
        orc.ilu0(U)


def orc_mod():
    import oracle
    return oracle


def test_ilu_precond_cuts_iterations_on_convection_diffusion(orc):
    """ILU(0) is the preconditioner the paper's experiments use (§5); on
    the 2-D convection-diffusion system it must converge to the same
    solution as M = I in far fewer iterations."""
    A = W.cd2d(32)
    b = W.row_sums(A)
    N = A.n_rows
    Q = orc.q_gauss(0, N, 4)
    r0 = orc.solve(A, b, np.zeros(N), Q, 3000, 1e-10)
    r1 = orc.solve(A, b, np.zeros(N), Q, 3000, 1e-10, ilu=orc.ilu0(A))
    assert r0.flag == 0 and r1.flag == 0
    assert r1.iter * 2 < r0.iter
    np.testing.assert_allclose(r1.x, 1.0, rtol=1e-7)
