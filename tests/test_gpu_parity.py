"""GPU parity: the CUDA library through its C ABI against the CPU oracle on
the same seeded inputs.

Tolerances (derived from the arithmetic, not fitted):
* shadow vectors: both sides evaluate the same generator; log and cos are
  correctly rounded to within 1 ulp on each side, so entries agree to a
  few ulp: |Q_gpu - Q_oracle| <= 4 eps max(1, |Q|).
* y = A x: both sides sum at most w products per row (w = longest row),
  so each differs from the exact sum by <= gamma_w sum|a||x| (Higham,
  Thm 3.1, gamma_w = w eps / (1 - w eps)); the difference of the two is at
  most twice that.  Q^H y: the same bound with N terms plus the propagated
  difference of y.
* solves: the recursive residuals of the first 8 iterations agree to
  max(1e-10, 4 N eps) relative: the oracle's inner products are sequential
  sums of N terms, each within gamma_N = N eps/(1 - N eps) of exact
  (relative to sum|u_i v_i|), and 8 steps amplify that by far less than
  the factor allowed; final solution within 1e-8 relative of the oracle's;
  true residual below tol = 1e-10.
* iteration counts: on short, well-conditioned solves (the 32x32 system,
  small complex systems) equal to the oracle's.  On long ill-conditioned
  solves the count is decided by rounding: the oracle's own count moves
  by several percent when one entry of b moves by one ulp.  There the GPU
  count must lie in the 99.9 % prediction interval of the oracle's counts
  over b and 16 one-ulp perturbations of b (tests/spread.py), and the
  index logic is checked bit-exactly instead at fixed iteration counts
  (tol = 0): the same (j, i) and the same Table 4.3 counters as the oracle
  after K steps.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle as O
from paper_1106_3678_gb300 import mlbicgstab as M
from paper_1106_3678_gb300 import workloads as W

from tests import spread

pytestmark = pytest.mark.gpu


def _par():
    """The oracle's multi-core build on every host core (results do not
    depend on the thread count)."""
    import os
    lib = O.load_par()
    O.par_threads(os.cpu_count() or 1)
    return lib
EPS = np.finfo(np.float64).eps


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1106_3678_gb300 import build
    build.build()
    M.load()


def _abs_spmv(A, x):
    return O.spmv(W.CSR(A.row_ptr, A.col, np.abs(A.val), A.n_rows), np.abs(x))


def _gamma(k):
    return k * EPS / (1 - k * EPS)


# ------------------------------------------------------------- shadow Q ----

@pytest.mark.parametrize("cplx", [False, True])
def test_shadow_vectors_match_oracle_generator(cplx):
    A = W.helmholtz3d_c(8, 6, 5) if cplx else W.cd2d(24)
    n = 5
    h = M.mlbicgstab_create(A, n=n, q_seed=1234)
    Qg = M.mlbicgstab_get_Q(h)
    Qo = O.q_gauss(1234, A.n_rows, n, complex_=cplx)
    assert Qg.shape == Qo.shape
    err = np.abs(Qg - Qo)
    assert np.all(err <= 4 * EPS * np.maximum(1.0, np.abs(Qo))), err.max()


def test_user_Q_is_used_verbatim():
    A = W.cd2d(16)
    Q = np.random.default_rng(3).standard_normal((A.n_rows, 3))
    h = M.mlbicgstab_create(A, n=3, Q=Q)
    np.testing.assert_array_equal(M.mlbicgstab_get_Q(h), Q)


# ------------------------------------------------- fused SpMV + Q^H y ------

def _check_spmv_qdot(A, n, seed=0, grid_rows=None):
    import torch
    cplx = np.iscomplexobj(A.val)
    rng = np.random.default_rng(seed)
    x = rng.standard_normal(A.n_rows)
    if cplx:
        x = x + 1j * rng.standard_normal(A.n_rows)
    h = M.mlbicgstab_create(A, n=n, q_seed=seed)
    dt = torch.complex128 if cplx else torch.float64
    xd = torch.tensor(x, dtype=dt, device="cuda")
    yd = torch.empty_like(xd)
    d = M.mlbicgstab_spmv_qdot(h, xd, yd)
    y = yd.cpu().numpy()
    yo = O.spmv(A, x)
    w = int(np.max(np.diff(A.row_ptr))) + 1
    bound = 2 * _gamma(w) * _abs_spmv(A, x)
    assert np.all(np.abs(y - yo) <= bound + 1e-300), np.max(np.abs(y - yo) - bound)
    Q = M.mlbicgstab_get_Q(h)
    do = Q.conj().T @ yo
    bd = (np.abs(Q).T @ np.abs(y - yo)) + 2 * _gamma(A.n_rows) * (np.abs(Q).T @ np.abs(yo))
    assert np.all(np.abs(d - do) <= bd), (d, do)
    return h


# n <= 4: every column fused into the product's epilogue (1, 2 or 4 at a
# time); larger n adds passes of up to 8 columns (4 for complex) over y
@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 13, 16, 64])
def test_spmv_qdot_cd2d(n):
    _check_spmv_qdot(W.cd2d(32), n)


@pytest.mark.parametrize("n", [1, 2, 9])
def test_spmv_qdot_complex_splits(n):
    _check_spmv_qdot(W.helmholtz3d_c(9, 8, 7), n, seed=n)


def test_spmv_qdot_after_set_n():
    """A handle created with n = 8 and set to 3 returns the 3 active inner
    products, equal to those of a handle created with n = 3."""
    import torch
    A = W.cd3d_lognormal(16)
    x = torch.tensor(np.random.default_rng(2).standard_normal(A.n_rows), device="cuda")
    y1, y2 = torch.empty_like(x), torch.empty_like(x)
    h8 = M.mlbicgstab_create(A, n=8, q_seed=0)
    M.mlbicgstab_set_n(h8, 3)
    d8 = M.mlbicgstab_spmv_qdot(h8, x, y1)
    d3 = M.mlbicgstab_spmv_qdot(M.mlbicgstab_create(A, n=3, q_seed=0), x, y2)
    assert d8.shape == (3,)
    np.testing.assert_array_equal(d8, d3)
    assert torch.equal(y1, y2)


def test_spmv_qdot_cd3d_several_slices_ragged_tail():
    # N = 23^3 = 12167: not a multiple of 32 (ragged last slice)
    _check_spmv_qdot(W.cd3d_lognormal(23), 8)


def test_spmv_qdot_irregular_rows():
    # random pattern with row lengths 1..40 plus the diagonal
    rng = np.random.default_rng(5)
    M_ = np.zeros((77, 77))
    for r in range(77):
        k = rng.integers(0, 40)
        cols = rng.choice(77, size=k, replace=False)
        M_[r, cols] = rng.standard_normal(k)
        M_[r, r] = 5.0
    _check_spmv_qdot(W.dense_to_csr(M_), 3)


def test_spmv_qdot_complex():
    _check_spmv_qdot(W.helmholtz3d_c(10, 9, 7), 6)


@pytest.mark.parametrize("cplx", [False, True])
@pytest.mark.parametrize("n", [1, 4, 9])
def test_spmv_qdot_async_fp64_equals_the_synchronous_call(n, cplx):
    """The asynchronous entry point runs the same kernel: y and d equal the
    synchronous call's bit for bit; d stays on the device with the status
    word 0 behind it."""
    import torch
    A = W.helmholtz3d_c(9, 8, 7) if cplx else W.cd3d_lognormal(21)
    dt = torch.complex128 if cplx else torch.float64
    h = M.mlbicgstab_create(A, n=n, q_seed=5)
    rng = np.random.default_rng(n)
    x = rng.standard_normal(A.n_rows) + (1j * rng.standard_normal(A.n_rows) if cplx else 0)
    xd = torch.tensor(x, dtype=dt, device="cuda")
    y1, y2 = torch.empty_like(xd), torch.empty_like(xd)
    d1 = M.mlbicgstab_spmv_qdot(h, xd, y1)
    k = 2 if cplx else 1
    dd = torch.full((n * k + 1,), float("nan"), dtype=torch.float64, device="cuda")
    for _ in range(2):   # back-to-back launches on the handle's stream
        M.mlbicgstab_spmv_qdot_async(h, xd, y2, dd)
    torch.cuda.synchronize()
    d2 = dd.cpu().numpy()
    assert d2[-1] == 0.0
    d2 = d2[:-1].view(np.complex128) if cplx else d2[:-1]
    np.testing.assert_array_equal(d2, d1)
    assert torch.equal(y1, y2)


@pytest.mark.parametrize("cplx", [False, True])
@pytest.mark.parametrize("n", [1, 4, 16])
def test_spmv_qdot_fp32_copies_of_a_refined_handle(n, cplx):
    """FP32 product and FP32 per-thread inner products (FP64 across threads
    and CTAs) against the oracle's FP64 product of the same FP32-rounded
    values.  y: each row sums at most w FP32 products, within gamma32_w of
    the exact sum of |a||x| (Higham, Thm 3.1, u = 2^-24), the oracle within
    gamma64_w.  d: the propagated y difference plus gamma32_N |q|^T |y|."""
    A = W.helmholtz3d_c(10, 9, 7) if cplx else W.cd3d_lognormal(23)
    h = M.mlbicgstab_create(A, n=n, q_seed=2, precision=M.MLB_PREC_FP32_REFINED)
    fp32_product_vs_oracle(h, A, n, cplx, 3 + n)


def fp32_product_vs_oracle(h, A, n, cplx, seed):
    """The FP32 fused product of a refined handle against the oracle's
    product of the FP32-rounded values, at the bounds described above."""
    import torch
    rng = np.random.default_rng(seed)
    x = rng.standard_normal(A.n_rows) + (1j * rng.standard_normal(A.n_rows) if cplx else 0)
    dt32, npt32 = (torch.complex64, np.complex64) if cplx else (torch.float32, np.float32)
    x32 = x.astype(npt32)
    xd = torch.tensor(x32, dtype=dt32, device="cuda")
    yd = torch.empty_like(xd)
    k = 2 if cplx else 1
    dd = torch.zeros(n * k + 1, dtype=torch.float64, device="cuda")
    M.mlbicgstab_spmv_qdot_async(h, xd, yd, dd)
    torch.cuda.synchronize()
    y = yd.cpu().numpy().astype(np.complex128 if cplx else np.float64)
    d = dd.cpu().numpy()
    assert d[-1] == 0.0
    d = d[:-1].view(np.complex128) if cplx else d[:-1]
    A32 = W.CSR(A.row_ptr, A.col, A.val.astype(npt32).astype(A.val.dtype), A.n_rows)
    xw = x32.astype(x.dtype)
    yo = O.spmv(A32, xw)
    w = int(np.max(np.diff(A.row_ptr))) + 1
    u32 = 2.0 ** -24
    g32 = lambda m: m * u32 / (1 - m * u32)
    bound_y = (g32(w) + _gamma(w)) * _abs_spmv(A32, xw) * (4 if cplx else 1)
    assert np.all(np.abs(y - yo) <= bound_y + 1e-300), np.max(np.abs(y - yo) - bound_y)
    Q32 = M.mlbicgstab_get_Q(h).astype(npt32).astype(x.dtype)
    do = Q32.conj().T @ y
    bd = (np.abs(Q32).T @ bound_y) + g32(A.n_rows) * (4 if cplx else 1) * (np.abs(Q32).T @ np.abs(y))
    assert np.all(np.abs(d - do) <= bd + np.abs(Q32).T @ np.abs(y - yo)), (d, do)


def test_spmv_qdot_async_rejects_fp32_on_an_fp64_handle():
    import torch
    A = W.cd2d(16)
    h = M.mlbicgstab_create(A, n=2)
    x = torch.ones(A.n_rows, dtype=torch.float32, device="cuda")
    y = torch.empty_like(x)
    d = torch.empty(3, dtype=torch.float64, device="cuda")
    with pytest.raises(M.MlbError) as e:
        M.mlbicgstab_spmv_qdot_async(h, x, y, d)
    assert e.value.code == M.MLB_ERR_UNSUPPORTED


def test_spmv_qdot_full_size_cd3d():
    """The 128^3 workload at full size, every row checked."""
    _check_spmv_qdot(W.cd3d_lognormal(128), 4)


# ------------------------------------------------------------- solves ------

def _gpu_solve(A, b, n, tol, maxit, q_seed=0, Q=None, kappa=0.0, max_outer=0,
               grid=0, hist=True, x0=None):
    h = M.mlbicgstab_create(A, n=n, q_seed=q_seed, Q=Q, kappa=kappa,
                            max_outer=max_outer, grid=grid)
    x = np.zeros(A.n_rows, dtype=b.dtype) if x0 is None else np.array(x0, copy=True)
    res, eh = M.mlbicgstab_solve(h, b, x, tol, maxit, hist_cap=(maxit + 1) if hist else 0)
    return h, x, res, eh


def _early_tol(N):
    return max(1e-10, 4 * N * EPS)


def _compare(A, b, n, tol=1e-10, maxit=2000, grid=0, kappa=0.0, Q=None,
             early=8, exact_iters=True):
    cplx = np.iscomplexobj(A.val)
    h, x, res, eh = _gpu_solve(A, b, n, tol, maxit, Q=Q, kappa=kappa, grid=grid)
    Qo = O.q_gauss(0, A.n_rows, n, complex_=cplx) if Q is None else Q
    ref = O.mlbicgstabt(A, b, np.zeros_like(b), Qo, maxit, tol, kappa,
                        err_hist=True)
    assert res.status == 0
    assert res.flag == ref.flag
    if exact_iters:
        assert res.iter == ref.iter
        assert (res.j, res.i) == (ref.j, ref.i)
        assert res.as_dict()["ops"] == ref.ops
    else:
        (lo, hi), counts = spread.oracle_window(A, b, Qo, tol, maxit, kappa, lib=_par())
        assert lo <= res.iter <= hi, (res.iter, lo, hi, counts)
        assert (res.j, res.i) == (O.gn(n, res.iter), O.rn(n, res.iter))
    k = min(early, ref.iter, res.iter) + 1
    np.testing.assert_allclose(eh[:k], ref.err_hist[:k], rtol=_early_tol(A.n_rows), atol=0)
    if ref.flag == 0:
        assert res.true_relres < tol
        rel = np.linalg.norm(x - ref.x) / np.linalg.norm(ref.x)
        assert rel <= 1e-8, rel
    return res, ref, x


@pytest.mark.parametrize("n", [1, 2, 3, 4, 8])
def test_solve_cd2d_matches_oracle(n):
    """The 32x32 convection-diffusion workload (N = 1024, one CTA)."""
    A = W.cd2d(32)
    _compare(A, W.row_sums(A), n)


@pytest.mark.parametrize("grid", [2, 5])
@pytest.mark.parametrize("n", [1, 4])
def test_solve_cd2d_multi_cta_grid_barrier(n, grid):
    """Same system on several CTAs: exercises the grid barrier and the
    cross-CTA reduction on a small case."""
    A = W.cd2d(32)
    _compare(A, W.row_sums(A), n, grid=grid)


@pytest.mark.parametrize("m,n", [(16, 4), (23, 8), (30, 3)])
def test_solve_cd3d_small_matches_oracle(m, n):
    """Log-normal 3-D systems spanning many slices, ragged last slice:
    long, ill-conditioned solves (iteration count compared with the
    oracle's rounding spread)."""
    A = W.cd3d_lognormal(m)
    b = W.uniform_rhs(A.n_rows, seed=2)
    _compare(A, b, n, maxit=20000, exact_iters=False)


@pytest.mark.parametrize("K", [37, 64, 101])
@pytest.mark.parametrize("n", [1, 3, 4, 8])
def test_index_logic_bit_exact_at_fixed_iterations(n, K):
    """tol = 0 and maxit = K: after exactly K steps the GPU reports the
    oracle's (j, i) = (g_n(K), r_n(K)) and the oracle's Table 4.3 counters;
    the residual histories agree in their first steps."""
    A = W.cd3d_lognormal(23)
    b = W.uniform_rhs(A.n_rows, seed=2)
    _, x, res, eh = _gpu_solve(A, b, n, 0.0, K)
    ref = O.mlbicgstabt(A, b, np.zeros(A.n_rows), O.q_gauss(0, A.n_rows, n), K, 0.0,
                        err_hist=True)
    assert (res.flag, res.iter, res.j, res.i) == (1, K, ref.j, ref.i)
    assert (res.j, res.i) == (O.gn(n, K), O.rn(n, K))
    assert res.as_dict()["ops"] == ref.ops
    np.testing.assert_allclose(eh[:9], ref.err_hist[:9], rtol=_early_tol(A.n_rows))


@pytest.mark.parametrize("n", [2, 4])
def test_solve_complex_matches_oracle(n):
    A = W.helmholtz3d_c(8, 8, 4, k=3.0)
    _compare(A, W.row_sums(A), n, maxit=3000)


def test_solve_kappa_guard_matches_oracle():
    A = W.cd2d(24, beta=(60.0, 10.0))
    _compare(A, W.row_sums(A), 3, kappa=0.7)


@pytest.mark.parametrize("N,n", [(12, 12), (10, 14), (9, 3)])
def test_finite_termination_on_gpu(N, n):
    A, Md, b = W.random_dense_system(N, seed=40 + N)
    Q = np.random.default_rng(N).standard_normal((N, n))
    h, x, res, _ = _gpu_solve(A, b, n, 1e-14, 4 * N, Q=Q, hist=False)
    assert res.flag == 0 and res.iter <= N
    xs = np.linalg.solve(Md, b)
    assert np.linalg.norm(x - xs) <= 1e-10 * np.linalg.norm(xs)


# ------------------------------------------------------- edge cases --------

def test_zero_rhs_and_exact_guess():
    A = W.cd2d(16)
    _, x, res, _ = _gpu_solve(A, np.zeros(A.n_rows), 4, 1e-10, 100)
    assert (res.iter, res.flag, res.err) == (0, 0, 0.0) and not x.any()
    _, x, res, _ = _gpu_solve(A, W.row_sums(A), 4, 1e-10, 100,
                              x0=np.ones(A.n_rows))
    assert res.iter == 0 and res.flag == 0


@pytest.mark.parametrize("n,maxit", [(4, 7), (4, 8), (3, 5), (1, 3)])
def test_iteration_limit(n, maxit):
    A = W.cd2d(16)
    b = W.row_sums(A)
    _, x, res, _ = _gpu_solve(A, b, n, 1e-14, maxit)
    ref = O.mlbicgstabt(A, b, np.zeros(A.n_rows), O.q_gauss(0, A.n_rows, n), maxit, 1e-14)
    assert (res.flag, res.iter, res.j, res.i) == (1, maxit, ref.j, ref.i)
    np.testing.assert_allclose(x, ref.x, rtol=1e-9, atol=1e-12)


def test_breakdown_c_zero():
    A = W.cd2d(6)
    N = A.n_rows
    b = np.zeros(N)
    b[7] = 1.0
    colk = np.zeros(N)
    for r in range(N):
        for k in range(A.row_ptr[r], A.row_ptr[r + 1]):
            if A.col[k] == 7:
                colk[r] = A.val[k]
    i, j = np.nonzero(colk)[0][:2]
    q = np.zeros(N)
    q[i], q[j] = colk[j], -colk[i]
    _, _, res, _ = _gpu_solve(A, b, 1, 1e-10, 50, Q=q[:, None])
    assert res.flag == -1 and res.iter == 0


def test_device_pointers_match_host_pointers():
    import torch
    A = W.cd2d(32)
    b = W.row_sums(A)
    h = M.mlbicgstab_create(A, n=4)
    xh = np.zeros(A.n_rows)
    r1, _ = M.mlbicgstab_solve(h, b, xh, 1e-10, 2000)
    bd = torch.tensor(b, device="cuda")
    xd = torch.zeros(A.n_rows, dtype=torch.float64, device="cuda")
    r2, _ = M.mlbicgstab_solve(h, bd, xd, 1e-10, 2000)
    assert r1.iter == r2.iter
    np.testing.assert_array_equal(xd.cpu().numpy(), xh)


def test_restart_on_true_residual():
    """max_outer > 0: the solve continues until the true residual meets
    tol, like the oracle's restart wrapper."""
    A = W.cd3d_lognormal(16)
    b = W.uniform_rhs(A.n_rows, seed=2)
    _, x, res, _ = _gpu_solve(A, b, 4, 1e-10, 20000, max_outer=10, hist=False)
    Q = O.q_gauss(0, A.n_rows, 4)
    ref = O.solve(A, b, np.zeros(A.n_rows), Q, 20000, 1e-10)
    assert ref.flag == 0 and ref.true_relres < 1e-10
    assert res.flag == 0 and res.true_relres < 1e-10
    (lo, hi), counts = spread.oracle_window(A, b, Q, 1e-10, 20000, restarts=True, lib=_par())
    assert lo <= res.iter <= hi, (res.iter, lo, hi, counts)
    assert np.linalg.norm(x - ref.x) <= 1e-8 * np.linalg.norm(ref.x)


# ------------------------------------------- full-size 128^3 workload -------

def test_full_size_cd3d_first_iterations_elementwise():
    """N = 2,097,152 (the benchmark workload, benchmark launch geometry):
    12 iterations on the GPU against 12 oracle iterations, x compared
    element by element."""
    A = W.cd3d_lognormal(128)
    b = W.uniform_rhs(A.n_rows, seed=2)
    n = 4
    h, x, res, eh = _gpu_solve(A, b, n, 1e-10, 12)
    ref = O.mlbicgstabt(A, b, np.zeros(A.n_rows), O.q_gauss(0, A.n_rows, n), 12,
                        1e-10, err_hist=True)
    assert (res.flag, res.iter, res.j, res.i) == (ref.flag, ref.iter, ref.j, ref.i)
    assert res.as_dict()["ops"] == ref.ops
    np.testing.assert_allclose(eh[:13], ref.err_hist[:13], rtol=_early_tol(A.n_rows))
    scale = np.max(np.abs(ref.x))
    assert np.max(np.abs(x - ref.x)) <= 1e-8 * scale


# ------------------------------------------------- failure detection -------

def test_barrier_wait_times_out_and_device_stays_usable():
    """A barrier participant that never arrives: every wait gives up after
    50 ms, the kernel returns, the host reads MLB_ERR_TIMEOUT, and the next
    solve runs normally."""
    assert M.mlbicgstab_selftest_barrier_timeout(4, 50_000_000) == M.MLB_ERR_TIMEOUT
    A = W.cd2d(16)
    _, _, res, _ = _gpu_solve(A, W.row_sums(A), 4, 1e-10, 1000, hist=False)
    assert res.flag == 0 and res.status == 0
