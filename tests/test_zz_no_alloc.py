"""Allocation-free fused y = A x, d = Q^H y (mlbicgstab_spmv_qdot_noalloc).

This entry point serves callers that cannot allocate device memory (a
framework pool that owns the device budget, a plug-in that may not
allocate, a latency-critical loop): it takes every array from the caller
and keeps its scratch in a fixed array of the library.  Its results are
checked through the C ABI against mlbicgstab_spmv_qdot, which works through
a handle that owns its memory, and against the CPU oracle's product and
inner products, each on two calls in a row: the second call shows that the
shared scratch array left by the first one does not leak into it.  A third
test counts device memory around 100 calls.

Tolerance: both paths sum at most w products per row (w = longest row), so
each is within gamma_w sum|a||x| of the exact product and the two differ by
at most twice that; for d the difference of y propagates through |Q|^T and
each N-term inner product adds at most gamma_N sum|q||y| (Higham, Thm 3.1).
"""
from __future__ import annotations

import numpy as np
import pytest

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


def _gamma(k):
    return k * EPS / (1 - k * EPS)


def _abs_product(A, x):
    rows = np.repeat(np.arange(A.n_rows), np.diff(A.row_ptr))
    out = np.zeros(A.n_rows)
    np.add.at(out, rows, np.abs(A.val) * np.abs(x[A.col]))
    return out


def _inputs(case):
    import torch
    if case == "real":
        A, n, dt = W.cd3d_lognormal(23), 8, torch.float64
    else:
        A, n, dt = W.helmholtz3d_c(10, 9, 7), 6, torch.complex128
    return A, n, dt


def _device_csr(A, dt):
    import torch
    rp = torch.tensor(A.row_ptr, dtype=torch.int64, device="cuda")
    ci = torch.tensor(A.col, dtype=torch.int32, device="cuda")
    av = torch.tensor(A.val, dtype=dt, device="cuda")
    return rp, ci, av


def _rand(rng, N, case):
    x = rng.standard_normal(N)
    if case == "complex":
        x = x + 1j * rng.standard_normal(N)
    return x


@pytest.mark.parametrize("case", ["real", "complex"])
def test_noalloc_matches_handle_entry_point_on_two_calls(case):
    import torch
    A, n, dt = _inputs(case)
    N = A.n_rows
    h = M.mlbicgstab_create(A, n=n, q_seed=3)
    Q = M.mlbicgstab_get_Q(h)                       # N x n
    rp, ci, av = _device_csr(A, dt)
    Qd = torch.tensor(np.ascontiguousarray(Q.T), dtype=dt, device="cuda")  # row q = q_q
    w = int(np.max(np.diff(A.row_ptr))) + 1
    rng = np.random.default_rng(11)
    for call in range(2):
        x = _rand(rng, N, case)
        xd = torch.tensor(x, dtype=dt, device="cuda")
        y_ref = torch.empty_like(xd)
        d_ref = M.mlbicgstab_spmv_qdot(h, xd, y_ref)
        y = torch.full_like(xd, float("nan"))
        d = torch.full((n,), float("nan"), dtype=dt, device="cuda")
        M.mlbicgstab_spmv_qdot_noalloc(rp, ci, av, xd, Qd, y, d)
        torch.cuda.synchronize()
        yn, yr = y.cpu().numpy(), y_ref.cpu().numpy()
        bound_y = 2 * _gamma(w) * _abs_product(A, x)
        assert np.all(np.abs(yn - yr) <= bound_y), (call, np.max(np.abs(yn - yr) - bound_y))
        dn = d.cpu().numpy()
        bound_d = (np.abs(Q).T @ np.abs(yn - yr)) + 2 * _gamma(N) * (np.abs(Q).T @ np.abs(yr))
        assert np.all(np.abs(dn - d_ref) <= bound_d), (call, dn, d_ref)
    h.destroy()


@pytest.mark.parametrize("case", ["real", "complex"])
@pytest.mark.parametrize("n", [1, 5, 20, 64])
def test_noalloc_matches_the_oracle_product_and_inner_products(case, n):
    """Element by element against the oracle: y = A x from the oracle's
    sparse product, d = Q^H y from those y values.  Each y_i differs from
    the oracle's by at most 2 gamma_w (|A||x|)_i (w = longest row); each d_k
    by the propagated y error plus 2 gamma_N (|q_k|^T |y|) (two N-term
    sums in different orders; Higham, Thm 3.1)."""
    import torch
    import oracle as O
    A, _, dt = _inputs(case)
    N = A.n_rows
    cplx = case == "complex"
    Q = O.q_gauss(9, N, n, complex_=cplx)          # N x n, oracle side
    rp, ci, av = _device_csr(A, dt)
    Qd = torch.tensor(np.ascontiguousarray(Q.T), dtype=dt, device="cuda")
    w = int(np.max(np.diff(A.row_ptr))) + 1
    rng = np.random.default_rng(100 + n)
    for call in range(2):
        x = _rand(rng, N, case)
        y_or = O.spmv(A, x)
        d_or = Q.conj().T @ y_or
        xd = torch.tensor(x, dtype=dt, device="cuda")
        y = torch.full_like(xd, float("nan"))
        d = torch.full((n,), float("nan"), dtype=dt, device="cuda")
        M.mlbicgstab_spmv_qdot_noalloc(rp, ci, av, xd, Qd, y, d)
        torch.cuda.synchronize()
        yn, dn = y.cpu().numpy(), d.cpu().numpy()
        bound_y = 2 * _gamma(w) * _abs_product(A, x)
        assert np.all(np.abs(yn - y_or) <= bound_y), (call, np.max(np.abs(yn - y_or) - bound_y))
        bound_d = (np.abs(Q).T @ bound_y) + 2 * _gamma(N) * (np.abs(Q).T @ np.abs(y_or))
        assert np.all(np.abs(dn - d_or) <= bound_d), (call, dn, d_or)


def test_noalloc_allocates_nothing_after_its_first_call():
    """Device free memory (cudaMemGetInfo) and the PyTorch caching
    allocator's counters do not move over 100 calls.  The first call sets
    up the scratch address, so the baseline is taken after it."""
    import torch
    A, n, dt = _inputs("real")
    N = A.n_rows
    rp, ci, av = _device_csr(A, dt)
    Qd = torch.randn((n, N), dtype=dt, device="cuda")
    xd = torch.randn(N, dtype=dt, device="cuda")
    y = torch.empty_like(xd)
    d = torch.empty(n, dtype=dt, device="cuda")
    M.mlbicgstab_spmv_qdot_noalloc(rp, ci, av, xd, Qd, y, d)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    st0 = torch.cuda.memory_stats()
    for _ in range(100):
        M.mlbicgstab_spmv_qdot_noalloc(rp, ci, av, xd, Qd, y, d)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    st1 = torch.cuda.memory_stats()
    assert free1 == free0, (free0, free1)
    for key in ("allocation.all.allocated", "segment.all.allocated", "allocated_bytes.all.allocated"):
        assert st1.get(key, 0) == st0.get(key, 0), key


def test_noalloc_rejects_sizes_beyond_its_scratch_limit():
    import torch
    A = W.cd2d(8)
    N = A.n_rows
    rp = torch.tensor(A.row_ptr, device="cuda")
    ci = torch.tensor(A.col, dtype=torch.int32, device="cuda")
    av = torch.tensor(A.val, device="cuda")
    x = torch.ones(N, dtype=torch.float64, device="cuda")
    y = torch.empty_like(x)
    Q = torch.ones((65, N), dtype=torch.float64, device="cuda")
    d = torch.empty(65, dtype=torch.float64, device="cuda")
    with pytest.raises(M.MlbError) as e:
        M.mlbicgstab_spmv_qdot_noalloc(rp, ci, av, x, Q, y, d)
    assert e.value.code == M.MLB_ERR_ARG
