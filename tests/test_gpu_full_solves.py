"""Complete solves on the GPU against complete solves of the oracle, up to
sizes whose working set exceeds the 129 MB L2 cache, on the launch
geometry the benchmark uses (all SMs for large N).

The oracle is its multi-core build (fixed-block reductions, results
independent of the thread count; pinned to the sequential oracle by
tests/test_oracle_par.py).  Bars: flag 0 on both sides, the
true relative residual ||b - A x||/||b|| below tol = 1e-10 on both sides
(the GPU's recomputed here with the oracle's product), and the GPU's x
within 1e-8 relative of the oracle's.  The iteration counts of these long
solves are decided by rounding (see tests/spread.py); here they are only
required to be consistent with the reported (j, i) = (g_n(k), r_n(k)).
"""
from __future__ import annotations

import os

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


@pytest.fixture(scope="module")
def par():
    lib = O.load_par()
    O.par_threads(os.cpu_count() or 1)
    return lib


def _full(par, A, b, n, tol=1e-10, maxit=40000, AH=None, precond=M.MLB_PRECOND_NONE, x_bound=1e-8):
    import torch
    cplx = np.iscomplexobj(A.val)
    dt = torch.complex128 if cplx else torch.float64
    h = M.mlbicgstab_create(A, AH=AH, n=n, q_seed=0, max_outer=10, precond=precond)
    bd = torch.tensor(b, dtype=dt, device="cuda")
    xd = torch.zeros_like(bd)
    res, _ = M.mlbicgstab_solve(h, bd, xd, tol, maxit)
    x = xd.cpu().numpy()
    Q = O.q_gauss(0, A.n_rows, n, complex_=cplx)
    kw = {"ilu": O.ilu0(A)} if precond == M.MLB_PRECOND_ILU0 else {}
    ref = O.solve(A, b, np.zeros_like(b), Q, maxit, tol, lib=par, **kw)
    assert ref.flag == 0 and ref.true_relres < tol, (ref.flag, ref.iter, ref.true_relres)
    assert res.status == 0 and res.flag == 0, res.as_dict()
    assert res.true_relres < tol
    assert O.true_relres(A, b, x, lib=par) < tol
    rel = np.linalg.norm(x - ref.x) / np.linalg.norm(ref.x)
    bound = x_bound(x, ref) if callable(x_bound) else x_bound
    assert rel <= bound, (rel, bound, res.iter, ref.iter)
    info = M.mlbicgstab_info(h)
    h.destroy()
    return res, ref, info


def test_full_solve_cd3d_64(par):
    A = W.cd3d_lognormal(64)
    res, ref, info = _full(par, A, W.uniform_rhs(A.n_rows, seed=2), 4)
    assert info["grid"] >= 64


def test_full_solve_cd3d_96_beyond_l2(par):
    """N = 884,736: matrix (74 MB) and solver state (141 MB) exceed L2;
    all 152 SMs."""
    A = W.cd3d_lognormal(96)
    res, ref, info = _full(par, A, W.uniform_rhs(A.n_rows, seed=2), 4)
    assert info["grid"] == 152


def test_full_solve_cd3d_96_ilu0_beyond_l2(par):
    A = W.cd3d_lognormal(96)
    _full(par, A, W.uniform_rhs(A.n_rows, seed=2), 4, precond=M.MLB_PRECOND_ILU0)


def test_full_solve_complex_helmholtz_64x64x16(par):
    """The damped shifted Laplacian family at a reduced size, n = 8, with
    A^H supplied as a separate CSR."""
    A = W.helmholtz3d_c(64, 64, 16)
    _full(par, A, W.row_sums(A), 8, AH=W.conj_transpose(A))


def test_full_solve_reservoir_without_preconditioner(par):
    """The 3x3-block reservoir family at a size where M = I converges
    (12 x 12 x 6 cells, N = 2,592, about 8,000 iterations).  This family is
    ill-conditioned (cond_2(A) ~ 2e6 here), so two solutions that both
    meet tol = 1e-10 need not agree to 1e-8: the oracle's own solution is
    ~2e-6 away from the exact one (x* = 1).  The bar is what the residuals
    imply: A (x - x_or) = r_or - r, so
        ||x - x_or|| <= ||A^{-1}||_2 (||r|| + ||r_or||),
    with ||A^{-1}||_2 = 1 / sigma_min(A) from a dense SVD, and the 1e-8
    bar wherever that bound is smaller."""
    A = W.bsr3_to_csr(W.reservoir_bsr3(12, 12, 6))
    b = W.row_sums(A)
    N = A.n_rows
    D = np.zeros((N, N))
    for r in range(N):
        k0, k1 = A.row_ptr[r], A.row_ptr[r + 1]
        np.add.at(D[r], A.col[k0:k1], A.val[k0:k1])
    inv_norm = 1.0 / np.linalg.svd(D, compute_uv=False)[-1]
    bn = np.linalg.norm(b)

    def bound(x, ref):
        rr = (O.true_relres(A, b, x, lib=par) + ref.true_relres) * bn
        return max(1e-8, 1.0001 * inv_norm * rr / np.linalg.norm(ref.x))

    _full(par, A, b, 8, x_bound=bound)
