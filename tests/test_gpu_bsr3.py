"""3x3-block (BSR(3)) matrices through the C ABI.

A BSR(3) input (mlb_matrix.block = 3) and a scalar CSR whose rows come in
triplets of consecutive columns (the same matrix expanded) are both stored
with one column index per three values; the products sum each row value by
value in column order, i.e. in the order of the expanded CSR row, so the
oracle on the expanded CSR is the reference (same rounding bounds as the
scalar tests).
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle as O
from paper_1106_3678_gb300 import mlbicgstab as M
from paper_1106_3678_gb300 import workloads as W
from tests import spread

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


def test_bsr_input_and_triplet_csr_share_the_block_storage():
    B = W.reservoir_bsr3(8, 8, 4)
    A = W.bsr3_to_csr(B)
    b = W.row_sums(A)
    hb = M.mlbicgstab_create(B, n=4)
    hc = M.mlbicgstab_create(A, n=4)
    assert M.mlbicgstab_info(hb)["entry_values"] == 3
    assert M.mlbicgstab_info(hc)["entry_values"] == 3
    assert M.mlbicgstab_info(hb)["nnz"] == A.nnz
    xb, xc = np.zeros(A.n_rows), np.zeros(A.n_rows)
    rb, hb_hist = M.mlbicgstab_solve(hb, b, xb, 0.0, 40, hist_cap=41)
    rc, hc_hist = M.mlbicgstab_solve(hc, b, xc, 0.0, 40, hist_cap=41)
    np.testing.assert_array_equal(xb, xc)
    np.testing.assert_array_equal(hb_hist, hc_hist)
    # a scalar matrix keeps one value per entry
    assert M.mlbicgstab_info(M.mlbicgstab_create(W.cd2d(12), n=2))["entry_values"] == 1


@pytest.mark.parametrize("n", [4, 8])
def test_bsr_early_iterations_match_oracle(n):
    B = W.reservoir_bsr3(10, 8, 6)
    A = W.bsr3_to_csr(B)
    N = A.n_rows
    b = W.uniform_rhs(N, seed=3)
    h = M.mlbicgstab_create(B, n=n, q_seed=0)
    K = 8
    x = np.zeros(N)
    res, eh = M.mlbicgstab_solve(h, b, x, 0.0, K, hist_cap=K + 1)
    # compared on the steps the method determines (tests/spread.py)
    ref, k = spread.unique_prefix(A, b, O.q_gauss(0, N, n), K)
    assert k >= 1
    assert (res.iter, res.j, res.i) == (ref.iter, ref.j, ref.i)
    assert res.as_dict()["ops"] == ref.ops
    np.testing.assert_allclose(eh[:k + 1], ref.err_hist[:k + 1], rtol=max(1e-10, 4 * N * EPS))
    if k == K:
        np.testing.assert_allclose(x, ref.x, rtol=0, atol=1e-9 * np.max(np.abs(ref.x)))


@pytest.mark.parametrize("precond", [M.MLB_PRECOND_ILU0, M.MLB_PRECOND_JACOBI])
def test_bsr_preconditioned_solve_matches_oracle(precond):
    B = W.reservoir_bsr3(12, 12, 6)
    A = W.bsr3_to_csr(B)
    N = A.n_rows
    b = W.row_sums(A)
    h = M.mlbicgstab_create(B, n=8, q_seed=0, precond=precond, max_outer=10)
    assert M.mlbicgstab_info(h)["entry_values"] == 3
    x = np.zeros(N)
    res, _ = M.mlbicgstab_solve(h, b, x, 1e-10, 20000)
    kw = {"ilu": O.ilu0(A)} if precond == M.MLB_PRECOND_ILU0 else {"mdiag": O.jacobi_diag(A)}
    ref = O.solve(A, b, np.zeros(N), O.q_gauss(0, N, 8), 20000, 1e-10, **kw)
    assert res.flag == 0 and ref.flag == 0
    assert res.true_relres < 1e-10 and O.true_relres(A, b, x) < 1e-10
    assert np.linalg.norm(x - ref.x) <= 1e-8 * np.linalg.norm(ref.x)


def test_bsr_refined_with_ilu0_matches_oracle():
    B = W.reservoir_bsr3(16, 16, 8)
    A = W.bsr3_to_csr(B)
    N = A.n_rows
    b = W.row_sums(A)
    h = M.mlbicgstab_create(B, n=8, q_seed=0, precond=M.MLB_PRECOND_ILU0, precision=M.MLB_PREC_FP32_REFINED)
    assert M.mlbicgstab_info(h)["entry_values"] == 3
    x = np.zeros(N)
    res, _ = M.mlbicgstab_solve(h, b, x, 1e-10, 20000)
    ref = O.solve(A, b, np.zeros(N), O.q_gauss(0, N, 8), 20000, 1e-10, ilu=O.ilu0(A))
    assert res.flag == 0 and res.true_relres < 1e-10 and O.true_relres(A, b, x) < 1e-10
    assert np.linalg.norm(x - ref.x) <= 1e-8 * np.linalg.norm(ref.x)


def test_bsr_handles_outside_the_single_solve_are_refused():
    import torch
    B = W.reservoir_bsr3(4, 4, 4)
    h = M.mlbicgstab_create(B, n=2)
    N = B.n_rows
    x = torch.ones(N, dtype=torch.float64, device="cuda")
    y = torch.empty_like(x)
    with pytest.raises(M.MlbError) as e:
        M.mlbicgstab_spmv_qdot(h, x, y)
    assert e.value.code == M.MLB_ERR_UNSUPPORTED
    with pytest.raises(M.MlbError) as e:
        M.mlbicgstab_solve_batch([h], [np.ones(N)], [np.zeros(N)], [1e-8], [10])
    assert e.value.code == M.MLB_ERR_UNSUPPORTED
