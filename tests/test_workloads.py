"""Synthetic input generators: sizes, structure and the properties the
stand-in workloads are defined by."""
from __future__ import annotations

import numpy as np
import pytest

from paper_1106_3678_gb300 import workloads as W
from tests import textbook as TB


def _check_csr(A):
    assert A.row_ptr[0] == 0 and A.row_ptr[-1] == A.nnz == len(A.col)
    assert np.all(np.diff(A.row_ptr) >= 0)
    assert A.col.min() >= 0 and A.col.max() < A.n_rows
    for r in range(0, A.n_rows, max(1, A.n_rows // 97)):
        c = A.col[A.row_ptr[r]:A.row_ptr[r + 1]]
        assert np.all(np.diff(c) > 0)


def test_cd2d_sizes_and_stencil():
    A = W.cd2d(32)
    _check_csr(A)
    assert (A.n_rows, A.nnz) == (1024, 4992)
    M = TB.dense(A)
    h = 1 / 33
    assert M[40, 40] == 4.0
    assert M[40, 41] == pytest.approx(-1 + 10 * h / 2)
    assert M[40, 39] == pytest.approx(-1 - 10 * h / 2)
    assert M[40, 72] == pytest.approx(-1 + 5 * h / 2)
    assert M[40, 8] == pytest.approx(-1 - 5 * h / 2)
    np.testing.assert_allclose(W.row_sums(A), M.sum(axis=1), atol=1e-14)


def test_cd3d_full_size_counts():
    A = W.cd3d_lognormal(128)
    assert (A.n_rows, A.nnz) == (2_097_152, 14_581_760)
    _check_csr(A)


def test_cd3d_symmetric_part_is_the_diffusion():
    """Central convection is skew: A + A^T keeps only the (SPD) diffusion."""
    A = W.cd3d_lognormal(6, seed=1)
    M = TB.dense(A)
    S = (M + M.T) / 2
    assert np.all(np.linalg.eigvalsh(S) > 0)
    K = (M - M.T) / 2
    h = 1 / 7
    assert np.max(np.abs(K)) == pytest.approx(50 * h / 2)


def test_reservoir_counts_and_dominance():
    B = W.reservoir_bsr3()
    assert (B.n_rows, B.nblocks) == (393_216, 901_120)
    small = W.reservoir_bsr3(5, 4, 3)
    C = W.bsr3_to_csr(small)
    _check_csr(C)
    M = TB.dense(C)
    d = np.abs(np.diag(M))
    off = np.abs(M).sum(axis=1) - d
    np.testing.assert_allclose(d, 1.05 * off, rtol=1e-12)


def test_helmholtz_counts_and_conj_transpose():
    A = W.helmholtz3d_c()
    assert (A.n_rows, A.nnz) == (4_194_304, 29_163_520)
    S = W.helmholtz3d_c(6, 5, 4)
    AH = W.conj_transpose(S)
    _check_csr(AH)
    np.testing.assert_array_equal(TB.dense(AH), TB.dense(S).conj().T)


def test_batch_sizes():
    sys_ = W.batch_cd(512, seed=5)
    Ns = np.array([A.n_rows for A, _ in sys_])
    assert len(sys_) == 512
    assert Ns.min() >= 900 and Ns.max() <= 110_000
    assert 9e6 < Ns.sum() < 13e6
    dims = [m["dim"] for _, m in sys_]
    assert 180 < dims.count(2) < 330


def test_iteration_window_is_a_prediction_interval():
    from tests import spread
    lo, hi = spread.window([100] * 17)
    assert (lo, hi) == (99.0, 101.0)
    c = [100, 104, 98, 101, 97, 103, 99, 100, 102, 96, 105, 100, 99, 101, 98, 100, 102]
    lo, hi = spread.window(c)
    m, s = np.mean(c), np.std(c, ddof=1)
    assert np.isclose(hi - m, 4.015 * s * np.sqrt(1 + 1 / 17))
    assert lo <= min(c) and hi >= max(c)
    b = np.arange(5.0)
    bb = spread.perturbed(b, 1)
    assert np.count_nonzero(bb != b) == 1 and np.all(bb >= b)
