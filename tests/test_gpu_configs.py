"""Full-size workloads through the C ABI against the oracle.

* 3x3-block reservoir system (N = 393,216, scalar CSR of 901,120 blocks):
  the first 12 iterations element by element, and the fused SpMV + Q^H y.
* complex damped shifted Laplacian, 256 x 256 x 64 (N = 4,194,304), with
  A^H supplied as a separate CSR: the first 12 iterations element by
  element; the same run with the library forming A^H must be bit-identical.
* 512 convection-diffusion systems of uneven size in one batch launch:
  every system converges (true residual < 1e-10); a sample is compared
  with the oracle's solution and with one-CTA single solves.

Tolerances as in test_gpu_parity (sequential-sum bound gamma_N for the
early residuals; 1e-8 relative for converged solutions).
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


def _early_tol(N):
    return max(1e-10, 4 * N * EPS)


def _first_iterations(A, b, n, K=12, AH=None):
    cplx = np.iscomplexobj(A.val)
    h = M.mlbicgstab_create(A, AH=AH, n=n, q_seed=0)
    x = np.zeros(A.n_rows, dtype=b.dtype)
    res, eh = M.mlbicgstab_solve(h, b, x, 1e-10, K, hist_cap=K + 1)
    ref = O.mlbicgstabt(A, b, np.zeros_like(b), O.q_gauss(0, A.n_rows, n, complex_=cplx), K,
                        1e-10, err_hist=True)
    assert (res.flag, res.iter, res.j, res.i) == (ref.flag, ref.iter, ref.j, ref.i)
    assert res.as_dict()["ops"] == ref.ops
    np.testing.assert_allclose(eh[:K + 1], ref.err_hist[:K + 1], rtol=_early_tol(A.n_rows))
    scale = np.max(np.abs(ref.x))
    assert np.max(np.abs(x - ref.x)) <= 1e-8 * scale
    return x


def test_reservoir_first_iterations_full_size():
    A = W.bsr3_to_csr(W.reservoir_bsr3())
    _first_iterations(A, W.row_sums(A), 8)


def test_helmholtz_complex_full_size_with_supplied_AH():
    A = W.helmholtz3d_c()
    AH = W.conj_transpose(A)
    b = W.row_sums(A)
    x1 = _first_iterations(A, b, 8, AH=AH)
    h = M.mlbicgstab_create(A, n=8, q_seed=0)          # library forms A^H
    x2 = np.zeros(A.n_rows, dtype=complex)
    M.mlbicgstab_solve(h, b, x2, 1e-10, 12)
    np.testing.assert_array_equal(x1, x2)


def test_batch_512_uneven_systems():
    import torch
    systems = W.batch_cd(512, seed=5)
    hs = [M.mlbicgstab_create(A, n=4, q_seed=0) for A, _ in systems]
    bs = [torch.tensor(W.row_sums(A), device="cuda") for A, _ in systems]
    xs = [torch.zeros(A.n_rows, dtype=torch.float64, device="cuda") for A, _ in systems]
    res = M.mlbicgstab_solve_batch(hs, bs, xs, [1e-10] * 512, [20000] * 512)
    assert all(r.status == 0 and r.flag == 0 and r.true_relres < 1e-10 for r in res)
    rng = np.random.default_rng(0)
    sample = sorted(rng.choice(512, size=12, replace=False))
    sizes = np.array([A.n_rows for A, _ in systems])
    sample = sorted(set(sample) | {int(np.argmax(sizes)), int(np.argmin(sizes))})
    for k in sample:
        A, _ = systems[k]
        b = W.row_sums(A)
        x = xs[k].cpu().numpy()
        assert O.true_relres(A, b, x) < 1e-10
        ref = O.solve(A, b, np.zeros(A.n_rows), O.q_gauss(0, A.n_rows, 4), 20000, 1e-10)
        assert ref.flag == 0
        assert np.linalg.norm(x - ref.x) <= 1e-8 * np.linalg.norm(ref.x), k
        # the same arithmetic as a single solve on as many CTAs as solved it
        # in the batch (one, or a team for the large systems)
        h1 = M.mlbicgstab_create(A, n=4, q_seed=0, grid=res[k].ctas)
        x1 = np.zeros(A.n_rows)
        r1, _ = M.mlbicgstab_solve(h1, b, x1, 1e-10, 20000)
        assert r1.iter == res[k].iter
        np.testing.assert_array_equal(x1, x)
    assert {r.ctas for r in res} == {1, 4}
