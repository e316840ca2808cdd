"""Sequences of systems with automatic choice of n (§5, "Choice of n").

* set_n: a handle created with n_max and set to n solves exactly like a
  handle created with n (Q(:,1:n) and F(:,1:n-1) are prefixes), bit for bit.
* solve_sequence: n follows the rule of mlbicgstab_next_n applied to the
  device times the call itself reports, every system converges and agrees
  with the oracle run at the n it used, and handles get their n back.
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


@pytest.mark.parametrize("cplx", [False, True])
def test_set_n_equals_handle_created_with_n(cplx):
    if cplx:
        A, _, b = W.random_dense_system(300, seed=31, complex_=True)
    else:
        A = W.cd2d(32)
        b = W.row_sums(A)
    N = A.n_rows
    h8 = M.mlbicgstab_create(A, n=8, q_seed=0)
    for n in (1, 3, 4, 8):
        M.mlbicgstab_set_n(h8, n)
        assert M.mlbicgstab_info(h8)["n_active"] == n
        hn = M.mlbicgstab_create(A, n=n, q_seed=0)
        x1 = np.zeros(N, dtype=b.dtype)
        x2 = np.zeros(N, dtype=b.dtype)
        r1, _ = M.mlbicgstab_solve(h8, b, x1, 1e-10, 2000)
        r2, _ = M.mlbicgstab_solve(hn, b, x2, 1e-10, 2000)
        assert (r1.iter, r1.flag, r1.j, r1.i) == (r2.iter, r2.flag, r2.j, r2.i)
        np.testing.assert_array_equal(x1, x2)
    with pytest.raises(M.MlbError):
        M.mlbicgstab_set_n(h8, 9)
    with pytest.raises(M.MlbError):
        M.mlbicgstab_set_n(h8, 0)


def test_sequence_follows_the_rule_and_matches_oracle():
    A = W.cd2d(32)
    N = A.n_rows
    rng = np.random.default_rng(33)
    count = 7
    bs = [rng.uniform(-1, 1, N) for _ in range(count)]
    xs = [np.zeros(N) for _ in range(count)]
    h = M.mlbicgstab_create(A, n=8, q_seed=0)
    M.mlbicgstab_set_n(h, 5)
    res, used = M.mlbicgstab_solve_sequence([h] * count, bs, xs, [1e-10] * count, [4000] * count,
                                            n0=4, step=2, n_min=2, n_max=8)
    assert M.mlbicgstab_info(h)["n_active"] == 5          # restored
    assert used[0] == 4 and used[1] == 4
    for s in range(1, count - 1):
        want = M.mlbicgstab_next_n(used[s], res[s - 1].kernel_ms, res[s].kernel_ms, 2, 2, 8)
        assert used[s + 1] == want, (s, used)
    Qfull = O.q_gauss(0, N, 8)
    for s in range(count):
        assert res[s].flag == 0 and res[s].true_relres < 1e-10
        ref = O.solve(A, bs[s], np.zeros(N), Qfull[:, :used[s]], 4000, 1e-10)
        assert ref.flag == 0
        assert np.linalg.norm(xs[s] - ref.x) <= 1e-8 * np.linalg.norm(ref.x)


def test_sequence_of_different_matrices_with_device_arrays():
    import torch
    systems = [A for A, _ in W.batch_cd(5, seed=34, n_min=400, n_max=2500)]
    hs = [M.mlbicgstab_create(A, n=6, q_seed=0) for A in systems]
    bs = [torch.tensor(W.row_sums(A), device="cuda") for A in systems]
    xs = [torch.zeros(A.n_rows, dtype=torch.float64, device="cuda") for A in systems]
    res, used = M.mlbicgstab_solve_sequence(hs, bs, xs, [1e-10] * 5, [4000] * 5, n0=3, step=1, n_min=1, n_max=6)
    assert all(1 <= n <= 6 for n in used) and used[:2] == [3, 3]
    for A, b, x, r in zip(systems, bs, xs, res):
        assert r.flag == 0
        assert O.true_relres(A, b.cpu().numpy(), x.cpu().numpy()) < 1e-10
    with pytest.raises(M.MlbError):   # a handle created with n < n_max
        M.mlbicgstab_solve_sequence(hs, bs, xs, [1e-10] * 5, [4000] * 5, n0=3, step=1, n_min=1, n_max=7)
