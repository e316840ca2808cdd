"""The autotuner: it picks a configuration among its candidates, solves after
tuning still agree with the oracle, the process-wide cache returns the same
choice for a second handle of the same shape (and the same bits), and
batches of tuned handles still match the oracle."""
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


def test_autotune_choice_cache_and_parity():
    A = W.cd2d(96)
    b = W.row_sums(A)
    N = A.n_rows
    h = M.mlbicgstab_create(A, n=4, q_seed=0)
    g_before = M.mlbicgstab_info(h)["grid"]
    r = M.mlbicgstab_autotune(h, iters=20, use_cache=False)
    assert r["from_cache"] == 0 and r["trials"] >= 4
    assert r["spt_cap"] in (15, 12, 8, 4)
    assert 1 <= r["grid"] <= max(g_before, 1)
    assert r["us_per_iter"] <= r["default_us_per_iter"]
    assert M.mlbicgstab_info(h)["grid"] == r["grid"]
    x = np.zeros(N)
    res, _ = M.mlbicgstab_solve(h, b, x, 1e-10, 4000)
    ref = O.solve(A, b, np.zeros(N), O.q_gauss(0, N, 4), 4000, 1e-10)
    assert res.flag == 0 and ref.flag == 0 and res.true_relres < 1e-10
    assert np.linalg.norm(x - ref.x) <= 1e-8 * np.linalg.norm(ref.x)
    h2 = M.mlbicgstab_create(A, n=4, q_seed=0)
    r2 = M.mlbicgstab_autotune(h2, iters=20, use_cache=True)
    assert r2["from_cache"] == 1 and (r2["grid"], r2["spt_cap"]) == (r["grid"], r["spt_cap"])
    x2 = np.zeros(N)
    res2, _ = M.mlbicgstab_solve(h2, b, x2, 1e-10, 4000)
    assert res2.iter == res.iter
    np.testing.assert_array_equal(x2, x)
    with pytest.raises(M.MlbError):
        M.mlbicgstab_autotune(h, iters=0)


def test_tuned_handles_in_a_batch_match_oracle():
    """Batches use each handle's tuned tile cap (the CTA count does not apply
    to a batch, which runs one CTA per system)."""
    systems = [A for A, _ in W.batch_cd(16, seed=41, n_min=500, n_max=5000)]
    hs = [M.mlbicgstab_create(A, n=4, q_seed=0) for A in systems]
    for h in hs:
        M.mlbicgstab_autotune(h, iters=10, use_cache=True)
    bs = [W.row_sums(A) for A in systems]
    xs = [np.zeros(A.n_rows) for A in systems]
    res = M.mlbicgstab_solve_batch(hs, bs, xs, [1e-10] * len(hs), [4000] * len(hs))
    for A, b, r, x in zip(systems, bs, res, xs):
        assert r.flag == 0 and r.true_relres < 1e-10
        ref = O.solve(A, b, np.zeros(A.n_rows), O.q_gauss(0, A.n_rows, 4), 4000, 1e-10)
        assert np.linalg.norm(x - ref.x) <= 1e-8 * np.linalg.norm(ref.x)


# ------------------------------------------- fused columns of the product --

def _qdot_vs_oracle(h, A, seed=0):
    """The handle's fused product against the oracle's y = A x and Q^H y
    (the same bounds as the parity tests of the product)."""
    import torch
    from tests.test_gpu_parity import _abs_spmv, _gamma
    cplx = np.iscomplexobj(A.val)
    rng = np.random.default_rng(seed)
    x = rng.standard_normal(A.n_rows) + (1j * rng.standard_normal(A.n_rows) if cplx else 0.0)
    dt = torch.complex128 if cplx else torch.float64
    xd = torch.tensor(x, dtype=dt, device="cuda")
    yd = torch.empty_like(xd)
    d = M.mlbicgstab_spmv_qdot(h, xd, yd)
    y = yd.cpu().numpy()
    yo = O.spmv(A, x)
    w = int(np.max(np.diff(A.row_ptr))) + 1
    assert np.all(np.abs(y - yo) <= 2 * _gamma(w) * _abs_spmv(A, x) + 1e-300)
    n = M.mlbicgstab_info(h)["n_active"]
    Q = M.mlbicgstab_get_Q(h)[:, :n]
    do = Q.conj().T @ yo
    bd = (np.abs(Q).T @ np.abs(y - yo)) + 2 * _gamma(A.n_rows) * (np.abs(Q).T @ np.abs(yo))
    assert np.all(np.abs(d - do) <= bd), (d, do)
    return d


@pytest.mark.parametrize("n,cplx", [(8, False), (4, False), (3, False), (5, True), (2, True)])
def test_every_fused_column_count_matches_oracle(n, cplx):
    """Each column count the tuner may choose (1, 2, 4; 4 real only; at
    most n) gives the product the oracle gives, on a matrix of several
    tiles per CTA with a ragged tail."""
    A = W.helmholtz3d_c(12, 11, 9) if cplx else W.cd3d_lognormal(23)
    h = M.mlbicgstab_create(A, n=n, q_seed=3)
    for ne in (1, 2, 4):
        if ne > n or (cplx and ne > 2):
            continue
        M.mlbicgstab_set_tuning(h, qd_fused=ne)
        assert M.mlbicgstab_get_tuning(h)["qd_fused"] == ne
        _qdot_vs_oracle(h, A, seed=ne)
    h.destroy()


@pytest.mark.parametrize("n,cplx", [(8, False), (4, False), (3, True)])
def test_every_fused_column_count_fp32_copies(n, cplx):
    """The same for the FP32 product on a refined handle's copies."""
    from tests.test_gpu_parity import fp32_product_vs_oracle
    A = W.helmholtz3d_c(10, 9, 7) if cplx else W.cd3d_lognormal(23)
    h = M.mlbicgstab_create(A, n=n, q_seed=2, precision=M.MLB_PREC_FP32_REFINED)
    for ne in (1, 2, 4):
        if ne > n or (cplx and ne > 2):
            continue
        M.mlbicgstab_set_tuning(h, qd_fused=ne)
        fp32_product_vs_oracle(h, A, n, cplx, 10 + ne)
    r = M.mlbicgstab_autotune(h, iters=5, use_cache=False)
    assert r["qd_fused"] in (1, 2, 4) and r["qd_us"] <= r["qd_default_us"]
    fp32_product_vs_oracle(h, A, n, cplx, 20)
    h.destroy()


def test_fused_column_choice_above_active_n_falls_back():
    A = W.cd3d_lognormal(16)
    h = M.mlbicgstab_create(A, n=8, q_seed=0)
    M.mlbicgstab_set_tuning(h, qd_fused=4)
    M.mlbicgstab_set_n(h, 2)
    _qdot_vs_oracle(h, A, seed=1)
    M.mlbicgstab_set_n(h, 1)
    _qdot_vs_oracle(h, A, seed=2)
    h.destroy()


def test_set_tuning_validates():
    A = W.helmholtz3d_c(6, 6, 6)
    h = M.mlbicgstab_create(A, n=4)
    t = M.mlbicgstab_get_tuning(h)
    assert t["batch_spt_cap"] == -1 and t["qd_fused"] == 0 and 1 <= t["spt_cap"] <= 15
    assert t["batch_team"] == 4
    for bad in (dict(qd_fused=4), dict(qd_fused=3), dict(spt_cap=0), dict(spt_cap=16),
                dict(batch_team=0), dict(batch_team=9),
                dict(batch_spt_cap=-2), dict(batch_spt_cap=16), dict(grid=0), dict(grid=100000)):
        with pytest.raises(M.MlbError):
            M.mlbicgstab_set_tuning(h, **bad)
    assert M.mlbicgstab_get_tuning(h) == t
    h.destroy()


def test_autotune_chooses_fused_columns_and_keeps_parity():
    A = W.cd3d_lognormal(40)
    h = M.mlbicgstab_create(A, n=8, q_seed=0)
    r = M.mlbicgstab_autotune(h, iters=10, use_cache=False)
    assert r["qd_fused"] in (1, 2, 4)
    assert 0 < r["qd_us"] <= r["qd_default_us"]
    assert M.mlbicgstab_get_tuning(h)["qd_fused"] == r["qd_fused"]
    _qdot_vs_oracle(h, A, seed=4)
    # a cached choice is applied to a second handle of the same shape
    h2 = M.mlbicgstab_create(A, n=8, q_seed=0)
    r2 = M.mlbicgstab_autotune(h2, iters=10, use_cache=True)
    assert r2["from_cache"] == 1 and r2["qd_fused"] == r["qd_fused"]
    # no product on a preconditioned handle: nothing chosen
    h3 = M.mlbicgstab_create(A, n=4, precond=M.MLB_PRECOND_JACOBI)
    assert M.mlbicgstab_autotune(h3, iters=5, use_cache=False)["qd_fused"] == 0
    for hh in (h, h2, h3):
        hh.destroy()


# ------------------------------------------------------- batch autotuner --

def _batch_vs_oracle(hs, systems, tol=1e-10, maxit=4000):
    bs = [W.row_sums(A) for A in systems]
    xs = [np.zeros(A.n_rows) for A in systems]
    res = M.mlbicgstab_solve_batch(hs, bs, xs, [tol] * len(hs), [maxit] * len(hs))
    for A, b, r, x in zip(systems, bs, res, xs):
        assert r.status == 0 and r.flag == 0 and r.true_relres < tol, r.as_dict()
        assert O.true_relres(A, b, x) < tol
        ref = O.solve(A, b, np.zeros(A.n_rows), O.q_gauss(0, A.n_rows, 4), maxit, tol)
        assert np.linalg.norm(x - ref.x) <= 1e-8 * np.linalg.norm(ref.x)
    return res


@pytest.mark.parametrize("cap", [0, 4, 15])
def test_batch_tile_caps_match_oracle(cap):
    """Every batch cap the batch tuner may choose, including 0 (the product
    reads the matrix with plain loads), solves to the oracle's x."""
    systems = [A for A, _ in W.batch_cd(10, seed=43, n_min=300, n_max=6000)]
    hs = [M.mlbicgstab_create(A, n=4, q_seed=0) for A in systems]
    for h in hs:
        M.mlbicgstab_set_tuning(h, batch_spt_cap=cap)
    _batch_vs_oracle(hs, systems)
    for h in hs:
        h.destroy()


def test_batch_autotune_per_size_class():
    systems = [A for A, _ in W.batch_cd(24, seed=44, n_min=300, n_max=20000)]
    hs = [M.mlbicgstab_create(A, n=4, q_seed=0) for A in systems]
    classes = {(int(np.floor(np.log2(A.n_rows))), int(round(A.nnz / A.n_rows))) for A in systems}
    r = M.mlbicgstab_autotune_batch(hs, tol=1e-8, maxit=3000, use_cache=False)
    assert r["classes"] == len(classes) and r["from_cache"] == 0
    assert r["trials"] >= 5 * len(classes) + 4
    assert r["default_ms"] > 0 and r["tuned_ms"] > 0
    caps = [M.mlbicgstab_get_tuning(h)["batch_spt_cap"] for h in hs]
    assert all(c in (15, 12, 8, 4, 0) for c in caps)
    assert r["team"] in (1, 2, 4, 8)
    assert all(M.mlbicgstab_get_tuning(h)["batch_team"] == r["team"] for h in hs)
    # one choice per class
    by_class = {}
    for A, c in zip(systems, caps):
        k = (int(np.floor(np.log2(A.n_rows))), int(round(A.nnz / A.n_rows)))
        assert by_class.setdefault(k, c) == c
    # single solves keep their own cap
    assert all(M.mlbicgstab_get_tuning(h)["spt_cap"] == 15 for h in hs)
    _batch_vs_oracle(hs, systems)
    # cached: the same caps, nothing timed but the two whole-batch launches
    hs2 = [M.mlbicgstab_create(A, n=4, q_seed=0) for A in systems]
    r2 = M.mlbicgstab_autotune_batch(hs2, tol=1e-8, maxit=3000, use_cache=True)
    assert r2["from_cache"] == r["classes"] and r2["trials"] == 0 and r2["team"] == r["team"]
    assert [M.mlbicgstab_get_tuning(h)["batch_spt_cap"] for h in hs2] == caps
    for h in hs + hs2:
        h.destroy()


def test_batch_autotune_rejects_a_repeated_handle():
    A = W.cd2d(20)
    h = M.mlbicgstab_create(A, n=4)
    with pytest.raises(M.MlbError):
        M.mlbicgstab_autotune_batch([h, h], tol=1e-8, maxit=5)
    h.destroy()
