"""Batched solves (one persistent launch, one CTA per system) through the C ABI.

A batch runs, for every system, exactly the arithmetic of a single solve on
one CTA (grid = 1): the same passes, the same reduction order.  So each
batch result must equal the single-CTA solve bit for bit (solution and
iteration count), and each solution must agree with the CPU oracle's to
1e-8 relative with a true residual below tol.
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


def _systems(count, seed, n_min=300, n_max=6000):
    out = []
    for A, meta in W.batch_cd(count, seed=seed, n_min=n_min, n_max=n_max):
        out.append((A, W.row_sums(A)))
    return out


@pytest.mark.parametrize("precision", [M.MLB_PREC_FP64, M.MLB_PREC_FP32_REFINED])
def test_batch_equals_single_cta_solves_and_oracle(precision):
    n, tol, maxit = 4, 1e-10, 4000
    systems = _systems(40, seed=21)
    hs = [M.mlbicgstab_create(A, n=n, q_seed=0, precision=precision) for A, _ in systems]
    bs = [b for _, b in systems]
    xs = [np.zeros(A.n_rows) for A, _ in systems]
    res = M.mlbicgstab_solve_batch(hs, bs, xs, [tol] * len(hs), [maxit] * len(hs))
    for k, ((A, b), r, x) in enumerate(zip(systems, res, xs)):
        assert r.status == 0 and r.flag == 0, (k, r.as_dict())
        assert r.true_relres < tol
        h1 = M.mlbicgstab_create(A, n=n, q_seed=0, precision=precision, grid=1)
        x1 = np.zeros(A.n_rows)
        r1, _ = M.mlbicgstab_solve(h1, b, x1, tol, maxit)
        assert (r.iter, r.outer, r.flag) == (r1.iter, r1.outer, r1.flag), k
        np.testing.assert_array_equal(x, x1)
        ref = O.solve(A, b, np.zeros(A.n_rows), O.q_gauss(0, A.n_rows, n), maxit, tol)
        assert ref.flag == 0
        assert np.linalg.norm(x - ref.x) <= 1e-8 * np.linalg.norm(ref.x), k


def test_batch_more_systems_than_ctas_and_device_pointers():
    import torch
    systems = _systems(400, seed=22, n_min=200, n_max=1500)
    hs = [M.mlbicgstab_create(A, n=2, q_seed=0) for A, _ in systems]
    bs = [torch.tensor(b, device="cuda") for _, b in systems]
    xs = [torch.zeros(A.n_rows, dtype=torch.float64, device="cuda") for A, _ in systems]
    res = M.mlbicgstab_solve_batch(hs, bs, xs, [1e-10] * 400, [3000] * 400)
    assert all(r.flag == 0 and r.true_relres < 1e-10 for r in res)
    for (A, b), x in list(zip(systems, xs))[::37]:
        assert O.true_relres(A, b, x.cpu().numpy()) < 1e-10


def test_batch_rejects_mixed_precision():
    A = W.cd2d(8)
    h1 = M.mlbicgstab_create(A, n=2)
    h2 = M.mlbicgstab_create(A, n=2, precision=M.MLB_PREC_FP32_REFINED)
    b = W.row_sums(A)
    with pytest.raises(M.MlbError) as e:
        M.mlbicgstab_solve_batch([h1, h2], [b, b], [np.zeros(64), np.zeros(64)],
                                 [1e-10, 1e-10], [100, 100])
    assert e.value.code == M.MLB_ERR_ARG


def test_batch_of_small_passes_is_race_free_and_deterministic():
    """Many refinement steps on small systems make many passes of a single
    tile, where the warps of a CTA can be a whole pass apart.  Each thread
    keeps its own tile counter, so every wait must complete (no status
    MLB_ERR_TIMEOUT) and repeated launches must give the same bits."""
    import torch
    systems = [A for A, _ in W.batch_cd(256, seed=23, n_min=300, n_max=3000)]
    bs = [torch.tensor(W.row_sums(A), device="cuda") for A in systems]
    runs = []
    for _ in range(3):
        hs = [M.mlbicgstab_create(A, n=4, q_seed=0, precision=M.MLB_PREC_FP32_REFINED, max_outer=40,
                                  inner_tol=1e-2, inner_maxit=50, timeout_ns=500_000_000) for A in systems]
        xs = [torch.zeros(A.n_rows, dtype=torch.float64, device="cuda") for A in systems]
        res = M.mlbicgstab_solve_batch(hs, bs, xs, [1e-10] * len(hs), [20000] * len(hs))
        assert all(r.status == 0 for r in res)
        runs.append(([x.cpu().numpy() for x in xs], [(r.iter, r.outer, r.flag) for r in res]))
    for xs_k, meta_k in runs[1:]:
        assert meta_k == runs[0][1]
        for a, b in zip(xs_k, runs[0][0]):
            np.testing.assert_array_equal(a, b)


# ------------------------------------------------- teams of CTAs in a batch --

def _check_batch_teams(systems, team, precision=M.MLB_PREC_FP64, precond=M.MLB_PRECOND_NONE, n=4,
                       tol=1e-10, maxit=6000, oracle_every=1):
    """Each system's batch result equals the single solve with grid = the
    CTAs that solved it in the batch (team size, or 1), bit for bit, and
    agrees with the oracle."""
    hs = [M.mlbicgstab_create(A, n=n, q_seed=0, precision=precision, precond=precond) for A in systems]
    M.mlbicgstab_set_tuning(hs[0], batch_team=team)
    bs = [W.row_sums(A) for A in systems]
    xs = [np.zeros(A.n_rows) for A in systems]
    res = M.mlbicgstab_solve_batch(hs, bs, xs, [tol] * len(hs), [maxit] * len(hs))
    ctas = [r.ctas for r in res]
    assert set(ctas) <= {1, team}
    for k, (A, b, r, x) in enumerate(zip(systems, bs, res, xs)):
        assert r.status == 0 and r.flag == 0 and r.true_relres < tol, (k, r.as_dict())
        h1 = M.mlbicgstab_create(A, n=n, q_seed=0, precision=precision, precond=precond, grid=r.ctas)
        assert M.mlbicgstab_info(h1)["grid"] == r.ctas
        x1 = np.zeros(A.n_rows)
        r1, _ = M.mlbicgstab_solve(h1, b, x1, tol, maxit)
        assert (r.iter, r.outer, r.flag) == (r1.iter, r1.outer, r1.flag), (k, r.ctas)
        np.testing.assert_array_equal(x, x1)
        h1.destroy()
        if k % oracle_every == 0:
            pc = {}
            if precond == M.MLB_PRECOND_ILU0:
                pc = dict(ilu=O.ilu0(A))
            ref = O.solve(A, b, np.zeros(A.n_rows), O.q_gauss(0, A.n_rows, n), maxit, tol, **pc)
            assert ref.flag == 0
            assert np.linalg.norm(x - ref.x) <= 1e-8 * np.linalg.norm(ref.x), k
    for h in hs:
        h.destroy()
    return ctas


@pytest.mark.parametrize("team", [2, 4, 8])
def test_batch_teams_fp64(team):
    systems = [A for A, _ in W.batch_cd(20, seed=45, n_min=500, n_max=40000)]
    ctas = _check_batch_teams(systems, team, oracle_every=3)
    assert ctas.count(team) >= 3 and ctas.count(1) >= 3


def test_batch_without_teams_is_one_cta_per_system():
    systems = [A for A, _ in W.batch_cd(8, seed=46, n_min=10000, n_max=30000)]
    ctas = _check_batch_teams(systems, 1, oracle_every=4)
    assert ctas == [1] * len(systems)


def test_batch_more_large_systems_than_teams():
    """Twice as many team systems as teams: teams take several systems in
    turn (the slots of the turns alternate)."""
    systems = [A for A, _ in W.batch_cd(40, seed=47, n_min=17000, n_max=20000)]
    ctas = _check_batch_teams(systems, 8, maxit=4000, oracle_every=8)
    assert ctas.count(8) == len(systems)   # 40 systems, 19 teams of 8 CTAs


def test_batch_teams_refined_and_ilu0():
    systems = [A for A, _ in W.batch_cd(10, seed=48, n_min=2000, n_max=30000)]
    ctas = _check_batch_teams(systems, 4, precision=M.MLB_PREC_FP32_REFINED, oracle_every=3)
    assert 4 in ctas
    # natural-order ILU(0) systems stay on one CTA; the multicolour ones
    # go to teams
    ctas = _check_batch_teams(systems, 4, precond=M.MLB_PRECOND_ILU0, oracle_every=3)
    assert set(ctas) == {1}
    ctas = _check_batch_teams(systems, 4, precond=M.MLB_PRECOND_ILU0_MC, oracle_every=100)
    assert 4 in ctas


def test_batch_teams_complex():
    systems = [W.helmholtz3d_c(m, m, 8, k=2.0) for m in (12, 20, 36, 40)]
    hs = [M.mlbicgstab_create(A, n=4, q_seed=0, AH=W.conj_transpose(A)) for A in systems]
    M.mlbicgstab_set_tuning(hs[0], batch_team=4)
    bs = [W.row_sums(A) for A in systems]
    xs = [np.zeros(A.n_rows, dtype=complex) for A in systems]
    res = M.mlbicgstab_solve_batch(hs, bs, xs, [1e-10] * 4, [6000] * 4)
    assert any(r.ctas == 4 for r in res)
    for A, b, r, x in zip(systems, bs, res, xs):
        assert r.status == 0 and r.flag == 0 and r.true_relres < 1e-10
        h1 = M.mlbicgstab_create(A, n=4, q_seed=0, AH=W.conj_transpose(A), grid=r.ctas)
        x1 = np.zeros(A.n_rows, dtype=complex)
        r1, _ = M.mlbicgstab_solve(h1, b, x1, 1e-10, 6000)
        assert r1.iter == r.iter
        np.testing.assert_array_equal(x, x1)
