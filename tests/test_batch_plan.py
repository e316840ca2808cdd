"""The batch work plan (host only, no GPU): which systems mlbicgstab_solve_batch
gives to teams of CTAs, in which order, and how many CTAs it launches.

The rule, as the header states it: estimated work w = (nnz + N) N^(1/3);
a system goes to a team when the team has more than one CTA, it is not
preconditioned by natural-order ILU(0), it has at least 2048 rows per team
CTA, and w exceeds a tenth of the average work per CTA; team systems come
first, then the others, each largest first (ties in input order); teams =
min(team systems, slots // team); grid = min(slots, teams * team + others).
"""
from __future__ import annotations

import numpy as np
import pytest

from paper_1106_3678_gb300 import build as B
from paper_1106_3678_gb300 import mlbicgstab as M
from paper_1106_3678_gb300 import workloads as W


@pytest.fixture(scope="module", autouse=True)
def _lib():
    B.build()
    M.load()


def _expected(N, nnz, pc, team, slots):
    N = np.asarray(N, dtype=np.int64)
    nnz = np.asarray(nnz, dtype=np.int64)
    tm = max(1, min(team, slots))
    w = (nnz + N).astype(float) * np.cbrt(N.astype(float))
    avg = w.sum() / slots
    big = [s for s in range(len(N)) if tm > 1 and pc[s] != M.MLB_PRECOND_ILU0 and N[s] >= 2048 * tm
           and w[s] > 0.1 * avg]
    small = [s for s in range(len(N)) if s not in big]
    key = lambda s: -w[s]
    order = sorted(big, key=key) + sorted(small, key=key)   # sorted() is stable
    teams = min(len(big), slots // tm)
    grid = min(slots, teams * tm + len(small))
    ctas = [tm if s in big else 1 for s in range(len(N))]
    return ctas, order, len(big), teams, grid


@pytest.fixture(scope="module")
def batch512():
    systems = [A for A, _ in W.batch_cd(512, seed=5)]
    return [A.n_rows for A in systems], [A.nnz for A in systems]


@pytest.mark.parametrize("team,slots", [(4, 152), (2, 152), (8, 152), (1, 152), (4, 16), (8, 3)])
def test_plan_of_the_512_system_batch(team, slots, batch512):
    N, nnz = batch512
    pc = [0] * len(N)
    got = M.mlbicgstab_batch_plan(N, nnz, pc, team=team, slots=slots)
    ctas, order, nbig, teams, grid = _expected(N, nnz, pc, team, slots)
    assert list(got["ctas"]) == ctas
    assert list(got["order"]) == order
    assert (got["nbig"], got["teams"], got["grid"]) == (nbig, teams, grid)
    assert sorted(got["order"]) == list(range(len(N)))
    if team == 4 and slots == 152:
        # the bench workload: 240 of the 271 systems of at least 8,192 rows
        # carry enough work for a team
        assert got["nbig"] == 240 and sum(1 for n in N if n >= 8192) == 271 and got["grid"] == 152


def test_natural_ilu0_systems_stay_on_one_cta_and_ties_keep_input_order():
    N = [40000, 40000, 40000, 1000, 1000, 50000]
    nnz = [7 * n for n in N]
    pc = [M.MLB_PRECOND_ILU0, M.MLB_PRECOND_NONE, M.MLB_PRECOND_ILU0_MC, 0, 0, M.MLB_PRECOND_JACOBI]
    got = M.mlbicgstab_batch_plan(N, nnz, pc, team=4, slots=152)
    assert list(got["ctas"]) == [1, 4, 4, 1, 1, 4]
    assert list(got["order"]) == [5, 1, 2, 0, 3, 4]
    assert (got["nbig"], got["teams"], got["grid"]) == (3, 3, 15)


def test_small_batches_and_few_slots():
    # one small system: no team, one CTA
    got = M.mlbicgstab_batch_plan([500], [2400], [0], team=4, slots=152)
    assert list(got["ctas"]) == [1] and (got["teams"], got["grid"]) == (0, 1)
    # more team systems than teams fit: teams take them in turns
    got = M.mlbicgstab_batch_plan([100000] * 10, [700000] * 10, [0] * 10, team=8, slots=20)
    assert got["nbig"] == 10 and got["teams"] == 2 and got["grid"] == 16
    # a team larger than the slots is clipped to the slots
    got = M.mlbicgstab_batch_plan([100000] * 2, [700000] * 2, [0] * 2, team=8, slots=4)
    assert list(got["ctas"]) == [4, 4] and got["teams"] == 1 and got["grid"] == 4


def test_plan_validates_its_arguments():
    with pytest.raises(M.MlbError):
        M.mlbicgstab_batch_plan([100], [500], [0], team=0)
    with pytest.raises(M.MlbError):
        M.mlbicgstab_batch_plan([100], [500], [0], slots=0)
    with pytest.raises(M.MlbError):
        M.mlbicgstab_batch_plan([0], [500], [0])
    with pytest.raises(M.MlbError):
        M.mlbicgstab_batch_plan([100], [-1], [0])
    with pytest.raises(M.MlbError):
        M.mlbicgstab_batch_plan([], [], [])
