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
