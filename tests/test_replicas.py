"""Multi-process host logic of replica runs, on CPU with gloo (world size 2).

Each rank reports its own step count and time; the job's time must be the
maximum over ranks and the throughput the sum of units over that time.  A
rank also solves a small system with the oracle (its own replica) so the
test covers ranks doing independent work between the collectives.
"""
from __future__ import annotations

import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(ws), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        import numpy as np

        import oracle as O
        from paper_1106_3678_gb300 import replicas as R
        from paper_1106_3678_gb300 import workloads as W
        assert R.world() == (ws, rank, rank)
        # every rank solves its own replica (same inputs, independent work)
        A = W.cd2d(8)
        b = W.row_sums(A)
        res = O.mlbicgstabt(A, b, np.zeros(A.n_rows), O.q_gauss(0, A.n_rows, 2), 200, 1e-10)
        steps = 3 + rank            # ranks did different amounts of work
        secs = 1.0 + 0.5 * rank     # and took different times
        thr, job = R.job_throughput(steps, secs)
        mx = R.max_over_ranks(float(res.iter) + rank)
        out[rank] = (thr, job, mx, res.iter, res.flag)
    finally:
        dist.destroy_process_group()


def test_replica_aggregation_gloo_two_ranks():
    ws = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        mp.start_processes(_worker, args=(ws, port, out), nprocs=ws, join=True, start_method="spawn")
        got = dict(out)
    assert sorted(got) == [0, 1]
    for rank in range(ws):
        thr, job, mx, it, flag = got[rank]
        assert job == 1.5                          # max over ranks of 1.0, 1.5
        assert thr == pytest.approx((3 + 4) / 1.5)  # sum of steps / max time
        assert flag == 0
        assert mx == max(got[r][3] + r for r in range(ws))
    assert got[0][3] == got[1][3]                  # identical replicas


def test_single_process_is_identity():
    from paper_1106_3678_gb300 import replicas as R
    if dist.is_initialized():
        pytest.skip("a process group is already initialised")
    assert R.max_over_ranks(2.5) == 2.5
    assert R.sum_over_ranks(2.5) == 2.5
    assert R.job_throughput(4, 2.0) == (2.0, 2.0)
