"""The multi-GPU form is weak scaling over independent runs: each rank runs
its own run (seed + rank) and the only collectives are the timing ones.
Their host logic runs here on CPU ranks (gloo, world size 2): the whole-job
throughput is every rank's work over the slowest rank's time."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        import bench
        # rank r: 10 + r ms device time, (r + 1) * 1e9 sim-days, e2e 2e9 in 0.5 + r s
        v, e, ms = bench.job_totals(10.0 + rank, (rank + 1) * 1e9, 2e9, 0.5 + rank, ws,
                                    device="cpu")
        out[rank] = (v, e, ms)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_job_totals_two_gloo_ranks():
    ws, port = 2, _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(ws, port, out), nprocs=ws, join=True)
        res = dict(out)
    for rank in range(ws):
        v, e, ms = res[rank]
        assert ms == 11.0                          # slowest rank's device time
        assert abs(v - 3e9 / 11e-3) < 1e-3 * v      # all ranks' sim-days over it
        assert abs(e - 4e9 / 1.5) < 1e-9 * e        # end to end: slowest host time


def test_single_rank_is_plain_ratio():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_totals(20.0, 4e9, 1e9, 0.25, 1) == (4e9 / 20e-3, 4e9, 20.0)


def test_each_rank_runs_its_own_run():
    sys.path.insert(0, ROOT)
    import bench
    from paper_2106_15508_gb300 import build as B
    from paper_2106_15508_gb300 import workloads as WL
    B.build()
    seeds = {bench.rank_config(WL.SMALL, r).seed for r in range(4)}
    assert len(seeds) == 4
