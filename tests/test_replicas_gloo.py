"""The multi-process host logic of the benchmark (replicas only: every rank
fits its own problem, no collective on the data path) on two gloo ranks on
the CPU: per-rank seeds and the whole-job rate over the slowest rank."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        assert bench.dist_env() == (ws, rank, rank)
        ms, rate = bench.aggregate_rate(10.0 * (rank + 1), steps=5, ws=ws)
        q.put((rank, bench.replica_seed(7, rank), ms, rate))
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_gloo_ranks():
    ws = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=100) for _ in range(ws))
    for p in procs:
        p.join(timeout=30)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [7, 8]                 # distinct replicas
    for _, _, ms, rate in out:
        assert ms == 20.0                                # the slowest rank's time
        assert rate == pytest.approx(ws * 5 / 0.020)     # all ranks' EM iterations


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate_rate(4.0, steps=2, ws=1) == (4.0, 500.0)
