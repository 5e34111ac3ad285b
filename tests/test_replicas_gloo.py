"""The multi-GPU path is N independent replicas (every rank solves its own
problem; no data-path collective): bench.py times each rank and reports the
slowest rank's time with the work of all ranks.  Checked here with two gloo
ranks on the CPU (no GPU needed)."""
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


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r: 10 + 5r ms for (r + 1) * 1e6 point-iterations
        ms, work = bench.aggregate(10.0 + 5.0 * rank, (rank + 1) * 1e6, world, device="cpu")
        out.put((rank, ms, work))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_replica_aggregation_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, work in res:
        assert ms == pytest.approx(15.0)      # the slowest rank
        assert work == pytest.approx(3e6)     # every rank's work


def test_single_rank_is_unchanged():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate(7.0, 42.0, 1) == (7.0, 42.0)
