"""The N > 1 path of bench.py on CPU: two gloo ranks (127.0.0.1) run the whole-job
aggregation - the slowest rank's time, all ranks' units - and the reference arm's
rank rule (only rank 0 works and prints). No GPU: the replicas share no data, so the
aggregation is the only collective the path has."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r took (r + 1) * 10 ms for (r + 1) * 1000 units
        ms, units = bench.aggregate(10.0 * (rank + 1), 1000.0 * (rank + 1), torch)
        w, r, _ = bench.dist_env()
        out.put((rank, ms, units, w, r))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_like_the_bench():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    results = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, units, w, r in results:
        assert (w, r) == (2, rank)
        assert ms == 20.0          # max over ranks
        assert units == 3000.0     # sum over ranks


def test_reference_arm_runs_on_rank_zero_only():
    sys.path.insert(0, ROOT)
    import bench

    class Args:
        ref_rows = 8
        steps = 1
        warmup = 3

    # a non-zero rank exits 0 at once, without starting the oracle
    assert bench.run_reference(Args(), 2, 1) == 0
