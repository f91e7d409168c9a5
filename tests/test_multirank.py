"""The N > 1 path of bench.py on CPU: world-size-2 gloo ranks, replicas only.

The suggest path has no exchange step, so N GPUs run N independent replicas;
the only collectives are the timing reductions: units summed over ranks, time
the slowest rank's.
"""
import os

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    value, seconds = bench.aggregate(units=1000 * (rank + 1), seconds=0.5 + rank, world=world)
    q.put((rank, value, seconds))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_aggregation_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + (os.getpid() % 1000)
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    out = sorted(q.get() for _ in range(2))
    for rank, value, seconds in out:
        assert seconds == pytest.approx(1.5)            # max over ranks
        assert value == pytest.approx(3000 / 1.5)       # all ranks' units / slowest time


def test_single_rank_aggregation():
    import bench
    assert bench.aggregate(500, 2.0, 1) == (250.0, 2.0)


def test_reference_arm_runs_on_cpu(capsys):
    """--impl reference times the oracle on the host and prints one JSON line."""
    import json
    import sys
    import bench
    argv = sys.argv
    sys.argv = ["bench.py", "--impl", "reference", "--config", "1", "--steps", "2", "--warmup", "3"]
    try:
        bench.main()
    finally:
        sys.argv = argv
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["e2e"]["h2d_bytes_per_step"] == 0
