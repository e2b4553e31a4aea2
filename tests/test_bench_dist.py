"""The multi-rank logic of bench.py (max-over-ranks timing, whole-job aggregation,
rank-0-only reference leg) on world_size-2 gloo process groups.  CPU only."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    d = bench.init_dist(world, "gloo")
    local_ms = 100.0 * (rank + 1)          # rank 1 is the slow one
    m = bench.max_over_ranks(d, local_ms)
    v = bench.aggregate_value(1024 * 1024, world, 5, m)
    bench.barrier(d)
    q.put((rank, m, v))
    d.destroy_process_group()


def test_max_over_ranks_and_aggregate_gloo():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, m, v in res:
        assert m == 200.0                                  # max over ranks
        assert v == pytest.approx(1024 * 1024 * 2 * 5 / 0.2)  # all ranks' units / max time


def test_reference_leg_nonzero_rank_exits_clean(capsys):
    import bench
    os.environ["RANK"] = "1"
    try:
        assert bench.run_reference(bench.argparse.Namespace(steps=1, warmup=3), 2, 1) == 0
    finally:
        os.environ.pop("RANK")
    assert capsys.readouterr().out == ""
