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


def test_reference_line_contract(capsys, monkeypatch):
    """The reference arm's JSON line: the oracle as the baseline program, the bench's
    metric, unit and direction, and an e2e object with no device copies."""
    import json

    import bench
    monkeypatch.setattr(bench, "oracle_sample", lambda p, target_s=15.0: (2300.0, 32, 14.0, 16))
    assert bench.run_reference(bench.argparse.Namespace(steps=2, warmup=3), 1, 0) == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC
    assert line["unit"] == bench.UNIT and line["higher_is_better"] is True
    assert line["value"] == 2300.0 and line["steps"] == 2 and line["warmup"] == 3
    assert line["vs_baseline"] is None and line["dtype"] == "f64" and line["n_gpus"] == 1
    assert line["config"]["workload"] == bench.WORKLOAD
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == line["value"] and cb["cores"] == 16
    assert "columns" in cb["sample"]
    assert line["e2e"] == {"value": 2300.0, "unit": bench.UNIT, "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}


def test_oracle_sample_runs_bounded():
    """The oracle timing leg on a short budget: whole columns of the n = 1024 planted
    matrix, a positive rate, the cores it used."""
    import bench
    from paper_2002_04989_gb300 import inputs
    v, cols, dt, cores = bench.oracle_sample(inputs.planted1024(), target_s=0.3)
    assert v > 0 and 1 <= cols <= 1023 and dt > 0 and cores >= 1
    assert abs(v - 1024 * cols / dt) <= 1e-6 * v
