"""The multi-GPU host logic of bench.py on CPU ranks (gloo, world size 2).

With N GPUs every rank computes its own product each step (replicas: the path has no exchange
step), the step takes the slowest rank's time (max over ranks), and the whole-job value is
that time divided by N products.  The reference arm prints on rank 0 only.
"""
import argparse
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    local = 1.0 + 0.5 * rank                     # rank 1 is the slower one
    m = bench.max_over_ranks(local, dist, "cpu")
    q.put((rank, m, bench.job_value(m, world)))
    dist.barrier()
    dist.destroy_process_group()


def test_step_time_is_max_over_ranks_and_value_is_per_product():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=180) for _ in range(2))
    for p in procs:
        p.join(timeout=120)
    assert [p.exitcode for p in procs] == [0, 0]
    assert res == [(0, 1.5, 0.75), (1, 1.5, 0.75)]


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(2.25) == 2.25 and bench.job_value(2.25, 1) == 2.25


def test_reference_arm_prints_on_rank_zero_only(capsys):
    import bench
    bench.run_reference(argparse.Namespace(gpus=2, steps=1, warmup=0), rank=1)
    assert capsys.readouterr().out == ""


def test_reference_arm_line_keeps_the_contract(capsys):
    """Rank 0 of the reference arm prints one JSON line: the oracle timed on the host cores on
    a bounded sample, with the metric, unit and config of the device arm."""
    import json
    import bench
    bench.run_reference(argparse.Namespace(gpus=1, steps=1, warmup=0), rank=0)
    lines = [ln for ln in capsys.readouterr().out.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == "ms"
    assert d["higher_is_better"] is False and d["n_gpus"] == 1 and d["steps"] == 1
    assert d["config"]["workload"] == bench.WORKLOAD and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1 and d["cpu_baseline"]["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
