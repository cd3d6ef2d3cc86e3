"""The multi-replica path of bench.py on CPU: two gloo ranks (127.0.0.1).
bench.py --gpus N runs N independent replicas of the batched workload (the
queries shard with no exchange); the only cross-rank step is the whole-job
reduction of the timed region (slowest rank) and of the work (sum), which
runs here on gloo exactly as it runs on NCCL; and the reference arm runs on
rank 0 alone."""
import os
import socket
import sys

import pytest

ROOT = os.path.abspath(os.path.join(os.path.dirname(__file__), ".."))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        # rank r: its timed region lasted 10 (r + 1) ms and 2 (r + 1) s, it did 100 (r + 1) and 7 units
        slow, tot = bench.reduce_over_ranks([10.0 * (rank + 1), 2.0 * (rank + 1)], [100 * (rank + 1), 7], world, "cpu")
        out.put((rank, slow, tot))
    finally:
        dist.destroy_process_group()


def test_two_ranks_reduce_to_slowest_time_and_total_work():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    got = [out.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, slow, tot in got:
        assert slow == [20.0, 4.0], (rank, slow)
        assert tot == [300.0, 14.0], (rank, tot)


def test_one_rank_keeps_its_values():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_over_ranks([1.5, 2.0], [3, 4], 1, "cpu") == ([1.5, 2.0], [3.0, 4.0])


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("LOCAL_RANK", "1")
    ns = type("A", (), dict(gpus=2, steps=1, warmup=0))()
    bench.run_reference(ns)
    assert capsys.readouterr().out == ""


def test_reference_arm_line_keeps_the_contract(monkeypatch, capsys):
    """Rank 0 of the reference arm prints one JSON line with the contract's
    keys, the oracle as its CPU baseline and the GPU arm's workload config."""
    import json
    sys.path.insert(0, ROOT)
    import bench
    for k, v in (("WORLD_SIZE", "1"), ("RANK", "0"), ("LOCAL_RANK", "0")):
        monkeypatch.setenv(k, v)
    ns = type("A", (), dict(gpus=1, steps=1, warmup=3))()
    bench.run_reference(ns)
    lines = [l for l in capsys.readouterr().out.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
                "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["value"] > 0
    assert d["steps"] == 1 and d["warmup"] == 3 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"] == bench.batch_config_dict(bench.batch_workload())
    assert d["config"]["workload"] == bench.BATCH_WORKLOAD
