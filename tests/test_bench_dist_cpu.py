"""Multi-rank bench logic on CPU: two gloo ranks (replicas of the encrypted
inference, no data-path exchange) agree on the slowest rank's time and on
the whole-job rate."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", init_method="env://", rank=rank, world_size=world)
    import bench
    w, r, local = bench.dist_setup()
    assert (w, r, local) == (world, rank, rank)
    ms = 1000.0 * (rank + 1)  # rank 1 is the slowest replica
    slowest = bench.max_over_ranks(ms, world, "cpu")
    rate = bench.job_rate(5160 * 7, world, slowest)
    out[rank] = (slowest, rate)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_max_time_and_job_rate():
    world = 2
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, join=True,
                       start_method="spawn")
    assert out[0] == out[1]
    slowest, rate = out[0]
    assert slowest == 2000.0
    assert rate == pytest.approx(5160 * 7 * 2 / 2.0)


def test_traffic_record_is_used_only_for_the_captured_kernel_source(tmp_path, monkeypatch):
    """bench.py reports the ncu DRAM traffic of a blind-rotation launch only
    while the kernel's source file still hashes to the value recorded with
    the capture, and only for the launch size that was captured."""
    import bench
    src = tmp_path / "k.cu"
    src.write_text("kernel v1\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setitem(bench.KERNEL_SOURCE, "tc", "k.cu")
    rec = tmp_path / "traffic.txt"
    monkeypatch.setattr(bench, "TRAFFIC_RECORD", str(rec))
    assert bench.recorded_traffic("tc", 9030.0)[0] is None  # no record
    rec.write_text("# header\narm=tc kernel=k sha16=%s cts_per_launch=9030 bytes_per_launch=123 "
                   "capture=x\n" % bench.source_sha16("k.cu"))
    assert bench.recorded_traffic("tc", 9030.0)[0] == 123.0
    assert bench.recorded_traffic("tc", 4096.0)[0] is None  # another launch size
    src.write_text("kernel v2\n")
    value, why = bench.recorded_traffic("tc", 9030.0)
    assert value is None and "changed" in why


def _run_bench(args, **env):
    import json
    import subprocess
    e = dict(os.environ)
    e.update({k: str(v) for k, v in env.items()})
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + args, cwd=ROOT, env=e,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return [json.loads(x) for x in r.stdout.splitlines() if x.startswith("{")]


def test_reference_arm_prints_one_oracle_line_on_rank_zero_only():
    """bench.py --impl reference times the oracle on the host cores and
    prints one line of the bench contract (its cpu_baseline and e2e describe
    this run); under torchrun the other ranks exit 0 without work."""
    import bench
    lines = _run_bench(["--impl", "reference", "--steps", "1", "--warmup", "0"])
    assert len(lines) == 1
    d = lines[0]
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["value"] > 0 and d["higher_is_better"] is True and d["n_gpus"] == 1
    assert (d["steps"], d["warmup"]) == (1, 0)
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    from paper_2309_09025_gb300 import synth
    assert d["config"]["workload"] == bench.workload_name(dict(synth.P630), 4, 7)
    assert _run_bench(["--impl", "reference", "--steps", "1", "--warmup", "0"],
                      RANK=1, WORLD_SIZE=2, LOCAL_RANK=1) == []
