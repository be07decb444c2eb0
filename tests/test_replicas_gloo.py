"""The N > 1 path of bench.py on the CPU: independent replicas, one per rank,
with no data-path collective; the only exchange is the maximum of the ranks'
timed regions (world_size 2, gloo, 127.0.0.1)."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, seconds, out_dir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    rate, t = bench.job_rate(seconds[rank], 1000, world, device="cpu")
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
        json.dump({"rate": rate, "t": t}, f)


def test_job_rate_takes_the_slowest_rank(tmp_path):
    mp = pytest.importorskip("torch.multiprocessing")
    seconds = [1.0, 2.5]
    mp.spawn(_rank_main, args=(2, _free_port(), seconds, str(tmp_path)), nprocs=2, join=True)
    for r in range(2):
        d = json.load(open(tmp_path / f"r{r}.json"))
        assert d["t"] == 2.5
        assert abs(d["rate"] - 2 * 1000 / 2.5) < 1e-9


def test_job_rate_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    rate, t = bench.job_rate(0.5, 100, 1)
    assert t == 0.5 and rate == 200.0


def test_reference_arm_under_torchrun_prints_once():
    """`bench.py --impl reference` launched as the driver launches N > 1:
    rank 0 alone times the oracle and prints one JSON line; the other rank
    exits 0 without work."""
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), "bench.py",
           "--impl", "reference", "--gpus", "2", "--steps", "2", "--warmup", "0", "--workload", "bubble160x80"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    # the line's contract: the metric and unit of the main line, the oracle
    # described as the CPU baseline, and an end-to-end figure with no copies
    sys.path.insert(0, ROOT)
    import bench
    assert d["metric"] == bench.METRIC and d["unit"] == bench.UNIT and d["higher_is_better"] is True
    assert d["steps"] == 2 and d["warmup"] == 0 and d["config"]["workload"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
