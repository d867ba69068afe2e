"""The multi-rank benchmark path on the CPU: world size 2 over gloo.

The path is "replicas only": every rank runs the whole workload, the step time
is the slowest rank's, and the value is the ranks' total work over it. The
reference arm under torchrun prints from rank 0 only."""
import importlib.util
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
torch = pytest.importorskip("torch")


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, world: int, port: int, out_dir: str):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    bench = _bench()
    ms = 100.0 + 25.0 * rank  # rank 1 is the slower replica
    slowest = bench.max_over_ranks(ms, dist, device="cpu")
    rate = bench.replica_rate(1000.0, world, slowest / 1e3)
    dist.barrier()
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump({"slowest": slowest, "rate": rate}, f)
    dist.destroy_process_group()


def test_replica_timing_takes_the_slowest_rank(tmp_path):
    port = _free_port()
    torch.multiprocessing.spawn(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    got = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(2)]
    for g in got:
        assert g["slowest"] == 125.0
        assert g["rate"] == pytest.approx(2 * 1000.0 / 0.125)


def test_single_process_figures_pass_through():
    bench = _bench()
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.replica_rate(10.0, 1, 2.0) == 5.0


def test_reference_arm_under_torchrun_prints_once():
    port = _free_port()
    out = subprocess.run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
                          "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
                          "--impl", "reference", "--gpus", "2", "--scale", "10", "--steps", "1", "--warmup", "0"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
