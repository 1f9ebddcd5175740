"""bench.py's contract on the CPU: the multi-rank job time (max over ranks, gloo, world size 2), the
whole-job value, and the reference arm's single JSON line (the oracle on the host cores)."""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = [12.5, 20.0][rank]
    t = bench.job_time_ms(ms, dist, "cpu")
    q.put((rank, t, bench.job_value(world, 1000, 4, t)))
    dist.barrier()
    dist.destroy_process_group()


def test_job_time_is_the_max_over_ranks_gloo():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # both ranks see the slower rank's time; the value counts both replicas' cells
    assert [t for _, t, _ in out] == [20.0, 20.0]
    assert out[0][2] == pytest.approx(2 * 1000 * 3 * 4 / 20e-3)


def test_single_rank_time_passes_through():
    assert bench.job_time_ms(7.0, None, "cpu") == 7.0
    assert bench.job_value(1, 1024 * 1024, 20, 14.0) == pytest.approx(1024 * 1024 * 60 / 14e-3)


def test_reference_arm_prints_one_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["higher_is_better"] is True and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0


def test_crop_is_the_corner_of_the_workload_and_needs_headline_only():
    W = bench._workloads()["mixed3d-64-r3"]
    C = bench.cropped(W, 16)
    assert C.n == [16, 16, 16] and C.ncell == 16 ** 3 and C.R == W.R and C.gate == W.gate
    assert torch.equal(C.make("cpu"), W.make("cpu")[:, :16, :16, :16])
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--crop", "16"], capture_output=True,
                       text=True, cwd=ROOT)
    assert r.returncode != 0 and "--crop needs --headline-only" in r.stderr
