"""The benchmark's contract on CPU: the reference arm (the FP64 oracle on the host cores)
prints one JSON line with the keys the contract fixes, alone and under torchrun with two
ranks (rank 0 alone prints); the GPU arm fails loudly when there is no GPU."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run(cmd, timeout=300):
    env = dict(os.environ, PYTHONPATH=ROOT)
    return subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True,
                          timeout=timeout)


def json_lines(out):
    lines = []
    for line in out.splitlines():
        line = line.strip()
        if line.startswith("{"):
            lines.append(json.loads(line))
    return lines


def check_reference_line(d, n_gpus):
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference"
    assert d["metric"] == "MLUPS" and d["unit"] == "MLUPS" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert d["n_gpus"] == n_gpus and d["steps"] == 2 and d["warmup"] == 1
    assert d["config"]["workload"].startswith("ellipse")
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"]
    assert cb["sample"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_arm_prints_one_contract_line():
    r = run([sys.executable, "bench.py", "--impl", "reference", "--steps", "2", "--warmup", "1"])
    assert r.returncode == 0, r.stderr[-2000:]
    lines = json_lines(r.stdout)
    assert len(lines) == 1
    check_reference_line(lines[0], 1)


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_reference_arm_under_torchrun_two_ranks():
    pytest.importorskip("torch")
    r = run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
             "--master-addr", "127.0.0.1", "--master-port", str(free_port()), "bench.py",
             "--impl", "reference", "--gpus", "2", "--steps", "2", "--warmup", "1"])
    assert r.returncode == 0, r.stderr[-2000:]
    lines = json_lines(r.stdout)
    assert len(lines) == 1  # rank 0 alone runs and prints
    check_reference_line(lines[0], 2)


def test_gpu_arm_fails_loudly_without_a_gpu():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    r = run([sys.executable, "bench.py", "--steps", "1", "--warmup", "1"])
    assert r.returncode != 0
    assert json_lines(r.stdout) == []  # no number without the CUDA path


def _ranks_body(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        # the slower rank's time decides; each rank ran its own replica of the lattice
        t = bench.max_over_ranks([10.0 + rank, 3.0 - rank], dist, device="cpu")
        q.put((rank, t, bench.whole_job_mlups(4096, 100, world, t[0] * 1e-3)))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_value_with_two_gloo_ranks():
    """The N > 1 path's host logic with two gloo ranks on CPU: every rank gets the
    slowest rank's time, and the whole-job rate counts every rank's updates over it."""
    pytest.importorskip("torch")
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    ps = [ctx.Process(target=_ranks_body, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = [q.get(timeout=120) for _ in ps]
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, v in out:
        assert t == [11.0, 3.0]
        assert abs(v - 4096 * 100 * 2 / 11e-3 / 1e6) < 1e-9
    assert bench_single_process_is_identity()


def bench_single_process_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    return bench.max_over_ranks([1.5, 2.5], None) == [1.5, 2.5]
