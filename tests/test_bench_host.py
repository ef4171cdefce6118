"""Host-side logic of bench.py on CPU: the replica path over a world-size-2 gloo
group (barrier, max-over-ranks duration, whole-job throughput) and the oracle arm
(rank 0 prints one JSON line, the other ranks exit without work)."""
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


def _replica(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    r, w, dist = bench.dist_setup(world, backend="gloo")
    bench.barrier(dist)
    t = bench.max_over_ranks(dist, 1.0 + 0.5 * r)  # rank 1 is the slower replica
    bench.barrier(dist)
    q.put((r, w, t, bench.job_throughput(12, w, t)))
    dist.destroy_process_group()


def test_replicas_take_max_time_and_sum_moves():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_replica, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[0] for o in out] == [0, 1]
    for r, w, t, v in out:
        assert w == 2
        assert t == 1.5            # every rank sees the slowest rank's time
        assert v == 12 * 2 / 1.5   # moves of both replicas over that time


def test_single_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.dist_setup(1) == (0, 1, None)
    assert bench.max_over_ranks(None, 3.0) == 3.0


def _run_reference(rank):
    env = dict(os.environ, RANK=str(rank), WORLD_SIZE="2", OMP_NUM_THREADS="2")
    return subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1",
                           "--warmup", "0", "--D", "2", "--chi", "8"], cwd=ROOT, env=env,
                          capture_output=True, text=True, timeout=300)


def test_reference_arm_rank0_prints_one_line():
    p = _run_reference(0)
    assert p.returncode == 0, p.stderr
    lines = [l for l in p.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference"
    assert line["unit"] == "moves/s" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle"
    assert line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": "moves/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    assert "D=2" in line["config"]["workload"] and "chi=8" in line["config"]["workload"]


def test_reference_arm_other_ranks_exit_without_output():
    p = _run_reference(1)
    assert p.returncode == 0, p.stderr
    assert p.stdout.strip() == ""


def test_tensor_core_utilisation_from_a_step_breakdown():
    sys.path.insert(0, ROOT)
    import bench
    breakdown = [{"name": "gemm_f64", "count": 10, "ms": 300.0, "flops": 1.2e11},
                 {"name": "tc_tf32_gemm", "count": 0, "ms": 0.0, "flops": 0.0},
                 {"name": "tc_bf16_gemm", "count": 528, "ms": 60.0, "flops": 4.5e12},
                 {"name": "jacobi_f64", "count": 1, "ms": 48.0, "flops": 0.0}]
    peaks = {"bf16_tflops_sustained": 1720.6}
    u = bench.tensor_core_util(breakdown, 308.0, peaks)
    assert list(u) == ["tc_bf16_gemm"]
    assert u["tc_bf16_gemm"]["achieved_tflops"] == pytest.approx(75.0)
    assert u["tc_bf16_gemm"]["frac"] == pytest.approx(75.0 / 1720.6)
    assert u["tc_bf16_gemm"]["share_of_step"] == pytest.approx(60.0 / 308.0)
    tf = bench.tensor_core_util([{"name": "tc_tf32_gemm", "count": 1, "ms": 1.0, "flops": 1e9}],
                                10.0, peaks)
    assert tf["tc_tf32_gemm"]["peak_tflops"] == pytest.approx(1720.6 * 1.1 / 2.25)
