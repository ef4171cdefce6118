"""Benchmark: CTM moves/s of the reduced-sequential move at D=8, chi=256, d=2.

One step = one CTM iteration: left, up, right and down moves (two column
absorptions each: reduced network, split isometries, sequential absorption,
normalisation) plus the FP64 convergence check (singular values of the 8
corners).  value = 4 * steps / device time (moves/s, whole job over N GPUs).

Inputs: A, B with i.i.d. N(0,1) entries, unit Frobenius norm (seeds 0, 1),
environment folded and grown to chi on the device before timing.  The working
set (16 environment tensors of up to chi*D*D*chi doubles, ~0.5 GB, plus GB of
intermediates) is larger than the 129 MB L2, so no flush is needed between
steps.

--impl reference times the CPU oracle (plain NumPy/LAPACK FP64) on a bounded
sample of the same workload (one reduced-sequential column absorption at the
same shapes) and scales it to moves/s.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

D_, CHI, PHYS = 8, 256, 2
WORKLOAD = "iPEPS 2-site {A,B} CTM iteration, d=2 D=8 chi=256 chi'=256, reduced-sequential"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="native", choices=["native", "reference"])
    p.add_argument("--precision", default=os.environ.get("CTM_BENCH_PRECISION", "bf16"))
    p.add_argument("--D", type=int, default=D_)
    p.add_argument("--chi", type=int, default=CHI)
    p.add_argument("--no-standard", action="store_true",
                   help="skip timing one FP64 standard move for comparison")
    p.add_argument("--no-cpu-baseline", action="store_true")
    return p.parse_args()


# ---------------------------------------------------------------------------
# distributed helpers (one process per GPU; independent replicas)
# ---------------------------------------------------------------------------
def dist_setup(n, backend="nccl"):
    """(rank, world, dist) for N > 1 under torchrun (one process per GPU), else (0, 1, None).
    The ranks are independent replicas: the process group carries only the barriers around the
    timed region and the max-over-ranks reduction of its duration."""
    import torch
    if n <= 1 or "RANK" not in os.environ:
        return 0, 1, None
    import torch.distributed as dist
    if backend == "nccl":
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    dist.init_process_group(backend)
    return dist.get_rank(), dist.get_world_size(), dist


def barrier(dist):
    if dist is not None:
        dist.barrier()


def max_over_ranks(dist, v):
    if dist is None:
        return v
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], device=dev, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(moves_per_rank, world, seconds_max):
    """Whole-job moves/s: the moves of all ranks over the slowest rank's time (weak scaling)."""
    return moves_per_rank * world / seconds_max


def bench_config(args, world):
    return {"workload": WORKLOAD.replace("D=8", f"D={args.D}").replace("chi=256", f"chi={args.chi}")
                                .replace("chi'=256", f"chi'={args.chi}"),
            "precision": args.precision, "parallelism": f"replicas{world}",
            "l2": "working set > L2 (no flush)"}


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# native arm
# ---------------------------------------------------------------------------
def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def fp64_gemm_peak():
    """cuBLAS DGEMM throughput on this GPU (TFLOP/s), the FP64 ALU denominator."""
    import torch
    n = 4096
    a = torch.randn(n, n, dtype=torch.float64, device="cuda")
    b = torch.randn(n, n, dtype=torch.float64, device="cuda")
    for _ in range(2):
        a @ b
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    best = 1e30
    for _ in range(3):
        e0.record()
        a @ b
        e1.record()
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1) / 1e3)
    return 2.0 * n ** 3 / best / 1e12


def run_native(args):
    import torch

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    # a side stream: the library can then capture steady-state moves in CUDA graphs
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        return _run_native(args)


def _run_native(args):
    import numpy as np
    import torch

    from paper_2306_08212_gb300 import ctm, inputs

    rank, world, dist = dist_setup(args.gpus)
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    ctm.load()
    stream = torch.cuda.current_stream()
    A, B = inputs.random_sites(PHYS, args.D, 0)
    env = ctm.Env(A, B, args.chi, precision=args.precision)
    ctx = env.ctx
    order = (ctm.LEFT, ctm.UP, ctm.RIGHT, ctm.DOWN)

    def step():
        for d in order:
            rc = ctm.ctm_move(ctx, d, ctm.REDUCED_SEQUENTIAL)
            if rc != ctm.OK:
                raise RuntimeError(ctm.ctm_last_error(ctx))
        # convergence check: FP64 singular values of the 8 corners
        rc, _ = ctm.ctm_corner_spectra(ctx, args.chi + 16)
        if rc != ctm.OK:
            raise RuntimeError(ctm.ctm_last_error(ctx))

    for _ in range(args.warmup):
        step()
    # untimed calibration step: every kernel class timed with CUDA events while
    # the context runs on its own stream alone (no side streams, no graphs), so
    # no two of its kernels overlap and each class's summed event time is its
    # own device time; also picks the contraction class with the most device time
    ctm.ctm_kernel_stats_reset(ctx, 0x1F | ctm.PROFILE_SERIAL)
    step()
    ctm.ctm_kernel_stats_reset(ctx, 0x1F | ctm.PROFILE_SERIAL)  # counters cleared
    c0 = torch.cuda.Event(enable_timing=True)
    c1 = torch.cuda.Event(enable_timing=True)
    c0.record(stream)
    step()
    c1.record(stream)
    torch.cuda.synchronize()
    calib_ms = c0.elapsed_time(c1)
    breakdown = ctm.ctm_kernel_stats(ctx)
    gemm_like = [k for k in breakdown if k["flops"] > 0]
    top = max(gemm_like, key=lambda k: k["ms"]) if gemm_like else None
    top_cls = {v: k for k, v in ctm.PROFILE_CLASSES.items()}[top["name"]] if top else None
    # timed region: events only around the launches of that class
    top_mask = (1 << top_cls) if top_cls is not None else 0
    ctm.ctm_kernel_stats_reset(ctx, top_mask)
    step()
    step()
    torch.cuda.synchronize()
    ctm.ctm_kernel_stats_reset(ctx, top_mask)
    launches0 = ctm.ctm_kernel_launches(ctx)
    clocks = Clocks(int(os.environ.get("LOCAL_RANK", "0")))
    barrier(dist)
    torch.cuda.synchronize()
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("ctm_timed")  # lets ncu capture exactly the timed steps
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    barrier(dist)
    clk = clocks.stop()
    t = e0.elapsed_time(e1) / 1e3
    t = max_over_ranks(dist, t)
    launches = ctm.ctm_kernel_launches(ctx) - launches0
    stats = ctm.ctm_kernel_stats(ctx)

    # end to end through the C ABI with host buffers: environment in (pinned
    # host -> device), one iteration, the 8 corner spectra out (device -> host)
    host_env = {}
    for kind in (0, 1):
        for k in range(1, 5):
            for x in (0, 1):
                t_np = env.tensor(kind, k, x)
                host_env[(kind, k, x)] = torch.from_numpy(t_np).pin_memory()
    h2d = sum(v.numel() * 8 for v in host_env.values())
    d2h = 8 * (args.chi + 0) * 8
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for (kind, k, x), v in host_env.items():
            dims = (ctm.ctypes.c_int * 4)(*(list(v.shape) + [0] * (4 - v.dim())))
            rc = ctm.load().ctm_set_tensor(ctx, kind, k, x,
                                           ctm.ctypes.cast(v.data_ptr(), ctm._D), dims)
            assert rc == ctm.OK, ctm.ctm_last_error(ctx)
        step()
    torch.cuda.synchronize()
    t_e2e = max_over_ranks(dist, time.perf_counter() - t0)

    std = None
    if not args.no_standard and rank == 0:
        std = standard_vs_reduced(args, A, B, host_env)

    if rank != 0:
        env.free()
        return None
    peaks, peaks_kind = measured_peaks()
    value = job_throughput(4 * args.steps, world, t)
    roof = roofline(args, stats, peaks, peaks_kind)
    line = {
        "metric": "CTM moves/s at D=8 chi=256: reduced-sequential mixed precision (vs FP64 standard)",
        "value": value,
        "unit": "moves/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": 1e3 * t / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": {"fp64": "f64", "tf32": "tf32/f32acc+f64", "bf16": "bf16/f32acc+f64"}[args.precision],
        "data": "synthetic: A,B ~ N(0,1) unit norm, seeds 0/1",
        "config": bench_config(args, world),
        "e2e": {"value": job_throughput(4 * args.steps, world, t_e2e), "unit": "moves/s",
                "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "kernel_classes": {k["name"]: {"launches": k["count"], "ms_per_step": k["ms"],
                                       "gflop_per_step": k["flops"] / 1e9}
                           for k in breakdown},
        "kernel_classes_method": ("one untimed calibration step on a single stream, eager "
                                  "(no side streams, no graphs): CUDA events around every "
                                  "launch of a class, summed"),
        "calibration_ms_per_step": calib_ms,
        "clocks": clk,
        "roofline": roof,
        "tensor_cores": tensor_core_util(breakdown, 1e3 * t / args.steps, peaks),
    }
    if std is not None:
        line["fp64_standard"] = std["fp64_standard"]
        line["equal_accuracy"] = std["equal_accuracy"]
        line["speedup_vs_fp64_standard"] = value / std["fp64_standard"]["value"]
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args)
    env.free()
    return line


def standard_vs_reduced(args, A, B, host_env, moves=("left", "up", "right")):
    """The FP64 standard move (Sec. II, O(chi^3 D^6)) beside the reduced-sequential move,
    both from the same environment (the bench context's after its timed steps): the
    standard rate from the 2nd and 3rd moves (the 1st is a warm-up), and the mean bond
    energy (Heisenberg S.S) after the same three moves in FP64 standard, FP64
    reduced-sequential and the bench's precision."""
    import numpy as np
    import torch

    from paper_2306_08212_gb300 import ctm
    sx = np.array([[0, 1], [1, 0]]) / 2
    sz = np.diag([0.5, -0.5])
    sy_sy = np.kron(np.array([[0, -1], [1, 0]]), np.array([[0, -1], [1, 0]])) / -4
    H = np.kron(sx, sx) + sy_sy + np.kron(sz, sz)

    def run(prec, mode):
        env = ctm.Env(A, B, args.chi, precision=ctm.PRECISIONS[prec] | ctm.INIT_NO_GROW)
        try:
            for (kind, k, x), v in host_env.items():
                env.set_tensor(kind, k, x, v.numpy())
            times = []
            for d in moves:
                torch.cuda.synchronize()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                env.move(d, mode)
                e1.record()
                torch.cuda.synchronize()
                times.append(e0.elapsed_time(e1) / 1e3)
            energy = float(np.mean([env.expect_bond(b, H) for b in range(4)]))
            return times, energy
        finally:
            env.free()

    t_std, e_std = run("fp64", "standard")
    t_seq64, e_seq64 = run("fp64", "reduced_sequential")
    _, e_seq = run(args.precision, "reduced_sequential")
    timed = t_std[1:]
    return {
        "fp64_standard": {"value": len(timed) / sum(timed), "unit": "moves/s",
                          "moves_timed": len(timed), "warmup_moves": 1,
                          "seconds_per_move": timed, "dtype": "f64"},
        "equal_accuracy": {
            "start": "the bench context's environment after its timed steps",
            "moves": list(moves), "observable": "mean Heisenberg S.S over the 4 bonds",
            "energy_fp64_standard": e_std, "energy_fp64_reduced_sequential": e_seq64,
            f"energy_{args.precision}_reduced_sequential": e_seq,
            "dE_vs_standard": e_seq - e_std,
            "dE_method_fp64": e_seq64 - e_std,
            "dE_precision": e_seq - e_seq64,
            "fp64_reduced_sequential_seconds_per_move": t_seq64},
    }


def tensor_core_util(breakdown, ms_per_step, peaks):
    """Tensor-core contraction classes of one step: their FLOPs over their own device time
    against the measured BF16 peak (TF32: x 1.1/2.25, the nominal ratio), and their share of
    the step's wall time."""
    out = {}
    for k in breakdown:
        if not k["name"].startswith("tc_") or k["ms"] <= 0:
            continue
        peak = peaks["bf16_tflops_sustained"] * (1.0 if "bf16" in k["name"] else 1.1 / 2.25)
        achieved = k["flops"] / (k["ms"] / 1e3) / 1e12
        out[k["name"]] = {"achieved_tflops": achieved, "peak_tflops": peak,
                          "frac": achieved / peak, "ms_per_step": k["ms"],
                          "share_of_step": k["ms"] / ms_per_step}
    return out


# DRAM bytes (read + write) per launch of a kernel class, from one ncu capture of this
# workload, valid only for the kernel source it was taken on: each entry names the source
# file and the first 16 hex digits of its SHA-256 at capture time; when the file has changed
# since, the bench reports traffic null.
# cholqr_f64: a launch of four 2048 x 256 problems (16.78 MB of FP64 inputs) read 16.93 MB
# and wrote 0.29 MB (ncu, D=8 chi=256 step): the inputs once, the outputs still in L2.  The
# step's 34 launches carry 96 such problems (four or two per launch) and 8 of 256 x 256 (the
# corner-spectra bases), 406.6 MB of inputs, so the mean launch moves 406.6 / 34 MB x
# (17.22 / 16.78).
TRAFFIC_PER_LAUNCH = {"cholqr_f64": ("paper_2306_08212_gb300/csrc/cholqr.cu", "fe352bb7bff5faf5",
                                     406.6e6 / 34.0 * 17.22 / 16.78)}


def measured_traffic(name):
    import hashlib
    entry = TRAFFIC_PER_LAUNCH.get(name)
    if entry is None:
        return None
    src, sha, nbytes = entry
    try:
        with open(os.path.join(ROOT, src), "rb") as f:
            if hashlib.sha256(f.read()).hexdigest()[:16] != sha:
                return None
    except OSError:
        return None
    return nbytes


def roofline(args, stats, peaks, peaks_kind):
    if not stats:
        return None
    top = max(stats, key=lambda s: s["ms"])
    if top["count"] == 0 or top["ms"] <= 0:
        return None
    avg_s = top["ms"] / top["count"] / 1e3
    flops_per_launch = top["flops"] / top["count"]
    achieved = flops_per_launch / avg_s / 1e12
    if top["name"].startswith("tc_bf16"):
        peak, bound, note = peaks["bf16_tflops_sustained"], "tensor", f"bf16 sustained ({peaks_kind})"
    elif top["name"].startswith("tc_tf32"):
        peak = peaks["bf16_tflops_sustained"] * (1.1 / 2.25)
        bound, note = "tensor", f"tf32 = bf16 sustained ({peaks_kind}) x 1.1/2.25"
    else:
        peak, bound, note = fp64_gemm_peak(), "alu", "fp64: cuBLAS DGEMM measured here"
    return {"kernel": top["name"], "bound": bound, "achieved": achieved, "peak": peak,
            "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": (measured_traffic(top["name"])
                        if (args.D, args.chi, args.precision) == (D_, CHI, "bf16") else None),
            "launches": top["count"], "avg_launch_us": avg_s * 1e6, "peak_source": note}


# ---------------------------------------------------------------------------
# CPU oracle (cpu_baseline leg and --impl reference)
# ---------------------------------------------------------------------------
def oracle_column_seconds(D, chi):
    """Seconds for one reduced-sequential column absorption of the oracle at (D, chi)."""
    import numpy as np

    from oracle import ctm_oracle as O
    from paper_2306_08212_gb300 import inputs
    A, B = inputs.random_sites(PHYS, D, 0)
    env = inputs.random_env_tensors(D, chi, seed=2)
    sites = {"a": A, "b": B}
    t0 = time.perf_counter()
    O.column_absorb(env, 0, sites, chi, chi, "reduced_sequential")
    return time.perf_counter() - t0


def cpu_baseline(args):
    sec = oracle_column_seconds(args.D, args.chi)
    return {"value": 1.0 / (2.0 * sec), "unit": "moves/s", "cores": os.cpu_count(),
            "kind": "oracle",
            "sample": f"one reduced-sequential column absorption (half a move) at D={args.D} "
                      f"chi={args.chi} on a seeded random environment, x2 per move"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return None
    times = []
    for _ in range(args.warmup):
        oracle_column_seconds(args.D, args.chi)
    for _ in range(args.steps):
        times.append(oracle_column_seconds(args.D, args.chi))
    t = sum(times)
    # one step = 4 moves = 8 column absorptions; the sample times one column each
    value = len(times) / (2.0 * t)
    cb = {"value": value, "unit": "moves/s", "cores": os.cpu_count(), "kind": "oracle",
          "sample": "one reduced-sequential column absorption per step at the bench shapes"}
    return {"impl": "reference",
            "metric": "CTM moves/s at D=8 chi=256: reduced-sequential mixed precision (vs FP64 standard)",
            "value": value, "unit": "moves/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "higher_is_better": True, "dtype": "f64",
            "config": bench_config(args, args.gpus), "cpu_baseline": cb,
            "e2e": {"value": value, "unit": "moves/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    if args.impl == "reference":
        line = run_reference(args)
    else:
        line = run_native(args)
    if line is not None:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
