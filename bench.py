"""Benchmark: particle-steps/s of RBM-1 on one GB300 (and the direct O(N^2)
step beside it) on the Thomson-sphere workload of Sec. 5.1 of
arXiv:1812.10575: N = 100000 points on S^2, K(x) = x/|x|^3, V = 0, sigma = 0,
positions projected back to the sphere after each step, p = 2, dt = 1e-4,
FP32.  Inputs are synthetic (uniform points on the sphere from a seeded
generator).

One timed step = one RBM-1 step: Philox keys, random division, in-batch
forces, Euler update, projection.  The state (1.6 MB) fits in L2, so L2 is
flushed before every timed step (a 256 MiB write, then a 256 MiB read so the
flush's dirty lines are written back before the step starts) and each step
is timed alone with CUDA events on the stream its kernels run on.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank advances its own replica of the workload (replica
index = rank; no data-path collective): weak scaling.  ``--impl reference``
times the CPU oracle on this host's cores instead (rank 0 only).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle-steps/s: RBM vs direct vs surrogate on 1 GB300 at stated W1 error"
UNIT = "particle-steps/s"
WORKLOAD = dict(workload="thomson_sphere_rbm1", n=100000, d=3, p=2, dt=1e-4, sigma=0.0, kernel="coulomb",
                potential="zero", renorm=True, dtype="f32", seed=0)
L2_FLUSH_BYTES = 256 << 20


def _env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


def _kernel_sources_digest() -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1812_10575_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(f.encode() + fh.read())
    return h.hexdigest()[:16]


def _measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, ValueError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            if self.thread is not None:
                self.thread.join(timeout=2)

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def _oracle_rbm_rate(n_particles, seconds, steps=None, warmup=0):
    """Time the CPU oracle's RBM-1 step on the workload (bounded sample)."""
    import oracle
    import workloads

    w = WORKLOAD
    prm = oracle.make_params(n_particles, w["d"], p=w["p"], dt=w["dt"], sigma=w["sigma"], seed=w["seed"],
                             k=w["kernel"], renorm=w["renorm"], precision="f32")
    X = workloads.sphere(n_particles, w["d"], seed=w["seed"]).astype(np.float32).astype(np.float64)
    for m in range(warmup):
        X = oracle.rbm_step(prm, X, m)
    done, t0 = 0, time.perf_counter()
    while True:
        X = oracle.rbm_step(prm, X, warmup + done)
        done += 1
        el = time.perf_counter() - t0
        if (steps is not None and done >= steps) or (steps is None and el >= seconds):
            break
    return n_particles * done / el, done, el, oracle.num_threads()


def run_reference(args):
    rank = _env_int("RANK", 0)
    if rank != 0:
        return 0
    n = WORKLOAD["n"]
    rate, done, el, cores = _oracle_rbm_rate(n, None, steps=args.steps, warmup=args.warmup)
    sample = (f"{done} oracle RBM-1 steps of the full N={n} Thomson workload (FP64 arithmetic, "
              f"FP32-equivalent noise), after {args.warmup} warm-up steps")
    line = {
        "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * el / done, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": dict(WORKLOAD), "impl": "reference",
        "cpu_baseline": {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def _traffic_for(kernel_name: str, digest: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel sources."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        data = json.load(f)
    ent = data.get(WORKLOAD["workload"], {}).get(kernel_name)
    if not ent or ent.get("sources") != digest:
        return None
    return ent.get("dram_bytes_per_launch")


def run_ours(args):
    import torch
    import torch.distributed as dist

    import paper_1812_10575_gb300 as rbm
    import workloads

    world = _env_int("WORLD_SIZE", 1)
    rank = _env_int("RANK", 0)
    local = _env_int("LOCAL_RANK", 0)
    if world > 1:
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = WORKLOAD
    n, d = w["n"], w["d"]
    stream = torch.cuda.current_stream()

    X0 = workloads.sphere(n, d, seed=w["seed"])
    x = torch.zeros(n, 4, dtype=torch.float32, device=dev)
    x[:, :3] = torch.from_numpy(X0).float().to(dev)
    kw = dict(p=w["p"], dt=w["dt"], sigma=w["sigma"], seed=w["seed"], k=w["kernel"], renorm=w["renorm"],
              replica=rank)
    sysm = rbm.System(x, d=d, stream=stream, **kw)
    sysm.set_tuning(graph_steps=1)
    flush_w = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    flush_r = torch.ones(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    sink = torch.empty((), dtype=torch.float32, device=dev)

    class _Flush:
        @staticmethod
        def zero_():
            flush_w.zero_()
            sink.copy_(flush_r.sum())

    flush = _Flush()

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    clocks = ClockSampler(local).__enter__()
    # warm-up: graph capture, caches; then about a second of steps so the
    # clock record covers the GPU under this load
    for _ in range(max(args.warmup, 3)):
        sysm.run(1)
    sysm.sync()
    soak = rbm.System(x.clone(), d=d, stream=stream, **kw)
    t_soak = time.perf_counter()
    while time.perf_counter() - t_soak < 1.0:
        soak.run(100)
        soak.sync()
    soak.close()

    # kernels per replayed one-step graph: the step's kernels, plus the
    # step-counter bump kernel unless the cooperative kernel advances it itself
    launches = sysm.launches_per_step("rbm") + (0 if sysm.tuning()["path"] == 2 else 1)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    barrier()
    if True:
        wall0 = time.perf_counter()
        for k in range(args.steps):
            flush.zero_()
            starts[k].record(stream)
            sysm.run(1)                    # one RBM-1 step (CUDA graph of one step)
            ends[k].record(stream)
        barrier()
        wall = time.perf_counter() - wall0
        step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
        # per-kernel CUDA-event timing of the same step, on the same stream
        per_kernel = {}
        for k in range(args.steps):
            flush.zero_()
            for name, ms in sysm.step_profiled("rbm"):
                per_kernel.setdefault(name, []).append(ms)
        barrier()
    sysm.sync()
    total_ms = float(sum(step_ms))
    if world > 1:
        t = torch.tensor([total_ms], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    value = world * n * args.steps / (total_ms * 1e-3)

    # direct O(N^2) step on the same system (a few steps: ~ms each)
    nd = min(args.steps, 5)
    dstart = [torch.cuda.Event(enable_timing=True) for _ in range(nd)]
    dend = [torch.cuda.Event(enable_timing=True) for _ in range(nd)]
    sysm.direct_step()
    sysm.sync()
    for k in range(nd):
        flush.zero_()
        dstart[k].record(stream)
        sysm.direct_step()
        dend[k].record(stream)
    sysm.sync()
    direct_ms = float(np.mean([s.elapsed_time(e) for s, e in zip(dstart, dend)]))
    direct_rate = n / (direct_ms * 1e-3)
    direct_kernel = {}
    for _ in range(2):
        for name, ms in sysm.step_profiled("direct"):
            direct_kernel.setdefault(name, []).append(ms)

    # end to end through the C ABI with host buffers (H2D + step + D2H each step)
    host = x.detach().cpu().pin_memory()
    sysm.step_host(host)
    e2e_ms = []
    for k in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sysm.step_host(host)
        e2e_ms.append(1e3 * (time.perf_counter() - t0))
    e2e_total = float(sum(e2e_ms))
    if world > 1:
        t = torch.tensor([e2e_total], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_total = float(t.item())
    e2e_value = world * n * args.steps / (e2e_total * 1e-3)
    row_bytes = 16

    # roofline of the dominant kernel
    peaks, peak_src = _measured_peaks()
    avg = {k: float(np.mean(v)) for k, v in per_kernel.items()}
    dom = max(avg, key=avg.get)
    # algorithmic bytes per particle (positions read + written once, one u32
    # permutation entry written and read): the floor any RBM-1 step moves
    step_floor = 2 * row_bytes + 8
    bytes_per_particle = {"k_rbm_coop": step_floor, "k_bucket_sort_step": 4 + 4 + 2 * row_bytes,
                          "k_bucket_scatter": 4, "k_straddle_fixup": 0, "k_bucket_scan": 0}
    alg_bytes = n * bytes_per_particle.get(dom, 0)
    achieved = alg_bytes / (avg[dom] * 1e-3) / 1e9
    digest = _kernel_sources_digest()
    roofline = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"], "traffic": _traffic_for(dom, digest),
                "algorithmic_bytes_per_launch": alg_bytes, "avg_launch_ms": avg[dom],
                "peak_source": f"{peak_src} (hbm_gbs)"}
    # the direct kernel is bound by the FP32 pipe: 17 flop per pair (Coulomb) over N^2 pairs
    fp32_peak = 152 * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    dk = float(np.mean(direct_kernel.get("k_direct", [direct_ms])))
    direct_tflops = 17.0 * n * n / (dk * 1e-3) / 1e12

    clocks.__exit__(None, None, None)
    clk = clocks.summary()
    clk["window"] = "sampled every 200 ms from the warm-up soak through the timed, profiled, direct and e2e phases"
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": dict(WORKLOAD, l2="flushed before every timed step (256 MiB write + 256 MiB read); "
                                    "each step timed alone",
                       parallelism=f"replicas x{world} (one independent system per GPU)"),
        "roofline": roofline,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": n * row_bytes,
                "d2h_bytes_per_step": n * row_bytes},
        "gpu_launches": launches * args.steps,
        "clocks": clk,
        "methods": {"rbm": value / world, "direct": direct_rate, "rbm_over_direct": (value / world) / direct_rate,
                    "direct_ms_per_step": direct_ms,
                    "direct_kernel": {"bound": "alu", "achieved": direct_tflops, "peak": fp32_peak,
                                      "unit": "TFLOP/s", "frac": direct_tflops / fp32_peak,
                                      "flop_per_pair": 17, "peak_source": "152 SMs x 128 FP32 lanes x 2 x max clock"}},
        "kernels_ms": avg,
        "wall_s_timed_region": wall,
        "kernel_sources": digest,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, done, el, cores = _oracle_rbm_rate(n, args.cpu_seconds)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": f"{done} oracle RBM-1 steps of the full N={n} workload in {el:.1f} s"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    sysm.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
