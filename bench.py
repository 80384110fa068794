"""Benchmark: particle-steps/s of RBM-1 on one GB300, with the direct O(N^2)
step beside it, on synthetic workloads shaped like the paper's
(arXiv:1812.10575) examples.  Default workload (the headline line): the
large-N system -- N = 2^26 particles in d = 3, V(x) = |x|^2/2, regularised
attraction K(x) = -x/(|x|^2 + 0.01), sigma = 0.2, X0 ~ N(0, I), p = 2,
dt = 1e-3, FP32 -- the regime where the direct method is out of reach
(Sec. 4.1, closing remarks; cost model of Sec. 2.1: O(pN) against O(N^2)).

One timed step = one RBM-1 step: Philox keys, random division, in-batch
forces, -grad V, Brownian increment, Euler-Maruyama update.  The state (1 GB
of positions) is larger than L2, so steps run back to back: K steps replayed
from one CUDA graph, timed with CUDA events on the stream the kernels run on.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload large_n|thomson|batched_opinion|dyson|large_n_sweep|surrogate|w1_sweep]
                    [--sizes 20,22 (large_n_sweep)] [--no-cpu-baseline]

Other workloads (one JSON line each, same keys):
  thomson         - the Thomson problem of Sec. 5.1: N = 100000 points on S^2,
                    K(x) = x/|x|^3, V = 0, sigma = 0, projection after each
                    step, p = 2, dt = 1e-4, FP32; the state (1.6 MB) fits in
                    L2, so L2 is flushed before every timed step and each step
                    is timed alone: latency-bound;
  batched_opinion - 4096 independent 2-D bounded-confidence opinion systems
                    (Sec. 5.2), N_r log-uniform in [256, 65536], sigma = 0.01,
                    dt = 1e-2, p = 2, one launch per step replayed from a
                    100-step CUDA graph; inputs (384 MB) exceed L2;
  dyson           - Dyson Brownian motion (Sec. 4.2), N = 1000, FP64,
                    splitting scheme, p = 2, dt = 1e-3;
  large_n_sweep   - the large-N system at N = 2^16 .. 2^26, p in {2, 4, 8},
                    RBM-1, RBM-r (up to 2^22, p = 2) and direct (up to 2^20);
  surrogate       - the learned mean-field surrogate, N = 2^22, d = 2,
                    Gaussian aggregation with confinement from a 4-cluster
                    mixture, sigma = 0.1, dt = 1e-3: whole 100-step cycles
                    (checkpoint training + 100 network steps), the network
                    step alone, RBM-1 and direct at the same N, and the
                    accuracy of each at N = 2^16 against the direct method;
  w1_sweep        - equal-accuracy comparison at N = 2^16: sliced W1 to a
                    direct reference at dt/16 for RBM-1, direct and the
                    surrogate at dt * {1, 1/2, 1/4, ...}, and the time to T
                    at W1 <= 1e-2 for each method.
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
L2_FLUSH_BYTES = 256 << 20

WORKLOADS = {
    "large_n": dict(workload="large_n_reg_attract", n=2**26, d=3, p=2, dt=1e-3, sigma=0.2, kernel="reg_attract",
                    potential="quadratic", v_coef=1.0, k_param=0.01, renorm=False, dtype="f32", seed=0,
                    scheme="euler", other_p=[4, 8], direct_n=2**20, cpu_sample_n=2**20,
                    surrogate=dict(train_every=100, fallback_tol=1e-2, n_queries=16384, iters_first=4000,
                                   iters_per_checkpoint=1000, max_rounds=4, lr=3e-3)),
    "thomson": dict(workload="thomson_sphere_rbm1", n=100000, d=3, p=2, dt=1e-4, sigma=0.0, kernel="coulomb",
                    potential="zero", v_coef=1.0, k_param=0.0, renorm=True, dtype="f32", seed=0, scheme="euler",
                    quality_steps=2000),
    "batched_opinion": dict(workload="batched_opinion_replicas", replicas=4096, n_lo=256, n_hi=65536, d=2, p=2,
                            dt=1e-2, sigma=0.01, kernel="bounded_conf", potential="zero", v_coef=1.0, k_param=0.25,
                            renorm=False, dtype="f32", seed=0, scheme="euler", graph_steps=100, ps=[2, 4],
                            eps=1e-2, horizon=1.0),
    "dyson": dict(workload="dyson_brownian_motion", n=1000, d=1, p=2, dt=1e-3, sigma=float(np.sqrt(1.0 / 1000)),
                  kernel="inv1d", potential="quadratic", v_coef=1.0, k_param=0.0, renorm=False, dtype="f64", seed=0,
                  scheme="split"),
    "large_n_sweep": dict(workload="large_n_reg_attract", d=3, dt=1e-3, sigma=0.2, kernel="reg_attract",
                          potential="quadratic", v_coef=1.0, k_param=0.01, renorm=False, dtype="f32", seed=0,
                          scheme="euler", sizes=[2**16, 2**18, 2**20, 2**22, 2**24, 2**26], ps=[2, 4, 8],
                          direct_max=2**20, rbmr_max=2**22),
    "surrogate": dict(workload="surrogate_mixture_aggregation", n=2**22, d=2, p=2, dt=1e-3, sigma=0.1,
                      kernel="gauss_agg", potential="quadratic", v_coef=1.0, k_param=0.0, renorm=False, dtype="f32",
                      seed=0, scheme="euler", train_every=100, n_queries=16384, iters_first=12000,
                      iters_per_checkpoint=2000, max_rounds=8, lr=3e-3, fallback_tol=1e-2, accuracy_n=2**16,
                      accuracy_steps=300),
    "w1_sweep": dict(workload="equal_accuracy_sweep", n=2**16, T=0.25, fine_steps=4096, eps=[1e-1, 3e-2, 1e-2, 3e-3],
                     rbm_refines=[512, 256, 128, 64, 32, 16, 8], ps=[2, 4, 8], direct_refines=[512, 256, 128, 64, 32],
                     surrogate_refines=[128, 64, 32], slices=16, seed=0, dtype="f32"),
}

# The two systems of the equal-W1 sweep (N = 2^16 for accuracy): the large-N
# workload (d = 3, regularised attraction) and the surrogate workload (d = 2,
# Gaussian aggregation from the 4-cluster mixture).
W1_SYSTEMS = {
    "large_n_reg_attract": dict(d=3, sigma=0.2, kernel="reg_attract", potential="quadratic", v_coef=1.0, k_param=0.01,
                                init="gaussian", surrogate=False),
    "surrogate_mixture_aggregation": dict(d=2, sigma=0.1, kernel="gauss_agg", potential="quadratic", v_coef=1.0,
                                          k_param=0.0, init="mixture", surrogate=True),
}


def _env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


# The source files each timed kernel is built from: a profile's counters stay
# valid while these files are unchanged.
KERNEL_SOURCES = {
    "k_rbm_coop": ["coop_step.cu", "rbm_grid.cuh", "rbm_batch.cuh", "rbm_device.cuh", "rbm_internal.h"],
    "k_rbm_batched": ["batched.cu", "rbm_batch.cuh", "rbm_device.cuh", "rbm_internal.h"],
    "k_sur_step": ["surrogate.cu", "tc.cuh", "rbm_device.cuh", "rbm_internal.h"],
    "k_bucket_sort_step": ["perm_step.cu", "rbm_batch.cuh", "rbm_device.cuh", "rbm_internal.h"],
    "k_rec_step": ["rec_step.cu", "rbm_batch.cuh", "rbm_device.cuh", "rbm_internal.h"],
    "k_direct": ["direct.cu", "rbm_device.cuh", "rbm_internal.h"],
    "k_rbmr_step": ["rbmr.cu", "rbm_grid.cuh", "rbm_device.cuh", "rbm_internal.h"],
}


def _kernel_sources_digest(kernel: str = "") -> str:
    """Digest of the kernel sources: of the files `kernel` is built from, or of
    every file when no kernel is named."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1812_10575_gb300", "csrc")
    files = KERNEL_SOURCES.get(kernel) or sorted(os.listdir(csrc))
    for f in sorted(files):
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

    def start(self):
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

    def stop(self):
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
        out = {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
               "reasons": sorted(reasons), "samples": len(sm),
               "window": "sampled every 200 ms from the warm-up soak through the timed, profiled, direct and e2e "
                         "phases"}
        return out


def _oprm(w, n, replica=0, precision=None):
    import oracle

    return oracle.make_params(n, w["d"], p=w["p"], dt=w["dt"], sigma=w["sigma"], seed=w["seed"], v=w["potential"],
                              v_coef=w["v_coef"], k=w["kernel"], k_param=w["k_param"], renorm=w["renorm"],
                              precision=precision or w["dtype"], replica=replica)


def _initial(w, n, seed=None):
    import workloads

    seed = w["seed"] if seed is None else seed
    if w["workload"].startswith("thomson"):
        return workloads.sphere(n, w["d"], seed=seed)
    if w["workload"].startswith("dyson"):
        return workloads.dyson(n, seed)
    if w["workload"].startswith("batched"):
        return workloads.unit_cube(n, w["d"], seed=seed)
    if w["workload"].startswith("surrogate"):
        return workloads.mixture(n, w["d"], seed=seed)
    return workloads.gaussian(n, w["d"], seed=seed)


def _oracle_step_fn(w):
    import oracle

    return oracle.rbm_split_step if w["scheme"] == "split" else oracle.rbm_step


def _oracle_rate(w, seconds=None, steps=None, warmup=0):
    """Time the CPU oracle's RBM-1 step on (a bounded sample of) the workload.
    Returns (particle-steps/s, steps done, seconds, threads, sample text)."""
    import oracle

    step = _oracle_step_fn(w)
    if w["workload"].startswith("batched"):
        import workloads

        sizes = workloads.replica_sizes(w["replicas"], w["n_lo"], w["n_hi"], seed=w["seed"])
        pick = list(range(0, len(sizes), max(1, len(sizes) // 16)))[:16]
        sample = f"replicas {pick[0]}..{pick[-1]} (16 of {len(sizes)}, {int(sum(sizes[pick]))} particles)"
        systems = [(_oprm(w, int(sizes[r]), replica=r), _initial(w, int(sizes[r]), seed=r)) for r in pick]
    else:
        n = w.get("cpu_sample_n", w["n"])
        if n == w["n"]:
            sample = f"the full N={n} system"
        else:
            sample = (f"a sample of the N={w['n']} system: its first {n} particles (rows 0..{n - 1} of the same "
                      f"X0 draw) stepped as a system of {n}")
        X = _initial(w, w["n"])[:n] if n != w["n"] else _initial(w, n)
        if w["dtype"] == "f32":
            X = X.astype(np.float32).astype(np.float64)
        systems = [(_oprm(w, n), X)]
    for m in range(warmup):
        systems = [(prm, step(prm, X, m)) for prm, X in systems]
    done, parts, t0 = 0, 0, time.perf_counter()
    while True:
        systems = [(prm, step(prm, X, warmup + done)) for prm, X in systems]
        parts += sum(prm.n for prm, _ in systems)
        done += 1
        el = time.perf_counter() - t0
        if (steps is not None and done >= steps) or (steps is None and el >= seconds):
            break
    return parts / el, done, el, oracle.num_threads(), sample


def run_reference(args, w):
    rank = _env_int("RANK", 0)
    if rank != 0:
        return 0
    rate, done, el, cores, sample = _oracle_rate(w, steps=args.steps, warmup=args.warmup)
    sample = f"{done} oracle RBM-1 steps of {sample} (FP64 arithmetic), after {args.warmup} warm-up steps"
    line = {
        "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * el / done, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": dict(w), "impl": "reference",
        "cpu_baseline": {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def _traffic_for(workload: str, kernel_name: str, digest: str, n=None):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current sources of that kernel (`digest`, of all sources, is kept
    for the line's record).  A capture taken at a smaller size `n` (the
    full-size launch is too large for a multi-pass capture) is scaled to the
    line's particles: the kernel's traffic grows in proportion to N."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        data = json.load(f)
    ent = data.get(workload, {}).get(kernel_name)
    if not ent or ent.get("sources") != _kernel_sources_digest(kernel_name):
        return None
    b = ent.get("dram_bytes_per_launch")
    if b is not None and n is not None and ent.get("n"):
        b = b * n / ent["n"]
    return b


def _issue_rate(workload: str, kernel_name: str, avg_ms: float, n, sm_mhz: float, num_sms: int = 152):
    """The kernel's instruction issue against the SMs' issue rate (four warp
    schedulers per SM, one warp instruction per scheduler and clock), from the
    warp instructions of the committed ncu capture (scaled by N like the
    traffic) and the launch's measured time; None without a capture taken on
    the current sources."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path) or avg_ms <= 0:
        return None
    with open(path) as f:
        ent = json.load(f).get(workload, {}).get(kernel_name)
    if not ent or ent.get("sources") != _kernel_sources_digest(kernel_name) or not ent.get("warp_inst_per_launch"):
        return None
    inst = ent["warp_inst_per_launch"] * (n / ent["n"] if n is not None and ent.get("n") else 1.0)
    achieved = inst / (avg_ms * 1e-3)
    peak = 4.0 * num_sms * sm_mhz * 1e6
    return {"warp_instructions_per_launch": inst, "achieved": achieved, "peak": peak,
            "unit": "warp instructions/s", "frac": achieved / peak,
            "peak_source": f"{num_sms} SMs x 4 schedulers x 1 warp instruction per clock x {sm_mhz:.0f} MHz "
                           "(median SM clock under load)"}


def max_over_ranks(dist, v, device):
    """The largest of every rank's v (the job's time is its slowest rank's)."""
    import torch

    t = torch.tensor([float(v)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_value(world, n_per_rank, steps, total_ms):
    """Whole-job particle-steps/s: every rank advances its own replica of N
    particles (no data-path collective), the job takes the slowest rank's time."""
    return world * n_per_rank * steps / (total_ms * 1e-3)


class Gpu:
    """Per-rank GPU context: device, stream, L2 flush, barrier."""

    def __init__(self):
        import torch
        import torch.distributed as dist

        self.torch, self.dist = torch, dist
        self.world = _env_int("WORLD_SIZE", 1)
        self.rank = _env_int("RANK", 0)
        self.local = _env_int("LOCAL_RANK", 0)
        if self.world > 1:
            os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
            dist.init_process_group("nccl")
        torch.cuda.set_device(self.local)
        self.dev = torch.device("cuda", self.local)
        self.stream = torch.cuda.current_stream()
        self.flush_w = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=self.dev)
        self.flush_r = torch.ones(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=self.dev)
        self.sink = torch.empty((), dtype=torch.float32, device=self.dev)

    def flush(self):
        self.flush_w.zero_()
        self.sink.copy_(self.flush_r.sum())

    def barrier(self):
        if self.world > 1:
            self.dist.barrier()
        self.torch.cuda.synchronize()

    def max_over_ranks(self, v):
        if self.world == 1:
            return v
        return max_over_ranks(self.dist, v, self.dev)

    def event(self):
        return self.torch.cuda.Event(enable_timing=True)

    def close(self):
        if self.world > 1:
            self.dist.destroy_process_group()


def _to_dev(g, X, d, dtype):
    torch = g.torch
    ld = 4 if d == 3 else d
    t = torch.zeros(X.shape[0], ld, dtype=torch.float64)
    t[:, :d] = torch.from_numpy(np.asarray(X, dtype=np.float64))
    return t.to(torch.float32 if dtype == "f32" else torch.float64).to(g.dev).contiguous()


def _run_shares(avg, steps):
    """Each kernel's share of a K-step run, from its per-launch time in the
    profiled step: the record path's scatter, last step and placement run
    once per run,
    its inner step and fix-up K - 1 times, every other kernel once per step."""
    reps = {}
    for k in avg:
        if k in ("k_rec_scatter", "k_rec_place") or k.endswith("_last"):
            reps[k] = 1
        elif k in ("k_rec_step", "k_rec_fixup"):
            reps[k] = max(steps - 1, 0)
        else:
            reps[k] = steps
    tot = sum(avg[k] * reps[k] for k in avg)
    return {k: avg[k] * reps[k] / tot for k in avg} if tot > 0 else {}


def _roofline(peaks, peak_src, kernel, alg_bytes, avg_ms, workload, digest, n=None):
    achieved = alg_bytes / (avg_ms * 1e-3) / 1e9 if avg_ms > 0 else 0.0
    return {"bound": "hbm", "kernel": kernel, "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": achieved / peaks["hbm_gbs"], "traffic": _traffic_for(workload, kernel, digest, n),
            "algorithmic_bytes_per_launch": alg_bytes, "avg_launch_ms": avg_ms,
            "peak_source": f"{peak_src} (hbm_gbs)"}


def _timed_run(g, sysm, steps, method="rbm"):
    """Milliseconds of `steps` steps replayed from the system's CUDA graph of
    `steps` steps (captured by an earlier call), CUDA events on the stream."""
    e0, e1 = g.event(), g.event()
    g.barrier()
    e0.record(g.stream)
    sysm.run(steps, method)
    e1.record(g.stream)
    g.barrier()
    return e0.elapsed_time(e1)


# Algorithmic work per unit, as the scope table counts it: bytes per
# particle-step of RBM-1 (positions read and written once at d words of the
# run's precision, one u32 permutation entry written and read) and flops per
# pair of the direct sum.
def rbm_floor_bytes(d, elem):
    return 2 * d * elem + 8


DIRECT_FLOP_PER_PAIR = {
    "coulomb": 19,       # 3 sub, 3 FMA (|x|^2), rsqrt, 2 mul, 3 FMA; FMA = 2
    "reg_attract": 16,   # 3 sub, 3 FMA (|x|^2), add, rcp (special-function unit, not counted), 3 FMA
    "inv1d": 6, "gauss_agg": 18, "smooth_test": 17, "bounded_conf": 16, "linear": 11,
}


_FMA_PEAK = {}


def _fma_peak():
    """Measured FP32 FMA throughput (TFLOP/s), scalar and packed two-lane,
    once per process (rbm_fp32_fma_peak)."""
    if not _FMA_PEAK:
        import paper_1812_10575_gb300 as rbm
        _FMA_PEAK.update(scalar=rbm.rbm_fp32_fma_peak(False), packed=rbm.rbm_fp32_fma_peak(True))
    return _FMA_PEAK


def _direct_kernel_roof(peaks, kernel, n, ms, dtype):
    flop = DIRECT_FLOP_PER_PAIR[kernel]
    derived = (152 * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12) / (1 if dtype == "f32" else 64)
    tf = flop * n * n / (ms * 1e-3) / 1e12
    if dtype == "f32":
        fma = _fma_peak()
        peak = max(fma["scalar"], fma["packed"])
        return {"bound": "alu", "achieved": tf, "peak": peak, "unit": "TFLOP/s", "frac": tf / peak,
                "flop_per_pair": flop,
                "peak_source": "measured: FP32 FMA loop (rbm_fp32_fma_peak), the better of scalar "
                               f"({fma['scalar']:.1f}) and packed two-lane ({fma['packed']:.1f}) FMA",
                "peak_derived": derived, "frac_of_derived": tf / derived,
                "derived_source": "152 SMs x 128 FP32 lanes x 2 x max SM clock"}
    return {"bound": "alu", "achieved": tf, "peak": derived, "unit": "TFLOP/s", "frac": tf / derived,
            "flop_per_pair": flop,
            "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x max SM clock / 64 (FP64)"}


def run_headline(args, w, g):
    """The large-N system at N = 2^26: RBM-1 steps replayed from a CUDA graph
    of K steps (the state exceeds L2: no flush needed), p = 4 and 8 at the
    same N, and the direct step with RBM-1 beside it at N = 2^20."""
    import paper_1812_10575_gb300 as rbm

    n, d = w["n"], w["d"]
    elem = 4
    X0 = _initial(w, n)
    kw = dict(dt=w["dt"], sigma=w["sigma"], seed=w["seed"], v=w["potential"], v_coef=w["v_coef"], k=w["kernel"],
              k_param=w["k_param"], renorm=w["renorm"], scheme=w["scheme"], replica=g.rank)
    steps = max(args.steps, 1)
    x = _to_dev(g, X0, d, w["dtype"])
    sysm = rbm.System(x, d=d, p=w["p"], stream=g.stream, **kw)
    sysm.set_tuning(graph_steps=steps)
    clocks = ClockSampler(g.local).start()
    sysm.run(max(args.warmup, 3) % steps)      # eager warm-up steps
    sysm.run(steps)                            # captures the K-step graph and replays it once
    sysm.sync()
    t_soak = time.perf_counter()
    while time.perf_counter() - t_soak < args.soak_seconds:
        sysm.run(steps)
        sysm.sync()
    launches = sysm.launches_per_step("rbm")
    wall0 = time.perf_counter()
    total_ms = g.max_over_ranks(_timed_run(g, sysm, steps))
    wall = time.perf_counter() - wall0
    value = weak_value(g.world, n, steps, total_ms)
    per_kernel = {}
    for _ in range(3):                         # one step, kernel by kernel, same stream
        for name, ms in sysm.step_profiled("rbm"):
            per_kernel.setdefault(name, []).append(ms)
    path = sysm.tuning()["path"]

    # end to end through the C ABI with host buffers (H2D + step + D2H)
    host = x.detach().cpu().pin_memory()
    sysm.step_host(host)
    n_e2e = min(steps, 10)
    g.torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(n_e2e):
        sysm.step_host(host)
    e2e_s = g.max_over_ranks(time.perf_counter() - t0)
    sysm.close()
    del host

    # p = 4 and 8 on the same system (the error scales as sqrt(dt/(p-1)), Sec. 3)
    others = {}
    for p in w["other_p"]:
        x.copy_(_to_dev(g, X0, d, w["dtype"]))
        s = rbm.System(x, d=d, p=p, stream=g.stream, **kw)
        s.set_tuning(graph_steps=steps)
        s.run(steps)
        s.sync()
        ms = _timed_run(g, s, steps)
        others[f"rbm_p{p}"] = {"particle_steps_per_s": n * steps / (ms * 1e-3), "ms_per_step": ms / steps}
        s.close()

    # the learned surrogate (3 -> 64 -> 64 -> 3 network) on the same system:
    # the first checkpoint (queries, direct forces at them, training), then
    # network steps while it is within its tolerance
    x.copy_(_to_dev(g, X0, d, w["dtype"]))
    s = rbm.System(x, d=d, p=w["p"], stream=g.stream, **kw)
    s.surrogate_config(**w["surrogate"])
    e0, e1 = g.event(), g.event()
    e0.record(g.stream)
    s.run(1, "surrogate")
    e1.record(g.stream)
    s.sync()
    first_ms = e0.elapsed_time(e1)
    sur_steps = min(steps, w["surrogate"]["train_every"] - 1)
    e0.record(g.stream)
    s.run(sur_steps, "surrogate")
    e1.record(g.stream)
    s.sync()
    sur_ms = e0.elapsed_time(e1) / sur_steps
    # a whole cycle: the next train_every steps, which hold one later checkpoint
    # (queries, direct forces at them, the drift check, retraining)
    every = w["surrogate"]["train_every"]
    e0.record(g.stream)
    s.run(every, "surrogate")
    e1.record(g.stream)
    s.sync()
    cycle_ms = e0.elapsed_time(e1)
    others["surrogate"] = {"particle_steps_per_s": n / (sur_ms * 1e-3), "ms_per_step": sur_ms,
                           "first_checkpoint_ms": first_ms, "steps_timed": sur_steps,
                           "cycle": {"steps": every, "ms": cycle_ms,
                                     "particle_steps_per_s": n * every / (cycle_ms * 1e-3)},
                           "stats": s.surrogate_stats(), "drift": s.surrogate_drift(),
                           "note": "network steps between checkpoints; `cycle` times train_every steps "
                                   "holding one later checkpoint (direct forces at the queries, drift check, "
                                   "retraining)"}
    s.close()
    del x
    g.torch.cuda.empty_cache()

    # the direct step (and RBM-1) on the first 2^20 particles
    nd = w["direct_n"]
    xd = _to_dev(g, X0[:nd], d, w["dtype"])
    sd = rbm.System(xd, d=d, p=w["p"], stream=g.stream, **kw)
    sd.direct_step()
    sd.sync()
    e0, e1 = g.event(), g.event()
    e0.record(g.stream)
    sd.direct_step()
    e1.record(g.stream)
    sd.sync()
    direct_ms = e0.elapsed_time(e1)
    direct_kernel = {}
    for name, ms in sd.step_profiled("direct"):
        direct_kernel.setdefault(name, []).append(ms)
    sd.set_tuning(graph_steps=steps)
    sd.run(steps)
    sd.sync()
    rbm_small_ms = _timed_run(g, sd, steps) / steps
    sd.close()
    clocks.stop()

    peaks, peak_src = _measured_peaks()
    avg = {k: float(np.mean(v)) for k, v in per_kernel.items()}
    # the record path's k_rec_step runs every step of a run but the last (which
    # runs k_rec_step_last): the steady-state kernel is the one to hold to the roofline
    dom = "k_rec_step" if "k_rec_step" in avg else max(avg, key=avg.get)
    digest = _kernel_sources_digest()
    floor = rbm_floor_bytes(d, elem)
    roof = _roofline(peaks, peak_src, dom, n * floor, avg[dom], w["workload"], digest, n)
    roof["bytes_per_particle_step"] = floor
    roof["bytes_note"] = ("2 x 12 B of positions (d = 3 FP32; the stored row is 16 B with its pad lane) + 4 B "
                          "permutation written + 4 B read")
    roof["step_frac"] = n * floor / (total_ms / steps * 1e-3) / 1e9 / peaks["hbm_gbs"]
    roof["kernel_shares"] = _run_shares(avg, steps)
    clk = clocks.summary()
    sms = g.torch.cuda.get_device_properties(g.torch.cuda.current_device()).multi_processor_count
    issue = _issue_rate(w["workload"], dom, avg[dom], n, clk.get("sm_mhz") or clk.get("sm_max_mhz") or 2070.0, sms)
    if issue is not None:
        roof["issue"] = issue
    dk = float(np.sum([np.mean(v) for v in direct_kernel.values()])) if direct_kernel else direct_ms
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": g.world, "steps": steps,
        "warmup": args.warmup, "ms_per_step": total_ms / steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": w["dtype"], "data": "synthetic",
        "config": dict(w, l2=f"inputs larger than L2 ({n * 16 / 1e9:.2f} GB of positions); K steps replayed back "
                             "to back from one CUDA graph",
                       parallelism=f"replicas x{g.world} (one independent system per GPU)", path=path),
        "roofline": roof,
        "e2e": {"value": g.world * n * n_e2e / e2e_s, "unit": UNIT, "h2d_bytes_per_step": n * 16,
                "d2h_bytes_per_step": n * 16, "steps": n_e2e},
        # per step the pipelined kernels; per graph replay the run's first
        # bucketing (the record path's scatter), the record path's placement
        # after the last step, and the step-counter bump
        "gpu_launches": launches * steps + (3 if path == 4 else 2),
        "clocks": clocks.summary(),
        "methods": dict(
            others, rbm_p2={"particle_steps_per_s": value / g.world, "ms_per_step": total_ms / steps},
            direct_at_n_direct={"n": nd, "particle_steps_per_s": nd / (direct_ms * 1e-3), "ms_per_step": direct_ms,
                                "kernel": _direct_kernel_roof(peaks, w["kernel"], nd, dk, w["dtype"])},
            rbm_at_n_direct={"n": nd, "particle_steps_per_s": nd / (rbm_small_ms * 1e-3),
                             "ms_per_step": rbm_small_ms},
            rbm_over_direct_at_n_direct=direct_ms / rbm_small_ms),
        "kernels_ms": avg, "direct_kernels_ms": {k: float(np.mean(v)) for k, v in direct_kernel.items()},
        "wall_s_timed_region": wall, "kernel_sources": digest,
    }
    return line


def run_single(args, w, g):
    """One system (thomson, dyson): each step timed alone after an L2 flush."""
    import paper_1812_10575_gb300 as rbm

    n, d = w["n"], w["d"]
    row_bytes = (4 if d == 3 else d) * (4 if w["dtype"] == "f32" else 8)
    x = _to_dev(g, _initial(w, n), d, w["dtype"])
    kw = dict(p=w["p"], dt=w["dt"], sigma=w["sigma"], seed=w["seed"], v=w["potential"], v_coef=w["v_coef"],
              k=w["kernel"], k_param=w["k_param"], renorm=w["renorm"], scheme=w["scheme"], replica=g.rank)
    sysm = rbm.System(x, d=d, stream=g.stream, **kw)
    clocks = ClockSampler(g.local).start()
    for _ in range(max(args.warmup, 3)):
        sysm.step()
    sysm.sync()
    soak = rbm.System(x.clone(), d=d, stream=g.stream, **kw)
    t_soak = time.perf_counter()
    while time.perf_counter() - t_soak < args.soak_seconds:
        soak.run(100)
        soak.sync()
    soak.close()

    # kernels per step (rbm_step; the bucketing of each step was done by the
    # step before it)
    launches = sysm.launches_per_step("rbm")
    starts = [g.event() for _ in range(args.steps)]
    ends = [g.event() for _ in range(args.steps)]
    g.barrier()
    wall0 = time.perf_counter()
    for k in range(args.steps):
        g.flush()
        starts[k].record(g.stream)
        sysm.step()                              # one RBM-1 step (rbm_step)
        ends[k].record(g.stream)
    g.barrier()
    wall = time.perf_counter() - wall0
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    per_kernel = {}
    for k in range(args.steps):                  # the same step, kernel by kernel, same stream
        g.flush()
        for name, ms in sysm.step_profiled("rbm"):
            per_kernel.setdefault(name, []).append(ms)
    g.barrier()
    total_ms = g.max_over_ranks(float(sum(step_ms)))
    value = weak_value(g.world, n, args.steps, total_ms)

    # direct O(N^2) step on the same system
    nd = min(args.steps, 5)
    sysm.direct_step()
    sysm.sync()
    dstart = [g.event() for _ in range(nd)]
    dend = [g.event() for _ in range(nd)]
    for k in range(nd):
        g.flush()
        dstart[k].record(g.stream)
        sysm.direct_step()
        dend[k].record(g.stream)
    sysm.sync()
    direct_ms = float(np.mean([s.elapsed_time(e) for s, e in zip(dstart, dend)]))
    direct_kernel = {}
    for _ in range(2):
        for name, ms in sysm.step_profiled("direct"):
            direct_kernel.setdefault(name, []).append(ms)

    # end to end through the C ABI with host buffers (H2D + step + D2H)
    host = x.detach().cpu().pin_memory()
    sysm.step_host(host)
    e2e_ms = []
    for k in range(args.steps):
        g.flush()
        g.torch.cuda.synchronize()
        t0 = time.perf_counter()
        sysm.step_host(host)
        e2e_ms.append(1e3 * (time.perf_counter() - t0))
    e2e_total = g.max_over_ranks(float(sum(e2e_ms)))
    clocks.stop()

    peaks, peak_src = _measured_peaks()
    avg = {k: float(np.mean(v)) for k, v in per_kernel.items()}
    dom = max(avg, key=avg.get)
    # algorithmic bytes per particle-step: positions read and written once,
    # one u32 permutation entry written and read
    floor = rbm_floor_bytes(d, 4 if w["dtype"] == "f32" else 8)
    digest = _kernel_sources_digest()
    roof = _roofline(peaks, peak_src, dom, n * floor, avg[dom], w["workload"], digest)
    roof["bytes_per_particle_step"] = floor
    dk = float(np.sum([np.mean(v) for v in direct_kernel.values()])) if direct_kernel else direct_ms
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": g.world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": w["dtype"], "data": "synthetic",
        "config": dict(w, l2="flushed before every timed step (256 MiB write + 256 MiB read); each step timed alone",
                       parallelism=f"replicas x{g.world} (one independent system per GPU)"),
        "roofline": roof,
        "e2e": {"value": g.world * n * args.steps / (e2e_total * 1e-3), "unit": UNIT,
                "h2d_bytes_per_step": n * row_bytes, "d2h_bytes_per_step": n * row_bytes},
        "gpu_launches": launches * args.steps,
        "clocks": clocks.summary(),
        "methods": {"rbm": value / g.world, "direct": n / (direct_ms * 1e-3),
                    "rbm_over_direct": (value / g.world) / (n / (direct_ms * 1e-3)), "direct_ms_per_step": direct_ms,
                    "direct_kernel": _direct_kernel_roof(peaks, w["kernel"], n, dk, w["dtype"])},
        "kernels_ms": avg, "direct_kernels_ms": {k: float(np.mean(v)) for k, v in direct_kernel.items()},
        "wall_s_timed_region": wall, "kernel_sources": digest,
    }
    if sysm.tuning()["path"] == 2:
        # the cooperative launch shape with no work (a step waits at no grid barrier)
        floor_us = sysm.latency_floor()
        kern_us = 1e3 * avg.get("k_rbm_coop", 0.0)
        line["latency_floor"] = {"floor_us": floor_us, "kernel_us": kern_us,
                                 "frac": floor_us / kern_us if kern_us > 0 else None,
                                 "what": "same cooperative launch (grid, block, shared memory) with no work (the "
                                         "step waits at no grid barrier); frac = floor / step kernel"}
        # the state is L2-resident: the step is bound by latency, not HBM
        line["roofline"] = dict(roof, bound="latency", latency_floor_frac=line["latency_floor"]["frac"],
                                note="state fits in L2; frac against HBM shown for reference only")
    sysm.close()
    if w.get("quality_steps"):
        line["quality"] = _thomson_quality(g, w, kw)
    return line


def _coulomb_energy(torch, X, chunk=512):
    """E = sum_{i<j} 1/|x_i - x_j| on the GPU with torch (a diagnostic of the
    run, not part of the timed path)."""
    e = torch.zeros((), dtype=torch.float64, device=X.device)
    for a in range(0, X.shape[0], chunk):
        dist = torch.cdist(X[a:a + chunk].double(), X.double())
        idx = torch.arange(a, min(a + chunk, X.shape[0]), device=X.device)
        dist[idx - a, idx] = float("inf")
        e += (1.0 / dist).sum()
    return float(e) / 2.0


def _sliced_w1_uniform(X, k=16, seed=0):
    """Mean over k random directions of W1 between the projections X v and
    U[-1, 1], the law of the projection of a uniform point of S^2 onto any
    axis (Archimedes): mean |y_(k) - q_k| with the uniform quantiles q_k."""
    rng = np.random.default_rng(seed)
    dirs = rng.standard_normal((k, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    n = X.shape[0]
    q = -1.0 + 2.0 * (np.arange(n) + 0.5) / n
    return float(np.mean([np.mean(np.abs(np.sort(X @ v) - q)) for v in dirs]))


def _thomson_quality(g, w, kw):
    """The Thomson run's own figures of merit after `quality_steps` steps of
    RBM-1 and of the direct method from the same X0: the Coulomb energy and
    the sliced W1 of the points to the uniform law on the sphere."""
    import paper_1812_10575_gb300 as rbm

    torch, n, d = g.torch, w["n"], w["d"]
    X0 = _initial(w, n)
    out = {"steps": w["quality_steps"], "T": w["quality_steps"] * w["dt"]}
    x0 = _to_dev(g, X0, d, w["dtype"])
    out["energy_x0"] = _coulomb_energy(torch, x0[:, :3])
    out["sliced_w1_uniform_x0"] = _sliced_w1_uniform(x0[:, :3].double().cpu().numpy())
    for method in ("rbm", "direct"):
        x = _to_dev(g, X0, d, w["dtype"])
        s = rbm.System(x, d=d, stream=g.stream, **kw)
        e0, e1 = g.event(), g.event()
        e0.record(g.stream)
        s.run(w["quality_steps"], method)
        e1.record(g.stream)
        s.sync()
        out[method] = {"energy": _coulomb_energy(torch, x[:, :3]),
                       "sliced_w1_uniform": _sliced_w1_uniform(x[:, :3].double().cpu().numpy()),
                       "seconds": e0.elapsed_time(e1) / 1e3}
        s.close()
    return out


def run_batched(args, w, g):
    """Batched replicas: K steps replayed from 100-step CUDA graphs; inputs exceed L2."""
    import paper_1812_10575_gb300 as rbm
    import workloads

    sizes = [int(v) for v in workloads.replica_sizes(w["replicas"], w["n_lo"], w["n_hi"], seed=w["seed"])]
    rows, d = sum(sizes), w["d"]
    row_bytes = d * 4
    x = _to_dev(g, _initial(w, rows), d, w["dtype"])
    kw = dict(p=w["p"], dt=w["dt"], sigma=w["sigma"], seed=w["seed"] + 1000 * g.rank, v=w["potential"],
              v_coef=w["v_coef"], k=w["kernel"], k_param=w["k_param"])
    rep = rbm.Replicas(x, sizes, d=d, stream=g.stream, **kw)
    # p by accuracy: least time to T with E(T) <= eps against the direct
    # method on one Brownian path (pilot: the replica closest to 16384)
    acc = rep.autotune_accuracy(w["ps"], w["eps"], w["horizon"], max_halvings=2, pilot_n=16384, trial_steps=2)
    tune = rep.autotune(trial_steps=2, table_path=None)
    steps = max(args.steps, 1)
    rep.set_graph_steps(min(w["graph_steps"], steps))
    clocks = ClockSampler(g.local).start()
    rep.run(max(args.warmup, 3))
    rep.sync()
    t_soak = time.perf_counter()
    while time.perf_counter() - t_soak < args.soak_seconds:
        rep.run(min(w["graph_steps"], steps))
        rep.sync()
    e0, e1 = g.event(), g.event()
    g.barrier()
    wall0 = time.perf_counter()
    e0.record(g.stream)
    rep.run(steps)
    e1.record(g.stream)
    g.barrier()
    wall = time.perf_counter() - wall0
    total_ms = g.max_over_ranks(e0.elapsed_time(e1))
    value = g.world * rows * steps / (total_ms * 1e-3)
    prof = {}
    for _ in range(3):
        for name, ms in rep.step_profiled():
            prof.setdefault(name, []).append(ms)
    clocks.stop()
    host = x.detach().cpu().pin_memory()
    n_e2e = 3
    t0 = time.perf_counter()
    for _ in range(n_e2e):
        rbm.rbm_step_host(rep.ctx, host)
    e2e_s = g.max_over_ranks(time.perf_counter() - t0)
    peaks, peak_src = _measured_peaks()
    avg = {k: float(np.mean(v)) for k, v in prof.items()}
    digest = _kernel_sources_digest()
    roof = _roofline(peaks, peak_src, "k_rbm_batched", rows * (2 * row_bytes + 8), total_ms / steps,
                     w["workload"], digest)
    roof["avg_launch_ms_profiled"] = avg.get("k_rbm_batched")
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": g.world, "steps": steps, "warmup": args.warmup,
        "ms_per_step": total_ms / steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": w["dtype"], "data": "synthetic",
        "replica_size_histogram": {f"[2^{k}, 2^{k + 1})": int(np.sum((np.array(sizes) >= 2 ** k) &
                                                                     (np.array(sizes) < 2 ** (k + 1))))
                                   for k in range(8, 17)},
        "config": dict(w, rows=rows, l2=f"inputs ({rows * row_bytes / 1e6:.0f} MB of positions) exceed L2; "
                                        "K steps replayed back to back from CUDA graphs",
                       parallelism=f"replicas x{g.world}", autotune=tune, p_by_accuracy=acc),
        "roofline": roof,
        "e2e": {"value": g.world * rows * n_e2e / e2e_s, "unit": UNIT, "h2d_bytes_per_step": rows * row_bytes,
                "d2h_bytes_per_step": rows * row_bytes},
        "gpu_launches": steps + (steps + min(w["graph_steps"], steps) - 1) // min(w["graph_steps"], steps),
        "clocks": clocks.summary(), "kernels_ms": avg, "wall_s_timed_region": wall, "kernel_sources": digest,
    }
    rep.close()
    return line


def run_large_n(args, w, g):
    """Throughput sweep over N and p (RBM) and N (direct up to 2^20)."""
    import paper_1812_10575_gb300 as rbm

    rows = []
    sizes = [1 << int(v) for v in args.sizes.split(",")] if args.sizes else w["sizes"]
    for n in sizes:
        X = _initial(w, n)
        for p in w["ps"]:
            x = _to_dev(g, X, w["d"], w["dtype"])
            s = rbm.System(x, d=w["d"], p=p, dt=w["dt"], sigma=w["sigma"], seed=w["seed"], v=w["potential"],
                           v_coef=w["v_coef"], k=w["kernel"], k_param=w["k_param"], stream=g.stream)
            s.set_tuning(graph_steps=100)        # the library's default graph length
            s.run(100)
            s.sync()
            e0, e1 = g.event(), g.event()
            e0.record(g.stream)
            s.run(100)
            e1.record(g.stream)
            s.sync()
            ms = e0.elapsed_time(e1) / 100
            ent = {"n": n, "p": p, "method": "rbm", "path": s.tuning()["path"], "ms_per_step": ms,
                   "particle_steps_per_s": n / (ms * 1e-3),
                   "hbm_frac_of_floor": n * rbm_floor_bytes(w["d"], 4) / (ms * 1e-3) / 1e9 / _measured_peaks()[0]["hbm_gbs"]}
            if p == w["ps"][0] and n <= w.get("rbmr_max", 0):
                # RBM-r: a step = floor(N/p) iterations in conflict-free rounds
                s.run(1, "rbmr")
                s.sync()
                e0.record(g.stream)
                s.run(5, "rbmr")
                e1.record(g.stream)
                s.sync()
                rms = e0.elapsed_time(e1) / 5
                ent["rbmr_ms_per_step"] = rms
                ent["rbmr_particle_steps_per_s"] = n / (rms * 1e-3)
                ent["rbmr_rounds_per_step"] = s.rbmr_info()["rounds_last"]
            if p == w["ps"][0] and n <= w["direct_max"]:
                s.direct_step()
                s.sync()
                e0.record(g.stream)
                s.direct_step()
                e1.record(g.stream)
                s.sync()
                dms = e0.elapsed_time(e1)
                ent["direct_ms_per_step"] = dms
                ent["direct_particle_steps_per_s"] = n / (dms * 1e-3)
            rows.append(ent)
            s.close()
    best = max(r["particle_steps_per_s"] for r in rows)
    return {"metric": METRIC, "value": best, "unit": UNIT, "n_gpus": g.world, "steps": 100, "warmup": 100,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": w["dtype"],
            "data": "synthetic", "config": dict(w, l2="state larger than L2 from N = 2^23"), "sweep": rows}


def _w1_marginals(A, B):
    """Wasserstein-1 distance of each coordinate's empirical distribution
    (equal sample sizes: the mean absolute difference of the sorted values)."""
    return [float(np.mean(np.abs(np.sort(A[:, k]) - np.sort(B[:, k])))) for k in range(A.shape[1])]


def run_surrogate(args, w, g):
    """The learned mean-field surrogate on the 4-cluster aggregation workload:
    whole 100-step cycles (checkpoint: queries, direct forces at them, Adam
    rounds until the held-out error is within tolerance; then 100 network
    steps replayed from a graph), the network step alone, RBM-1 and one direct
    step at the same N, and the accuracy of each method at N = 2^16 against
    the direct method with the same Brownian increments."""
    import paper_1812_10575_gb300 as rbm

    n, d = w["n"], w["d"]
    kw = dict(p=w["p"], dt=w["dt"], sigma=w["sigma"], seed=w["seed"], v=w["potential"], v_coef=w["v_coef"],
              k=w["kernel"], k_param=w["k_param"], replica=g.rank)
    cfg = dict(train_every=w["train_every"], fallback_tol=w["fallback_tol"], n_queries=w["n_queries"],
               iters_first=w["iters_first"], iters_per_checkpoint=w["iters_per_checkpoint"],
               max_rounds=w["max_rounds"], lr=w["lr"])
    every = w["train_every"]
    X0 = _initial(w, n)
    x = _to_dev(g, X0, d, "f32")
    sysm = rbm.System(x, d=d, stream=g.stream, **kw)
    sysm.surrogate_config(**cfg)
    clocks = ClockSampler(g.local).start()
    e0, e1 = g.event(), g.event()
    e0.record(g.stream)
    sysm.run(every, "surrogate")                 # first checkpoint (training from scratch) + one cycle
    e1.record(g.stream)
    sysm.sync()
    first_cycle_ms = e0.elapsed_time(e1)
    st0 = sysm.surrogate_stats()
    cycles = max(2, -(-args.steps // every))
    starts = [g.event() for _ in range(cycles)]
    ends = [g.event() for _ in range(cycles)]
    g.barrier()
    wall0 = time.perf_counter()
    for k in range(cycles):
        starts[k].record(g.stream)
        sysm.run(every, "surrogate")             # checkpoint + `every` steps
        ends[k].record(g.stream)
    g.barrier()
    wall = time.perf_counter() - wall0
    cyc_ms = [a.elapsed_time(b) for a, b in zip(starts, ends)]
    st1 = sysm.surrogate_stats()
    total_ms = g.max_over_ranks(float(sum(cyc_ms)))
    value = g.world * n * every * cycles / (total_ms * 1e-3)

    # the network step alone, kernel by kernel (inputs 32 MiB: L2 flushed
    # first), with the trained network forced active: the drift schedule may
    # have handed the last interval to the RBM-1 fallback, whose gated
    # network step does no work
    theta, norm = sysm.surrogate_params()
    sysm.surrogate_config(**dict(cfg, fallback_tol=1e30, iters_first=0, iters_per_checkpoint=0))
    sysm.surrogate_set_params(theta, norm)
    sysm.run(1, "surrogate")                     # a checkpoint without training: the network takes the steps
    sysm.sync()
    profiled_active = bool(sysm.surrogate_stats()["active"])
    per_kernel = {}
    for _ in range(max(args.warmup, 3) + 5):
        g.flush()
        for name, ms in sysm.step_profiled("surrogate"):
            per_kernel.setdefault(name, []).append(ms)
    avg = {k: float(np.mean(v[3:])) for k, v in per_kernel.items()}
    step_ms = float(sum(avg.values()))
    # the same step through the C ABI with host buffers
    host = x.detach().cpu().pin_memory()
    sysm.step_host(host, "surrogate")
    e2e_ms = []
    for _ in range(5):
        g.torch.cuda.synchronize()
        t0 = time.perf_counter()
        sysm.step_host(host, "surrogate")
        e2e_ms.append(1e3 * (time.perf_counter() - t0))
    e2e_total = g.max_over_ranks(float(np.mean(e2e_ms)))
    launches = sysm.launches_per_step("surrogate")
    sysm.close()

    # RBM-1 and one direct step at the same N
    xr = _to_dev(g, X0, d, "f32")
    rb = rbm.System(xr, d=d, stream=g.stream, **kw)
    rb.run(every)
    rb.sync()
    e0.record(g.stream)
    rb.run(every)
    e1.record(g.stream)
    rb.sync()
    rbm_ms = e0.elapsed_time(e1) / every
    e0.record(g.stream)
    rb.direct_step()
    e1.record(g.stream)
    rb.sync()
    direct_ms = e0.elapsed_time(e1)
    rb.close()
    clocks.stop()

    # accuracy at N = 2^16 after `accuracy_steps` steps, same X0 and increments
    na, steps = w["accuracy_n"], w["accuracy_steps"]
    Xa = _initial(w, na)
    # the surrogate as configured (retrained every train_every steps) and
    # retrained every 25 steps in rounds of 1000 Adam iterations
    variants = {"rbm": None, "surrogate": cfg,
                "surrogate_every25": dict(cfg, train_every=25, iters_per_checkpoint=1000)}
    out, stats, secs = {}, {}, {}
    for method in ("direct",) + tuple(variants):
        xa = _to_dev(g, Xa, d, "f32")
        sa = rbm.System(xa, d=d, stream=g.stream, **kw)
        if variants.get(method):
            sa.surrogate_config(**variants[method])
        g.torch.cuda.synchronize()
        t0 = time.perf_counter()
        sa.run(steps, "surrogate" if variants.get(method) else method)
        sa.sync()
        secs[method] = time.perf_counter() - t0
        out[method] = xa[:, :d].double().cpu().numpy()
        if variants.get(method):
            stats[method] = sa.surrogate_stats()
        sa.close()
    acc = {"direct": {"wall_s": secs["direct"]}}
    for method in variants:
        diff = out[method] - out["direct"]
        acc[method] = {"E_T": float(np.sqrt(np.mean(np.sum(diff ** 2, axis=1)))),
                       "w1_marginals_vs_direct": _w1_marginals(out[method], out["direct"]),
                       "wall_s": secs[method]}
        if method in stats:
            acc[method]["stats"] = stats[method]

    # launches in the timed cycles: the network step and the gated RBM-1
    # kernels per step; per checkpoint the query sample and the direct sum
    # (2); per round 2 per Adam iteration, the step-count bump, the network
    # forces at the queries and the error check
    adam = st1["adam_steps"] - st0["adam_steps"]
    rounds = adam // max(1, w["iters_per_checkpoint"])
    gpu_launches = cycles * (every * launches + 3) + 2 * adam + 3 * rounds
    peaks, peak_src = _measured_peaks()
    dom = "k_sur_step"
    # special-function unit: 2 operations per tanh (exponential, reciprocal),
    # 128 tanh per particle, plus 4 for the Gaussian pair (log, sqrt, sin, cos)
    mufu_per_particle = 2 * 128 + 4
    mufu_peak = 152 * 16 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    achieved = mufu_per_particle * n / (avg[dom] * 1e-3) / 1e12
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": g.world, "steps": every * cycles,
        "warmup": every, "ms_per_step": total_ms / (every * cycles), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 (bf16 tensor-core operands)", "data": "synthetic",
        "config": dict(w, l2="state 32 MiB: L2 not flushed inside a cycle (a cycle is one graph); "
                             "flushed before each profiled network step",
                       parallelism=f"replicas x{g.world} (one independent system per GPU)"),
        "roofline": {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": mufu_peak,
                     "unit": "T special-function ops/s", "frac": achieved / mufu_peak,
                     "traffic": _traffic_for(w["workload"], dom, _kernel_sources_digest()),
                     "ops_per_particle": mufu_per_particle, "avg_launch_ms": avg[dom],
                     "peak_source": "152 SMs x 16 special-function results per clock x max SM clock"},
        "e2e": {"value": g.world * n / (e2e_total * 1e-3), "unit": UNIT, "h2d_bytes_per_step": n * 8,
                "d2h_bytes_per_step": n * 8, "note": "one network step through rbm_step_host"},
        "gpu_launches": gpu_launches,
        "clocks": clocks.summary(),
        "methods": {"surrogate_cycle": value / g.world, "surrogate_step_only": n / (step_ms * 1e-3),
                    "rbm": n / (rbm_ms * 1e-3), "direct": n / (direct_ms * 1e-3),
                    "surrogate_step_ms": step_ms, "rbm_ms_per_step": rbm_ms, "direct_ms_per_step": direct_ms,
                    "cycle_ms": cyc_ms, "first_cycle_ms": first_cycle_ms,
                    "adam_steps_per_cycle": adam / cycles,
                    "stats_after": st1, "profiled_network_active": profiled_active},
        "accuracy": dict(acc, n=na, steps=steps),
        "kernels_ms": avg, "launches_per_network_step": launches,
        "wall_s_timed_region": wall, "kernel_sources": _kernel_sources_digest(),
    }
    return line


def _sliced_w1(A, B, k, seed=0):
    """Mean over k random unit directions (and the coordinate axes) of the
    1-D Wasserstein-1 distance of the projected samples (equal sizes)."""
    rng = np.random.default_rng(seed)
    dirs = rng.standard_normal((k, A.shape[1]))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    dirs = np.concatenate([np.eye(A.shape[1]), dirs])
    return float(np.mean([np.mean(np.abs(np.sort(A @ v) - np.sort(B @ v))) for v in dirs]))


def _rms_gap(A, B):
    """E(T) of eq. "errorformula": the root mean square over particles of the
    distance between two runs of the same particles."""
    return float(np.sqrt(np.mean(np.sum((A - B) ** 2, axis=1))))


def run_w1_sweep(args, w, g):
    """Equal-accuracy comparison on one Brownian path.  For each system: a
    direct reference with the fine step dt_f = T / fine_steps, then RBM-1
    (p = 2, 4, 8), the direct method and the surrogate at dt = r dt_f with
    noise refinement r, so every run is driven by the reference's Brownian
    increments (the synchronous coupling of Sec. 3, eq. "coupling"; the
    fine-step direct reference of Sec. 4.1).  For each run: E(T) (eq.
    "errorformula") and the sliced W1 of the final empirical distribution to
    the reference's, the time to T (CUDA events over the run's eager steps)
    and particle-steps/s; for each method and tolerance eps the least time to
    T of a run with E(T) <= eps."""
    import paper_1812_10575_gb300 as rbm
    import workloads

    n, T, nf = w["n"], w["T"], w["fine_steps"]
    dt_f = T / nf
    out = {}
    clocks = ClockSampler(g.local).start()
    for name, sy in W1_SYSTEMS.items():
        d = sy["d"]
        X0 = workloads.gaussian(n, d, seed=w["seed"]) if sy["init"] == "gaussian" else \
            workloads.mixture(n, d, seed=w["seed"])

        def final(method, r, p=2):
            x = _to_dev(g, X0, d, "f32")
            s = rbm.System(x, d=d, p=p, dt=dt_f * r, sigma=sy["sigma"], seed=w["seed"], v=sy["potential"],
                           v_coef=sy["v_coef"], k=sy["kernel"], k_param=sy["k_param"], stream=g.stream)
            s.set_tuning(graph_steps=1 << 30)    # eager steps: no graph capture inside the timed run
            s.set_noise_refinement(r)
            if method == "surrogate":
                s.surrogate_config(train_every=25, fallback_tol=1e-2, n_queries=16384, iters_first=12000,
                                   iters_per_checkpoint=1000, max_rounds=8, lr=3e-3)
            steps = nf // r
            e0, e1 = g.event(), g.event()
            g.torch.cuda.synchronize()
            e0.record(g.stream)
            s.run(steps, method)
            e1.record(g.stream)
            s.sync()
            ms = e0.elapsed_time(e1)
            st = s.surrogate_stats() if method == "surrogate" else None
            X = x[:, :d].double().cpu().numpy()
            s.close()
            return X, ms, steps, st

        Xref, ref_ms, ref_steps, _ = final("direct", 1)
        runs = {f"rbm_p{p}": ("rbm", w["rbm_refines"], p) for p in w["ps"]}
        runs["direct"] = ("direct", w["direct_refines"], 2)
        if sy["surrogate"]:
            runs["surrogate"] = ("surrogate", w["surrogate_refines"], 2)
        res = {"T": T, "dt_fine": dt_f,
               "reference": {"method": "direct", "dt": dt_f, "steps": ref_steps, "seconds": ref_ms / 1e3}}
        for label, (method, refines, p) in runs.items():
            curve = []
            for r in refines:
                X, ms, steps, st = final(method, r, p)
                ent = {"dt": dt_f * r, "refine": r, "steps": steps, "E_T": _rms_gap(X, Xref),
                       "sliced_w1": _sliced_w1(X, Xref, w["slices"]), "seconds_to_T": ms / 1e3,
                       "particle_steps_per_s": n * steps / (ms * 1e-3)}
                if st:
                    ent["surrogate_steps"], ent["fallback_steps"] = st["surrogate_steps"], st["fallback_steps"]
                curve.append(ent)
            at_eps = {}
            for eps in w["eps"]:
                ok = [c for c in curve if c["E_T"] <= eps]
                best = min(ok, key=lambda c: c["seconds_to_T"]) if ok else None
                at_eps[f"{eps:g}"] = ({"seconds_to_T": best["seconds_to_T"], "dt": best["dt"],
                                       "particle_steps_per_s": best["particle_steps_per_s"]} if best else None)
            res[label] = {"curve": curve, "at_eps": at_eps}
        speedup = {}
        for eps in w["eps"]:
            k = f"{eps:g}"
            dsec = res["direct"]["at_eps"][k]
            rsec = [res[f"rbm_p{p}"]["at_eps"][k] for p in w["ps"]]
            rsec = [v["seconds_to_T"] for v in rsec if v]
            if dsec and rsec:
                speedup[k] = dsec["seconds_to_T"] / min(rsec)
        res["rbm_over_direct_time_to_T"] = speedup
        out[name] = res
    clocks.stop()
    head = out["large_n_reg_attract"]
    best = head["rbm_p2"]["at_eps"].get("0.01")
    value = best["particle_steps_per_s"] if best else 0.0
    return {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": g.world, "steps": None, "warmup": 0,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": dict(w, systems=W1_SYSTEMS, l2="state 1-2 MB (L2-resident); whole runs timed with events",
                           value_is="RBM-1 (p = 2) particle-steps/s of the cheapest run with E(T) <= 1e-2, "
                                    "large-N system at N = 2^16"),
            "clocks": clocks.summary(), "sweeps": out}


def run_ours(args, w):
    g = Gpu()
    if w["workload"].startswith("batched"):
        line = run_batched(args, w, g)
    elif w["workload"].startswith("surrogate"):
        line = run_surrogate(args, w, g)
    elif w["workload"].startswith("equal_accuracy"):
        line = run_w1_sweep(args, w, g)
    elif "sizes" in w:
        line = run_large_n(args, w, g)
    elif w["workload"].startswith("large_n"):
        line = run_headline(args, w, g)
    else:
        line = run_single(args, w, g)
    if g.rank == 0 and g.world == 1 and not args.no_cpu_baseline and "sweep" not in line and "sweeps" not in line:
        rate, done, el, cores, sample = _oracle_rate(w, seconds=args.cpu_seconds)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": f"{done} oracle RBM-1 steps of {sample} in {el:.1f} s"}
    if g.rank == 0:
        print(json.dumps(line), flush=True)
    g.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="large_n", choices=sorted(WORKLOADS))
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--soak-seconds", type=float, default=1.0,
                    help="untimed load before the timed steps (brings the clocks up; 0 for short profiling runs)")
    ap.add_argument("--sizes", default="", help="large_n_sweep only: comma-separated log2 N (default 16,18,20,22,24,26)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    w = WORKLOADS[args.workload]
    if args.impl == "reference":
        return run_reference(args, w)
    return run_ours(args, w)


if __name__ == "__main__":
    sys.exit(main())
