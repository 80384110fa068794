"""ctypes binding of ``include/rbm.h``: argument marshalling only.

Every function here has the name of the C entry point it calls and does no
arithmetic of the method; all work runs in the CUDA kernels of ``librbm.so``.
Positions are caller-owned CUDA tensors of shape ``(N, ld)`` (``ld = d`` for
d = 1, 2 and 4 for d = 3) in float32 or float64; PyTorch provides the device
memory and the stream only.

If ``librbm.so`` is missing or cannot be loaded the binding raises: there is
no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

RBM_OK = 0
RBM_ERR_INVALID = -1
RBM_ERR_CUDA = -2
RBM_ERR_NOMEM = -3
RBM_ERR_TIMEOUT = -4
RBM_ERR_NONFINITE = -5
RBM_ERR_STATE = -6
RBM_ERR_UNSUPPORTED = -7

RBM_F32, RBM_F64 = 0, 1
RBM_V_ZERO, RBM_V_QUADRATIC = 0, 1
KERNELS = {"inv1d": 0, "coulomb": 1, "bounded_conf": 2, "gauss_agg": 3, "reg_attract": 4, "smooth_test": 5,
           "linear": 6}
POTENTIALS = {"zero": 0, "quadratic": 1}
RBM_METHOD_RBM, RBM_METHOD_DIRECT = 0, 1
METHODS = {"rbm": 0, "direct": 1, "surrogate": 2, "rbmr": 3}
RBM_SCHEME_EULER, RBM_SCHEME_SPLIT, RBM_SCHEME_VERLET = 0, 1, 2
SCHEMES = {"euler": 0, "split": 1, "verlet": 2}
RBM_FLAG_RENORM_SPHERE = 1
RBM_FLAG_GBM_NOISE = 2

# Every symbol include/rbm.h declares.
EXPORTS = (
    "rbm_init", "rbm_step", "rbm_direct_step", "rbm_run", "rbm_step_host", "rbm_get_step", "rbm_set_step",
    "rbm_set_tuning", "rbm_get_tuning", "rbm_sync", "rbm_free", "rbm_status_string", "rbm_last_error",
    "rbm_permutation", "rbm_forces", "rbm_direct_forces_at", "rbm_step_profiled", "rbm_launches_per_step",
    "rbm_permutation_noalloc", "rbm_batched_init", "rbm_batched_set_launch", "rbm_autotune",
    "rbm_surrogate_config", "rbm_surrogate_train", "rbm_surrogate_stats", "rbm_surrogate_params",
    "rbm_surrogate_set_params", "rbm_surrogate_forces", "rbm_surrogate_gradient",
    "rbm_rbmr_sets", "rbm_rbmr_info", "rbm_verlet_set_velocity", "rbm_verlet_get_previous",
    "rbm_verlet_set_previous", "rbm_surrogate_state_size", "rbm_surrogate_save", "rbm_surrogate_load",
    "rbm_latency_floor", "rbm_fp32_fma_peak", "rbm_set_noise_refinement", "rbm_get_noise_refinement", "rbm_surrogate_drift",
    "rbm_set_batch_size", "rbm_autotune_accuracy",
)
N_SURROGATE_PARAMS = 4482     # the d = 2 network


def surrogate_param_count(d: int = 2) -> int:
    """Parameters of the d -> 64 -> 64 -> d network: 4224 + 129 d."""
    return 4224 + 129 * int(d)


class RbmParams(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int64),
        ("d", ctypes.c_int32),
        ("p", ctypes.c_int32),
        ("dt", ctypes.c_double),
        ("sigma", ctypes.c_double),
        ("seed", ctypes.c_uint64),
        ("dtype", ctypes.c_int32),
        ("v", ctypes.c_int32),
        ("v_coef", ctypes.c_double),
        ("k", ctypes.c_int32),
        ("k_param", ctypes.c_double),
        ("flags", ctypes.c_uint32),
        ("scheme", ctypes.c_int32),
        ("replica", ctypes.c_uint32),
    ]


class RbmTuning(ctypes.Structure):
    _fields_ = [
        ("bucket_bits", ctypes.c_int32),
        ("slot_cap", ctypes.c_int32),
        ("sort_cap", ctypes.c_int32),
        ("block", ctypes.c_int32),
        ("direct_block", ctypes.c_int32),
        ("graph_steps", ctypes.c_int32),
        ("path", ctypes.c_int32),
        ("wait_limit_us", ctypes.c_int32),
        ("test_skip_arrival", ctypes.c_int32),
    ]


class RbmError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = f"{where}: {rbm_status_string(status)} ({status})"
        detail = rbm_last_error() if status == RBM_ERR_CUDA else ""
        super().__init__(msg + (f" [{detail}]" if detail else ""))


_lib = None


def load(path: str | None = None) -> ctypes.CDLL:
    """Load ``librbm.so`` (building it first if it is stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if path is None:
        path = _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"librbm.so not found at {path}")
    L = ctypes.CDLL(path)
    vp = ctypes.c_void_p
    i32, i64 = ctypes.c_int32, ctypes.c_int64
    P = ctypes.POINTER(RbmParams)
    TP = ctypes.POINTER(RbmTuning)
    sig = {
        "rbm_init": [P, vp, vp, ctypes.POINTER(vp)],
        "rbm_step": [vp],
        "rbm_direct_step": [vp],
        "rbm_run": [vp, i64, i32],
        "rbm_step_host": [vp, vp, i32],
        "rbm_get_step": [vp, ctypes.POINTER(i64)],
        "rbm_set_step": [vp, i64],
        "rbm_set_tuning": [vp, TP],
        "rbm_get_tuning": [vp, TP],
        "rbm_sync": [vp],
        "rbm_free": [vp],
        "rbm_permutation": [vp, vp],
        "rbm_forces": [vp, i32, vp],
        "rbm_direct_forces_at": [vp, vp, i64, vp],
        "rbm_launches_per_step": [vp, i32, ctypes.POINTER(i32)],
        "rbm_rbmr_sets": [vp, i64, vp],
        "rbm_verlet_set_velocity": [vp, vp],
        "rbm_latency_floor": [vp, ctypes.POINTER(ctypes.c_float)],
        "rbm_fp32_fma_peak": [i32, ctypes.POINTER(ctypes.c_double), vp],
        "rbm_set_noise_refinement": [vp, i32],
        "rbm_set_batch_size": [vp, i32],
        "rbm_autotune_accuracy": [vp, ctypes.POINTER(i32), i32, ctypes.c_double, ctypes.c_double, i32, i64, i32,
                                  ctypes.c_char_p, ctypes.POINTER(i32), ctypes.POINTER(ctypes.c_double),
                                  ctypes.POINTER(i32), ctypes.c_char_p, i32],
        "rbm_surrogate_drift": [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i32), ctypes.POINTER(i32),
                                ctypes.POINTER(i64)],
        "rbm_get_noise_refinement": [vp, ctypes.POINTER(i32)],
        "rbm_verlet_get_previous": [vp, vp, ctypes.POINTER(i32)],
        "rbm_verlet_set_previous": [vp, vp, i32],
        "rbm_surrogate_state_size": [vp, ctypes.POINTER(i64)],
        "rbm_surrogate_save": [vp, vp, i64],
        "rbm_surrogate_load": [vp, vp, i64],
        "rbm_rbmr_info": [vp, ctypes.POINTER(i64), ctypes.POINTER(i32)],
        "rbm_permutation_noalloc": [i64, ctypes.c_uint64, ctypes.c_uint32, i64, vp, vp],
        "rbm_batched_init": [P, i32, ctypes.POINTER(i64), vp, vp, ctypes.POINTER(vp)],
        "rbm_batched_set_launch": [vp, i32, i32],
        "rbm_autotune": [vp, i32, ctypes.c_char_p, ctypes.c_char_p, i32],
        "rbm_surrogate_config": [vp, i32, ctypes.c_double, i64, i32, i32, i32, ctypes.c_double],
        "rbm_surrogate_train": [vp, i32],
        "rbm_surrogate_stats": [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i64), ctypes.POINTER(i64),
                                ctypes.POINTER(i32), ctypes.POINTER(i64)],
        "rbm_surrogate_params": [vp, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float)],
        "rbm_surrogate_set_params": [vp, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float)],
        "rbm_surrogate_forces": [vp, vp, i64, vp],
        "rbm_surrogate_gradient": [vp, vp, vp, i64, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_double)],
        "rbm_step_profiled": [vp, i32, ctypes.POINTER(ctypes.c_float), i32, ctypes.POINTER(i32), ctypes.c_char_p,
                              i32],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = ctypes.c_int32
    L.rbm_status_string.argtypes = [i32]
    L.rbm_status_string.restype = ctypes.c_char_p
    L.rbm_last_error.argtypes = []
    L.rbm_last_error.restype = ctypes.c_char_p
    _lib = L
    return L


def library_path() -> str:
    return _build.LIB


def _check(status: int, where: str) -> None:
    if status != RBM_OK:
        raise RbmError(status, where)


def rbm_status_string(status: int) -> str:
    return load().rbm_status_string(int(status)).decode()


def rbm_last_error() -> str:
    return load().rbm_last_error().decode()


def make_params(n, d, p=2, dt=1e-3, sigma=0.0, seed=0, dtype="f32", v="zero", v_coef=1.0, k="linear",
                k_param=0.0, renorm=False, scheme="euler", replica=0, gbm=False) -> RbmParams:
    return RbmParams(
        n=int(n), d=int(d), p=int(p), dt=float(dt), sigma=float(sigma), seed=int(seed),
        dtype=RBM_F32 if dtype in ("f32", "float32") else RBM_F64,
        v=POTENTIALS[v] if isinstance(v, str) else int(v), v_coef=float(v_coef),
        k=KERNELS[k] if isinstance(k, str) else int(k), k_param=float(k_param),
        flags=(RBM_FLAG_RENORM_SPHERE if renorm else 0) | (RBM_FLAG_GBM_NOISE if gbm else 0),
        scheme=SCHEMES[scheme] if isinstance(scheme, str) else int(scheme), replica=int(replica),
    )


def _stream_handle(stream) -> int:
    if stream is None:
        import torch

        return int(torch.cuda.current_stream().cuda_stream)
    return int(getattr(stream, "cuda_stream", stream))


def _dev_ptr(t) -> int:
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return int(t.data_ptr())


def rbm_init(params: RbmParams, x, stream=None) -> ctypes.c_void_p:
    ctx = ctypes.c_void_p()
    _check(load().rbm_init(ctypes.byref(params), ctypes.c_void_p(_dev_ptr(x)),
                           ctypes.c_void_p(_stream_handle(stream)), ctypes.byref(ctx)), "rbm_init")
    return ctx


def rbm_batched_init(params: RbmParams, sizes, x, stream=None) -> ctypes.c_void_p:
    """``sizes``: replica sizes; ``x``: (sum(sizes), ld) CUDA tensor."""
    n = (ctypes.c_int64 * len(sizes))(*[int(v) for v in sizes])
    ctx = ctypes.c_void_p()
    _check(load().rbm_batched_init(ctypes.byref(params), len(sizes), n, ctypes.c_void_p(_dev_ptr(x)),
                                   ctypes.c_void_p(_stream_handle(stream)), ctypes.byref(ctx)), "rbm_batched_init")
    return ctx


def rbm_batched_set_launch(ctx, threads: int, bucket_target: int) -> None:
    _check(load().rbm_batched_set_launch(ctx, int(threads), int(bucket_target)), "rbm_batched_set_launch")


def rbm_autotune(ctx, trial_steps: int = 3, table_path: str | None = None) -> str:
    rep = ctypes.create_string_buffer(1024)
    _check(load().rbm_autotune(ctx, int(trial_steps), table_path.encode() if table_path else None, rep, 1024),
           "rbm_autotune")
    return rep.value.decode()


def rbm_surrogate_config(ctx, train_every=100, fallback_tol=1e-2, n_queries=65536, iters_first=8000,
                         iters_per_checkpoint=1000, max_rounds=8, lr=3e-3) -> None:
    _check(load().rbm_surrogate_config(ctx, int(train_every), float(fallback_tol), int(n_queries), int(iters_first),
                                       int(iters_per_checkpoint), int(max_rounds), float(lr)), "rbm_surrogate_config")


def rbm_surrogate_train(ctx, iters: int) -> None:
    _check(load().rbm_surrogate_train(ctx, int(iters)), "rbm_surrogate_train")


def rbm_surrogate_stats(ctx) -> dict:
    err = ctypes.c_double()
    ns, nf = ctypes.c_int64(), ctypes.c_int64()
    act = ctypes.c_int32()
    na = ctypes.c_int64()
    _check(load().rbm_surrogate_stats(ctx, ctypes.byref(err), ctypes.byref(ns), ctypes.byref(nf), ctypes.byref(act),
                                      ctypes.byref(na)), "rbm_surrogate_stats")
    return {"rel_err": err.value, "surrogate_steps": ns.value, "fallback_steps": nf.value, "active": bool(act.value),
            "adam_steps": na.value}


def rbm_surrogate_params(ctx, d=2):
    import numpy as np

    th = np.zeros(surrogate_param_count(d), dtype=np.float32)
    nm = np.zeros(d + 2, dtype=np.float32)
    _check(load().rbm_surrogate_params(ctx, th.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                       nm.ctypes.data_as(ctypes.POINTER(ctypes.c_float))), "rbm_surrogate_params")
    return th, nm


def rbm_surrogate_set_params(ctx, theta, norm=None, d=2) -> None:
    """Load parameters (4224 + 129 d floats) and, unless None, the
    normalisation (mu (d values), s, sF), which is then kept at the first
    checkpoint."""
    import numpy as np

    th = np.ascontiguousarray(np.asarray(theta, dtype=np.float32))
    if th.size != surrogate_param_count(d):
        raise ValueError(f"expected {surrogate_param_count(d)} parameters")
    nm_ptr = None
    if norm is not None:
        nm = np.ascontiguousarray(np.asarray(norm, dtype=np.float32))
        if nm.size != d + 2:
            raise ValueError(f"expected {d + 2} normalisation values")
        nm_ptr = nm.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
    _check(load().rbm_surrogate_set_params(ctx, th.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), nm_ptr),
           "rbm_surrogate_set_params")


def rbm_surrogate_forces(ctx, q, f) -> None:
    _check(load().rbm_surrogate_forces(ctx, ctypes.c_void_p(_dev_ptr(q)), int(q.shape[0]),
                                       ctypes.c_void_p(_dev_ptr(f))), "rbm_surrogate_forces")


def rbm_surrogate_gradient(ctx, x, f_target, d=2):
    import numpy as np

    g = np.zeros(surrogate_param_count(d), dtype=np.float32)
    loss = ctypes.c_double()
    _check(load().rbm_surrogate_gradient(ctx, ctypes.c_void_p(_dev_ptr(x)), ctypes.c_void_p(_dev_ptr(f_target)),
                                         int(x.shape[0]), g.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                         ctypes.byref(loss)), "rbm_surrogate_gradient")
    return g, loss.value


def rbm_step(ctx) -> None:
    _check(load().rbm_step(ctx), "rbm_step")


def rbm_direct_step(ctx) -> None:
    _check(load().rbm_direct_step(ctx), "rbm_direct_step")


def rbm_run(ctx, steps: int, method="rbm") -> None:
    _check(load().rbm_run(ctx, int(steps), METHODS.get(method, method)), "rbm_run")


def rbm_step_host(ctx, x_host, method="rbm") -> None:
    """``x_host``: a CPU tensor (pinned for speed) of the positions' shape."""
    if x_host.is_cuda or not x_host.is_contiguous():
        raise ValueError("expected a contiguous host tensor")
    _check(load().rbm_step_host(ctx, ctypes.c_void_p(int(x_host.data_ptr())), METHODS.get(method, method)),
           "rbm_step_host")


def rbm_get_step(ctx) -> int:
    m = ctypes.c_int64()
    _check(load().rbm_get_step(ctx, ctypes.byref(m)), "rbm_get_step")
    return m.value


def rbm_set_step(ctx, m: int) -> None:
    _check(load().rbm_set_step(ctx, int(m)), "rbm_set_step")


def rbm_set_tuning(ctx, tuning: RbmTuning) -> None:
    _check(load().rbm_set_tuning(ctx, ctypes.byref(tuning)), "rbm_set_tuning")


def rbm_get_tuning(ctx) -> RbmTuning:
    t = RbmTuning()
    _check(load().rbm_get_tuning(ctx, ctypes.byref(t)), "rbm_get_tuning")
    return t


def rbm_sync(ctx) -> None:
    _check(load().rbm_sync(ctx), "rbm_sync")


def rbm_free(ctx) -> None:
    _check(load().rbm_free(ctx), "rbm_free")


def rbm_permutation(ctx, perm) -> None:
    """``perm``: int32 CUDA tensor of N entries (holds uint32 ids)."""
    _check(load().rbm_permutation(ctx, ctypes.c_void_p(_dev_ptr(perm))), "rbm_permutation")


def rbm_forces(ctx, method, f) -> None:
    _check(load().rbm_forces(ctx, METHODS.get(method, method), ctypes.c_void_p(_dev_ptr(f))), "rbm_forces")


def rbm_direct_forces_at(ctx, q, f) -> None:
    _check(load().rbm_direct_forces_at(ctx, ctypes.c_void_p(_dev_ptr(q)), int(q.shape[0]),
                                       ctypes.c_void_p(_dev_ptr(f))), "rbm_direct_forces_at")


def rbm_step_profiled(ctx, method="rbm"):
    """One step with per-kernel CUDA-event timing: returns [(name, ms), ...]."""
    ms = (ctypes.c_float * 16)()
    nk = ctypes.c_int32()
    names = ctypes.create_string_buffer(512)
    _check(load().rbm_step_profiled(ctx, METHODS.get(method, method), ms, 16, ctypes.byref(nk), names, 512),
           "rbm_step_profiled")
    return list(zip(names.value.decode().split(";"), [ms[i] for i in range(nk.value)]))


def rbm_permutation_noalloc(n: int, seed: int, replica: int, m: int, perm, stream=None) -> None:
    """Random division of step ``m`` into ``perm`` (int32 CUDA tensor of n
    entries) with no device allocation (n <= 65536); see include/rbm.h."""
    if perm.numel() < n:
        raise ValueError("perm holds fewer than n entries")
    _check(load().rbm_permutation_noalloc(int(n), int(seed), int(replica), int(m),
                                          ctypes.c_void_p(_dev_ptr(perm)), ctypes.c_void_p(_stream_handle(stream))),
           "rbm_permutation_noalloc")


def rbm_rbmr_sets(ctx, m, sets) -> None:
    """RBM-r sets of step ``m`` into ``sets`` (a CUDA int32 tensor of K x p)."""
    _check(load().rbm_rbmr_sets(ctx, int(m), ctypes.c_void_p(int(sets.data_ptr()))), "rbm_rbmr_sets")


def rbm_verlet_set_velocity(ctx, v) -> None:
    """Velocities V_0 (a CUDA tensor shaped like the positions) for the
    Verlet scheme; the next step is the Taylor start."""
    _check(load().rbm_verlet_set_velocity(ctx, ctypes.c_void_p(int(v.data_ptr()))), "rbm_verlet_set_velocity")


def rbm_verlet_get_previous(ctx, prev) -> bool:
    """X_{n-1} (or V_0 while the Taylor start is pending) into ``prev``; returns
    whether the Taylor start is pending."""
    pend = ctypes.c_int32()
    _check(load().rbm_verlet_get_previous(ctx, ctypes.c_void_p(int(prev.data_ptr())), ctypes.byref(pend)),
           "rbm_verlet_get_previous")
    return bool(pend.value)


def rbm_verlet_set_previous(ctx, prev, taylor_pending) -> None:
    _check(load().rbm_verlet_set_previous(ctx, ctypes.c_void_p(int(prev.data_ptr())), int(bool(taylor_pending))),
           "rbm_verlet_set_previous")


def rbm_surrogate_save(ctx) -> bytes:
    """The surrogate's state as bytes (checkpoint/resume)."""
    n = ctypes.c_int64()
    _check(load().rbm_surrogate_state_size(ctx, ctypes.byref(n)), "rbm_surrogate_state_size")
    buf = ctypes.create_string_buffer(n.value)
    _check(load().rbm_surrogate_save(ctx, buf, n.value), "rbm_surrogate_save")
    return buf.raw


def rbm_surrogate_load(ctx, state: bytes) -> None:
    buf = ctypes.create_string_buffer(state, len(state))
    _check(load().rbm_surrogate_load(ctx, buf, len(state)), "rbm_surrogate_load")


def rbm_latency_floor(ctx) -> float:
    """Microseconds of the cooperative step's launch shape with no work (a step in the common case waits at no grid barrier)."""
    us = ctypes.c_float()
    _check(load().rbm_latency_floor(ctx, ctypes.byref(us)), "rbm_latency_floor")
    return us.value


def rbm_fp32_fma_peak(packed: bool = False, stream=None) -> float:
    """Measured FP32 FMA throughput (TFLOP/s) of the current device: scalar or
    packed two-lane FMA chains (see include/rbm.h)."""
    tf = ctypes.c_double()
    _check(load().rbm_fp32_fma_peak(1 if packed else 0, ctypes.byref(tf), ctypes.c_void_p(_stream_handle(stream))),
           "rbm_fp32_fma_peak")
    return tf.value


def rbm_set_noise_refinement(ctx, r: int) -> None:
    """Share one Brownian path with runs of step dt/r (see include/rbm.h)."""
    _check(load().rbm_set_noise_refinement(ctx, int(r)), "rbm_set_noise_refinement")


def rbm_get_noise_refinement(ctx) -> int:
    r = ctypes.c_int32()
    _check(load().rbm_get_noise_refinement(ctx, ctypes.byref(r)), "rbm_get_noise_refinement")
    return r.value


def rbm_set_batch_size(ctx, p: int) -> None:
    _check(load().rbm_set_batch_size(ctx, int(p)), "rbm_set_batch_size")


def rbm_autotune_accuracy(ctx, ps, eps, horizon, max_halvings=3, pilot_n=16384, trial_steps=3,
                          table_path=None) -> dict:
    """Batch size (and step) by the least time to T at E(T) <= eps (see include/rbm.h)."""
    arr = (ctypes.c_int32 * len(ps))(*[int(v) for v in ps])
    p, dt, met = ctypes.c_int32(), ctypes.c_double(), ctypes.c_int32()
    buf = ctypes.create_string_buffer(4096)
    _check(load().rbm_autotune_accuracy(ctx, arr, len(ps), float(eps), float(horizon), int(max_halvings),
                                        int(pilot_n), int(trial_steps),
                                        table_path.encode() if table_path else None, ctypes.byref(p),
                                        ctypes.byref(dt), ctypes.byref(met), buf, len(buf)),
           "rbm_autotune_accuracy")
    return {"p": p.value, "dt": dt.value, "met": bool(met.value), "report": buf.value.decode()}


def rbm_surrogate_drift(ctx) -> dict:
    """The surrogate's drift-aware schedule (see include/rbm.h)."""
    e, iv, fo, nf = ctypes.c_double(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64()
    _check(load().rbm_surrogate_drift(ctx, ctypes.byref(e), ctypes.byref(iv), ctypes.byref(fo), ctypes.byref(nf)),
           "rbm_surrogate_drift")
    return {"drift_err": e.value, "interval": iv.value, "forced_off": bool(fo.value), "forced_intervals": nf.value}


def rbm_rbmr_info(ctx) -> dict:
    k, r = ctypes.c_int64(), ctypes.c_int32()
    _check(load().rbm_rbmr_info(ctx, ctypes.byref(k), ctypes.byref(r)), "rbm_rbmr_info")
    return {"iterations_per_step": k.value, "rounds_last": r.value}


def rbm_launches_per_step(ctx, method="rbm") -> int:
    n = ctypes.c_int32()
    _check(load().rbm_launches_per_step(ctx, METHODS.get(method, method), ctypes.byref(n)),
           "rbm_launches_per_step")
    return n.value
