"""Plain FP64 CPU oracle of RBM-1 and of the direct step (arXiv:1812.10575).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA library in ``paper_1812_10575_gb300``: the arithmetic lives in
``rbm_oracle.c`` (plain C, compiled here with gcc) and this module only
marshals numpy arrays into it.

Positions are ``(N, d)`` float64 arrays.  Parameters mirror the problem
statement of Sec. 1 (V, K, sigma) and Algorithm "randomdiv" (p, tau) of the
paper; see ``rbm_oracle.h`` for the field list.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "liboracle.so")
_SRC = os.path.join(_HERE, "rbm_oracle.c")

V_KINDS = {"zero": 0, "quadratic": 1}
K_KINDS = {
    "inv1d": 0,
    "coulomb": 1,
    "bounded_conf": 2,
    "gauss_agg": 3,
    "reg_attract": 4,
    "smooth_test": 5,
    "linear": 6,
}


class OrcParams(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int64),
        ("d", ctypes.c_int32),
        ("p", ctypes.c_int32),
        ("dt", ctypes.c_double),
        ("sigma", ctypes.c_double),
        ("seed", ctypes.c_uint64),
        ("v_kind", ctypes.c_int32),
        ("k_kind", ctypes.c_int32),
        ("v_coef", ctypes.c_double),
        ("k_param", ctypes.c_double),
        ("renorm", ctypes.c_int32),
        ("ubits", ctypes.c_int32),
        ("decide_f32", ctypes.c_int32),
        ("replica", ctypes.c_uint32),
        ("gbm", ctypes.c_int32),
        ("noise_refine", ctypes.c_int32),
    ]


def build(force: bool = False) -> str:
    """Compile ``rbm_oracle.c`` into ``_build/liboracle.so`` (gcc, -O2, OpenMP).

    ``-ffp-contract=off`` keeps C's evaluation rules (no implicit fused
    multiply-adds), so the oracle gives the same results on x86-64 and Arm.
    """
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "rbm_oracle.h"))
    ):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = [
        "gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared", "-fopenmp",
        "-ffp-contract=off", _SRC, "-o", tmp, "-lm",
    ]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_lib = None
_lock = threading.Lock()


def lib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            P = ctypes.POINTER(OrcParams)
            u32p = ctypes.POINTER(ctypes.c_uint32)
            u64p = ctypes.POINTER(ctypes.c_uint64)
            dp = ctypes.POINTER(ctypes.c_double)
            L.orc_philox4x32_10.argtypes = [u32p, u32p, u32p]
            L.orc_perm_keys.argtypes = [P, ctypes.c_int64, u64p]
            L.orc_permutation.argtypes = [P, ctypes.c_int64, u32p]
            L.orc_normals.argtypes = [P, ctypes.c_int64, dp]
            L.orc_kernel_pair.argtypes = [P, dp, dp, dp]
            L.orc_direct_interaction.argtypes = [P, dp, dp]
            L.orc_rbm_interaction.argtypes = [P, dp, u32p, dp]
            L.orc_euler_update.argtypes = [P, dp, dp, ctypes.c_int64]
            L.orc_rbm_step.argtypes = [P, dp, ctypes.c_int64]
            L.orc_rbm_split_step.argtypes = [P, dp, ctypes.c_int64]
            L.orc_split_pair_solve.argtypes = [P, dp, dp, dp, dp]
            L.orc_direct_step.argtypes = [P, dp, ctypes.c_int64]
            L.orc_rbm_verlet_step.argtypes = [P, dp, dp, ctypes.c_int64, ctypes.c_int]
            L.orc_direct_verlet_step.argtypes = [P, dp, dp, ctypes.c_int]
            L.orc_rbmr_iterations_per_step.argtypes = [P]
            L.orc_rbmr_iterations_per_step.restype = ctypes.c_int64
            L.orc_rbmr_set.argtypes = [P, ctypes.c_int64, u32p]
            L.orc_rbmr_iteration.argtypes = [P, dp, ctypes.c_int64]
            L.orc_rbmr_step.argtypes = [P, dp, ctypes.c_int64]
            L.orc_direct_forces_at.argtypes = [P, dp, dp, ctypes.c_int64, dp]
            L.orc_direct_step_sampled.argtypes = [P, dp, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64),
                                                  ctypes.c_int64, dp]
            L.orc_num_threads.restype = ctypes.c_int
            for f in (L.orc_philox4x32_10, L.orc_perm_keys, L.orc_permutation, L.orc_normals,
                      L.orc_kernel_pair, L.orc_direct_interaction, L.orc_rbm_interaction,
                      L.orc_euler_update, L.orc_rbm_step, L.orc_rbm_split_step, L.orc_split_pair_solve, L.orc_direct_step,
                      L.orc_direct_forces_at, L.orc_direct_step_sampled):
                f.restype = None
            _lib = L
    return _lib


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def make_params(n, d, p=2, dt=1e-3, sigma=0.0, seed=0, v="zero", v_coef=1.0, k="linear",
                k_param=0.0, renorm=False, precision="f64", replica=0, gbm=False, noise_refine=1) -> OrcParams:
    """Build an :class:`OrcParams`.

    ``precision`` names the precision of the run the oracle is compared with:
    ``"f64"`` uses 53-bit uniforms and FP64 kernel decisions, ``"f32"`` uses
    24-bit uniforms and takes kernel decisions on the FP32 squared norm.  The
    arithmetic itself is always FP64.  ``noise_refine`` = r draws each step's
    Brownian increment as the normalised sum of the r increments of a run with
    step dt/r (path coupling across step sizes).
    """
    if precision not in ("f64", "f32"):
        raise ValueError(precision)
    return OrcParams(
        n=int(n), d=int(d), p=int(p), dt=float(dt), sigma=float(sigma), seed=int(seed),
        v_kind=V_KINDS[v] if isinstance(v, str) else int(v),
        k_kind=K_KINDS[k] if isinstance(k, str) else int(k),
        v_coef=float(v_coef), k_param=float(k_param), renorm=int(bool(renorm)),
        ubits=53 if precision == "f64" else 24, decide_f32=int(precision == "f32"),
        replica=int(replica), gbm=int(bool(gbm)), noise_refine=int(noise_refine),
    )


def philox4x32_10(ctr, key) -> np.ndarray:
    """Philox4x32-10 of one counter (4 x u32) and key (2 x u32)."""
    c = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint32))
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_ptr(c, ctypes.c_uint32), _ptr(k, ctypes.c_uint32), _ptr(out, ctypes.c_uint32))
    return out


def perm_keys(prm: OrcParams, m: int) -> np.ndarray:
    keys = np.zeros(prm.n, dtype=np.uint64)
    lib().orc_perm_keys(ctypes.byref(prm), int(m), _ptr(keys, ctypes.c_uint64))
    return keys


def permutation(prm: OrcParams, m: int) -> np.ndarray:
    perm = np.zeros(prm.n, dtype=np.uint32)
    lib().orc_permutation(ctypes.byref(prm), int(m), _ptr(perm, ctypes.c_uint32))
    return perm


def normals(prm: OrcParams, m: int) -> np.ndarray:
    z = np.zeros((prm.n, prm.d), dtype=np.float64)
    lib().orc_normals(ctypes.byref(prm), int(m), _ptr(z, ctypes.c_double))
    return z


def _x(X, prm):
    X = np.ascontiguousarray(np.asarray(X, dtype=np.float64))
    if X.shape != (prm.n, prm.d):
        raise ValueError(f"positions must be ({prm.n}, {prm.d}), got {X.shape}")
    return X


def kernel_pair(prm: OrcParams, xi, xj) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(xi, dtype=np.float64).reshape(prm.d))
    b = np.ascontiguousarray(np.asarray(xj, dtype=np.float64).reshape(prm.d))
    out = np.zeros(prm.d, dtype=np.float64)
    lib().orc_kernel_pair(ctypes.byref(prm), _ptr(a, ctypes.c_double), _ptr(b, ctypes.c_double),
                          _ptr(out, ctypes.c_double))
    return out


def direct_interaction(prm: OrcParams, X) -> np.ndarray:
    X = _x(X, prm)
    F = np.zeros_like(X)
    lib().orc_direct_interaction(ctypes.byref(prm), _ptr(X, ctypes.c_double), _ptr(F, ctypes.c_double))
    return F


def rbm_interaction(prm: OrcParams, X, perm) -> np.ndarray:
    X = _x(X, prm)
    perm = np.ascontiguousarray(np.asarray(perm, dtype=np.uint32))
    if perm.shape != (prm.n,):
        raise ValueError("perm must have N entries")
    F = np.zeros_like(X)
    lib().orc_rbm_interaction(ctypes.byref(prm), _ptr(X, ctypes.c_double), _ptr(perm, ctypes.c_uint32),
                              _ptr(F, ctypes.c_double))
    return F


def euler_update(prm: OrcParams, X, FK, m: int) -> np.ndarray:
    Y = _x(X, prm).copy()
    FK = _x(FK, prm)
    lib().orc_euler_update(ctypes.byref(prm), _ptr(Y, ctypes.c_double), _ptr(FK, ctypes.c_double), int(m))
    return Y


def rbm_step(prm: OrcParams, X, m: int) -> np.ndarray:
    """One RBM-1 step from step index ``m``; returns the new positions."""
    Y = _x(X, prm).copy()
    lib().orc_rbm_step(ctypes.byref(prm), _ptr(Y, ctypes.c_double), int(m))
    return Y


def rbm_split_step(prm: OrcParams, X, m: int) -> np.ndarray:
    """One RBM-1 step of the splitting scheme (p = 2, K = 1/x, Coulomb or -c x)."""
    if prm.p != 2 or prm.k_kind not in (K_KINDS["inv1d"], K_KINDS["coulomb"], K_KINDS["linear"]):
        raise ValueError("the splitting scheme needs p = 2 and K = 1/x, x/|x|^3 or -c x")
    Y = _x(X, prm).copy()
    lib().orc_rbm_split_step(ctypes.byref(prm), _ptr(Y, ctypes.c_double), int(m))
    return Y


def split_pair_solve(prm: OrcParams, xi, xj):
    a = np.ascontiguousarray(np.asarray(xi, dtype=np.float64).reshape(prm.d))
    b = np.ascontiguousarray(np.asarray(xj, dtype=np.float64).reshape(prm.d))
    yi = np.zeros(prm.d); yj = np.zeros(prm.d)
    lib().orc_split_pair_solve(ctypes.byref(prm), _ptr(a, ctypes.c_double), _ptr(b, ctypes.c_double),
                               _ptr(yi, ctypes.c_double), _ptr(yj, ctypes.c_double))
    return yi, yj


def direct_step(prm: OrcParams, X, m: int) -> np.ndarray:
    """One direct forward-Euler step from step index ``m``; returns the new positions."""
    Y = _x(X, prm).copy()
    lib().orc_direct_step(ctypes.byref(prm), _ptr(Y, ctypes.c_double), int(m))
    return Y


def verlet_run(prm: OrcParams, X0, V0, m0: int, steps: int, method: str = "rbm"):
    """Verlet scheme of the second-order system (Appendix A, Sec. 4.1):
    ``steps`` steps from positions X0 and velocities V0 at step index m0 (the
    first step is the Taylor start); returns (X_n, X_{n-1})."""
    X = _x(X0, prm).copy()
    P = _x(V0, prm).copy()
    for s in range(steps):
        if method == "rbm":
            lib().orc_rbm_verlet_step(ctypes.byref(prm), _ptr(X, ctypes.c_double), _ptr(P, ctypes.c_double),
                                      int(m0 + s), int(s == 0))
        else:
            lib().orc_direct_verlet_step(ctypes.byref(prm), _ptr(X, ctypes.c_double), _ptr(P, ctypes.c_double),
                                         int(s == 0))
    return X, P


def rbmr_iterations_per_step(prm: OrcParams) -> int:
    """RBM-r iterations per step: floor(N/p), at least 1."""
    return int(lib().orc_rbmr_iterations_per_step(ctypes.byref(prm)))


def rbmr_set(prm: OrcParams, k: int) -> np.ndarray:
    """The p members (slot order) of RBM-r iteration ``k``."""
    out = np.zeros(prm.p, dtype=np.uint32)
    lib().orc_rbmr_set(ctypes.byref(prm), int(k), _ptr(out, ctypes.c_uint32))
    return out


def rbmr_iteration(prm: OrcParams, X, k: int) -> np.ndarray:
    """One RBM-r iteration (Algorithm "fullyrandom"); returns the new positions."""
    Y = _x(X, prm).copy()
    lib().orc_rbmr_iteration(ctypes.byref(prm), _ptr(Y, ctypes.c_double), int(k))
    return Y


def rbmr_step(prm: OrcParams, X, m: int) -> np.ndarray:
    """One RBM-r step m -> m+1: iterations m K .. m K + K - 1, K = floor(N/p)."""
    Y = _x(X, prm).copy()
    lib().orc_rbmr_step(ctypes.byref(prm), _ptr(Y, ctypes.c_double), int(m))
    return Y


def run(prm: OrcParams, X, m0: int, steps: int, method: str = "rbm") -> np.ndarray:
    step = {"rbm": rbm_step, "direct": direct_step, "split": rbm_split_step, "rbmr": rbmr_step}[method]
    Y = _x(X, prm).copy()
    for s in range(steps):
        Y = step(prm, Y, m0 + s)
    return Y


def direct_step_sampled(prm: OrcParams, X, m: int, idx) -> np.ndarray:
    """New positions of particles ``idx`` after one direct step from ``X``."""
    X = _x(X, prm)
    idx = np.ascontiguousarray(np.asarray(idx, dtype=np.int64))
    Y = np.zeros((len(idx), prm.d))
    lib().orc_direct_step_sampled(ctypes.byref(prm), _ptr(X, ctypes.c_double), int(m),
                                  idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), len(idx),
                                  _ptr(Y, ctypes.c_double))
    return Y


def direct_forces_at(prm: OrcParams, X, Q) -> np.ndarray:
    X = _x(X, prm)
    Q = np.ascontiguousarray(np.asarray(Q, dtype=np.float64).reshape(-1, prm.d))
    F = np.zeros_like(Q)
    lib().orc_direct_forces_at(ctypes.byref(prm), _ptr(X, ctypes.c_double), _ptr(Q, ctypes.c_double),
                               int(Q.shape[0]), _ptr(F, ctypes.c_double))
    return F


def num_threads() -> int:
    return int(lib().orc_num_threads())
