"""Helpers of the GPU tests: layout conversion between the oracle's (N, d)
float64 arrays and the library's (N, ld) device tensors, and the parity
tolerances.  No arithmetic of the method lives here."""
from __future__ import annotations

import numpy as np
import pytest

EPS32 = float(np.finfo(np.float32).eps)


def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def ld_of(d: int) -> int:
    return 4 if d == 3 else d


def to_dev(X: np.ndarray, dtype: str = "f64", pad_value: float = 0.0):
    torch = torch_cuda()
    n, d = X.shape
    t = torch.full((n, ld_of(d)), pad_value, dtype=torch.float64)
    t[:, :d] = torch.from_numpy(np.asarray(X, dtype=np.float64))
    t = t.to(torch.float32 if dtype == "f32" else torch.float64)
    return t.cuda().contiguous()


def from_dev(x, d: int) -> np.ndarray:
    return x[:, :d].double().cpu().numpy()


def as_run_precision(X: np.ndarray, dtype: str) -> np.ndarray:
    """The exact values an FP32 run starts from (float64 copies of float32)."""
    return X.astype(np.float32).astype(np.float64) if dtype == "f32" else np.asarray(X, dtype=np.float64)


def rel_err(got: np.ndarray, ref: np.ndarray) -> np.ndarray:
    """Per-particle |got - ref| / max(|ref|, 1)."""
    return np.linalg.norm(got - ref, axis=1) / np.maximum(np.linalg.norm(ref, axis=1), 1.0)


def assert_close_per_particle(got, ref, tol, extra=None, what=""):
    """|got_i - ref_i| <= tol * max(|ref_i|, 1) + extra_i for every particle."""
    diff = np.linalg.norm(got - ref, axis=1)
    bound = tol * np.maximum(np.linalg.norm(ref, axis=1), 1.0)
    if extra is not None:
        bound = bound + extra
    bad = np.nonzero(~(diff <= bound))[0]
    if len(bad):
        i = bad[np.argmax((diff - bound)[bad])]
        raise AssertionError(f"{what}: {len(bad)} of {len(diff)} particles off; worst {i}: diff {diff[i]:.3e} "
                             f"bound {bound[i]:.3e} got {got[i]} ref {ref[i]}")
