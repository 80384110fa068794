"""The FP32 build at equilibrium.

- A contracting system (V = |x|^2/2 dominates the smooth attraction
  K = -x/(|x|^2 + 0.01)) run to T = 5 from the same X0 with the same
  Brownian increments as the FP64 oracle: rounding differences stay bounded
  (the flow contracts), so the FP32 empirical law must agree with the
  oracle's within 1e-3 in Wasserstein-1 (sliced, 1-D W1 of the projections
  on the axes and on random directions) and in the second moment.
- The Dyson Brownian motion at the paper's N = 1e5 (Sec. 4.2, splitting
  scheme) against its closed forms: the semicircle of radius sqrt(2)
  (eq. "semicircle") and m2 = (1 + 1/N)/2.
"""
import numpy as np
import pytest

import oracle
import paper_1812_10575_gb300 as rbm
import workloads
from gpu_util import as_run_precision, from_dev, to_dev, torch_cuda

pytestmark = pytest.mark.gpu


def _sliced_w1(A, B, k=16, seed=0):
    rng = np.random.default_rng(seed)
    dirs = rng.standard_normal((k, A.shape[1]))
    dirs = np.concatenate([np.eye(A.shape[1]), dirs / np.linalg.norm(dirs, axis=1, keepdims=True)])
    return max(float(np.mean(np.abs(np.sort(A @ v) - np.sort(B @ v)))) for v in dirs)


def test_fp32_equilibrium_matches_fp64_oracle():
    torch_cuda()
    n, d, steps = 10000, 3, 5000
    kw = dict(p=2, dt=1e-3, sigma=0.2, v="quadratic", k="reg_attract", k_param=0.01)
    X = as_run_precision(workloads.gaussian(n, d, seed=3), "f32")
    x = to_dev(X, "f32")
    s = rbm.System(x, d=d, seed=11, **kw)
    s.run(steps)
    s.sync()
    got = from_dev(x, d)
    ref = oracle.run(oracle.make_params(n, d, seed=11, precision="f32", **kw), X, 0, steps)
    assert _sliced_w1(got, ref) < 1e-3
    assert abs(np.mean(np.sum(got ** 2, axis=1)) - np.mean(np.sum(ref ** 2, axis=1))) < 1e-3


def _semicircle_cdf(x, r2):
    r = np.sqrt(r2)
    x = np.clip(x, -r, r)
    return 0.5 + x * np.sqrt(np.maximum(r2 - x * x, 0.0)) / (np.pi * r2) + np.arcsin(x / r) / np.pi


def test_dyson_fp32_equilibrium_at_paper_size():
    """N = 1e5, dt = 1e-3, sigma^2 = 1/N, splitting scheme, T = 5 from N(0,1)."""
    torch_cuda()
    n = 100000
    X = as_run_precision(workloads.dyson(n, 0), "f32")
    x = to_dev(X, "f32")
    s = rbm.System(x, d=1, p=2, dt=1e-3, sigma=float(np.sqrt(1.0 / n)), v="quadratic", k="inv1d", seed=1,
                   scheme="split")
    s.run(5000)
    s.sync()
    got = from_dev(x, 1).ravel()
    xs = np.linspace(-2.0, 2.0, 40001)
    femp = np.searchsorted(np.sort(got), xs, side="right") / n
    w1 = np.trapezoid(np.abs(femp - _semicircle_cdf(xs, 2.0)), xs)
    assert w1 < 5e-3, w1
    # sampling std of m2 is about 0.5 / sqrt(N) = 1.6e-3, plus an O(dt) bias
    assert abs(np.mean(got ** 2) - (1.0 + 1.0 / n) / 2.0) < 5e-3
