"""The accuracy-aware autotuner (rbm_autotune_accuracy) and rbm_set_batch_size.

The error of RBM-1 decays like sqrt(dt / (p - 1)) (Sec. 3) while a step costs
more with p, so the tuner picks the batch size (and the step) with the least
time to T at E(T) <= eps, E(T) of eq. "errorformula" against the direct method
on one Brownian path.  Checked here:

- the error the tuner acts on, recomputed independently through the public
  API (pilot system, direct reference at dt / 2^(H+1), noise refinement): the
  chosen (p, dt) meets eps and, for that p, the next coarser step does not;
- with a loose eps the coarsest step is taken; with an unreachable one the
  result says so;
- positions and step index are left as they were, and the chosen p is
  applied (later steps equal a fresh context built with that p, bit for bit),
  for a single system and for batched replicas;
- a stored result is read back from the table instead of searching.
"""
import os
import tempfile

import numpy as np
import pytest

import paper_1812_10575_gb300 as rbm
import workloads
from gpu_util import from_dev, to_dev, torch_cuda

pytestmark = pytest.mark.gpu

KW = dict(dt=2e-3, sigma=0.3, v="quadratic", v_coef=1.0, k="reg_attract", k_param=0.05, seed=5)
H, T, PILOT = 2, 0.1, 4096


def _gap(a, b):
    return float(np.sqrt(np.mean(np.sum((a - b) ** 2, axis=1))))


def _pilot_error(X, d, p, dt):
    """E(T) of RBM-1 (p, dt) against the direct method at dt_ctx / 2^(H+1) on
    the first PILOT particles, one Brownian path."""
    Xp = X[:PILOT]
    dt_ref = KW["dt"] / 2 ** (H + 1)
    xr = to_dev(Xp, "f64")
    ref = rbm.System(xr, d=d, p=2, **dict(KW, dt=dt_ref))
    ref.run(int(round(T / dt_ref)), "direct")
    ref.sync()
    xs = to_dev(Xp, "f64")
    s = rbm.System(xs, d=d, p=p, **dict(KW, dt=dt))
    s.set_noise_refinement(int(round(dt / dt_ref)))
    s.run(int(round(T / dt)))
    s.sync()
    return _gap(from_dev(xs, d), from_dev(xr, d))


def test_tuner_meets_eps_with_the_cheapest_step_and_applies_p():
    torch = torch_cuda()
    n, d = 20000, 2
    X = workloads.gaussian(n, d, seed=3)
    e2 = _pilot_error(X, d, 2, KW["dt"])
    eps = 0.6 * e2                                  # p = 2 at the context's step is not enough
    x = to_dev(X, "f64")
    s = rbm.System(x, d=d, p=2, **KW)
    s.m = 11
    before = x.clone()
    res = s.autotune_accuracy([2, 4, 8], eps, T, max_halvings=H, pilot_n=PILOT, trial_steps=2)
    assert res["met"], res
    assert torch.equal(x, before) and s.m == 11
    e = _pilot_error(X, d, res["p"], res["dt"])
    assert e <= eps * (1 + 1e-9), (e, eps, res)
    if res["dt"] < KW["dt"] * (1 - 1e-12):        # a finer step was needed for this p
        assert _pilot_error(X, d, res["p"], 2 * res["dt"]) > eps, res
    # the chosen p is applied: later steps equal a fresh context with that p
    y = before.clone()
    t = rbm.System(y, d=d, p=res["p"], **KW)
    t.m = 11
    s.run(3)
    t.run(3)
    s.sync()
    t.sync()
    assert torch.equal(x, y)


def test_tuner_loose_and_unreachable_eps_and_table():
    torch_cuda()
    n, d = 20000, 2
    X = workloads.gaussian(n, d, seed=4)
    x = to_dev(X, "f64")
    s = rbm.System(x, d=d, p=2, **KW)
    loose = s.autotune_accuracy([2, 4], 1e3, T, max_halvings=H, pilot_n=PILOT, trial_steps=2)
    assert loose["met"] and loose["dt"] == KW["dt"], loose
    hard = s.autotune_accuracy([2, 4], 1e-14, T, max_halvings=H, pilot_n=PILOT, trial_steps=2)
    assert not hard["met"] and hard["p"] in (2, 4), hard
    with tempfile.TemporaryDirectory() as tmp:
        path = os.path.join(tmp, "table.txt")
        first = s.autotune_accuracy([2, 4], 1e3, T, max_halvings=H, pilot_n=PILOT, trial_steps=2, table_path=path)
        again = s.autotune_accuracy([2, 4], 1e3, T, max_halvings=H, pilot_n=PILOT, trial_steps=2, table_path=path)
        assert again["report"].startswith("table") and (again["p"], again["dt"]) == (first["p"], first["dt"])


def test_tuner_on_batched_replicas_leaves_state_and_applies_p():
    torch = torch_cuda()
    sizes = [int(v) for v in workloads.replica_sizes(24, 256, 4096, seed=2)] + [4096]
    X = workloads.unit_cube(sum(sizes), 2, seed=1)
    kw = dict(dt=1e-2, sigma=0.01, k="bounded_conf", k_param=0.25, seed=2)
    x = to_dev(X, "f32")
    rep = rbm.Replicas(x, sizes, d=2, p=2, **kw)
    rep.m = 5
    before = x.clone()
    res = rep.autotune_accuracy([2, 4], 1e3, 0.2, max_halvings=1, pilot_n=4096, trial_steps=2)
    assert res["met"] and res["p"] in (2, 4), res
    assert torch.equal(x, before) and rep.m == 5
    y = before.clone()
    other = rbm.Replicas(y, sizes, d=2, p=res["p"], **kw)
    other.m = 5
    rep.run(2)
    other.run(2)
    rep.sync()
    other.sync()
    assert torch.equal(x, y)
    with pytest.raises(rbm.RbmError):
        rep.set_batch_size(33)                      # batched contexts take p <= 32
