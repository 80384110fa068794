"""Checkpoint/resume: the RNG is counter-based, so a run's state is the
positions, the step index, the parameters and, where a method keeps more,
its own buffers (the Verlet scheme's X_{n-1}, the surrogate's network and
Adam state).  200 steps in one context must equal 100 steps, a save through
host memory, a fresh context and 100 more steps, bit for bit."""
import numpy as np
import pytest

import paper_1812_10575_gb300 as rbm
import workloads
from gpu_util import to_dev, torch_cuda

pytestmark = pytest.mark.gpu


def _resume(X, d, dtype, kw, method="rbm", path=None, first=100, second=100, graph_steps=None):
    torch = torch_cuda()
    tuning = {}
    if path is not None:
        tuning["path"] = path
    if graph_steps is not None:
        tuning["graph_steps"] = graph_steps
    whole = rbm.System(to_dev(X, dtype), d=d, **kw)
    if tuning:
        whole.set_tuning(**tuning)
    whole.run(first + second, method)
    whole.sync()
    a = rbm.System(to_dev(X, dtype), d=d, **kw)
    if tuning:
        a.set_tuning(**tuning)
    a.run(first, method)
    a.sync()
    saved_x, saved_m = a.x.cpu().clone(), a.m          # the checkpoint, in host memory
    a.close()
    b = rbm.System(saved_x.cuda(), d=d, **kw)
    if tuning:
        b.set_tuning(**tuning)
    b.m = saved_m
    b.run(second, method)
    b.sync()
    assert b.m == whole.m == first + second
    assert torch.equal(b.x, whole.x)


@pytest.mark.parametrize("path", [1, 2, 3, 4])
def test_rbm_resume_bit_identical(path):
    n = 1500 if path == 3 else 20000
    X = workloads.gaussian(n, 3, seed=1)
    _resume(X, 3, "f32", dict(p=2, dt=1e-3, sigma=0.2, v="quadratic", k="reg_attract", k_param=0.01, seed=3),
            path=path, graph_steps=30)


def test_split_scheme_resume_bit_identical():
    X = workloads.dyson(1000, 0)
    _resume(X, 1, "f64", dict(p=2, dt=1e-3, sigma=float(np.sqrt(1e-3)), v="quadratic", k="inv1d", seed=2,
                              scheme="split"))


def test_direct_and_rbmr_resume_bit_identical():
    X = workloads.gaussian(3000, 2, seed=4)
    kw = dict(p=2, dt=1e-3, sigma=0.1, v="quadratic", k="gauss_agg", seed=5)
    _resume(X, 2, "f32", kw, method="direct", first=7, second=8)
    _resume(X, 2, "f32", kw, method="rbmr", first=12, second=13)


def test_verlet_resume_bit_identical():
    torch = torch_cuda()
    n, d = 4000, 1
    kw = dict(p=2, dt=2.0 ** -6, k="smooth_test", scheme="verlet", seed=6)
    X = workloads.semicircle(n, 2.0, seed=7)
    V = np.random.default_rng(8).normal(size=(n, d))
    whole = rbm.System(to_dev(X, "f32"), d=d, **kw)
    whole.verlet_set_velocity(to_dev(V, "f32"))
    whole.run(64)
    a = rbm.System(to_dev(X, "f32"), d=d, **kw)
    a.verlet_set_velocity(to_dev(V, "f32"))
    a.run(32)
    prev, pending = a.verlet_get_previous()
    assert not pending
    saved = (a.x.cpu().clone(), prev.cpu().clone(), a.m)
    a.close()
    b = rbm.System(saved[0].cuda(), d=d, **kw)
    b.m = saved[2]
    b.verlet_set_previous(saved[1].cuda(), False)
    b.run(32)
    whole.sync()
    b.sync()
    assert torch.equal(b.x, whole.x)


def test_surrogate_resume_bit_identical():
    """Checkpoints at steps 0, 100 and 200; the save at step 150 carries the
    network, its Adam moments and the schedule into a fresh context."""
    torch = torch_cuda()
    n = 16384
    kw = dict(p=2, dt=1e-3, sigma=0.1, v="quadratic", k="gauss_agg", seed=9)
    cfg = dict(train_every=100, fallback_tol=1e-2, n_queries=4096, iters_first=2000, iters_per_checkpoint=500,
               max_rounds=2, lr=3e-3)
    X = workloads.mixture(n, 2, seed=10)
    whole = rbm.System(to_dev(X, "f32"), d=2, **kw)
    whole.surrogate_config(**cfg)
    whole.run(300, "surrogate")
    a = rbm.System(to_dev(X, "f32"), d=2, **kw)
    a.surrogate_config(**cfg)
    a.run(150, "surrogate")
    a.sync()
    saved = (a.x.cpu().clone(), a.m, a.surrogate_save())
    a.close()
    b = rbm.System(saved[0].cuda(), d=2, **kw)
    b.surrogate_config(**cfg)
    b.surrogate_load(saved[2])
    b.m = saved[1]
    b.run(150, "surrogate")
    whole.sync()
    b.sync()
    assert torch.equal(b.x, whole.x)
    sa, sb = whole.surrogate_stats(), b.surrogate_stats()
    assert sa == sb, (sa, sb)
    with pytest.raises(rbm.RbmError):
        b.surrogate_load(saved[2][:100])            # a short buffer is refused
