"""Path coupling across step sizes on the GPU (rbm_set_noise_refinement):
each step's Brownian increment is the normalised sum of the r increments of
a run with step dt/r, as the oracle draws it (``noise_refine``).

- FP64 runs with refinement within 1e-10 per particle of the oracle after
  10 steps: RBM-1 on each of the three step paths, the direct step, and a
  batched replica set;
- a pure Brownian motion stepped at 4 dt with refinement 4 lands where the
  run at dt lands (both on the GPU; FP64 to rounding, FP32 within a few ulp);
- RBM-r refuses a refined step, graphs captured before a change are not
  replayed with the old value, and bad values are rejected.
"""
import numpy as np
import pytest

import oracle
import paper_1812_10575_gb300 as rbm
import workloads
from gpu_util import assert_close_per_particle, from_dev, to_dev, torch_cuda

pytestmark = pytest.mark.gpu

KW = dict(p=2, dt=2e-3, sigma=0.3, v="quadratic", v_coef=1.0, k="reg_attract", k_param=0.01)


@pytest.mark.parametrize("path,n", [(1, 5000), (2, 5000), (3, 700)])
@pytest.mark.parametrize("r", [2, 5])
def test_rbm_fp64_ten_steps_with_refinement(path, n, r):
    torch_cuda()
    d = 3
    X = workloads.gaussian(n, d, seed=8)
    x = to_dev(X, "f64")
    s = rbm.System(x, d=d, seed=4, **KW)
    s.set_tuning(path=path, graph_steps=4)
    s.set_noise_refinement(r)
    s.run(10)                                   # two 4-step graph replays and two eager steps
    s.sync()
    ref = oracle.run(oracle.make_params(n, d, seed=4, noise_refine=r, **KW), X, 0, 10, "rbm")
    assert_close_per_particle(from_dev(x, d), ref, 1e-10, what=f"path {path} r {r}")


def test_direct_fp64_ten_steps_with_refinement():
    torch_cuda()
    n, d = 1500, 2
    X = workloads.gaussian(n, d, seed=8)
    x = to_dev(X, "f64")
    s = rbm.System(x, d=d, seed=4, **KW)
    s.set_noise_refinement(3)
    s.run(10, "direct")
    s.sync()
    ref = oracle.run(oracle.make_params(n, d, seed=4, noise_refine=3, **KW), X, 0, 10, "direct")
    assert_close_per_particle(from_dev(x, d), ref, 1e-10, what="direct")


def test_batched_fp64_with_refinement():
    torch_cuda()
    sizes = [2, 5, 300, 1001, 2048, 5000]
    d = 2
    X = workloads.unit_cube(sum(sizes), d, seed=0)
    x = to_dev(X, "f64")
    kw = dict(p=2, dt=1e-2, sigma=0.05, k="bounded_conf", k_param=0.25)
    rep = rbm.Replicas(x, sizes, d=d, seed=3, **kw)
    rep.set_noise_refinement(4)
    rep.run(6)
    rep.sync()
    got = from_dev(x, d)
    lo = 0
    for r, n in enumerate(sizes):
        prm = oracle.make_params(n, d, seed=3, replica=r, noise_refine=4, **kw)
        assert_close_per_particle(got[lo:lo + n], oracle.run(prm, X[lo:lo + n], 0, 6), 1e-10, what=f"replica {r}")
        lo += n


@pytest.mark.parametrize("dtype,tol", [("f64", 1e-12), ("f32", 4e-6)])
@pytest.mark.parametrize("method", ["rbm", "direct"])
def test_pure_brownian_motion_coarse_equals_fine_on_gpu(dtype, tol, method):
    torch_cuda()
    n, d, dt = 20000, 3, 1e-3
    X = workloads.gaussian(n, d, seed=1)
    kw = dict(p=2, sigma=0.5, v="zero", k="linear", k_param=0.0, seed=9)
    xf = to_dev(X, dtype)
    fine = rbm.System(xf, d=d, dt=dt, **kw)
    fine.run(24, method)
    fine.sync()
    xc = to_dev(X, dtype)
    coarse = rbm.System(xc, d=d, dt=4 * dt, **kw)
    coarse.set_noise_refinement(4)
    coarse.run(6, method)
    coarse.sync()
    a, b = from_dev(xc, d), from_dev(xf, d)
    assert np.max(np.abs(a - b)) <= tol * max(1.0, np.max(np.abs(b)))


def test_refinement_guards_and_graph_rebuild():
    torch = torch_cuda()
    n, d = 4000, 2
    X = workloads.gaussian(n, d, seed=2)
    x = to_dev(X, "f64")
    s = rbm.System(x, d=d, seed=1, **KW)
    s.set_tuning(graph_steps=5)
    s.run(5)                                    # captures a graph with r = 1
    s.set_noise_refinement(2)
    assert rbm.rbm_get_noise_refinement(s.ctx) == 2
    s.run(5)                                    # must not replay the r = 1 graph
    s.sync()
    prm1 = oracle.make_params(n, d, seed=1, **KW)
    prm2 = oracle.make_params(n, d, seed=1, noise_refine=2, **KW)
    ref = oracle.run(prm2, oracle.run(prm1, X, 0, 5), 5, 5)
    assert_close_per_particle(from_dev(x, d), ref, 1e-10, what="after the change")
    with pytest.raises(rbm.RbmError):
        s.set_noise_refinement(0)
    with pytest.raises(rbm.RbmError):
        s.run(1, "rbmr")                        # RBM-r draws its own increments
    s.set_noise_refinement(1)
    s.run(1, "rbmr")
    s.sync()
    del torch
