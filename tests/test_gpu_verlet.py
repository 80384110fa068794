"""The second-order system (Appendix A) by the Verlet scheme on the GPU
(RBM_SCHEME_VERLET) against the FP64 oracle: RBM-1 on both step paths and the
direct step, graph replay, FP32 per step, and the argument checks."""
import numpy as np
import pytest

import oracle
import paper_1812_10575_gb300 as rbm
import workloads
from gpu_util import EPS32, as_run_precision, assert_close_per_particle, from_dev, to_dev, torch_cuda

pytestmark = pytest.mark.gpu

PAPER_1D = dict(p=2, dt=2.0 ** -6, sigma=0.0, k="smooth_test")   # Sec. 4.1's second-order example


def _start(n, d, seed=0, dtype="f64"):
    X = workloads.semicircle(n, 2.0, seed=seed) if d == 1 else workloads.gaussian(n, d, seed=seed)
    V = np.random.default_rng(seed + 100).normal(size=(n, d))
    return as_run_precision(X, dtype), as_run_precision(V, dtype)


@pytest.mark.parametrize("path", [2, 1])
@pytest.mark.parametrize("case", [dict(n=2000, d=1, **PAPER_1D),
                                  dict(n=5000, d=3, p=4, dt=1e-2, sigma=0.0, v="quadratic", k="reg_attract",
                                       k_param=0.1)],
                         ids=["paper-1d", "d3-p4"])
def test_verlet_rbm_fp64_ten_steps(case, path):
    torch_cuda()
    case = dict(case)
    n, d = case.pop("n"), case.pop("d")
    X, V = _start(n, d, seed=1)
    x, v = to_dev(X, "f64"), to_dev(V, "f64")
    s = rbm.System(x, d=d, seed=9, scheme="verlet", **case)
    s.set_tuning(path=path)
    if s.tuning()["path"] != path:
        pytest.skip("step path not available at this size")
    s.verlet_set_velocity(v)
    s.run(10)
    s.sync()
    Xr, _ = oracle.verlet_run(oracle.make_params(n, d, seed=9, **case), X, V, 0, 10, method="rbm")
    assert_close_per_particle(from_dev(x, d), Xr, 1e-10, what=f"path {path}")


def test_verlet_direct_fp64_five_steps():
    torch_cuda()
    n, d = 1500, 2
    kw = dict(p=2, dt=1e-2, sigma=0.0, v="quadratic", k="gauss_agg")
    X, V = _start(n, d, seed=2)
    x, v = to_dev(X, "f64"), to_dev(V, "f64")
    s = rbm.System(x, d=d, seed=3, scheme="verlet", **kw)
    s.verlet_set_velocity(v)
    for _ in range(5):
        s.direct_step()
    s.sync()
    Xr, _ = oracle.verlet_run(oracle.make_params(n, d, seed=3, **kw), X, V, 0, 5, method="direct")
    assert_close_per_particle(from_dev(x, d), Xr, 1e-10, what="direct")


def test_verlet_graph_replay_equals_eager_and_restart():
    """25 steps from graphs equal 25 eager steps; setting the velocities again
    makes the next step a Taylor start at the new step index."""
    torch = torch_cuda()
    n, d = 3000, 1
    X, V = _start(n, d, seed=4, dtype="f32")
    xa, xb, v = to_dev(X, "f32"), to_dev(X, "f32"), to_dev(V, "f32")
    a = rbm.System(xa, d=d, seed=5, scheme="verlet", **PAPER_1D)
    b = rbm.System(xb, d=d, seed=5, scheme="verlet", **PAPER_1D)
    a.set_tuning(graph_steps=10)
    a.verlet_set_velocity(v)
    b.verlet_set_velocity(v)
    a.run(25)
    for _ in range(25):
        b.step()
    a.sync()
    b.sync()
    assert torch.equal(xa, xb)
    # restart at step 25 with zero velocity: one step is x + dt^2 F / 2
    X25 = from_dev(xa, d)
    a.verlet_set_velocity(torch.zeros_like(xa))
    a.step()
    a.sync()
    prm = oracle.make_params(n, d, seed=5, precision="f32", **PAPER_1D)
    FK = oracle.rbm_interaction(prm, X25, oracle.permutation(prm, 25))
    want = X25 + 0.5 * PAPER_1D["dt"] ** 2 * FK
    assert_close_per_particle(from_dev(xa, d), want, 1e-6, what="restart")


def test_verlet_fp32_one_step():
    torch_cuda()
    n, d = 4096, 3
    kw = dict(p=2, dt=1e-2, sigma=0.0, v="quadratic", k="reg_attract", k_param=0.1)
    X, V = _start(n, d, seed=6, dtype="f32")
    x, v = to_dev(X, "f32"), to_dev(V, "f32")
    s = rbm.System(x, d=d, seed=7, scheme="verlet", **kw)
    s.verlet_set_velocity(v)
    s.step()
    s.sync()
    prm = oracle.make_params(n, d, seed=7, precision="f32", **kw)
    Xr, _ = oracle.verlet_run(prm, X, V, 0, 1, method="rbm")
    extra = 8.0 * EPS32 * (np.abs(X).max(axis=1) + kw["dt"] * np.abs(V).max(axis=1) + 1.0)
    assert_close_per_particle(from_dev(x, d), Xr, 1e-5, extra=extra, what="fp32 Verlet")


def test_verlet_argument_checks():
    torch = torch_cuda()
    x = to_dev(workloads.gaussian(100, 2, seed=0), "f64")
    with pytest.raises(rbm.RbmError) as e:
        rbm.System(x, d=2, p=2, sigma=0.1, scheme="verlet")      # the system carries no noise
    assert e.value.status == -1
    s = rbm.System(x, d=2, p=2, scheme="verlet")
    with pytest.raises(rbm.RbmError) as e:
        s.step()                                                 # no velocities yet
    assert e.value.status == -6
    euler = rbm.System(x.clone(), d=2, p=2)
    with pytest.raises(rbm.RbmError) as e:
        euler.verlet_set_velocity(torch.zeros_like(x))
    assert e.value.status == -6
