"""RBM-r (Algorithm "fullyrandom") on the GPU against the sequential FP64
oracle: the sets bit-exact, whole steps (floor(N/p) iterations each, run in
conflict-free rounds on the GPU) within the FP64 bar, the FP32 build per
step, p = N against the direct step, and graph replay against eager steps."""
import numpy as np
import pytest

import oracle
import paper_1812_10575_gb300 as rbm
import workloads
from gpu_util import EPS32, as_run_precision, assert_close_per_particle, from_dev, to_dev, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,p", [(2, 2), (7, 3), (1000, 2), (4099, 8), (300, 32), (32, 32)])
def test_rbmr_sets_bit_exact(n, p):
    torch_cuda()
    X = workloads.gaussian(n, 2, seed=0)
    s = rbm.System(to_dev(X, "f64"), d=2, p=p, seed=13)
    prm = oracle.make_params(n, 2, p=p, seed=13)
    K = oracle.rbmr_iterations_per_step(prm)
    assert s.rbmr_info()["iterations_per_step"] == K
    for m in (0, 5):
        got = s.rbmr_sets(m).cpu().numpy().view(np.uint32)
        want = np.stack([oracle.rbmr_set(prm, m * K + j) for j in range(K)])
        assert np.array_equal(got, want), (n, p, m)


CASES = [
    dict(n=1000, d=2, p=2, dt=1e-2, sigma=0.1, v="quadratic", k="gauss_agg"),
    dict(n=1000, d=3, p=3, dt=1e-3, sigma=0.2, v="quadratic", k="reg_attract", k_param=0.01),
    dict(n=777, d=1, p=8, dt=1e-3, sigma=0.1, v="quadratic", k="smooth_test"),
    dict(n=640, d=2, p=32, dt=1e-2, sigma=0.05, v="zero", k="bounded_conf", k_param=0.25),
    dict(n=500, d=3, p=2, dt=1e-4, sigma=0.0, v="zero", k="coulomb", renorm=True),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c['k']}-d{c['d']}-p{c['p']}")
def test_rbmr_fp64_three_steps(case):
    torch_cuda()
    case = dict(case)
    n, d = case.pop("n"), case.pop("d")
    X = workloads.sphere(n, 3, seed=1) if case.get("renorm") else workloads.gaussian(n, d, seed=1)
    x = to_dev(X, "f64")
    s = rbm.System(x, d=d, seed=21, **case)
    s.run(3, "rbmr")
    s.sync()
    info = s.rbmr_info()
    assert info["rounds_last"] >= 1
    prm = oracle.make_params(n, d, seed=21, **case)
    ref = oracle.run(prm, X, 0, 3, method="rbmr")
    assert_close_per_particle(from_dev(x, d), ref, 1e-10, what=str(case))
    assert s.m == 3


def test_rbmr_fp32_one_step():
    torch_cuda()
    n, d = 4096, 3
    kw = dict(p=2, dt=1e-3, sigma=0.2, v="quadratic", k="reg_attract", k_param=0.01)
    X = as_run_precision(workloads.gaussian(n, d, seed=2), "f32")
    x = to_dev(X, "f32")
    s = rbm.System(x, d=d, seed=4, **kw)
    s.run(1, "rbmr")
    s.sync()
    prm = oracle.make_params(n, d, seed=4, precision="f32", **kw)
    ref = oracle.rbmr_step(prm, X, 0)
    # a particle may be moved several times within the step, each move adding
    # its FP32 rounding; 4 moves of at most a few ulp of |x| and of dt |F|
    extra = 64.0 * EPS32 * (np.abs(ref).max(axis=1) + 1.0)
    assert_close_per_particle(from_dev(x, d), ref, 1e-5, extra=extra, what="fp32 RBM-r step")


def test_rbmr_p_equals_n_is_the_direct_step():
    """p = N, sigma = 0: one iteration per step, its set is everyone: a direct step."""
    torch_cuda()
    n, d = 24, 2
    kw = dict(p=n, dt=1e-2, sigma=0.0, v="quadratic", k="reg_attract", k_param=0.1)
    X = workloads.gaussian(n, d, seed=3)
    x = to_dev(X, "f64")
    s = rbm.System(x, d=d, seed=2, **kw)
    s.run(1, "rbmr")
    s.sync()
    assert s.rbmr_info() == {"iterations_per_step": 1, "rounds_last": 1}
    ref = oracle.direct_step(oracle.make_params(n, d, seed=2, **kw), X, 0)
    assert_close_per_particle(from_dev(x, d), ref, 1e-12, what="p = N")


def test_rbmr_graph_replay_equals_eager():
    torch = torch_cuda()
    n, d = 3000, 2
    kw = dict(p=4, dt=1e-2, sigma=0.1, seed=8, v="quadratic", k="gauss_agg")
    X = workloads.gaussian(n, d, seed=4)
    xa, xb = to_dev(X, "f32"), to_dev(X, "f32")
    a, b = rbm.System(xa, d=d, **kw), rbm.System(xb, d=d, **kw)
    a.set_tuning(graph_steps=10)
    a.run(25, "rbmr")               # 2 graph replays + 5 eager steps
    for _ in range(25):
        b.run(1, "rbmr")
    a.sync()
    b.sync()
    assert a.m == 25 and torch.equal(xa, xb)


def test_rbmr_rejects_what_it_does_not_do():
    torch = torch_cuda()
    X = workloads.sphere(100, 3, seed=5)
    s = rbm.System(to_dev(X, "f64"), d=3, p=2, scheme="split", k="coulomb", dt=1e-4)
    with pytest.raises(rbm.RbmError) as e:
        s.run(1, "rbmr")
    assert e.value.status == -7
    big = rbm.System(torch.zeros(100, 2, dtype=torch.float64, device="cuda"), d=2, p=40)
    with pytest.raises(rbm.RbmError):
        big.run(1, "rbmr")
