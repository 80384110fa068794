"""The wealth model (Sec. 5.2) on the GPU: multiplicative noise with the
Euler-Maruyama step and with the splitting scheme (exact pair exchange,
exact geometric step) against the FP64 oracle, and the paper's run (N = 1e5,
tau = 1e-3, T = 3, X0 = |N(0, 1)|) against the inverse Gamma equilibrium of
eq. "rhoinfty"."""
import numpy as np
import pytest
from scipy import stats

import oracle
import paper_1812_10575_gb300 as rbm
from gpu_util import EPS32, as_run_precision, assert_close_per_particle, from_dev, to_dev, torch_cuda

pytestmark = pytest.mark.gpu

WEALTH = dict(p=2, dt=1e-3, sigma=float(np.sqrt(2.0)), k="linear", k_param=1.0, gbm=True)


def _x0(n, seed=0):
    return np.abs(np.random.default_rng(seed).normal(size=(n, 1)))


@pytest.mark.parametrize("scheme,method", [("split", "split"), ("euler", "rbm")])
def test_wealth_fp64_ten_steps(scheme, method):
    torch_cuda()
    n = 3001
    X = _x0(n, 1)
    x = to_dev(X, "f64")
    s = rbm.System(x, d=1, seed=2, scheme=scheme, **WEALTH)
    s.run(10)
    s.sync()
    ref = oracle.run(oracle.make_params(n, 1, seed=2, **WEALTH), X, 0, 10, method=method)
    assert_close_per_particle(from_dev(x, 1), ref, 1e-10, what=scheme)


def test_wealth_direct_euler_fp64():
    torch_cuda()
    n = 1000
    X = _x0(n, 3)
    x = to_dev(X, "f64")
    s = rbm.System(x, d=1, seed=4, **WEALTH)
    for _ in range(3):
        s.direct_step()
    s.sync()
    ref = oracle.run(oracle.make_params(n, 1, seed=4, **WEALTH), X, 0, 3, method="direct")
    assert_close_per_particle(from_dev(x, 1), ref, 1e-10, what="direct")


def test_wealth_equilibrium_inverse_gamma():
    """FP32, N = 1e5, T = 3 with the splitting scheme: the empirical law is
    the inverse Gamma law of shape kappa/D + 1 = 2 and scale kappa eta / D."""
    torch_cuda()
    n = 100000
    X = as_run_precision(_x0(n, 5), "f32")
    x = to_dev(X, "f32")
    s = rbm.System(x, d=1, seed=6, scheme="split", **WEALTH)
    s.run(3000)
    s.sync()
    got = from_dev(x, 1).ravel()
    ks = stats.kstest(got, stats.invgamma(a=2.0, scale=X.mean()).cdf)
    assert ks.statistic < 0.01, ks
    assert np.all(got > 0)


def test_wealth_rejected_where_undefined():
    torch_cuda()
    s = rbm.System(to_dev(_x0(100), "f64"), d=1, **WEALTH)
    with pytest.raises(rbm.RbmError) as e:
        s.run(1, "rbmr")
    assert e.value.status == -7
