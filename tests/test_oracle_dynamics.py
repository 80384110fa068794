"""Pins of the oracle's time stepping against what the paper and the
mathematics fix:

- Sec. 4.1 / Fig. "errdepN": RBM-1 (p=2) vs a fine direct forward-Euler
  reference for K(x) = x/(1+x^2), beta in {0,1}: error ~ sqrt(tau), the
  log-log slope close to 1/2;
- Sec. 4.2: the Dyson Brownian motion (K = 1/x, V = x^2/2, sigma^2 = 1/N)
  through the splitting scheme: the second moment obeys
  dm2/dt = -2 m2 + 1 + 1/N, the transient from a radius-2 semicircle follows
  eq. "analyticaldis" and the equilibrium is the semicircle of radius sqrt 2
  (eq. "semicircle");
- closed forms of the Euler recursion: Ornstein-Uhlenbeck variance,
  linear kernel contraction for RBM pairs and for the direct step;
- the exact pair solves of the splitting scheme against a fine numerical
  integration of the pair ODE;
- projection onto the sphere (Sec. 5.1).
"""
import numpy as np
import pytest

import oracle
import workloads


def semicircle_cdf(x, r2):
    r = np.sqrt(r2)
    x = np.clip(x, -r, r)
    return 0.5 + x * np.sqrt(np.maximum(r2 - x * x, 0.0)) / (np.pi * r2) + np.arcsin(x / r) / np.pi


def w1_to_cdf(samples, cdf, lo=-8.0, hi=8.0, n=160001):
    xs = np.linspace(lo, hi, n)
    s = np.sort(np.asarray(samples).ravel())
    femp = np.searchsorted(s, xs, side="right") / len(s)
    return np.trapezoid(np.abs(femp - cdf(xs)), xs)


@pytest.mark.slow
@pytest.mark.parametrize("beta", [0.0, 1.0])
def test_error_decays_like_sqrt_tau(beta):
    n = 500
    X0 = workloads.semicircle(n, 2.0, seed=1)
    ref = oracle.make_params(n, 1, p=2, dt=2.0**-12, v="quadratic", v_coef=beta, k="smooth_test")
    Xref = oracle.run(ref, X0, 0, 2**12, "direct")
    taus = [2.0**-7, 2.0**-6, 2.0**-5, 2.0**-4]
    errs = []
    for tau in taus:
        prm = oracle.make_params(n, 1, p=2, dt=tau, v="quadratic", v_coef=beta, k="smooth_test", seed=3)
        Y = oracle.run(prm, X0, 0, int(round(1.0 / tau)))
        errs.append(np.sqrt(np.mean((Y - Xref) ** 2)))     # eq. "errorformula"
    slope = np.polyfit(np.log(taus), np.log(errs), 1)[0]
    assert 0.35 < slope < 0.65, (errs, slope)
    assert errs[0] < 0.1


def _dyson(n, seed=0):
    return oracle.make_params(n, 1, p=2, dt=1e-3, sigma=np.sqrt(1.0 / n), v="quadratic", v_coef=1.0,
                              k="inv1d", seed=seed)


def test_dyson_second_moment_closed_form():
    n = 1000
    X0 = workloads.dyson(n, 0)
    prm = _dyson(n)
    X1 = oracle.run(prm, X0, 0, 1000, "split")
    minf = (1.0 + 1.0 / n) / 2.0
    m20 = np.mean(X0 ** 2)
    closed = minf + (m20 - minf) * np.exp(-2.0)
    assert abs(np.mean(X1 ** 2) - closed) < 5e-3


def test_dyson_transient_matches_analytic_density():
    n = 10000
    X0 = workloads.semicircle(n, 2.0, seed=2)
    X = oracle.run(_dyson(n, seed=5), X0, 0, 500, "split")
    s = 1.0 + np.exp(-1.0)                    # sigma(t) = 1 + e^{-2t}, t = 0.5
    assert w1_to_cdf(X, lambda x: semicircle_cdf(x, 2.0 * s)) < 0.015


@pytest.mark.slow
def test_dyson_equilibrium_is_semicircle_radius_sqrt2():
    n = 1000
    X = oracle.run(_dyson(n), workloads.dyson(n, 0), 0, 5000, "split")
    assert w1_to_cdf(X, lambda x: semicircle_cdf(x, 2.0)) < 0.04
    assert abs(np.mean(X ** 2) - (1.0 + 1.0 / n) / 2.0) < 0.03


def test_ou_variance_recursion():
    """K = 0, V = |x|^2/2: v' = (1-tau)^2 v + sigma^2 tau, from v0 = 0."""
    n, tau, sigma = 40000, 0.05, 0.7
    prm = oracle.make_params(n, 2, p=2, dt=tau, sigma=sigma, v="quadratic", v_coef=1.0, k="linear",
                             k_param=0.0, seed=8)
    X = np.zeros((n, 2))
    v = 0.0
    for m in range(30):
        X = oracle.rbm_step(prm, X, m)
        v = (1 - tau) ** 2 * v + sigma ** 2 * tau
    assert abs(X.var() - v) < 6 * v * np.sqrt(2.0 / (2 * n))
    assert abs(X.mean()) < 6 * np.sqrt(v / (2 * n))


def test_linear_kernel_pair_contraction_and_direct_contraction():
    n, d, tau, c = 200, 2, 0.01, 1.5
    X = np.random.default_rng(9).standard_normal((n, d))
    prm = oracle.make_params(n, d, p=2, dt=tau, k="linear", k_param=c)
    perm = oracle.permutation(prm, 0)
    Y = oracle.rbm_step(prm, X, 0)
    for q in range(n // 2):
        i, j = perm[2 * q], perm[2 * q + 1]
        np.testing.assert_allclose(Y[i] - Y[j], (X[i] - X[j]) * (1 - 2 * c * tau), rtol=1e-12)
        np.testing.assert_allclose(Y[i] + Y[j], X[i] + X[j], rtol=1e-12, atol=1e-14)
    Z = oracle.direct_step(prm, X, 0)
    mean = X.mean(axis=0)
    np.testing.assert_allclose(Z - mean, (X - mean) * (1 - c * tau * n / (n - 1)), rtol=1e-11, atol=1e-13)


def _integrate_pair(kname, xi, xj, tau, steps=200000):
    """Classical RK4 of dX^i = K(X^i - X^j), dX^j = K(X^j - X^i) over [0, tau]."""
    def f(a, b):
        x = a - b
        r = np.linalg.norm(x)
        return (1.0 / x) if kname == "inv1d" else x / r ** 3
    a, b = np.array(xi, float), np.array(xj, float)
    h = tau / steps
    for _ in range(steps):
        k1a, k1b = f(a, b), f(b, a)
        k2a, k2b = f(a + h / 2 * k1a, b + h / 2 * k1b), f(b + h / 2 * k1b, a + h / 2 * k1a)
        k3a, k3b = f(a + h / 2 * k2a, b + h / 2 * k2b), f(b + h / 2 * k2b, a + h / 2 * k2a)
        k4a, k4b = f(a + h * k3a, b + h * k3b), f(b + h * k3b, a + h * k3a)
        a, b = a + h / 6 * (k1a + 2 * k2a + 2 * k3a + k4a), b + h / 6 * (k1b + 2 * k2b + 2 * k3b + k4b)
    return a, b


@pytest.mark.parametrize("kname,d,xi,xj", [("inv1d", 1, [0.3], [0.25]), ("inv1d", 1, [-1.0], [0.2]),
                                           ("coulomb", 3, [0.1, 0.2, 0.0], [0.0, 0.25, 0.1])])
def test_split_pair_solve_is_the_exact_pair_flow(kname, d, xi, xj):
    tau = 1e-3
    prm = oracle.make_params(2, d, p=2, dt=tau, k=kname)
    yi, yj = oracle.split_pair_solve(prm, xi, xj)
    ai, aj = _integrate_pair(kname, xi, xj, tau, steps=4000)
    np.testing.assert_allclose(yi, ai, rtol=1e-9, atol=1e-11)
    np.testing.assert_allclose(yj, aj, rtol=1e-9, atol=1e-11)


def test_renormalisation_projects_to_sphere():
    n = 1000
    X = workloads.sphere(n, seed=3)
    prm = oracle.make_params(n, 3, p=2, dt=1e-4, k="coulomb", renorm=True)
    Y = oracle.rbm_step(prm, X, 0)
    np.testing.assert_allclose(np.linalg.norm(Y, axis=1), 1.0, rtol=4e-16 * 4)
