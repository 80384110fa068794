"""Pins of the wealth model (Sec. 5.2, eq. "wealth" with phi(y) = y^2/2, so
K(x) = -kappa x, and multiplicative noise sqrt(2D) Y dB) in the oracle: the
exact pair exchange, the exact geometric Brownian sub-step, and the inverse
Gamma equilibrium of eq. "rhoinfty"."""
import numpy as np
from scipy import stats

import oracle


def test_pair_exchange_shrinks_the_gap_about_the_mean():
    """K(x) = -c x, p = 2: d(delta)/dt = -2 c delta, the pair's sum fixed."""
    c, dt = 0.8, 0.05
    prm = oracle.make_params(2, 1, p=2, dt=dt, k="linear", k_param=c)
    yi, yj = oracle.split_pair_solve(prm, np.array([3.0]), np.array([0.5]))
    np.testing.assert_allclose(yi + yj, 3.5, rtol=1e-15)
    np.testing.assert_allclose(yi - yj, 2.5 * np.exp(-2 * c * dt), rtol=1e-14)


def test_geometric_step_is_lognormal_with_mean_one():
    """No interaction: one splitting step from x = 1 is exp(-s^2/2 + s z),
    s = sigma sqrt(tau): log y ~ N(-s^2/2, s^2) and E y = 1."""
    n, dt, sigma = 200000, 0.05, np.sqrt(2.0)
    prm = oracle.make_params(n, 1, p=2, dt=dt, sigma=sigma, k="linear", k_param=0.0, gbm=True, seed=3)
    Y = oracle.rbm_split_step(prm, np.ones((n, 1)), 0).ravel()
    s2 = sigma * sigma * dt
    ly = np.log(Y)
    assert abs(ly.mean() + s2 / 2) < 5 * np.sqrt(s2 / n)
    assert abs(ly.var() - s2) < 5 * s2 * np.sqrt(2.0 / n)
    assert abs(Y.mean() - 1.0) < 5 * np.sqrt((np.exp(s2) - 1) / n)


def test_euler_noise_is_proportional_to_wealth():
    """Euler-Maruyama with multiplicative noise: a particle at 0 never moves
    when nothing acts on it, one at x moves by sigma sqrt(tau) x z."""
    prm = oracle.make_params(4, 1, p=2, dt=0.01, sigma=1.0, k="linear", k_param=0.0, gbm=True, seed=4)
    X = np.array([[0.0], [0.0], [2.0], [2.0]])
    Y = oracle.rbm_step(prm, X, 0)
    z = oracle.normals(prm, 0)
    np.testing.assert_array_equal(Y[:2], 0.0)
    np.testing.assert_allclose(Y[2:], X[2:] * (1.0 + 0.1 * z[2:]), rtol=1e-15)


def test_equilibrium_is_inverse_gamma():
    """kappa = D = 1, X0 = |N(0, 1)|, tau = 1e-3, T = 3 (the paper's run, with
    N = 2e4): the empirical law matches rho_inf of eq. "rhoinfty", the inverse
    Gamma law of shape kappa/D + 1 = 2 and scale kappa eta / D, eta the mean
    wealth."""
    n, dt, T = 20000, 1e-3, 3.0
    X0 = np.abs(np.random.default_rng(0).normal(size=(n, 1)))
    prm = oracle.make_params(n, 1, p=2, dt=dt, sigma=np.sqrt(2.0), k="linear", k_param=1.0, gbm=True, seed=1)
    X = oracle.run(prm, X0, 0, int(round(T / dt)), method="split").ravel()
    ks = stats.kstest(X, stats.invgamma(a=2.0, scale=X0.mean()).cdf)
    assert ks.statistic < 0.015, ks
