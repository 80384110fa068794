"""Pins of the RBM-r oracle (Sec. 2.2, Algorithm "fullyrandom"): the random
sets, one iteration against closed forms, conservation laws, the p = N case
against the direct step, and the stationary law of an Ornstein-Uhlenbeck
process that every iteration advances by tau."""
import itertools

import numpy as np
import pytest
from scipy import stats

import oracle


def test_sets_hold_p_distinct_ids_in_range():
    for n, p in [(2, 2), (5, 3), (40, 32), (1000, 8)]:
        prm = oracle.make_params(n, 2, p=p, seed=3)
        for k in range(200):
            s = oracle.rbmr_set(prm, k)
            assert len(set(s.tolist())) == p and s.max() < n


@pytest.mark.parametrize("p", [2, 3])
def test_sets_are_uniform_over_p_subsets(p):
    """Every unordered p-subset of 5 particles equally likely (chi-square)."""
    n, draws = 5, 20000
    prm = oracle.make_params(n, 1, p=p, seed=11)
    subsets = {c: i for i, c in enumerate(itertools.combinations(range(n), p))}
    counts = np.zeros(len(subsets))
    for k in range(draws):
        counts[subsets[tuple(sorted(oracle.rbmr_set(prm, k).tolist()))]] += 1
    assert stats.chisquare(counts).pvalue > 1e-3


def test_slot_order_is_uniform():
    """Each member equally likely in slot 0 (the draw order is random too)."""
    prm = oracle.make_params(4, 1, p=2, seed=2)
    first = np.bincount([oracle.rbmr_set(prm, k)[0] for k in range(8000)], minlength=4)
    assert stats.chisquare(first).pvalue > 1e-3


def test_linear_kernel_pair_contracts_by_one_minus_two_c_tau():
    """K(x) = -c x, V = 0, sigma = 0, p = 2: the pair's mean stays, their
    difference shrinks by (1 - 2 c tau); nobody else moves."""
    c, dt = 0.7, 0.05
    prm = oracle.make_params(10, 3, p=2, dt=dt, k="linear", k_param=c, seed=4)
    X = np.random.default_rng(0).normal(size=(10, 3))
    k = 17
    i, j = oracle.rbmr_set(prm, k)
    Y = oracle.rbmr_iteration(prm, X, k)
    np.testing.assert_allclose(Y[i] + Y[j], X[i] + X[j], rtol=0, atol=1e-14)
    np.testing.assert_allclose(Y[i] - Y[j], (1 - 2 * c * dt) * (X[i] - X[j]), rtol=1e-14, atol=1e-15)
    others = [q for q in range(10) if q not in (i, j)]
    assert np.array_equal(Y[others], X[others])


def test_p_equals_n_iteration_is_the_direct_step():
    """p = N: the only N-subset is everyone, one iteration per step, so with
    sigma = 0 an RBM-r step is the direct Euler step."""
    n = 9
    prm = oracle.make_params(n, 2, p=n, dt=1e-2, v="quadratic", k="reg_attract", k_param=0.1, seed=5)
    X = np.random.default_rng(1).normal(size=(n, 2))
    assert oracle.rbmr_iterations_per_step(prm) == 1
    np.testing.assert_allclose(oracle.rbmr_step(prm, X, 0), oracle.direct_step(prm, X, 0), rtol=1e-13, atol=1e-15)


def test_odd_kernel_conserves_the_mean():
    """V = 0, sigma = 0 and K odd: every iteration's forces cancel in pairs."""
    prm = oracle.make_params(50, 3, p=4, dt=1e-3, k="coulomb", seed=6)
    X = np.random.default_rng(2).normal(size=(50, 3))
    Y = oracle.run(prm, X, 0, 5, method="rbmr")
    np.testing.assert_allclose(Y.mean(axis=0), X.mean(axis=0), atol=1e-12)
    assert not np.allclose(Y, X)


def test_ou_stationary_variance():
    """V = |x|^2/2, no interaction (K = -0 x), sigma = 1: each update is
    x <- (1 - tau) x + sqrt(tau) z, whose stationary variance is 1/(2 - tau)
    however often a particle is picked."""
    n, dt = 4000, 0.05
    prm = oracle.make_params(n, 1, p=2, dt=dt, sigma=1.0, v="quadratic", k="linear", k_param=0.0, seed=7)
    Y = oracle.run(prm, np.zeros((n, 1)), 0, 150, method="rbmr")
    var = Y.var()
    se = np.sqrt(2.0 / n) / (2 - dt)
    assert abs(var - 1 / (2 - dt)) < 5 * se, (var, 1 / (2 - dt))


def test_iterations_run_in_order():
    """A particle in two consecutive sets moves twice, the second time from
    where the first left it: running the two iterations one after the other
    differs from applying both to the starting positions."""
    prm = oracle.make_params(3, 1, p=2, dt=0.1, k="linear", k_param=1.0, seed=8)
    X = np.array([[0.0], [1.0], [3.0]])
    k = next(k for k in range(100) if set(oracle.rbmr_set(prm, k)) & set(oracle.rbmr_set(prm, k + 1)))
    seq = oracle.rbmr_iteration(prm, oracle.rbmr_iteration(prm, X, k), k + 1)
    a, b = oracle.rbmr_iteration(prm, X, k), oracle.rbmr_iteration(prm, X, k + 1)
    simultaneous = X + (a - X) + (b - X)
    assert not np.allclose(seq, simultaneous)
