"""Pins of the Verlet oracle for the second-order system (Appendix A, eq.
"Hamil1"; the Verlet scheme of Sec. 4.1): free flight, the harmonic
oscillator's exact discrete solution, momentum conservation, RBM-1 with p = N
against the direct method, and the paper's slope-1/2 error decay (Fig.
"second")."""
import numpy as np
import pytest

import oracle
import workloads


def test_free_flight_is_exact():
    """b = 0, K = 0: X_n = X_0 + n tau V_0."""
    rng = np.random.default_rng(0)
    X0, V0 = rng.normal(size=(20, 3)), rng.normal(size=(20, 3))
    tau, n = 0.03, 25
    prm = oracle.make_params(20, 3, p=4, dt=tau, k="linear", k_param=0.0)
    X, P = oracle.verlet_run(prm, X0, V0, 0, n)
    np.testing.assert_allclose(X, X0 + n * tau * V0, rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(P, X0 + (n - 1) * tau * V0, rtol=1e-13, atol=1e-13)


def test_harmonic_oscillator_discrete_solution():
    """b(x) = -x, K = 0: X_{n+1} = (2 - tau^2) X_n - X_{n-1} has the solution
    X_n = X_0 cos(n theta) + tau V_0 sin(n theta) / sin(theta),
    cos(theta) = 1 - tau^2/2, fixed by X_0 and the Taylor start X_1."""
    rng = np.random.default_rng(1)
    X0, V0 = rng.normal(size=(8, 2)), rng.normal(size=(8, 2))
    tau, n = 0.1, 200
    prm = oracle.make_params(8, 2, p=2, dt=tau, v="quadratic", v_coef=1.0, k="linear", k_param=0.0)
    X, _ = oracle.verlet_run(prm, X0, V0, 0, n, method="direct")
    theta = np.arccos(1 - tau * tau / 2)
    want = X0 * np.cos(n * theta) + tau * V0 * np.sin(n * theta) / np.sin(theta)
    np.testing.assert_allclose(X, want, rtol=1e-10, atol=1e-10)


@pytest.mark.parametrize("method", ["rbm", "direct"])
def test_odd_kernel_conserves_momentum(method):
    """b = 0 and K odd: the centre of mass moves with the mean initial velocity."""
    rng = np.random.default_rng(2)
    X0, V0 = rng.normal(size=(30, 2)), rng.normal(size=(30, 2))
    tau, n = 0.01, 40
    prm = oracle.make_params(30, 2, p=3, dt=tau, k="smooth_test", seed=3)
    X, _ = oracle.verlet_run(prm, X0, V0, 0, n, method=method)
    np.testing.assert_allclose(X.mean(axis=0), X0.mean(axis=0) + n * tau * V0.mean(axis=0), atol=1e-12)


def test_rbm_with_p_equal_n_is_direct():
    rng = np.random.default_rng(4)
    X0, V0 = rng.normal(size=(12, 1)), rng.normal(size=(12, 1))
    prm = oracle.make_params(12, 1, p=12, dt=0.05, v="quadratic", k="smooth_test", seed=5)
    a, pa = oracle.verlet_run(prm, X0, V0, 0, 10, method="rbm")
    b, pb = oracle.verlet_run(prm, X0, V0, 0, 10, method="direct")
    assert np.array_equal(a, b) and np.array_equal(pa, pb)


@pytest.mark.slow
def test_rbm_error_decays_like_sqrt_tau():
    """Fig. "second": K(x) = x/(1 + x^2), b = 0, X_0 from the semicircle of
    radius 2, V_0 ~ N(0, 1), T = 1, p = 2; the error of RBM-1 against the
    direct method at a fine step (the paper's eq. "errorformula", averaged
    over random divisions) decays with slope about 1/2 in tau."""
    n, T = 500, 1.0
    X0 = workloads.semicircle(n, 2.0, seed=6)
    V0 = np.random.default_rng(7).normal(size=(n, 1))
    ref_tau = 2.0 ** -11
    prm_ref = oracle.make_params(n, 1, p=2, dt=ref_tau, k="smooth_test")
    Xref, _ = oracle.verlet_run(prm_ref, X0, V0, 0, int(round(T / ref_tau)), method="direct")
    taus = [2.0 ** -k for k in range(3, 8)]
    errs = []
    for tau in taus:
        e2 = []
        for seed in range(8):
            prm = oracle.make_params(n, 1, p=2, dt=tau, k="smooth_test", seed=100 + seed)
            X, _ = oracle.verlet_run(prm, X0, V0, 0, int(round(T / tau)), method="rbm")
            e2.append(np.mean((X - Xref) ** 2))
        errs.append(np.sqrt(np.mean(e2)))
    slope = np.polyfit(np.log(taus), np.log(errs), 1)[0]
    assert 0.35 < slope < 0.65, (slope, errs)
