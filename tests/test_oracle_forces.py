"""Pins of the oracle's interaction forces.

- hand-computed kernel values (tests/golden/worked_kernels.txt);
- Lemma "averagefunc" (Sec. 3) by brute force over all N! permutations:
  the RBM-1 force averaged over the random division equals the direct force,
  and its variance equals (1/(p-1) - 1/(N-1)) Lambda_i;
- RBM-1 with p = N is the direct step (eq. "firstalgorithm" vs eq.
  "interactingps"), bit for bit;
- odd kernels conserve the mean (pair forces cancel);
- K = 1/x: sum_i x_i F_i = N/2 for every division (each batch adds |C|/2).
"""
import itertools
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
ALL_K = ["inv1d", "coulomb", "bounded_conf", "gauss_agg", "reg_attract", "smooth_test", "linear"]


def _worked_rows():
    rows = []
    with open(os.path.join(GOLDEN, "worked_kernels.txt")) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if not line:
                continue
            a, b, c = line.split("|")
            kname, kparam, d, *xi = a.split()
            rows.append((kname, float(kparam), int(d), [float(v) for v in xi],
                         [float(v) for v in b.split()], [float(v) for v in c.split()]))
    return rows


@pytest.mark.parametrize("kname,kparam,d,xi,xj,expect", _worked_rows())
@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_kernel_worked_values(kname, kparam, d, xi, xj, expect, precision):
    prm = oracle.make_params(2, d, k=kname, k_param=kparam, precision=precision)
    got = oracle.kernel_pair(prm, xi, xj)
    np.testing.assert_allclose(got, expect, rtol=1e-14, atol=1e-15)


def _dims(kname):
    return [1] if kname == "inv1d" else [1, 2, 3]


@pytest.mark.parametrize("kname", ALL_K)
@pytest.mark.parametrize("n,p", [(6, 2), (6, 3), (6, 6)])
def test_lemma_averagefunc_bruteforce(kname, n, p):
    d = _dims(kname)[-1]
    rng = np.random.default_rng(hash((kname, n, p)) % 2**32)
    X = rng.standard_normal((n, d))
    prm = oracle.make_params(n, d, p=p, k=kname, k_param=0.8 if kname != "reg_attract" else 0.01)
    direct = oracle.direct_interaction(prm, X)
    perms = list(itertools.permutations(range(n)))
    forces = np.stack([oracle.rbm_interaction(prm, X, np.array(pm, dtype=np.uint32)) for pm in perms])
    mean = forces.mean(axis=0)
    np.testing.assert_allclose(mean, direct, rtol=1e-12, atol=1e-12)
    # variance: E|chi_i|^2 = (1/(p-1) - 1/(N-1)) Lambda_i
    var = ((forces - direct[None]) ** 2).sum(axis=2).mean(axis=0)
    Kij = np.zeros((n, n, d))
    for i in range(n):
        for j in range(n):
            if i != j:
                Kij[i, j] = oracle.kernel_pair(prm, X[i], X[j])
    lam = np.zeros(n)
    for i in range(n):
        for j in range(n):
            if j != i:
                lam[i] += np.sum((Kij[i, j] - direct[i]) ** 2)
    lam /= (n - 2)
    np.testing.assert_allclose(var, (1.0 / (p - 1) - 1.0 / (n - 1)) * lam, rtol=1e-10, atol=1e-12)


def test_singleton_last_batch_feels_no_interaction():
    n, p = 7, 2
    X = np.random.default_rng(1).standard_normal((n, 2))
    prm = oracle.make_params(n, 2, p=p, k="gauss_agg")
    perm = oracle.permutation(prm, 4)
    F = oracle.rbm_interaction(prm, X, perm)
    assert np.all(F[perm[-1]] == 0.0)
    assert np.all(np.abs(F[perm[:-1]]).sum(axis=1) > 0)


@pytest.mark.parametrize("kname", ALL_K)
def test_rbm_with_p_equal_n_is_the_direct_step(kname):
    d = _dims(kname)[-1]
    n = 50
    X = np.random.default_rng(3).standard_normal((n, d))
    prm = oracle.make_params(n, d, p=n, dt=1e-3, sigma=0.3, v="quadratic", v_coef=0.7, k=kname, k_param=0.9)
    a = oracle.rbm_step(prm, X, 12)
    b = oracle.direct_step(prm, X, 12)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("kname", ["coulomb", "bounded_conf", "gauss_agg", "reg_attract", "smooth_test", "linear"])
@pytest.mark.parametrize("p", [2, 3, 4])
def test_odd_kernel_conserves_mean(kname, p):
    n, d = 301, 3
    X = np.random.default_rng(4).standard_normal((n, d))
    prm = oracle.make_params(n, d, p=p, dt=1e-2, sigma=0.0, v="zero", k=kname, k_param=0.9)
    Y = X
    for m in range(5):
        Y = oracle.rbm_step(prm, Y, m)
    scale = np.abs(Y).max() * 5 * np.finfo(float).eps * n
    np.testing.assert_allclose(Y.mean(axis=0), X.mean(axis=0), atol=scale)
    Z = oracle.direct_step(prm, X, 0)
    np.testing.assert_allclose(Z.mean(axis=0), X.mean(axis=0), atol=scale)


@pytest.mark.parametrize("n,p", [(1000, 2), (1000, 4), (999, 4), (11, 3)])
def test_dyson_virial_identity(n, p):
    """K = 1/x: each batch C adds sum_{i != j in C} x_i/(x_i-x_j)/(|C|-1) = |C|/2."""
    X = np.random.default_rng(5).standard_normal((n, 1))
    prm = oracle.make_params(n, 1, p=p, k="inv1d")
    F = oracle.rbm_interaction(prm, X, oracle.permutation(prm, 2))
    last = n % p
    expect = n / 2.0 - (0.5 if last == 1 else 0.0)
    assert abs(np.sum(X * F) - expect) < 1e-9 * n * np.abs(X * F).max()
    Fd = oracle.direct_interaction(prm, X)
    assert abs(np.sum(X * Fd) - n / 2.0) < 1e-9 * n * np.abs(X * Fd).max()


def test_direct_forces_at_particles_equals_direct_interaction():
    n, d = 64, 2
    X = np.random.default_rng(6).standard_normal((n, d))
    prm = oracle.make_params(n, d, k="gauss_agg")
    np.testing.assert_array_equal(oracle.direct_forces_at(prm, X, X), oracle.direct_interaction(prm, X))
