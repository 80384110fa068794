"""Pins of the oracle's path coupling across step sizes (``noise_refine``):
a run with step dt and refinement r draws each step's Brownian increment as
the normalised sum of the r increments a run with step dt/r draws over the
same interval, so runs with different dt see one Brownian path (the
synchronous coupling of Sec. 3, eq. "coupling", extended to the fine-step
reference of Sec. 4.1).

What fixes it, independently of the formula:
- a pure Brownian motion (no force) is the sum of its increments, so the
  coarse run must land exactly where the fine run lands at the same time;
  a wrong fine-step index or a wrong scale fails this;
- Euler-Maruyama has strong order 1 for additive noise (Kloeden & Platen,
  Thm. 10.3.5 with constant diffusion): on one Brownian path the gap to a
  fine run shrinks linearly in dt; with independent paths it does not shrink;
- each refined increment is still standard normal.
"""
import numpy as np

import oracle
import workloads


def _no_force(n, d, dt, r, seed=5):
    return oracle.make_params(n, d, p=2, dt=dt, sigma=0.7, seed=seed, v="zero", k="linear", k_param=0.0,
                              noise_refine=r)


def test_pure_brownian_motion_is_the_sum_of_its_fine_increments():
    n, d, dt = 257, 3, 1e-3
    X0 = workloads.gaussian(n, d, seed=2)
    fine = oracle.run(_no_force(n, d, dt, 1), X0, 0, 24, "direct")
    for r in (2, 3, 4, 8):
        coarse = oracle.run(_no_force(n, d, dt * r, r), X0, 0, 24 // r, "direct")
        assert np.max(np.abs(coarse - fine)) < 1e-12, r
    # the RBM step with no interaction moves by the same increments
    coarse = oracle.run(_no_force(n, d, dt * 4, 4), X0, 0, 6, "rbm")
    assert np.max(np.abs(coarse - fine)) < 1e-12


def test_without_refinement_the_paths_differ():
    n, d, dt = 257, 2, 1e-3
    X0 = workloads.gaussian(n, d, seed=2)
    fine = oracle.run(_no_force(n, d, dt, 1), X0, 0, 8, "direct")
    plain = oracle.run(_no_force(n, d, dt * 4, 1), X0, 0, 2, "direct")
    assert np.sqrt(np.mean((plain - fine) ** 2)) > 0.01


def _ou_gap(refine_coupled, n=4000, T=0.5, seed=9):
    """RMS gap at T between Euler-Maruyama runs of dX = -X dt + dB at steps
    T/8, T/16, T/32 and a fine run at step T/512, on one Brownian path
    (refinement 512 dt_f / dt) or on independent ones (no refinement)."""
    X0 = workloads.gaussian(n, 1, seed=1)
    dt_f = T / 512
    ref = oracle.make_params(n, 1, p=2, dt=dt_f, sigma=1.0, seed=seed, v="quadratic", v_coef=1.0, k="linear",
                             k_param=0.0, noise_refine=1)
    Xf = oracle.run(ref, X0, 0, 512, "direct")
    gaps, dts = [], []
    for steps in (8, 16, 32):
        r = 512 // steps
        prm = oracle.make_params(n, 1, p=2, dt=T / steps, sigma=1.0, seed=seed, v="quadratic", v_coef=1.0,
                                 k="linear", k_param=0.0, noise_refine=r if refine_coupled else 1)
        Xc = oracle.run(prm, X0, 0, steps, "direct")
        gaps.append(np.sqrt(np.mean((Xc - Xf) ** 2)))
        dts.append(T / steps)
    return np.array(dts), np.array(gaps)


def test_coupled_euler_maruyama_converges_with_strong_order_one():
    dts, gaps = _ou_gap(True)
    slope = np.polyfit(np.log(dts), np.log(gaps), 1)[0]
    assert 0.8 < slope < 1.2, (gaps, slope)
    assert gaps[-1] < 0.01


def test_independent_paths_do_not_converge():
    dts, gaps = _ou_gap(False)
    # the gap is the spread of two independent OU paths, about sqrt(2 Var) ~ 0.9
    assert np.all(gaps > 0.5), gaps


def test_refined_increment_is_standard_normal():
    n = 200000
    for r in (1, 4, 16):
        prm = oracle.make_params(n, 2, p=2, dt=1e-3, sigma=1.0, seed=11, noise_refine=r)
        z = oracle.normals(prm, 3)
        assert abs(z.mean()) < 0.01
        assert abs(z.var() - 1.0) < 0.01
        assert abs(np.corrcoef(z[:, 0], z[:, 1])[0, 1]) < 0.01
    # a refined draw is not the plain draw of the same step
    a = oracle.normals(oracle.make_params(1000, 2, seed=11, noise_refine=1), 3)
    b = oracle.normals(oracle.make_params(1000, 2, seed=11, noise_refine=4), 3)
    assert np.max(np.abs(a - b)) > 0.1
