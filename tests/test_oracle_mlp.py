"""Pins of the surrogate-network oracle (oracle/mlp.py): the gradient against
central finite differences, a hand-built network with a known output, the
bfloat16 rounding against torch's own conversion, and Adam's first step."""
import numpy as np
import pytest

from oracle import mlp


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    theta = mlp.init_params(3) * 0.7 + rng.normal(0, 0.05, mlp.N_PARAMS)
    x = rng.normal(0, 1.5, (40, 2))
    t = rng.normal(0, 1, (40, 2))
    norm = np.array([0.1, -0.2, 1.3, 0.8])
    _, g = mlp.loss_and_grad(theta, x, t, norm, emulate_bf16=False)
    idx = rng.choice(mlp.N_PARAMS, 120, replace=False)
    h = 1e-6
    for i in idx:
        e = np.zeros(mlp.N_PARAMS)
        e[i] = h
        lp, _ = mlp.loss_and_grad(theta + e, x, t, norm, emulate_bf16=False)
        lm, _ = mlp.loss_and_grad(theta - e, x, t, norm, emulate_bf16=False)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 + 1e-6 * abs(fd), (i, fd, g[i])


def test_hand_built_network_computes_known_function():
    """W1 = [[1,0],[-1,0],[0,1],[0,-1],0...], W2 = I, W3 picks |x0| - |x1|
    through relu(x) + relu(-x) = |x|; with mu = 0, s = 1, sF = 2."""
    p = {k: np.zeros(s) for k, s in mlp.SIZES}
    p["W1"][0] = [1, 0]
    p["W1"][1] = [-1, 0]
    p["W1"][2] = [0, 1]
    p["W1"][3] = [0, -1]
    p["W2"] = np.eye(mlp.H)
    p["W3"][0, :4] = [1, 1, -1, -1]
    p["W3"][1, :4] = [0, 0, 1, 1]
    p["b3"] = [0.5, 0.0]
    theta = mlp.pack(p)
    x = np.array([[0.75, -2.5], [-1.5, 0.25]])
    f = mlp.predict_force(theta, x, np.array([0.0, 0.0, 1.0, 2.0]))
    # y0 = |x0| - |x1| + 0.5, y1 = |x1|; F = 2 y (all values exact in bfloat16)
    np.testing.assert_array_equal(f, [[2 * (0.75 - 2.5 + 0.5), 2 * 2.5], [2 * (1.5 - 0.25 + 0.5), 2 * 0.25]])


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    v = np.random.default_rng(1).normal(0, 10, 10000)
    v = np.concatenate([v, [0.0, -0.0, 1.0, 3.0e38, 1e-40, 1.00390625, 1.01171875]])
    ref = torch.tensor(v, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(mlp.bf16(v), ref)


def test_adam_first_step_moves_each_parameter_by_lr():
    """At t = 1 the bias-corrected step is lr * g/(|g| + eps) ~ lr sign(g)."""
    g = np.array([0.3, -2.0, 1e-3, 0.0])
    th, m, v = mlp.adam_step(np.zeros(4), np.zeros(4), np.zeros(4), g, 1, lr=0.01)
    np.testing.assert_allclose(th[:3], -0.01 * np.sign(g[:3]), rtol=1e-4)
    assert th[3] == 0.0
