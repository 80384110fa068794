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


def test_saturated_network_computes_known_function():
    """Weights large enough that every tanh saturates to exactly +-1 or sits
    at tanh(0) = 0, so the output is a known step function of the input; W2 is
    not symmetric, so a transposed W2 changes the answer.  All weights are
    exact in bfloat16.  mu = (0.5, -0.25), s = 2, sF = 4."""
    p = {k: np.zeros(s) for k, s in mlp.SIZES}
    p["W1"][0] = [256, 0]           # h1[0] = sign(x0 - 0.5)
    p["W1"][1] = [0, 256]           # h1[1] = sign(x1 + 0.25)
    p["W1"][2] = [256, 256]         # h1[2] = sign(x0 + x1 - 0.25)
    p["b1"][3] = 64                 # h1[3] = 1
    p["W2"][5, 0] = 512             # h2[5] = h1[0]
    p["W2"][6, 1] = -512            # h2[6] = -h1[1]
    p["W2"][7, 2] = 512
    p["W2"][7, 3] = 512             # h2[7] = 1 if h1[2] = 1 else tanh(0) = 0
    p["W3"][0, 5:8] = [1, 2, 0.5]
    p["W3"][1, 5:8] = [-1, 0, 4]
    p["b3"] = [0.25, -0.5]
    theta = mlp.pack(p)
    x = np.array([[1.5, 0.75], [-1.0, 0.5], [0.0, -2.0], [3.0, -1.0]])
    f = mlp.predict_force(theta, x, np.array([0.5, -0.25, 2.0, 4.0]))
    # (h2[5], h2[6], h2[7]) = (+1, -1, 1), (-1, -1, 0), (-1, +1, 0), (+1, +1, 1)
    want = 4 * np.array([[1 - 2 + 0.5 + 0.25, -1 + 4 - 0.5],
                         [-1 - 2 + 0.25, 1 - 0.5],
                         [-1 + 2 + 0.25, 1 - 0.5],
                         [1 + 2 + 0.5 + 0.25, -1 + 4 - 0.5]])
    np.testing.assert_array_equal(f, want)


def test_tanh_layers_at_closed_form_points():
    """tanh(ln a) = (a^2 - 1)/(a^2 + 1): an input of ln 2 gives h1 = 3/5 and
    W2 = ln 3 / 0.6 gives h2 = tanh(ln 3) = 4/5 (FP64, no bfloat16)."""
    p = {k: np.zeros(s) for k, s in mlp.SIZES}
    p["W1"][9] = [0, 1]
    p["W2"][4, 9] = np.log(3.0) / 0.6
    p["W3"][:, 4] = [1.0, -3.0]
    p["b3"] = [0.5, 0.0]
    f = mlp.predict_force(mlp.pack(p), np.array([[7.0, np.log(2.0)]]), np.array([0.0, 0.0, 1.0, 2.0]),
                          emulate_bf16=False)
    np.testing.assert_allclose(f, [[2 * (0.8 + 0.5), 2 * (-2.4)]], rtol=1e-13)


def test_small_inputs_see_the_linearised_network():
    """Zero biases and |z| ~ 1e-4: tanh(z) = z - z^3/3 + ..., so the force is
    sF W3 W2 W1 (x - mu)/s to relative O(z^2)."""
    rng = np.random.default_rng(5)
    p = {k: np.zeros(s) for k, s in mlp.SIZES}
    p["W1"] = rng.normal(0, 1, (mlp.H, 2))
    p["W2"] = rng.normal(0, 0.3, (mlp.H, mlp.H))
    p["W3"] = rng.normal(0, 1, (2, mlp.H))
    mu, s, sF = np.array([1.0, -2.0]), 3.0, 0.7
    x = mu + s * rng.normal(0, 1e-5, (5, 2))
    f = mlp.predict_force(mlp.pack(p), x, np.array([mu[0], mu[1], s, sF]), emulate_bf16=False)
    lin = sF * ((x - mu) / s) @ (p["W3"] @ p["W2"] @ p["W1"]).T
    np.testing.assert_allclose(f, lin, rtol=1e-6)


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


def test_three_dimensional_gradient_matches_finite_differences():
    rng = np.random.default_rng(5)
    d = 3
    theta = mlp.init_params(4, d=3) * 0.7 + rng.normal(0, 0.05, mlp.n_params(3))
    assert len(theta) == 4611 and mlp.dim_of(theta) == 3
    x = rng.normal(0, 1.5, (40, d))
    t = rng.normal(0, 1, (40, d))
    norm = np.array([0.1, -0.2, 0.3, 1.3, 0.8])
    _, g = mlp.loss_and_grad(theta, x, t, norm, emulate_bf16=False)
    idx = np.concatenate([np.arange(0, 192, 7), rng.choice(len(theta), 60, replace=False),
                          np.arange(len(theta) - 195, len(theta))])   # W1, random, W3 and b3
    h = 1e-6
    for i in idx:
        e = np.zeros(len(theta))
        e[i] = h
        lp, _ = mlp.loss_and_grad(theta + e, x, t, norm, emulate_bf16=False)
        lm, _ = mlp.loss_and_grad(theta - e, x, t, norm, emulate_bf16=False)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 + 1e-6 * abs(fd), (i, fd, g[i])


def test_three_dimensional_saturated_network_uses_every_coordinate():
    """d = 3: hidden units that switch on the third coordinate and on mu_z,
    and an output row per coordinate (a swapped coordinate or a normalisation
    read from the d = 2 layout fails).  mu = (0, 0, 1), s = 2, sF = 3."""
    p = {k: np.zeros(s) for k, s in mlp.sizes(3)}
    p["W1"][0] = [0, 0, 256]        # h1[0] = sign(z - 1)
    p["W1"][1] = [256, 0, 0]        # h1[1] = sign(x)
    p["W2"][2, 0] = 512             # h2[2] = h1[0]
    p["W2"][3, 1] = 512             # h2[3] = h1[1]
    p["W3"][0, 2] = 1
    p["W3"][1, 3] = 2
    p["W3"][2, 2:4] = [1, 1]
    p["b3"] = [0.5, 0, -0.25]
    theta = mlp.pack(p)
    x = np.array([[1.0, 5.0, 2.0], [-1.0, 0.0, 0.5], [2.0, -3.0, 0.0]])
    f = mlp.predict_force(theta, x, np.array([0.0, 0.0, 1.0, 2.0, 3.0]))
    h = np.array([[1, 1], [-1, -1], [-1, 1]])      # (h2[2], h2[3]) per row
    want = 3 * np.stack([h[:, 0] + 0.5, 2 * h[:, 1], h[:, 0] + h[:, 1] - 0.25], axis=1)
    np.testing.assert_array_equal(f, want)
