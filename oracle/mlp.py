"""FP64 oracle of the mean-field surrogate: a d -> 64 -> 64 -> d tanh MLP (d = 2, 3) that
approximates the interaction force F(x) = 1/(N-1) sum_j K(x - X^j) (the mean-
field force K * mu of eq. "nonlinearfp" in arXiv:1812.10575, evaluated on the
empirical measure), its mean-squared-error gradient and one Adam step.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  The paper has no
surrogate; this module fixes the definitions the CUDA path must match:

  xh = (x - mu) / s                               input normalisation
  z1 = W1 xh + b1,       h1 = tanh(z1)            (64)
  z2 = W2 h1 + b2,       h2 = tanh(z2)            (64)
  y  = W3 h2 + b3                                 (d)
  F(x) = sF * y                                   output scale
  loss = 1/B sum_s |y_s - t_s|^2,  t_s = F_target,s / sF

Weights enter every product rounded to bfloat16 (the precision the tensor-core
kernels read them in); the hidden activations that feed the 64 x 64 products
(h1 forward; h1 and dz2 in the weight gradient; dz2 in dh1) are rounded to
bfloat16 as well.  Rounding is round-to-nearest-even of the float32 value.
Everything else is FP64.  Parameter vector layout (float32 masters, 4224 +
129 d: 4482 for d = 2, 4611 for d = 3): W1[64][d], b1[64], W2[64][64], b2[64],
W3[d][64], b3[d].  Normalisation vector: mu (d), s, sF.
"""
from __future__ import annotations

import numpy as np

H = 64


def sizes(d=2):
    return [("W1", (H, d)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (d, H)), ("b3", (d,))]


def n_params(d=2):
    return sum(int(np.prod(s)) for _, s in sizes(d))


SIZES = sizes(2)
N_PARAMS = n_params(2)


def dim_of(theta):
    """d of a parameter vector (its length is 4224 + 129 d)."""
    d = (len(theta) - 4224) // 129
    if d not in (2, 3) or n_params(d) != len(theta):
        raise ValueError(f"not a parameter vector of the d -> 64 -> 64 -> d network: {len(theta)}")
    return d


def unpack(theta):
    theta = np.asarray(theta, dtype=np.float64)
    out, o = {}, 0
    for name, shape in sizes(dim_of(theta)):
        k = int(np.prod(shape))
        out[name] = theta[o:o + k].reshape(shape)
        o += k
    return out


def pack(p):
    d = np.asarray(p["b3"]).size
    return np.concatenate([np.asarray(p[name], dtype=np.float64).ravel() for name, _ in sizes(d)])


def bf16(a):
    """Round to bfloat16 (nearest, ties to even) through float32; returns float64."""
    f = np.asarray(a, dtype=np.float64).astype(np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    nan = np.isnan(f)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    out = r.view(np.float32).astype(np.float64)
    out[nan] = np.nan
    return out


def forward(theta, x, norm, emulate_bf16=True):
    """Returns the output y (B x d) and the activations needed by backward."""
    p = unpack(theta)
    d = p["b3"].size
    q = bf16 if emulate_bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    mu, s = np.asarray(norm[:d], dtype=np.float64), float(norm[d])
    xh = (np.asarray(x, dtype=np.float64) - mu) / s
    z1 = xh @ q(p["W1"]).T + p["b1"]
    h1 = np.tanh(z1)
    z2 = q(h1) @ q(p["W2"]).T + p["b2"]
    h2 = np.tanh(z2)
    y = h2 @ q(p["W3"]).T + p["b3"]
    return y, dict(xh=xh, z1=z1, h1=h1, z2=z2, h2=h2)


def predict_force(theta, x, norm, emulate_bf16=True):
    y, _ = forward(theta, x, norm, emulate_bf16)
    return float(norm[len(norm) - 1]) * y


def loss_and_grad(theta, x, f_target, norm, emulate_bf16=True):
    """MSE loss and its gradient with respect to the float parameters."""
    p = unpack(theta)
    q = bf16 if emulate_bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    y, a = forward(theta, x, norm, emulate_bf16)
    t = np.asarray(f_target, dtype=np.float64) / float(norm[len(norm) - 1])
    B = y.shape[0]
    r = y - t
    loss = float(np.sum(r * r) / B)
    dy = 2.0 * r / B                                   # B x d
    g = {}
    g["W3"] = dy.T @ a["h2"]                           # d x 64
    g["b3"] = dy.sum(axis=0)
    dh2 = dy @ q(p["W3"])                              # B x 64
    dz2 = dh2 * (1.0 - a["h2"] * a["h2"])             # tanh' = 1 - tanh^2
    g["W2"] = q(dz2).T @ q(a["h1"])                    # 64 x 64
    g["b2"] = dz2.sum(axis=0)
    dh1 = q(dz2) @ q(p["W2"])                          # B x 64
    dz1 = dh1 * (1.0 - a["h1"] * a["h1"])
    g["W1"] = dz1.T @ a["xh"]                          # 64 x d
    g["b1"] = dz1.sum(axis=0)
    return loss, pack(g)


def lr_at(lr, it, iters, round_=0):
    """Rate of iteration it (0-based) of training round `round_` (0-based) of
    `iters` Adam steps: a geometric decay from lr/2^round_ to lr/(100 2^round_)
    over the round."""
    return lr * 0.5 ** round_ * 0.01 ** (it / max(iters - 1, 1))


def adam_step(theta, m, v, grad, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015) at step t >= 1; returns (theta, m, v)."""
    m = beta1 * np.asarray(m, dtype=np.float64) + (1.0 - beta1) * grad
    v = beta2 * np.asarray(v, dtype=np.float64) + (1.0 - beta2) * grad * grad
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    theta = np.asarray(theta, dtype=np.float64) - lr * mhat / (np.sqrt(vhat) + eps)
    return theta, m, v


def init_params(seed=0, d=2):
    """Initial parameters: each weight and bias of a layer uniform in
    +-c/sqrt(fan_in), c = 3 for the input layer and 1 otherwise (a seeded
    draw; the CUDA path draws its own start and tests load the same values
    into both sides)."""
    g = np.random.default_rng(np.random.SeedSequence([int(seed), 0x4D4C50]))
    p = {}
    for name, shape in sizes(d):
        fan_in = d if name in ("W1", "b1") else H
        c = 3.0 if name in ("W1", "b1") else 1.0
        p[name] = g.uniform(-1, 1, shape) * c / np.sqrt(fan_in)
    return pack(p).astype(np.float32).astype(np.float64)
