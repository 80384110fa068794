"""The learned mean-field surrogate (rbm_surrogate_*): its tensor-core forward
and gradient against the FP64 oracle (oracle/mlp.py, same bfloat16 operand
rounding), its training on the method's own trajectory, and what it gains over
RBM-1 at equal dt under the synchronous coupling of eq. "coupling"
(same X0, same Brownian increments).

Workload (aggregation with confinement): d = 2, V = |x|^2/2,
K(x) = -x exp(-|x|^2/2), sigma = 0.1, dt = 1e-3, X0 a 4-component Gaussian
mixture with means on the radius-3 circle and std 0.5.
"""
import numpy as np
import pytest

import oracle
from oracle import mlp
import paper_1812_10575_gb300 as rbm
import workloads
from gpu_util import from_dev, to_dev, torch_cuda

pytestmark = pytest.mark.gpu

AGG = dict(p=2, dt=1e-3, sigma=0.1, v="quadratic", k="gauss_agg")


def _system(n, seed=0, **extra):
    X = workloads.mixture(n, 2, seed=seed).astype(np.float32).astype(np.float64)
    x = to_dev(X, "f32")
    kw = dict(AGG)
    kw.update(extra)
    return rbm.System(x, d=2, **kw), x, X


def _params(seed):
    rng = np.random.default_rng(seed)
    theta = mlp.init_params(seed) + rng.normal(0, 0.02, mlp.N_PARAMS)
    return theta.astype(np.float32), np.array([0.3, -0.2, 2.5, 0.7], dtype=np.float32)


def test_surrogate_forward_matches_oracle():
    torch = torch_cuda()
    s, x, X = _system(1024)
    s.surrogate_config(n_queries=1024)
    theta, norm = _params(1)
    s.surrogate_set_params(theta, norm)
    Q = np.random.default_rng(2).normal(0, 3, (1000, 2)).astype(np.float32)
    f = s.surrogate_forces(torch.from_numpy(Q).cuda()).cpu().numpy().astype(np.float64)
    s.sync()
    ref = mlp.predict_force(theta, Q, norm, emulate_bf16=True)
    scale = np.sqrt(np.mean(ref ** 2))
    err = np.abs(f - ref).max() / scale
    assert err < 2e-3, err
    assert np.median(np.abs(f - ref)) / scale < 1e-5


def test_surrogate_gradient_matches_oracle():
    torch = torch_cuda()
    s, x, X = _system(1024)
    s.surrogate_config(n_queries=1024)
    theta, norm = _params(3)
    s.surrogate_set_params(theta, norm)
    rng = np.random.default_rng(4)
    xs = rng.normal(0, 3, (777, 2)).astype(np.float32)          # a ragged last tile
    ts = rng.normal(0, 1, (777, 2)).astype(np.float32)
    g, loss = s.surrogate_gradient(torch.from_numpy(xs).cuda(), torch.from_numpy(ts).cuda())
    ref_loss, ref_g = mlp.loss_and_grad(theta, xs, ts, norm, emulate_bf16=True)
    assert abs(loss - ref_loss) <= 1e-5 * abs(ref_loss)
    p_g, p_r = mlp.unpack(g), mlp.unpack(ref_g)
    for name, _ in mlp.SIZES:
        rel = np.linalg.norm(p_g[name] - p_r[name]) / max(np.linalg.norm(p_r[name]), 1e-30)
        assert rel < 1e-2, (name, rel)


def test_surrogate_network_step_at_full_size_sampled():
    """The network step at the size the benchmark times (N = 2^22, FP32,
    d = 2): every particle's force from the tensor-core network, then the
    Euler-Maruyama update.  The weights stay fixed (a checkpoint with no
    training iterations and a tolerance that always keeps the network), and
    4096 sampled particles after one step must match the oracle's network
    forward (same bfloat16 operand rounding) and update: 1e-5 relative plus
    dt times the forward's bar (2e-3 of the force scale)."""
    torch_cuda()
    n = 1 << 22
    s, x, X = _system(n, seed=5)
    s.surrogate_config(train_every=100, fallback_tol=1e30, n_queries=1024, iters_first=0, iters_per_checkpoint=0,
                       max_rounds=1, lr=1e-3)
    theta, norm = _params(6)
    s.surrogate_set_params(theta, norm)
    s.run(1, "surrogate")
    s.sync()
    st = s.surrogate_stats()
    assert st["surrogate_steps"] == 1 and st["fallback_steps"] == 0 and st["adam_steps"] == 0, st
    got = from_dev(x, 2)
    idx = np.sort(np.random.default_rng(7).choice(n, 4096, replace=False))
    prm = oracle.make_params(n, 2, seed=0, precision="f32", **AGG)
    FK = np.zeros_like(X)
    FK[idx] = mlp.predict_force(theta, X[idx].astype(np.float32), norm, emulate_bf16=True)
    ref = oracle.euler_update(prm, X, FK, 0)
    scale = np.sqrt(np.mean(FK[idx] ** 2))
    diff = np.linalg.norm(got[idx] - ref[idx], axis=1)
    bound = 1e-5 * np.maximum(np.linalg.norm(ref[idx], axis=1), 1.0) + AGG["dt"] * 2e-3 * scale
    assert np.all(diff <= bound), (diff.max(), bound.min())


def _sampled_ids(nq, n, m=0, seed=0, replica=0):
    """Query ids of a checkpoint at step m: floor(w0 n / 2^32) of the Philox
    block at counter (q, m, replica, stream 2)."""
    key = [seed & 0xFFFFFFFF, seed >> 32]
    return np.array([(int(oracle.philox4x32_10([q, m, replica, 2 * 256], key)[0]) * n) >> 32 for q in range(nq)])


def test_surrogate_training_call_matches_oracle():
    """One checkpoint of 3 Adam iterations from loaded parameters: the queries
    are the Philox-chosen particles, the targets their direct-sum forces, the
    update full-batch Adam with the rate decaying lr -> lr/10 -> lr/100; the
    parameters and the held-out error match the FP64 oracle's."""
    torch_cuda()
    n, nq, iters, lr = 2048, 1024, 3, 3e-3
    s, x, X = _system(n, seed=4)
    s.surrogate_config(n_queries=nq, lr=lr)
    theta, norm = _params(5)
    s.surrogate_set_params(theta, norm)
    s.surrogate_train(iters)
    th_gpu, norm_gpu = s.surrogate_params()
    st = s.surrogate_stats()
    np.testing.assert_array_equal(norm_gpu, norm)          # a given normalisation is kept

    ids = _sampled_ids(nq, n)
    Q = X[ids]
    F = oracle.direct_forces_at(oracle.make_params(n, 2, k="gauss_agg"), X, Q)
    ntr = 3 * nq // 4
    th = theta.astype(np.float64)
    m = v = np.zeros(mlp.N_PARAMS)
    for it in range(iters):
        _, g = mlp.loss_and_grad(th, Q[:ntr], F[:ntr], norm, emulate_bf16=True)
        th, m, v = mlp.adam_step(th, m, v, g, it + 1, lr=mlp.lr_at(lr, it, iters))
    d_orc, d_gpu = th - theta, th_gpu.astype(np.float64) - theta
    assert np.linalg.norm(d_gpu - d_orc) <= 0.05 * np.linalg.norm(d_orc)
    # elements whose gradient sign is decided by bfloat16-level noise may differ
    assert np.mean(np.abs(d_gpu - d_orc) > 0.05 * lr) < 0.02
    pred = mlp.predict_force(th, Q[ntr:], norm)
    rel = np.sqrt(np.sum((pred - F[ntr:]) ** 2) / np.sum(F[ntr:] ** 2))
    assert abs(st["rel_err"] - rel) <= 0.02 * rel + 1e-5, (st["rel_err"], rel)


SCHEDULE = dict(train_every=100, fallback_tol=1e-2, iters_first=12000, iters_per_checkpoint=2000, max_rounds=8,
                lr=3e-3)


def test_surrogate_trains_and_takes_over():
    """N = 2^16 and 2^14 queries: the first checkpoint trains until the
    held-out error is within 1e-2, so the network drives the whole first
    interval (100 steps)."""
    torch_cuda()
    s, x, X = _system(65536, seed=1)
    s.surrogate_config(n_queries=16384, **SCHEDULE)
    s.run(100, "surrogate")
    st = s.surrogate_stats()
    assert st["rel_err"] <= 1e-2 and st["active"], st
    assert st["surrogate_steps"] == 100 and st["fallback_steps"] == 0, st
    assert s.m == 100
    assert s.surrogate_drift()["drift_err"] == -1.0       # no later checkpoint yet
    got = from_dev(x, 2)
    assert np.all(np.isfinite(got))


def _drift_schedule(every, tol_ok, steps):
    """Checkpoint steps of the documented drift-aware schedule when every
    drift measurement is above the tolerance (tol_ok False) or within half
    of it (True)."""
    lo = max(1, every // 16)
    at, interval, m = [0], every, 0
    while True:
        m += interval
        if m >= steps:
            return at
        at.append(m)
        interval = min(every, 2 * interval) if tol_ok else max(lo, interval // 2)


def test_surrogate_drift_shortens_the_interval_and_falls_back():
    """The aggregation workload moves its clusters at speed ~|x|, so the
    network fitted at step 0 is ~50% off at step 100.  The checkpoint at step
    100 measures that drift on its fresh queries (it agrees with the error of
    the stale network over all particles, measured through the ABI); the
    interval then halves at every checkpoint down to train_every / 16 = 6
    steps, and since the drift over 6 steps still exceeds 1e-2 the RBM-1
    fallback takes over."""
    torch = torch_cuda()
    s, x, X = _system(65536, seed=2)
    s.surrogate_config(n_queries=16384, **dict(SCHEDULE, iters_per_checkpoint=500, max_rounds=2))
    s.run(100, "surrogate")
    s.sync()
    fd = s.forces("direct")                     # the network of step 0 at the positions of step 100
    fs = s.surrogate_forces(x.contiguous())
    stale = float(torch.sqrt(((fs - fd) ** 2).sum() / (fd ** 2).sum()))
    s.run(1, "surrogate")                       # checkpoint at step 100
    dr = s.surrogate_drift()
    assert dr["drift_err"] > 0.1 and abs(dr["drift_err"] - stale) <= 0.05 * stale, (dr, stale)
    assert dr["interval"] == 50 and not dr["forced_off"], dr
    s.run(199, "surrogate")                     # to step 300
    dr, st = s.surrogate_drift(), s.surrogate_stats()
    assert dr["forced_off"] and dr["interval"] == 6 and dr["forced_intervals"] >= 1, dr
    assert st["fallback_steps"] > 0 and st["surrogate_steps"] + st["fallback_steps"] == 300, st


def test_surrogate_gains_over_rbm_at_equal_dt():
    """E(T) = sqrt(mean |X_method - X_direct|^2) (eq. "errorformula") after 300
    steps from the same X0 with the same Brownian increments, N = 2^16.  The
    confinement carries the clusters towards the origin at speed ~|x|, so a
    network fitted to the force field of one instant is off by ~12% after 25
    steps and ~50% after 100; retrained every 25 steps (rounds of 1000 Adam
    iterations) its trajectory error is less than half the random-batch one."""
    torch_cuda()
    n, steps = 65536, 300
    ref, xr, X = _system(n, seed=2)
    rb, xb, _ = _system(n, seed=2)
    su, xs, _ = _system(n, seed=2)
    ref.run(steps, "direct")
    rb.run(steps, "rbm")
    su.surrogate_config(n_queries=16384, **dict(SCHEDULE, train_every=25, iters_per_checkpoint=1000))
    su.run(steps, "surrogate")
    for sysm in (ref, rb, su):
        sysm.sync()
    st = su.surrogate_stats()
    Xd, Xb, Xs = from_dev(xr, 2), from_dev(xb, 2), from_dev(xs, 2)
    e_rbm = np.sqrt(np.mean(np.sum((Xb - Xd) ** 2, axis=1)))
    e_sur = np.sqrt(np.mean(np.sum((Xs - Xd) ** 2, axis=1)))
    assert st["surrogate_steps"] >= 250 and st["surrogate_steps"] + st["fallback_steps"] == steps, st
    assert e_sur < 0.5 * e_rbm, (e_sur, e_rbm, st)


def test_surrogate_force_error_at_checkpoint_and_after():
    """Right after a checkpoint the network's force at every particle is
    within the tolerance of the direct sum (the held-out estimate holds on the
    whole system) and ~100x closer than the random-batch force (p = 2); the
    error then grows as the clusters move."""
    torch = torch_cuda()
    s, x, X = _system(65536, seed=2)
    s.surrogate_config(n_queries=16384, **SCHEDULE)
    s.run(100, "surrogate")                     # checkpoint at step 0 ... step 99
    s.surrogate_train(0)                        # fresh queries, no training: error after 100 steps
    drifted = s.surrogate_stats()["rel_err"]
    s.surrogate_train(4000)                     # retrained on the current positions
    s.sync()
    fd = s.forces("direct")
    fr = s.forces("rbm")
    fs = s.surrogate_forces(x.contiguous())

    def rel(a):
        return float(torch.sqrt(((a - fd) ** 2).sum() / (fd ** 2).sum()))

    assert rel(fs) <= 1.5e-2, rel(fs)
    assert rel(fs) < 0.02 * rel(fr), (rel(fs), rel(fr))
    assert drifted > 0.1, drifted


def test_surrogate_falls_back_when_tolerance_is_unreachable():
    torch_cuda()
    s, x, X = _system(4096, seed=3)
    s.surrogate_config(train_every=50, fallback_tol=1e-9, n_queries=2048, iters_first=10, iters_per_checkpoint=5,
                       max_rounds=3)
    s.run(120, "surrogate")
    st = s.surrogate_stats()
    assert not st["active"] and st["surrogate_steps"] == 0 and st["fallback_steps"] == 120, st
    # every checkpoint runs all its rounds; the drift is never within the
    # tolerance, so the interval halves from 50 down to 3 steps
    later = len(_drift_schedule(50, False, 120)) - 1
    assert st["adam_steps"] == 10 + 2 * 5 + later * 3 * 5, (st, later)
    # the fallback steps are exactly RBM-1 steps
    t, y, _ = _system(4096, seed=3)
    t.run(120, "rbm")
    s.sync()
    t.sync()
    assert np.array_equal(x.cpu().numpy(), y.cpu().numpy())


# ---------------------------------------------------------------------------
# d = 3: the 3 -> 64 -> 64 -> 3 network on the large-N system (V = |x|^2/2,
# K(x) = -x/(|x|^2 + 0.01), sigma = 0.2, X0 ~ N(0, I)); rows of 4 floats.
# ---------------------------------------------------------------------------
LARGE = dict(p=2, dt=1e-3, sigma=0.2, v="quadratic", k="reg_attract", k_param=0.01)


def _system3(n, seed=0):
    X = workloads.gaussian(n, 3, seed=seed).astype(np.float32).astype(np.float64)
    x = to_dev(X, "f32")
    return rbm.System(x, d=3, **LARGE), x, X


def _params3(seed):
    rng = np.random.default_rng(seed)
    theta = mlp.init_params(seed, d=3) + rng.normal(0, 0.02, mlp.n_params(3))
    return theta.astype(np.float32), np.array([0.1, -0.2, 0.05, 1.1, 0.4], dtype=np.float32)


def _rows(torch, A):
    t = torch.zeros(A.shape[0], 4, dtype=torch.float32)
    t[:, :3] = torch.from_numpy(np.asarray(A, dtype=np.float32))
    return t.cuda()


def test_surrogate_3d_forward_matches_oracle():
    torch = torch_cuda()
    s, x, X = _system3(1024)
    s.surrogate_config(n_queries=1024)
    theta, norm = _params3(1)
    s.surrogate_set_params(theta, norm)
    got_theta, got_norm = s.surrogate_params()
    assert np.array_equal(got_theta, theta) and np.array_equal(got_norm, norm)
    Q = np.random.default_rng(2).normal(0, 1.5, (1000, 3)).astype(np.float32)
    f = s.surrogate_forces(_rows(torch, Q)).cpu().numpy()[:, :3].astype(np.float64)
    s.sync()
    ref = mlp.predict_force(theta, Q, norm, emulate_bf16=True)
    scale = np.sqrt(np.mean(ref ** 2))
    assert np.abs(f - ref).max() / scale < 2e-3
    assert np.median(np.abs(f - ref)) / scale < 1e-5


def test_surrogate_3d_gradient_matches_oracle():
    torch = torch_cuda()
    s, x, X = _system3(1024)
    s.surrogate_config(n_queries=1024)
    theta, norm = _params3(3)
    s.surrogate_set_params(theta, norm)
    rng = np.random.default_rng(4)
    xs = rng.normal(0, 1.5, (777, 3)).astype(np.float32)          # a ragged last tile
    ts = rng.normal(0, 0.5, (777, 3)).astype(np.float32)
    g, loss = s.surrogate_gradient(_rows(torch, xs), _rows(torch, ts))
    ref_loss, ref_g = mlp.loss_and_grad(theta, xs, ts, norm, emulate_bf16=True)
    assert abs(loss - ref_loss) <= 1e-5 * abs(ref_loss)
    p_g, p_r = mlp.unpack(g), mlp.unpack(ref_g)
    for name, _ in mlp.sizes(3):
        rel = np.linalg.norm(p_g[name] - p_r[name]) / max(np.linalg.norm(p_r[name]), 1e-30)
        assert rel < 1e-2, (name, rel)


def test_surrogate_3d_network_step_sampled():
    """One network step at N = 2^20 with fixed weights: sampled particles
    against the oracle's forward and update; the pad lane is preserved."""
    torch = torch_cuda()
    n = 1 << 20
    s, x, X = _system3(n, seed=5)
    x[:, 3] = 7.0
    s.surrogate_config(train_every=100, fallback_tol=1e30, n_queries=1024, iters_first=0, iters_per_checkpoint=0,
                       max_rounds=1, lr=1e-3)
    theta, norm = _params3(6)
    s.surrogate_set_params(theta, norm)
    s.run(1, "surrogate")
    s.sync()
    assert s.surrogate_stats()["surrogate_steps"] == 1
    assert bool(torch.all(x[:, 3] == 7.0))
    got = from_dev(x, 3)
    idx = np.sort(np.random.default_rng(7).choice(n, 4096, replace=False))
    prm = oracle.make_params(n, 3, seed=0, precision="f32", **LARGE)
    FK = np.zeros_like(X)
    FK[idx] = mlp.predict_force(theta, X[idx].astype(np.float32), norm, emulate_bf16=True)
    ref = oracle.euler_update(prm, X, FK, 0)
    scale = np.sqrt(np.mean(FK[idx] ** 2))
    diff = np.linalg.norm(got[idx] - ref[idx], axis=1)
    bound = 1e-5 * np.maximum(np.linalg.norm(ref[idx], axis=1), 1.0) + LARGE["dt"] * 2e-3 * scale
    assert np.all(diff <= bound), (diff.max(), bound.min())


def test_surrogate_3d_trains_and_drives_the_first_interval():
    torch_cuda()
    s, x, X = _system3(65536, seed=1)
    s.surrogate_config(n_queries=16384, **SCHEDULE)
    s.run(100, "surrogate")
    st = s.surrogate_stats()
    assert st["rel_err"] <= 1e-2 and st["active"] and st["surrogate_steps"] == 100, st
    assert np.all(np.isfinite(from_dev(x, 3)))
