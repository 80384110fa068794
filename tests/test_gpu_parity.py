"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Bars (each test states which it checks):
  - permutation: bit-exact (integer work);
  - FP64 runs: every particle within 1e-10 * max(|x|, 1) of the oracle after
    10 steps;
  - FP32 runs: per step, every particle within 1e-5 * max(|x|, 1) plus the
    rounding of the interaction force, 32 eps32 dt |F^K_i| (divided by the
    pre-projection norm when positions are projected onto the sphere): a
    particle whose batch partner is very close feels a force so large that
    FP32 rounding of that force alone exceeds 1e-5; the bound follows the
    FP32 evaluation error of K (a few ulp) scaled by dt.
The oracle starts from exactly the values the run starts from (FP32 runs: the
float32 values), and for FP32 runs takes its kernel decisions on the FP32
squared norm and draws 24-bit uniforms, as the CUDA path does.
"""
import numpy as np
import pytest

import oracle
import paper_1812_10575_gb300 as rbm
import workloads
from gpu_util import EPS32, as_run_precision, assert_close_per_particle, from_dev, to_dev, torch_cuda

pytestmark = pytest.mark.gpu

ALL_K = ["inv1d", "coulomb", "bounded_conf", "gauss_agg", "reg_attract", "smooth_test", "linear"]
KPARAM = {"bounded_conf": 0.6, "reg_attract": 0.01, "linear": 0.8}


def kparam(k):
    return KPARAM.get(k, 0.0)


def _system(X, d, dtype, **kw):
    x = to_dev(X, dtype)
    return rbm.System(x, d=d, **kw), x


def _oprm(n, d, dtype, **kw):
    kw = dict(kw)
    kw.pop("scheme", None)
    return oracle.make_params(n, d, precision=dtype, **kw)


# ---------------------------------------------------------------------------
# permutation: bit-exact
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("path", [1, 2, 3])
@pytest.mark.parametrize("n,seed,m,r", [(2, 0, 0, 0), (3, 1, 5, 0), (7, 3, 9, 2), (513, 0, 1, 0), (1000, 0, 0, 0),
                                        (1001, 5, 17, 3), (4097, 9, 2**31 + 5, 1), (100000, 0, 123, 0),
                                        (300001, 2**40 + 7, 7, 0), (900000, 3, 1, 0)])
def test_permutation_bit_exact(n, seed, m, r, path):
    torch = torch_cuda()
    X = np.zeros((n, 1))
    s, _ = _system(X, 1, "f32", p=2, seed=seed, replica=r)
    s.set_tuning(path=path)
    assert s.tuning()["path"] == (1 if path == 3 and n > 2048 else path)   # one block: N <= 2048 only
    s.m = m
    perm = s.permutation().cpu().numpy().view(np.uint32)
    s.sync()
    expect = oracle.permutation(oracle.make_params(n, 1, seed=seed, replica=r), m)
    assert np.array_equal(perm, expect)
    assert s.m == m
    del torch


@pytest.mark.parametrize("tuning", [dict(path=1, bucket_bits=3, slot_cap=4, sort_cap=8),     # spill + counting
                                    dict(path=1, bucket_bits=6, slot_cap=8, sort_cap=4096),  # spill list in smem
                                    dict(path=1, bucket_bits=0, sort_cap=4096),              # one bucket
                                    dict(path=1, bucket_bits=12),                            # separate scan
                                    dict(path=2),                                            # cooperative kernel
                                    dict(path=2, slot_cap=8)])                               # ... regrouped compactly
@pytest.mark.parametrize("p", [2, 5, 40])
def test_permutation_and_step_under_forced_bucket_paths(tuning, p):
    n, d = 3000, 2
    X = workloads.gaussian(n, d, seed=4)
    kw = dict(p=p, dt=1e-2, sigma=0.1, seed=11, v="quadratic", k="gauss_agg")
    s, x = _system(X, d, "f64", **kw)
    s.set_tuning(**tuning)
    s.m = 3
    perm = s.permutation().cpu().numpy().view(np.uint32)
    prm = _oprm(n, d, "f64", **kw)
    assert np.array_equal(perm, oracle.permutation(prm, 3))
    s.step()
    s.sync()
    assert_close_per_particle(from_dev(x, d), oracle.rbm_step(prm, X, 3), 1e-12, what=str(tuning))


# ---------------------------------------------------------------------------
# interaction forces of one step (RBM and direct), FP64
# ---------------------------------------------------------------------------
def _cases():
    out = []
    for k in ALL_K:
        dims = [1] if k == "inv1d" else [1, 2, 3]
        for d in dims:
            for p in ([2, 3, 8, 33] if d == dims[-1] else [2, 4]):
                out.append((k, d, p))
    return out


@pytest.mark.parametrize("path", [1, 2, 3])
@pytest.mark.parametrize("k,d,p", _cases())
def test_rbm_and_direct_forces_fp64(k, d, p, path):
    n = 997
    X = workloads.gaussian(n, d, seed=d * 31 + p)
    kw = dict(p=p, seed=p, k=k, k_param=kparam(k))
    s, x = _system(X, d, "f64", **kw)
    s.set_tuning(path=path)
    s.m = 5
    f_rbm = from_dev(s.forces("rbm"), d)
    f_dir = from_dev(s.forces("direct"), d)
    perm = s.permutation().cpu().numpy().view(np.uint32)
    s.sync()
    prm = _oprm(n, d, "f64", **kw)
    assert np.array_equal(perm, oracle.permutation(prm, 5))
    assert_close_per_particle(f_rbm, oracle.rbm_interaction(prm, X, perm), 1e-12, what="rbm forces")
    assert_close_per_particle(f_dir, oracle.direct_interaction(prm, X), 1e-12, what="direct forces")


# ---------------------------------------------------------------------------
# FP64 trajectories: 10 steps within 1e-10
# ---------------------------------------------------------------------------
FP64_RUNS = [
    # Dyson Brownian motion (Sec. 4.2): N = 1000, V = x^2/2, K = 1/x, sigma^2 = 1/N, p = 2, dt = 1e-3
    ("dyson-split", 1000, 1, dict(p=2, dt=1e-3, sigma=np.sqrt(1e-3), v="quadratic", k="inv1d", scheme="split")),
    ("dyson-euler", 1000, 1, dict(p=2, dt=1e-3, sigma=np.sqrt(1e-3), v="quadratic", k="inv1d")),
    ("smooth-p4", 1001, 1, dict(p=4, dt=2**-7, v="quadratic", k="smooth_test")),
    ("gauss-p8", 1003, 2, dict(p=8, dt=1e-2, sigma=0.3, v="quadratic", k="gauss_agg")),
    ("bounded-p3", 1000, 2, dict(p=3, dt=1e-2, sigma=0.01, k="bounded_conf", k_param=0.25)),
    ("regattract-p2", 999, 3, dict(p=2, dt=1e-3, sigma=0.2, v="quadratic", k="reg_attract", k_param=0.01)),
    ("thomson-renorm", 1000, 3, dict(p=2, dt=1e-4, k="coulomb", renorm=True)),
    ("thomson-split", 1000, 3, dict(p=2, dt=1e-4, k="coulomb", renorm=True, scheme="split")),
    ("linear-p40", 1000, 2, dict(p=40, dt=1e-2, sigma=0.1, k="linear", k_param=1.0)),
]


def _initial(name, n, d):
    if name.startswith("dyson"):
        return workloads.dyson(n, 0)
    if name.startswith("thomson"):
        return workloads.sphere(n, d, seed=1)
    if name.startswith("bounded"):
        return workloads.unit_cube(n, d, seed=2)
    return workloads.gaussian(n, d, seed=3)


@pytest.mark.parametrize("path", [1, 2, 3])
@pytest.mark.parametrize("name,n,d,kw", FP64_RUNS, ids=[r[0] for r in FP64_RUNS])
def test_rbm_fp64_ten_steps(name, n, d, kw, path):
    X = _initial(name, n, d)
    s, x = _system(X, d, "f64", seed=0, **kw)
    s.set_tuning(path=path)
    s.run(10)
    s.sync()
    prm = _oprm(n, d, "f64", seed=0, **kw)
    ref = oracle.run(prm, X, 0, 10, "split" if kw.get("scheme") == "split" else "rbm")
    assert_close_per_particle(from_dev(x, d), ref, 1e-10, what=name)


DIRECT_10 = [r for r in FP64_RUNS if "split" not in r[0] and "p40" not in r[0] and r[0] != "dyson-euler"]


@pytest.mark.parametrize("name,n,d,kw", DIRECT_10, ids=[r[0] for r in DIRECT_10])
def test_direct_fp64_ten_steps(name, n, d, kw):
    X = _initial(name, n, d)
    kw = dict(kw)
    s, x = _system(X, d, "f64", seed=0, **kw)
    s.run(10, "direct")
    s.sync()
    ref = oracle.run(_oprm(n, d, "f64", seed=0, **kw), X, 0, 10, "direct")
    assert_close_per_particle(from_dev(x, d), ref, 1e-10, what=name)


def test_direct_fp64_dyson_euler_per_step():
    """Direct forward Euler on K = 1/x with sigma^2 = 1/N is chaotic at
    dt = 1e-3: two particles closer than ~1e-6 receive kicks of order one, so
    rounding differences grow by orders of magnitude within a few steps and a
    10-step trajectory comparison measures the conditioning, not the kernel.
    Each step is therefore compared from the GPU's own state, within 1e-10."""
    name, n, d, kw = [r for r in FP64_RUNS if r[0] == "dyson-euler"][0]
    X = _initial(name, n, d)
    s, x = _system(X, d, "f64", seed=0, **kw)
    prm = _oprm(n, d, "f64", seed=0, **kw)
    cur = X
    for m in range(10):
        s.direct_step()
        s.sync()
        got = from_dev(x, d)
        assert_close_per_particle(got, oracle.direct_step(prm, cur, m), 1e-10, what=f"dyson direct step {m}")
        cur = got


def test_p_equal_n_rbm_equals_direct_on_gpu():
    n, d = 700, 2
    X = workloads.gaussian(n, d, seed=9)
    kw = dict(p=n, dt=1e-3, sigma=0.2, v="quadratic", k="gauss_agg")
    a, xa = _system(X, d, "f64", **kw)
    b, xb = _system(X, d, "f64", **kw)
    a.step()
    b.direct_step()
    a.sync()
    b.sync()
    assert_close_per_particle(from_dev(xa, d), from_dev(xb, d), 1e-12, what="p = N")


# ---------------------------------------------------------------------------
# FP32: per-step parity
# ---------------------------------------------------------------------------
def _fp32_bound(prm, X, FK, m):
    """32 eps32 dt |F^K_i| (/ |u_i| with the projection, u the unprojected update)."""
    extra = 32.0 * EPS32 * prm.dt * np.linalg.norm(FK, axis=1)
    if prm.renorm:
        import copy

        p2 = copy.copy(prm)
        p2.renorm = 0
        u = oracle.euler_update(p2, X, FK, m)
        extra = extra / np.maximum(np.linalg.norm(u, axis=1), 1e-30) + 8 * EPS32
    return extra


FP32_RUNS = [
    # Thomson problem (Sec. 5.1): N = 1e5 on S^2, K = x/|x|^3, V = 0, sigma = 0, projection, p = 2, dt = 1e-4
    ("thomson-1e5", 100000, 3, dict(p=2, dt=1e-4, k="coulomb", renorm=True)),
    ("opinion-p4", 20000, 2, dict(p=4, dt=1e-2, sigma=0.01, k="bounded_conf", k_param=0.25)),
    ("aggregation", 65536, 2, dict(p=2, dt=1e-3, sigma=0.1, v="quadratic", k="gauss_agg")),
    ("regattract-p8", 65536, 3, dict(p=8, dt=1e-3, sigma=0.2, v="quadratic", k="reg_attract", k_param=0.01)),
    ("dyson-f32", 1000, 1, dict(p=2, dt=1e-3, sigma=np.sqrt(1e-3), v="quadratic", k="inv1d")),
]


def _initial32(name, n, d):
    if name.startswith("thomson"):
        return workloads.sphere(n, d, seed=0)
    if name.startswith("opinion"):
        return workloads.unit_cube(n, d, seed=0)
    if name.startswith("aggregation"):
        return workloads.mixture(n, d, seed=0)
    if name.startswith("dyson"):
        return workloads.dyson(n, 0)
    return workloads.gaussian(n, d, seed=0)


@pytest.mark.parametrize("path", [1, 2, 3])
@pytest.mark.parametrize("name,n,d,kw", FP32_RUNS, ids=[r[0] for r in FP32_RUNS])
def test_rbm_fp32_per_step(name, n, d, kw, path):
    X = as_run_precision(_initial32(name, n, d), "f32")
    s, x = _system(X, d, "f32", seed=1, **kw)
    s.set_tuning(path=path)
    prm = _oprm(n, d, "f32", seed=1, **kw)
    cur = X
    for m in range(3):
        s.step()
        s.sync()
        got = from_dev(x, d)
        perm = oracle.permutation(prm, m)
        FK = oracle.rbm_interaction(prm, cur, perm)
        ref = oracle.euler_update(prm, cur, FK, m)
        assert_close_per_particle(got, ref, 1e-5, extra=_fp32_bound(prm, cur, FK, m), what=f"{name} step {m}")
        cur = got


@pytest.mark.parametrize("p", [2, 16])
def test_cooperative_path_at_millions_of_particles(p):
    """N = 5e6 on the single-kernel path (about 5000 buckets, more than the
    152 x 32 warps of one pass): the permutation bit-exact and one FP32 step
    within the per-step bar; p = 16 needs more than 7 picks for a straddling
    batch, so the general mode's boundary loop runs."""
    n, d = 5_000_000, 3
    kw = dict(p=p, dt=1e-3, sigma=0.2, v="quadratic", k="reg_attract", k_param=0.01)
    X = as_run_precision(workloads.gaussian(n, d, seed=7), "f32")
    s, x = _system(X, d, "f32", seed=3, **kw)
    s.set_tuning(path=2)                      # beyond the automatic crossover
    assert s.tuning()["path"] == 2
    prm = _oprm(n, d, "f32", seed=3, **kw)
    perm = oracle.permutation(prm, 0)
    assert np.array_equal(s.permutation().cpu().numpy().view(np.uint32), perm)
    s.step()
    s.sync()
    FK = oracle.rbm_interaction(prm, X, perm)
    ref = oracle.euler_update(prm, X, FK, 0)
    assert_close_per_particle(from_dev(x, d), ref, 1e-5, extra=_fp32_bound(prm, X, FK, 0), what=f"p = {p}")


@pytest.mark.parametrize("log2n", [24, 26])
def test_multi_kernel_path_at_large_n_full_size(log2n):
    """The large-N sweep's N = 2^24 and N = 2^26 (its largest) entries (d = 3,
    FP32, regularised attraction, p = 2) on the multi-kernel bucket-sort path
    (the per-id path; the library picks the record path there, which
    tests/test_gpu_rec.py checks at N = 2^26): the whole permutation
    bit-exact and one step of every particle within the FP32 bar."""
    n, d = 1 << log2n, 3
    kw = dict(p=2, dt=1e-3, sigma=0.2, v="quadratic", k="reg_attract", k_param=0.01)
    X = as_run_precision(workloads.gaussian(n, d, seed=7), "f32")
    s, x = _system(X, d, "f32", seed=3, **kw)
    s.set_tuning(path=1)
    assert s.tuning()["path"] == 1
    prm = _oprm(n, d, "f32", seed=3, **kw)
    perm = oracle.permutation(prm, 0)
    assert np.array_equal(s.permutation().cpu().numpy().view(np.uint32), perm)
    s.step()
    s.sync()
    FK = oracle.rbm_interaction(prm, X, perm)
    ref = oracle.euler_update(prm, X, FK, 0)
    assert_close_per_particle(from_dev(x, d), ref, 1e-5, extra=_fp32_bound(prm, X, FK, 0), what=f"N = 2^{log2n}")


def test_direct_fp32_full_size_sampled():
    """Thomson N = 1e5, FP32, the launch the benchmark times: 256 sampled particles."""
    n, d = 100000, 3
    kw = dict(p=2, dt=1e-4, k="coulomb", renorm=True)
    X = as_run_precision(workloads.sphere(n, d, seed=0), "f32")
    s, x = _system(X, d, "f32", seed=1, **kw)
    s.direct_step()
    s.sync()
    got = from_dev(x, d)
    prm = _oprm(n, d, "f32", seed=1, **kw)
    idx = np.random.default_rng(0).choice(n, 256, replace=False)
    ref = oracle.direct_step_sampled(prm, X, 0, idx)
    FK = oracle.direct_forces_at(prm, X, X[idx])
    # an FP32 sum of N-1 terms rounds within (N eps32) times the sum of their
    # magnitudes; for K = x/|x|^3 that is sum_j |X^i - X^j|^-2 / (N-1)
    r2 = ((X[idx, None, :] - X[None, :, :]) ** 2).sum(axis=2)
    absmean = np.where(r2 > 0, 1.0 / np.where(r2 > 0, r2, 1.0), 0.0).sum(axis=1) / (n - 1)
    extra = 32.0 * EPS32 * prm.dt * np.linalg.norm(FK, axis=1) + n * EPS32 * prm.dt * absmean
    assert_close_per_particle(got[idx], ref, 1e-5, extra=extra, what="direct thomson")


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_direct_forces_at_queries(dtype):
    n, d, nq = 5000, 2, 777
    X = as_run_precision(workloads.mixture(n, d, seed=1), dtype)
    Q = as_run_precision(workloads.gaussian(nq, d, seed=2) * 3.0, dtype)
    s, x = _system(X, d, dtype, k="gauss_agg")
    f = from_dev(s.direct_forces_at(to_dev(Q, dtype)), d)
    s.sync()
    ref = oracle.direct_forces_at(_oprm(n, d, dtype, k="gauss_agg"), X, Q)
    tol = 1e-12 if dtype == "f64" else 2e-5
    assert_close_per_particle(f, ref, tol, what="forces at queries")


# ---------------------------------------------------------------------------
# behaviour of the boundary
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("path", [1, 2, 3])
def test_graph_replay_equals_eager_steps(path):
    n, d = (2000 if path == 3 else 20000), 3
    X = workloads.gaussian(n, d, seed=5)
    kw = dict(p=2, dt=1e-3, sigma=0.2, v="quadratic", k="reg_attract", k_param=0.01)
    a, xa = _system(X, d, "f32", **kw)
    b, xb = _system(X, d, "f32", **kw)
    a.set_tuning(graph_steps=7, path=path)
    b.set_tuning(path=path)
    a.run(23)                       # 3 graph replays + 2 eager steps
    for _ in range(23):
        b.step()
    a.sync()
    b.sync()
    assert a.m == 23 and b.m == 23
    assert np.array_equal(xa.cpu().numpy(), xb.cpu().numpy())


@pytest.mark.parametrize("path", [1, 2])
def test_lookahead_bucketing_survives_mixed_calls(path):
    """The bucket-sort and cooperative paths bucket the next step's ids at the
    end of each step.  A sequence that mixes graph replays, eager steps, a
    permutation and a force query at the current step, and a jump back in
    the step index must equal the same sequence run eagerly step by step, bit
    for bit, and every permutation must be the oracle's."""
    torch = torch_cuda()
    n, d = 20000, 3
    X = as_run_precision(workloads.gaussian(n, d, seed=12), "f32")
    kw = dict(p=2, dt=1e-3, sigma=0.2, v="quadratic", k="reg_attract", k_param=0.01, seed=13)
    prm = _oprm(n, d, "f32", **kw)

    def sequence(s):
        perms = []
        s.run(7)                              # graphs of 5 steps + 2 eager ones (or all eager)
        perms.append((s.m, s.permutation().cpu().numpy().view(np.uint32).copy()))
        s.step()
        s.m = 3                               # back in the step index
        s.step()
        f = s.forces().cpu().clone()
        perms.append((s.m, s.permutation().cpu().numpy().view(np.uint32).copy()))
        s.run(11)
        s.step()
        s.sync()
        return perms, f

    a, xa = _system(X, d, "f32", **kw)
    b, xb = _system(X, d, "f32", **kw)
    a.set_tuning(path=path, graph_steps=5)
    b.set_tuning(path=path, graph_steps=1000)
    assert a.tuning()["path"] == path and b.tuning()["path"] == path
    pa, fa = sequence(a)
    pb, fb = sequence(b)
    assert torch.equal(xa, xb)
    assert torch.equal(fa, fb)
    for (ma, perm_a), (mb, perm_b) in zip(pa, pb):
        assert ma == mb
        assert np.array_equal(perm_a, perm_b)
        assert np.array_equal(perm_a, oracle.permutation(prm, ma))
    assert a.m == b.m == 4 + 11 + 1


def test_latency_floor_of_the_cooperative_launch():
    """rbm_latency_floor times the cooperative step's launch shape with no
    work: positive, below the step kernel's own time, and leaving positions
    and step index alone; contexts on another path get RBM_ERR_STATE."""
    torch = torch_cuda()
    n, d = 100000, 3
    X = as_run_precision(workloads.sphere(n, d, seed=2), "f32")
    s, x = _system(X, d, "f32", p=2, dt=1e-4, k="coulomb", renorm=True)
    s.set_tuning(path=2)
    s.step()
    s.sync()
    before, m = x.clone(), s.m
    floor_us = s.latency_floor()
    assert 0.0 < floor_us < 1000.0
    assert torch.equal(x, before) and s.m == m
    step_us = 1e3 * sum(ms for name, ms in s.step_profiled() if name == "k_rbm_coop")
    assert floor_us < step_us
    t, _ = _system(X, d, "f32", p=2, dt=1e-4, k="coulomb", renorm=True)
    t.set_tuning(path=1)
    with pytest.raises(rbm.RbmError) as e:
        t.latency_floor()
    assert e.value.status == -6


def test_pad_lane_preserved_and_step_host_matches():
    torch = torch_cuda()
    n, d = 4096, 3
    X = workloads.sphere(n, d, seed=2)
    kw = dict(p=2, dt=1e-4, k="coulomb", renorm=True)
    x = to_dev(X, "f32", pad_value=7.25)
    s = rbm.System(x, d=d, **kw)
    host = x.cpu().pin_memory()
    ref = x.clone()
    t = rbm.System(ref, d=d, **kw)
    s.step_host(host)          # H2D, step, D2H
    t.step()
    t.sync()
    assert np.array_equal(host.numpy(), ref.cpu().numpy())
    assert np.all(host.numpy()[:, 3] == 7.25)
    pageable = host.clone()    # not pinned: the copy-engine path
    s.step_host(pageable)
    t.step()
    t.sync()
    assert np.array_equal(pageable.numpy(), ref.cpu().numpy())
    del torch


def test_nonfinite_positions_are_reported():
    n, d = 1000, 2
    X = workloads.gaussian(n, d, seed=1)
    X[17, 0] = np.nan
    s, _ = _system(X, d, "f32", p=2, k="gauss_agg")
    s.step()
    with pytest.raises(rbm.RbmError) as e:
        s.sync()
    assert e.value.status == -5
    with pytest.raises(rbm.RbmError) as e2:
        s.step()
    assert e2.value.status == -6


def test_invalid_parameters_rejected():
    torch = torch_cuda()
    x = torch.zeros(100, 1, device="cuda", dtype=torch.float64)
    for bad in [dict(p=1), dict(p=101), dict(dt=0.0), dict(sigma=-1.0), dict(k="inv1d", d=2),
                dict(scheme="split", p=3, k="inv1d"), dict(scheme="split", k="gauss_agg")]:
        kw = dict(p=2, k="inv1d", d=1)
        kw.update(bad)
        d = kw.pop("d")
        with pytest.raises(rbm.RbmError) as e:
            rbm.System(x if d == 1 else torch.zeros(100, d, device="cuda", dtype=torch.float64), d=d, **kw)
        assert e.value.status == -1
    for rows in (0, 1):                       # no system to divide into batches
        with pytest.raises(rbm.RbmError) as e:
            rbm.System(torch.zeros(rows, 1, device="cuda", dtype=torch.float64), d=1, p=2, k="inv1d")
        assert e.value.status == -1


def test_cooperative_compact_regrouping_equals_slots():
    """Buckets that outgrow their slots (slot_cap forced small) take the
    compact regrouping behind one more grid barrier; six steps, launches
    alternating the bucket-total buffers, must equal the default run bit for
    bit, and the permutation must stay the oracle's."""
    torch = torch_cuda()
    n, d = 60000, 3
    X = as_run_precision(workloads.gaussian(n, d, seed=5), "f32")
    kw = dict(p=2, dt=1e-3, sigma=0.2, v="quadratic", k="reg_attract", k_param=0.01, seed=8)
    a, xa = _system(X, d, "f32", **kw)
    b, xb = _system(X, d, "f32", **kw)
    a.set_tuning(path=2)
    b.set_tuning(path=2, slot_cap=100)
    assert a.tuning()["slot_cap"] == 2048 and b.tuning()["slot_cap"] == 100
    for _ in range(6):
        a.step()
        b.step()
    assert torch.equal(xa, xb)
    b.m = 4
    perm = b.permutation().cpu().numpy().view(np.uint32)
    b.sync()
    assert np.array_equal(perm, oracle.permutation(_oprm(n, d, "f32", **kw), 4))


def test_cooperative_barrier_wait_runs_out_and_is_reported():
    """A bounded grid-barrier wait that runs out: block 0 of the cooperative
    step is told (host-side hook) to leave before the first barrier, the other
    blocks' waits end after 20 ms and the step reports RBM_ERR_TIMEOUT.  The
    first phase writes no positions, so the state is untouched."""
    n, d = 50000, 2
    X = workloads.gaussian(n, d, seed=1)
    s, x = _system(X, d, "f32", p=2, k="gauss_agg")
    s.set_tuning(path=2, wait_limit_us=20000, test_skip_arrival=1)
    before = x.clone()
    s.step()
    with pytest.raises(rbm.RbmError) as e:
        s.sync()
    assert e.value.status == -4
    assert np.array_equal(before.cpu().numpy(), x.cpu().numpy())
    s.close()
    # a fresh context on the same device works normally afterwards
    t, y = _system(X, d, "f32", p=2, k="gauss_agg")
    t.set_tuning(path=2)
    t.step()
    t.sync()
