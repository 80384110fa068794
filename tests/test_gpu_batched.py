"""Batched replicas through the C ABI (rbm_batched_init): every replica must
follow exactly the trajectory of a single system with replica index r.

- permutation of every replica bit-exact against the oracle (counter word 2 = r);
- FP64 runs within 1e-10 per particle after 10 steps, FP32 runs per step
  within the FP32 bar of test_gpu_parity (1e-5 plus the force-rounding term);
- a batched replica equals the same replica run as a single system, bit for bit;
- CUDA-graph replay equals eager steps; the autotuner leaves the state alone.
"""
import os
import tempfile

import numpy as np
import pytest

import oracle
import paper_1812_10575_gb300 as rbm
import workloads
from gpu_util import EPS32, as_run_precision, assert_close_per_particle, from_dev, to_dev, torch_cuda

pytestmark = pytest.mark.gpu

OPINION = dict(dt=1e-2, sigma=0.01, k="bounded_conf", k_param=0.25)


def _sizes(count, lo, hi, seed):
    return [int(v) for v in workloads.replica_sizes(count, lo, hi, seed=seed)]


def _replicas(sizes, d, dtype, data_seed=0, **kw):
    """kw (including the Philox seed) goes to the library; data_seed draws X0."""
    X = as_run_precision(workloads.unit_cube(sum(sizes), d, seed=data_seed), dtype)
    x = to_dev(X, dtype)
    return rbm.Replicas(x, sizes, d=d, **kw), x, X


def _slices(sizes):
    offs = np.concatenate([[0], np.cumsum(sizes)])
    return [(int(offs[r]), int(offs[r + 1])) for r in range(len(sizes))]


@pytest.mark.parametrize("p", [2, 4])
def test_batched_permutations_bit_exact(p):
    torch_cuda()
    sizes = [2, 3, 5, 257, 1000, 4097, 30000, 65536] + _sizes(40, 256, 4096, seed=3)
    rep, x, X = _replicas(sizes, 2, "f32", p=p, seed=7, **OPINION)
    rep.m = 11
    perm = rep.permutation().cpu().numpy().view(np.uint32)
    rep.sync()
    for r, (lo, hi) in enumerate(_slices(sizes)):
        expect = oracle.permutation(oracle.make_params(hi - lo, 2, p=p, seed=7, replica=r), 11)
        assert np.array_equal(perm[lo:hi], expect), f"replica {r} (N={hi - lo})"


@pytest.mark.parametrize("p", [2, 4])
def test_batched_fp64_ten_steps(p):
    torch_cuda()
    sizes = [2, 3, 7, 300, 1001, 2500] + _sizes(10, 256, 2048, seed=5)
    kw = dict(p=p, seed=3, **OPINION)
    rep, x, X = _replicas(sizes, 2, "f64", **kw)
    rep.run(10)
    rep.sync()
    got = from_dev(x, 2)
    for r, (lo, hi) in enumerate(_slices(sizes)):
        prm = oracle.make_params(hi - lo, 2, p=p, dt=OPINION["dt"], sigma=OPINION["sigma"], seed=3,
                                 k="bounded_conf", k_param=0.25, replica=r)
        ref = oracle.run(prm, X[lo:hi], 0, 10)
        assert_close_per_particle(got[lo:hi], ref, 1e-10, what=f"replica {r}")


def test_batched_fp32_per_step_opinion_workload():
    """The batched opinion workload (2-D bounded confidence, R = 0.25, sigma =
    0.01, dt = 1e-2, X0 uniform in [0,1]^2, p = 2), 64 replicas of log-uniform
    size in [256, 8192]."""
    torch_cuda()
    sizes = _sizes(64, 256, 8192, seed=1)
    kw = dict(p=2, seed=0, **OPINION)
    rep, x, X = _replicas(sizes, 2, "f32", **kw)
    cur = X
    for m in range(2):
        rep.step()
        rep.sync()
        got = from_dev(x, 2)
        for r, (lo, hi) in enumerate(_slices(sizes)):
            prm = oracle.make_params(hi - lo, 2, p=2, dt=OPINION["dt"], sigma=OPINION["sigma"], seed=0,
                                     k="bounded_conf", k_param=0.25, replica=r, precision="f32")
            FK = oracle.rbm_interaction(prm, cur[lo:hi], oracle.permutation(prm, m))
            ref = oracle.euler_update(prm, cur[lo:hi], FK, m)
            extra = 32.0 * EPS32 * prm.dt * np.linalg.norm(FK, axis=1)
            assert_close_per_particle(got[lo:hi], ref, 1e-5, extra=extra, what=f"replica {r} step {m}")
        cur = got


def test_batched_full_opinion_workload_sampled():
    """The full batched workload as the benchmark times it: 4096 replicas of
    log-uniform size in [256, 65536] (5.1e7 particles, FP32, d = 2), with the
    launch shape the autotuner picks there (1024 threads, mean buckets of
    1024).  Permutations of 64 sampled replicas (the largest and the smallest
    among them) bit-exact, and one step of 24 of them within the FP32 bar."""
    torch_cuda()
    sizes = _sizes(4096, 256, 65536, seed=0)
    kw = dict(p=2, seed=0, **OPINION)
    rep, x, X = _replicas(sizes, 2, "f32", **kw)
    rep.set_launch(1024, 1024)
    perm = rep.permutation().cpu().numpy().view(np.uint32)
    rep.step()
    rep.sync()
    got = from_dev(x, 2)
    order = np.argsort(sizes)
    pick = sorted(set(order[::64].tolist()) | {int(order[0]), int(order[-1])})
    slices = _slices(sizes)
    for k, r in enumerate(pick):
        lo, hi = slices[r]
        prm = oracle.make_params(hi - lo, 2, p=2, dt=OPINION["dt"], sigma=OPINION["sigma"], seed=0,
                                 k="bounded_conf", k_param=0.25, replica=r, precision="f32")
        expect = oracle.permutation(prm, 0)
        assert np.array_equal(perm[lo:hi], expect), f"replica {r} (N={hi - lo})"
        if k % 3 == 0 or r in (int(order[0]), int(order[-1])):
            FK = oracle.rbm_interaction(prm, X[lo:hi], expect)
            ref = oracle.euler_update(prm, X[lo:hi], FK, 0)
            extra = 32.0 * EPS32 * prm.dt * np.linalg.norm(FK, axis=1)
            assert_close_per_particle(got[lo:hi], ref, 1e-5, extra=extra, what=f"replica {r}")


@pytest.mark.parametrize("p,bucket_target", [(8, 64), (32, 64), (4, 2048)])
def test_batched_bucket_shapes_fp64(p, bucket_target):
    """Small buckets (a batch straddles almost every bucket boundary, stepped
    after the buckets) and buckets of mean ~2048 (some beyond the
    shared-memory sort: the replica takes the general mode) give the oracle's
    trajectory."""
    torch_cuda()
    sizes = [4100, 6000, 300, 33, 40, 2049, 2100, 31]
    kw = dict(p=p, seed=5, **OPINION)
    rep, x, X = _replicas(sizes, 2, "f64", data_seed=4, **kw)
    rep.set_launch(256, bucket_target)
    rep.run(5)
    rep.sync()
    got = from_dev(x, 2)
    for r, (lo, hi) in enumerate(_slices(sizes)):
        prm = oracle.make_params(hi - lo, 2, p=p, dt=OPINION["dt"], sigma=OPINION["sigma"], seed=5,
                                 k="bounded_conf", k_param=0.25, replica=r)
        ref = oracle.run(prm, X[lo:hi], 0, 5)
        assert_close_per_particle(got[lo:hi], ref, 1e-10, what=f"replica {r} (N={hi - lo})")


def test_batched_replica_equals_single_system_bitwise():
    torch = torch_cuda()
    sizes = [700, 5000, 1234, 4]
    kw = dict(p=4, dt=1e-2, sigma=0.05, seed=9, v="quadratic", k="gauss_agg")
    Xall = workloads.gaussian(sum(sizes), 3, seed=2)
    x = to_dev(Xall, "f32")
    rep = rbm.Replicas(x, sizes, d=3, **kw)
    rep.run(5)
    rep.sync()
    for r, (lo, hi) in enumerate(_slices(sizes)):
        y = to_dev(Xall[lo:hi], "f32")
        single = rbm.System(y, d=3, replica=r, **kw)
        for _ in range(5):
            single.step()
        single.sync()
        assert torch.equal(x[lo:hi], y), f"replica {r}"


def test_batched_graph_replay_equals_eager():
    torch = torch_cuda()
    sizes = _sizes(300, 256, 4096, seed=4)
    a, xa, X = _replicas(sizes, 2, "f32", p=2, seed=1, **OPINION)
    b, xb, _ = _replicas(sizes, 2, "f32", p=2, seed=1, **OPINION)
    a.set_graph_steps(10)
    a.run(25)          # 2 graph replays + 5 eager steps
    for _ in range(25):
        b.step()
    a.sync()
    b.sync()
    assert a.m == 25
    assert torch.equal(xa, xb)


def test_autotune_keeps_state_and_uses_table():
    torch = torch_cuda()
    sizes = _sizes(200, 256, 8192, seed=6)
    rep, x, X = _replicas(sizes, 2, "f32", p=2, seed=2, **OPINION)
    before = x.clone()
    with tempfile.TemporaryDirectory() as tmp:
        table = os.path.join(tmp, "tune.txt")
        report = rep.autotune(trial_steps=2, table_path=table)
        assert report.startswith("searched")
        assert torch.equal(before, x) and rep.m == 0
        again = rep.autotune(trial_steps=2, table_path=table)
        assert again.startswith("table")
    ref, xr, _ = _replicas(sizes, 2, "f32", p=2, seed=2, **OPINION)
    rep.run(3)
    ref.run(3)
    rep.sync()
    ref.sync()
    assert torch.equal(x, xr)          # the launch shape does not change the result


def test_batched_rejects_direct_and_bad_sizes():
    torch = torch_cuda()
    x = torch.zeros(10, 2, device="cuda")
    with pytest.raises(ValueError):
        rbm.Replicas(x, [5, 4], d=2, p=2)          # sizes do not add up to the rows (binding check)
    prm = rbm.make_params(10, 2, p=2)
    with pytest.raises(rbm.RbmError) as e0:
        rbm.rbm_batched_init(prm, [5, 4], x)       # the library's own check of the same
    assert e0.value.status == -1
    with pytest.raises(rbm.RbmError):
        rbm.Replicas(x, [9, 1], d=2, p=2)          # a replica of one particle
    rep = rbm.Replicas(x, [5, 5], d=2, p=2)
    with pytest.raises(rbm.RbmError) as e:
        rbm.rbm_direct_step(rep.ctx)
    assert e.value.status == -7
