"""The record path of large systems (path 4: FP32, d = 3, p <= 32): the
positions move through the steps of one call as bucketed records and are
written back by id after the call's last step.

- a run of steps on the record path equals the same steps on the per-id
  bucket-sort path bit for bit (both evaluate each batch with the same
  arithmetic on the same rows in the same order), for p from 2 to 32, sizes
  that leave a ragged last batch, bucket geometries down to sub-buckets of a
  few records (batches crossing many of them), graph replays and eager runs;
  at N = 2^20 + 3 keys that agree in all the bits a sub-bucket sorts on (the
  top 37 of 64) occur about four times per step, so the full-key order of
  such ties is exercised as well;
- rbm_step_profiled (two steps, each kernel timed) equals two steps of a
  run, and a step launches four kernels;
- against the oracle: every particle within the FP32 bar after one step, and
  after a 5-step run within a bound that adds the per-step bars;
- every kernel family's step instance (the family fixed at compile time on
  the plain Euler-Maruyama configuration) equals the per-id path bit for bit;
- the pad lane of every row is left as the caller wrote it;
- a step of positions in host memory (rbm_step_host) beyond 16 MB, where the
  rows are copied in and scattered, and placed and copied out, in chunks on
  two streams, equals the same step on device-resident positions bit for bit
  (pinned and pageable host buffers, pad lanes kept), over several calls;
- the full-size large-N system (N = 2^26, the benchmarked launch
  configuration): one step of every particle within the FP32 bar of the
  oracle.
"""
import numpy as np
import pytest

import oracle
import paper_1812_10575_gb300 as rbm
import workloads
from gpu_util import EPS32, as_run_precision, assert_close_per_particle, from_dev, to_dev, torch_cuda

pytestmark = pytest.mark.gpu

KW = dict(dt=1e-3, sigma=0.2, v="quadratic", v_coef=1.0, k="reg_attract", k_param=0.01)


def _x(X, torch, pad_seed=None):
    x = to_dev(X, "f32")
    if pad_seed is not None:
        g = torch.Generator(device="cpu").manual_seed(pad_seed)
        x[:, 3] = torch.randn(x.shape[0], generator=g).to(x.device)
    return x


def _run(torch, X, path, steps, p, seed=3, graph_steps=0, bucket_bits=0, **kw):
    x = _x(X, torch, pad_seed=11)
    s = rbm.System(x, d=3, p=p, seed=seed, **dict(KW, **kw))
    s.set_tuning(path=path, graph_steps=graph_steps, bucket_bits=bucket_bits)
    assert s.tuning()["path"] == path
    s.run(steps)
    s.sync()
    out = x.cpu().numpy()
    s.close()
    return out


@pytest.mark.parametrize("n,p,bits", [(5000, 2, 0), (5001, 3, 0), (100000, 2, 0), (100003, 7, 0),
                                      (70001, 32, 0), (5003, 5, 10), (4099, 32, 9), (20000, 2, 12),
                                      (300007, 2, 13), (100003, 7, 14), (70001, 32, 16),
                                      (1048579, 3, 0)])
def test_record_path_run_equals_per_id_path_bitwise(n, p, bits):
    torch = torch_cuda()
    X = as_run_precision(workloads.gaussian(n, 3, seed=2), "f32")
    got = _run(torch, X, 4, 6, p, bucket_bits=bits)
    ref = _run(torch, X, 1, 6, p)
    assert np.array_equal(got.view(np.uint32), ref.view(np.uint32)), \
        f"{np.sum(np.any(got != ref, axis=1))} rows differ"


@pytest.mark.parametrize("n,bits", [(20000, 12), (300007, 13), (100003, 14)])
def test_record_path_profiled_steps_equal_run(n, bits):
    torch = torch_cuda()
    X = as_run_precision(workloads.gaussian(n, 3, seed=9), "f32")
    out = []
    for profiled in (False, True):
        x = _x(X, torch, pad_seed=3)
        s = rbm.System(x, d=3, p=3, seed=2, **KW)
        s.set_tuning(path=4, bucket_bits=bits)
        assert s.launches_per_step() == 4
        if profiled:
            names = [k for k, _ in s.step_profiled()]       # two steps, one kernel after another
            assert names.count("k_rec_split") == 2 and names.count("k_rec_step_last") == 1
        else:
            s.run(2)
        s.sync()
        assert s.m == 2
        out.append(x.cpu().numpy())
        s.close()
    assert np.array_equal(out[0].view(np.uint32), out[1].view(np.uint32))


def test_record_path_graph_replays_equal_eager_run():
    torch = torch_cuda()
    n = 50000
    X = as_run_precision(workloads.gaussian(n, 3, seed=4), "f32")
    a = _run(torch, X, 4, 23, 2, graph_steps=10)       # two 10-step graphs, then a 3-step run
    b = _run(torch, X, 4, 23, 2, graph_steps=1000)     # one eager 23-step run
    c = _run(torch, X, 1, 23, 2)
    assert np.array_equal(a.view(np.uint32), b.view(np.uint32))
    assert np.array_equal(a.view(np.uint32), c.view(np.uint32))


@pytest.mark.parametrize("kw", [dict(), dict(scheme="split", k="coulomb", v="zero", sigma=0.0, renorm=True),
                                dict(gbm=True, sigma=0.3)], ids=["euler", "split-thomson", "gbm"])
def test_record_path_schemes_equal_per_id_path(kw):
    torch = torch_cuda()
    n = 30000
    X0 = workloads.sphere(n, 3, seed=1) if kw.get("renorm") else workloads.gaussian(n, 3, seed=1)
    X = as_run_precision(X0, "f32")
    assert np.array_equal(_run(torch, X, 4, 5, 2, **kw).view(np.uint32),
                          _run(torch, X, 1, 5, 2, **kw).view(np.uint32))


@pytest.mark.parametrize("k,k_param", [("coulomb", 0.0), ("bounded_conf", 0.5), ("gauss_agg", 0.0),
                                       ("smooth_test", 0.0), ("linear", 0.7), ("reg_attract", 0.01)])
def test_record_path_every_kernel_family_equals_per_id_path(k, k_param):
    """The step kernels instantiated per kernel family (plain Euler-Maruyama
    configuration) give the per-id path's bits for every family."""
    torch = torch_cuda()
    n = 30011
    X = as_run_precision(workloads.gaussian(n, 3, seed=3), "f32")
    kw = dict(k=k, k_param=k_param, sigma=0.3)
    assert np.array_equal(_run(torch, X, 4, 4, 3, **kw).view(np.uint32),
                          _run(torch, X, 1, 4, 3, **kw).view(np.uint32))


def _fp32_bound(prm, X, FK, m):
    return 32.0 * EPS32 * prm.dt * np.linalg.norm(FK, axis=1)


def test_record_path_against_oracle_one_step_and_run():
    torch = torch_cuda()
    n, p = 60001, 3
    X = as_run_precision(workloads.gaussian(n, 3, seed=6), "f32")
    prm = oracle.make_params(n, 3, p=p, seed=5, precision="f32", **KW)
    x = _x(X, torch, pad_seed=1)
    pad = x[:, 3].clone()
    s = rbm.System(x, d=3, p=p, seed=5, **KW)
    s.set_tuning(path=4)
    s.step()
    s.sync()
    FK = oracle.rbm_interaction(prm, X, oracle.permutation(prm, 0))
    ref1 = oracle.euler_update(prm, X, FK, 0)
    got1 = from_dev(x, 3)
    assert_close_per_particle(got1, ref1, 1e-5, extra=_fp32_bound(prm, X, FK, 0), what="one step")
    assert torch.equal(x[:, 3], pad)
    # a 5-step run from the GPU's state against 5 oracle steps from the same state
    cur, bound = got1, np.zeros(n)
    for m in range(1, 6):
        FK = oracle.rbm_interaction(prm, cur, oracle.permutation(prm, m))
        bound = bound + 1e-5 * np.maximum(np.linalg.norm(cur, axis=1), 1.0) + _fp32_bound(prm, cur, FK, m)
        cur = oracle.euler_update(prm, cur, FK, m)
    s.run(5)
    s.sync()
    assert_close_per_particle(from_dev(x, 3), cur, 0.0, extra=2.0 * bound, what="5-step run")
    assert torch.equal(x[:, 3], pad)


@pytest.mark.parametrize("n,bits", [(1048579, 0), (1100007, 13)])
def test_record_path_host_step_equals_device_step(n, bits):
    torch = torch_cuda()
    X = as_run_precision(workloads.gaussian(n, 3, seed=6), "f32")
    x = _x(X, torch, pad_seed=5)
    ref = x.clone()
    s = rbm.System(x, d=3, p=3, seed=4, **KW)
    t = rbm.System(ref, d=3, p=3, seed=4, **KW)
    for sysm in (s, t):
        sysm.set_tuning(path=4, bucket_bits=bits)
        assert sysm.tuning()["path"] == 4
    host = x.cpu().pin_memory()
    assert host.numel() * 4 > (16 << 20)     # beyond the mapped-copy size: the chunked copies
    for _ in range(2):
        s.step_host(host)
        t.step()
        t.sync()
        assert np.array_equal(host.numpy().view(np.uint32), ref.cpu().numpy().view(np.uint32))
    pageable = host.clone()
    s.step_host(pageable)
    t.step()
    t.sync()
    assert np.array_equal(pageable.numpy().view(np.uint32), ref.cpu().numpy().view(np.uint32))
    assert s.m == 3 and t.m == 3
    s.close()
    t.close()


def test_record_path_full_size_large_n():
    """N = 2^26, the large-N system as the benchmark runs it (path chosen by
    the library): one step of every particle within the FP32 bar."""
    torch = torch_cuda()
    n, d = 1 << 26, 3
    kw = dict(p=2, **KW)
    X = as_run_precision(workloads.gaussian(n, d, seed=7), "f32")
    x = to_dev(X, "f32")
    s = rbm.System(x, d=d, seed=3, **kw)
    assert s.tuning()["path"] == 4
    s.step()
    s.sync()
    prm = oracle.make_params(n, d, seed=3, precision="f32", **kw)
    FK = oracle.rbm_interaction(prm, X, oracle.permutation(prm, 0))
    ref = oracle.euler_update(prm, X, FK, 0)
    assert_close_per_particle(from_dev(x, d), ref, 1e-5, extra=_fp32_bound(prm, X, FK, 0), what="N = 2^26")
    del torch
