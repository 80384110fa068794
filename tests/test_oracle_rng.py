"""Pins of the oracle's counter-based RNG and Brownian increments.

Philox4x32-10 is not in the paper (any uniform shuffle and Gaussian source
serve, Sec. 2.1); it is pinned to its published known answer and to an
independent implementation (Triton's), and the Gaussians to the normal law.
"""
import os

import numpy as np
import pytest
from scipy import stats

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _kat_rows():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            v = [int(t, 16) for t in line.split()]
            rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,expect", _kat_rows())
def test_philox_known_answer(ctr, key, expect):
    assert list(oracle.philox4x32_10(ctr, key)) == expect


def test_philox_matches_triton_implementation():
    """Triton ships its own Philox4x32-10 (triton.language.random); run it in
    the CPU interpreter on random counters and keys and compare word by word."""
    pytest.importorskip("triton")
    import subprocess
    import sys
    import textwrap

    code = textwrap.dedent(
        """
        import os, sys, json
        os.environ["TRITON_INTERPRET"] = "1"
        import numpy as np, torch, triton, triton.language as tl
        @triton.jit
        def k(out, c0p, c1p, c2p, c3p, seed, BLOCK: tl.constexpr):
            i = tl.arange(0, BLOCK)
            a, b, c, d = tl.philox(seed, tl.load(c0p + i), tl.load(c1p + i), tl.load(c2p + i), tl.load(c3p + i), 10)
            tl.store(out + i * 4 + 0, a); tl.store(out + i * 4 + 1, b)
            tl.store(out + i * 4 + 2, c); tl.store(out + i * 4 + 3, d)
        cases = json.loads(sys.stdin.read())
        res = []
        for seed, ctrs in cases:
            c = np.array(ctrs, dtype=np.uint32).view(np.int32)
            out = torch.zeros(4 * len(ctrs), dtype=torch.int32)
            cols = [torch.from_numpy(np.ascontiguousarray(c[:, j])) for j in range(4)]
            k[(1,)](out, *cols, seed, BLOCK=len(ctrs))
            res.append((out.numpy().view(np.uint32).reshape(-1, 4)).tolist())
        print(json.dumps(res))
        """
    )
    rng = np.random.default_rng(7)
    cases = []
    for _ in range(3):
        seed = int(rng.integers(0, 2**63))
        ctrs = rng.integers(0, 2**32, size=(16, 4), dtype=np.uint64).astype(np.uint32)
        cases.append((seed, ctrs.tolist()))
    import json

    env = dict(os.environ, TRITON_INTERPRET="1")
    p = subprocess.run([sys.executable, "-c", code], input=json.dumps(cases), capture_output=True,
                       text=True, env=env, timeout=600)
    if p.returncode != 0:
        pytest.skip("triton interpreter unavailable: " + p.stderr.strip().splitlines()[-1])
    got = json.loads(p.stdout.strip().splitlines()[-1])
    for (seed, ctrs), outs in zip(cases, got):
        key = [seed & 0xFFFFFFFF, seed >> 32]
        for c, o in zip(ctrs, outs):
            assert list(oracle.philox4x32_10(c, key)) == o


def test_philox_bytes_uniform():
    prm = oracle.make_params(200000, 1, seed=123)
    keys = oracle.perm_keys(prm, 5)
    b = keys.view(np.uint8)
    counts = np.bincount(b, minlength=256)
    chi2, pval = stats.chisquare(counts)
    assert pval > 1e-4


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_normals_are_standard_gaussian(precision):
    prm = oracle.make_params(100000, 3, seed=11, precision=precision)
    z = oracle.normals(prm, 3)
    for k in range(3):
        col = z[:, k]
        assert abs(col.mean()) < 5.0 / np.sqrt(len(col))
        assert abs(col.var() - 1.0) < 5.0 * np.sqrt(2.0 / len(col))
        assert stats.kstest(col, "norm").pvalue > 1e-4
    c = np.corrcoef(z.T)
    assert np.all(np.abs(c - np.eye(3)) < 5.0 / np.sqrt(z.shape[0]))


def test_normals_differ_by_step_and_replica():
    a = oracle.normals(oracle.make_params(1000, 2, seed=1), 0)
    b = oracle.normals(oracle.make_params(1000, 2, seed=1), 1)
    c = oracle.normals(oracle.make_params(1000, 2, seed=1, replica=1), 0)
    assert not np.allclose(a, b) and not np.allclose(a, c)
    assert abs(np.corrcoef(a[:, 0], b[:, 0])[0, 1]) < 0.15
