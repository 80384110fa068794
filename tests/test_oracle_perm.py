"""Pins of the oracle's random division (Sec. 2.1, Algorithm "randomdiv";
Lemma "averagefunc" in Sec. 3 for the co-occurrence probabilities)."""
import itertools
import math

import numpy as np
import pytest
from scipy import stats

import oracle


@pytest.mark.parametrize("n,seed,m,r", [(1, 0, 0, 0), (2, 1, 0, 0), (7, 3, 9, 0), (1000, 0, 0, 0),
                                        (1001, 5, 17, 3), (4096, 2**40 + 7, 2**31 + 5, 1)])
def test_permutation_is_key_order(n, seed, m, r):
    prm = oracle.make_params(n, 1, seed=seed, replica=r)
    perm = oracle.permutation(prm, m)
    keys = oracle.perm_keys(prm, m)
    assert sorted(perm.tolist()) == list(range(n))
    # numpy's lexsort of (id, key) is the same order computed another way
    expect = np.lexsort((np.arange(n), keys))
    assert np.array_equal(perm, expect.astype(np.uint32))


def test_permutations_uniform_over_all_orders():
    """N = 4: every one of the 4! orders is equally likely (chi-square over steps)."""
    prm = oracle.make_params(4, 1, seed=99)
    index = {p: k for k, p in enumerate(itertools.permutations(range(4)))}
    counts = np.zeros(24)
    for m in range(24000):
        counts[index[tuple(oracle.permutation(prm, m).tolist())]] += 1
    assert stats.chisquare(counts).pvalue > 1e-4


@pytest.mark.parametrize("n,p", [(6, 2), (6, 3), (8, 4)])
def test_pair_and_triple_cooccurrence(n, p):
    """P(i,j same batch) = (p-1)/(N-1), P(i,j,k) = (p-1)(p-2)/((N-1)(N-2))
    (proof of Lemma "averagefunc")."""
    prm = oracle.make_params(n, 1, seed=5)
    steps = 20000
    pair = 0
    triple = 0
    for m in range(steps):
        perm = oracle.permutation(prm, m)
        batch_of = np.empty(n, dtype=int)
        batch_of[perm] = np.arange(n) // p
        pair += batch_of[0] == batch_of[1]
        triple += (batch_of[0] == batch_of[1]) and (batch_of[0] == batch_of[2])
    p2 = (p - 1) / (n - 1)
    p3 = (p - 1) * (p - 2) / ((n - 1) * (n - 2))
    assert abs(pair / steps - p2) < 5 * math.sqrt(p2 * (1 - p2) / steps)
    assert abs(triple / steps - p3) < 5 * math.sqrt(max(p3 * (1 - p3), 1e-9) / steps) + 1e-12
