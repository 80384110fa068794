"""The allocation-free random division (rbm_permutation_noalloc).

Callers whose device memory is owned by someone else (an application's own
memory manager, a fixed budget) or that must never block on an allocation
cannot use rbm_init, which allocates scratch with cudaMalloc.  For them the
library computes the random division of a step from a fixed scratch array in
device memory.  This test calls that entry point through the C ABI twice in a
row and checks each result, bit for bit, against the permutation the regular
entry point (rbm_permutation on a context) gives for the same n, seed,
replica and step.  It lives in a file of its own that pytest collects last.
"""
import numpy as np
import pytest

import paper_1812_10575_gb300 as rbm
from gpu_util import torch_cuda

pytestmark = pytest.mark.gpu


def _regular_permutation(torch, n, seed, replica, m):
    x = torch.zeros(n, 1, dtype=torch.float32, device="cuda")
    s = rbm.System(x, d=1, p=2, seed=seed, replica=replica)
    s.m = m
    perm = s.permutation()
    s.sync()
    out = perm.cpu().numpy().view(np.uint32).copy()
    s.close()
    return out


def test_noalloc_permutation_matches_regular_entry_point_twice():
    torch = torch_cuda()
    stream = torch.cuda.current_stream()
    cases = [(65536, 2**33 + 5, 1, 7),   # the largest n the fixed scratch holds
             (1000, 17, 0, 8)]           # a smaller system right after it
    for n, seed, replica, m in cases:
        perm = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        rbm.rbm_permutation_noalloc(n, seed, replica, m, perm, stream)
        torch.cuda.synchronize()
        got = perm.cpu().numpy().view(np.uint32)
        expect = _regular_permutation(torch, n, seed, replica, m)
        assert np.array_equal(got, expect), f"n={n} m={m}"


def test_noalloc_calls_take_no_device_memory():
    """After a first call, further calls leave the device's free memory
    unchanged (no cudaMalloc or cudaMallocAsync on this path), and their
    permutations stay right."""
    torch = torch_cuda()
    stream = torch.cuda.current_stream()
    n, seed, replica = 50000, 99, 2
    outs = [torch.full((n,), -1, dtype=torch.int32, device="cuda") for _ in range(4)]
    rbm.rbm_permutation_noalloc(n, seed, replica, 0, outs[0], stream)
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    for m in range(1, 4):
        rbm.rbm_permutation_noalloc(n, seed, replica, m, outs[m], stream)
    torch.cuda.synchronize()
    free_after = torch.cuda.mem_get_info()[0]
    assert free_after == free_before
    for m in (0, 3):
        got = outs[m].cpu().numpy().view(np.uint32)
        assert np.array_equal(got, _regular_permutation(torch, n, seed, replica, m)), f"m={m}"


def test_noalloc_rejects_n_above_maximum():
    torch = torch_cuda()
    perm = torch.empty(65537, dtype=torch.int32, device="cuda")
    with pytest.raises(rbm.RbmError) as e:
        rbm.rbm_permutation_noalloc(65537, 0, 0, 0, perm)
    assert e.value.status == -1
    assert "exceeds the maximum" in rbm.rbm_last_error()
