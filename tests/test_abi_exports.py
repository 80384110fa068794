"""The C-ABI library without a GPU: it loads, exports every function
include/rbm.h declares, its structs have the layout the Python binding
assumes, and parameter errors come back synchronously without touching CUDA."""
import ctypes
import os
import re
import subprocess
import tempfile

import pytest

import paper_1812_10575_gb300 as rbm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rbm.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(rbm_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_what_the_binding_lists():
    assert declared_functions() == sorted(rbm.EXPORTS)


def test_library_exports_every_declared_function():
    lib = rbm.load()
    out = subprocess.run(["nm", "-D", "--defined-only", rbm.library_path()], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\bT (rbm_[a-z0-9_]+)$", out, flags=re.M))
    for name in declared_functions():
        assert name in exported, name
        getattr(lib, name)


def test_struct_layout_matches_header():
    src = r"""
#include <stdio.h>
#include <stddef.h>
#include "rbm.h"
#define F(s, f) printf(#s "." #f " %zu\n", offsetof(s, f))
int main(void) {
  printf("rbm_params %zu\n", sizeof(rbm_params));
  F(rbm_params, n); F(rbm_params, d); F(rbm_params, p); F(rbm_params, dt); F(rbm_params, sigma);
  F(rbm_params, seed); F(rbm_params, dtype); F(rbm_params, v); F(rbm_params, v_coef); F(rbm_params, k);
  F(rbm_params, k_param); F(rbm_params, flags); F(rbm_params, scheme); F(rbm_params, replica);
  printf("rbm_tuning %zu\n", sizeof(rbm_tuning));
  F(rbm_tuning, bucket_bits); F(rbm_tuning, slot_cap); F(rbm_tuning, sort_cap); F(rbm_tuning, block);
  F(rbm_tuning, direct_block); F(rbm_tuning, graph_steps); F(rbm_tuning, path); F(rbm_tuning, wait_limit_us);
  F(rbm_tuning, test_skip_arrival);
  return 0;
}
"""
    with tempfile.TemporaryDirectory() as tmp:
        c = os.path.join(tmp, "layout.c")
        exe = os.path.join(tmp, "layout")
        open(c, "w").write(src)
        subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        lines = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split("\n")
    got = dict(line.split() for line in lines if line.strip())
    assert int(got["rbm_params"]) == ctypes.sizeof(rbm.RbmParams)
    assert int(got["rbm_tuning"]) == ctypes.sizeof(rbm.RbmTuning)
    for cls, cname in ((rbm.RbmParams, "rbm_params"), (rbm.RbmTuning, "rbm_tuning")):
        for field, _ in cls._fields_:
            assert int(got[f"{cname}.{field}"]) == getattr(cls, field).offset, field


@pytest.mark.parametrize("bad", [dict(n=1), dict(d=4), dict(p=1), dict(dt=0.0), dict(sigma=-1.0),
                                 dict(k=99), dict(k="inv1d", d=2), dict(scheme="split", p=3, k="inv1d")])
def test_invalid_parameters_return_synchronously(bad):
    kw = dict(n=100, d=1, p=2, dt=1e-3, k="inv1d")
    kw.update(bad)
    n, d = kw.pop("n"), kw.pop("d")
    prm = rbm.make_params(n, d, **kw)
    ctx = ctypes.c_void_p()
    fake_aligned_device_pointer = ctypes.c_void_p(1 << 20)
    status = rbm.load().rbm_init(ctypes.byref(prm), fake_aligned_device_pointer, None, ctypes.byref(ctx))
    assert status == -1
    assert not ctx.value


def test_status_strings():
    assert rbm.rbm_status_string(0) == "ok"
    assert rbm.rbm_status_string(-5) == "non-finite position"
    assert rbm.rbm_status_string(12345) == "unknown status"


def test_noalloc_rejects_large_n_without_gpu():
    status = rbm.load().rbm_permutation_noalloc(1 << 20, 0, 0, 0, ctypes.c_void_p(1 << 20), None)
    assert status == -1
    assert "exceeds the maximum" in rbm.rbm_last_error()


@pytest.mark.parametrize("n,m,reason", [(1, 0, "at least 2"), (100, -1, "must not be negative")])
def test_noalloc_rejections_set_the_error_text_without_gpu(n, m, reason):
    lib = rbm.load()
    # leave an unrelated message first: the rejection must replace it
    assert lib.rbm_permutation_noalloc(1 << 20, 0, 0, 0, ctypes.c_void_p(1 << 20), None) == -1
    status = lib.rbm_permutation_noalloc(n, 0, 0, m, ctypes.c_void_p(1 << 20), None)
    assert status == -1
    assert reason in rbm.rbm_last_error()


def test_noalloc_rejects_null_output_without_gpu():
    assert rbm.load().rbm_permutation_noalloc(100, 0, 0, 0, None, None) == -1
    assert "null pointer" in rbm.rbm_last_error()


@pytest.mark.parametrize("packed,null", [(2, False), (-1, False), (0, True)])
def test_fma_peak_rejects_bad_arguments_without_gpu(packed, null):
    out = ctypes.c_double()
    status = rbm.load().rbm_fp32_fma_peak(packed, None if null else ctypes.byref(out), None)
    assert status == -1
    assert "rbm_fp32_fma_peak" in rbm.rbm_last_error()
