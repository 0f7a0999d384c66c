"""The C-ABI library: it builds, loads, exports every symbol include/nmf.h
declares, and validates arguments on the host (no kernel is launched here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "nmf.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(nmf_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def built():
    from paper_2106_15214_gb300 import build, binding
    build.build()
    return binding.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("nmf_create", "nmf_step_joint", "nmf_step_alternating", "nmf_loss", "nmf_grad",
                 "nmf_set_csr", "nmf_batch_create", "nmf_destroy"):
        assert must in names


def test_library_exports_every_declared_symbol(built):
    from paper_2106_15214_gb300 import binding
    for name in declared_functions():
        assert hasattr(built, name), name
    assert set(declared_functions()) <= set(binding.EXPORTS) | {"nmf_status_string"}


def test_status_strings(built):
    for code in range(8):
        assert built.nmf_status_string(code).decode().startswith("NMF_")


def test_host_validation(built):
    ctx = ctypes.c_void_p()
    assert built.nmf_create(0, 5, 2, 1.0, ctypes.byref(ctx)) == 1          # F < 1
    assert built.nmf_create(5, 5, 0, 1.0, ctypes.byref(ctx)) == 1          # K < 1
    assert built.nmf_create(5, 5, 2, float("nan"), ctypes.byref(ctx)) == 1 # beta not finite
    assert built.nmf_create(5, 5, 200, 1.0, ctypes.byref(ctx)) == 6        # K above the kernels' limit
    assert built.nmf_create(5, 7, 2, 1.5, ctypes.byref(ctx)) == 0
    try:
        assert built.nmf_set_options(ctx, 9, 0, 1, 0.0, 1, None) == 1      # bad precision
        assert built.nmf_set_options(ctx, 1, 0, 1, -1.0, 1, None) == 1     # negative kappa
        assert built.nmf_set_options(ctx, 1, 0, 1, 0.0, 1, None) == 0
        assert built.nmf_set_subiterations(ctx, 0) == 1
        assert built.nmf_set_dense(ctx, ctypes.c_void_p(16), 3) == 1       # ldv < N
        loss = ctypes.c_double()
        assert built.nmf_step_joint(ctx, 1, ctypes.byref(loss)) == 7       # no data yet
        assert built.nmf_step_joint(ctx, 0, None) == 1
        assert built.nmf_set_csr(ctx, 4, ctypes.c_void_p(16), ctypes.c_void_p(16), ctypes.c_void_p(16)) == 1  # beta != 1
        built.nmf_set_floor.argtypes = [ctypes.c_void_p, ctypes.c_double]
        assert built.nmf_set_floor(ctx, float("nan")) == 1
        assert built.nmf_set_floor(ctx, float("inf")) == 1
        assert built.nmf_set_floor(ctx, 1e-20) == 0
        assert built.nmf_set_floor(ctx, -1.0) == 0                      # back to the default
        assert built.nmf_set_floor(None, 0.0) == 1
        cap = ctypes.c_int32(0)
        assert built.nmf_autotune(ctx, 0, ctypes.byref(cap)) == 1          # trials < 1
        assert built.nmf_autotune(ctx, 2, ctypes.byref(cap)) == 7          # no data yet
        assert built.nmf_autotune(None, 2, None) == 1
        assert built.nmf_set_options(ctx, 2, 0, 1, 0.0, 1, None) == 0      # TF32 single problem
        assert built.nmf_autotune(ctx, 2, ctypes.byref(cap)) == 6          # the tensor-core path has its own model
    finally:
        built.nmf_destroy(ctx)
    built.nmf_destroy(None)


def test_barrier_test_validation(built):
    """nmf_set_barrier_test accepts bounds of 1 ms .. 10 s and 0 or 1 extra arrivals."""
    ctx = ctypes.c_void_p()
    assert built.nmf_create(20, 30, 3, 1.0, ctypes.byref(ctx)) == 0
    try:
        assert built.nmf_set_barrier_test(ctx, 999_999, 0) == 1
        assert built.nmf_set_barrier_test(ctx, 1_000_000, 2) == 1
        assert built.nmf_set_barrier_test(ctx, 20_000_000_000, 0) == 1
        assert built.nmf_set_barrier_test(ctx, 1_000_000, -1) == 1
        assert built.nmf_set_barrier_test(ctx, 1_000_000, 1) == 0
        assert built.nmf_set_barrier_test(ctx, 1_000_000_000, 0) == 0
        assert built.nmf_set_barrier_test(None, 1_000_000_000, 0) == 1
    finally:
        built.nmf_destroy(ctx)


def test_batch_validation(built):
    ctx = ctypes.c_void_p()
    F = (ctypes.c_int64 * 2)(4, 5)
    N = (ctypes.c_int64 * 2)(6, 0)
    K = (ctypes.c_int32 * 2)(2, 2)
    assert built.nmf_batch_create(2, F, N, K, 1.5, ctypes.byref(ctx)) == 1
    N[1] = 3
    assert built.nmf_batch_create(2, F, N, K, 1.5, ctypes.byref(ctx)) == 0
    built.nmf_destroy(ctx)


def test_binding_rejects_missing_library(tmp_path):
    from paper_2106_15214_gb300 import binding
    saved = binding._lib
    binding._lib = None
    try:
        with pytest.raises(RuntimeError):
            binding.load(str(tmp_path / "nope.so"))
    finally:
        binding._lib = saved
