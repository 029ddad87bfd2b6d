"""The C-ABI library builds for sm_103a, loads, and exports every entry
point include/wc4d.h declares; the Python binding wraps each of them.
No GPU needed (no compute call is made)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "wc4d.h")


def declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(wc4d_[a-zA-Z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2101_07249_gb300 import _build
    path = _build.build()
    import paper_2101_07249_gb300 as w
    return w.load(path)


def test_header_declares_the_inner_loop_calls():
    names = declared()
    for must in ("wc4d_create", "wc4d_hvp", "wc4d_sketch", "wc4d_pcg", "wc4d_inner_loop", "wc4d_lmp_apply",
                 "wc4d_set_propagator", "wc4d_set_covariance", "wc4d_set_background_obs", "wc4d_destroy"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    nm = subprocess.run(["nm", "-D", "--defined-only", os.path.join(ROOT, "paper_2101_07249_gb300", "libwc4d.so")],
                        capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (wc4d_\w+)", nm))
    missing = [n for n in declared() if n not in exported]
    assert not missing, missing
    for n in declared():
        assert getattr(lib, n) is not None


def test_binding_wraps_every_entry_point():
    import paper_2101_07249_gb300 as w
    assert set(declared()) == set(w.EXPORTS)
    for n in declared():
        assert callable(getattr(w, n)), n


def test_create_rejects_bad_problems_without_touching_the_gpu(lib):
    """Argument checks happen before any CUDA call."""
    import ctypes as C
    import paper_2101_07249_gb300 as w
    p = w.Problem()
    p.n, p.N, p.sigma_o2, p.obs_stride = 1, 3, 0.01, 1      # n < 2
    ctx = C.c_void_p()
    assert lib.wc4d_create(C.byref(ctx), C.byref(p), None) == w.EINVAL
    p.n, p.sigma_o2 = 16, -1.0                                # sigma_o2 <= 0
    assert lib.wc4d_create(C.byref(ctx), C.byref(p), None) == w.EINVAL
    p.sigma_o2, p.n = 0.01, 16384                             # n too large for the on-chip FFT
    assert lib.wc4d_create(C.byref(ctx), C.byref(p), None) == w.EINVAL
    assert lib.wc4d_hvp(None, None, None, 1, 1, 0) == w.EINVAL


def test_wait_controls_reject_a_null_context_without_touching_the_gpu(lib):
    """wc4d_set_wait_limit and wc4d_sync check their arguments before any
    CUDA call: a null context is EINVAL, whatever the limit."""
    import paper_2101_07249_gb300 as w
    assert lib.wc4d_sync(None) == w.EINVAL
    assert lib.wc4d_set_wait_limit(None, 0) == w.EINVAL
    assert lib.wc4d_set_wait_limit(None, -1) == w.EINVAL
