"""The binding's checks of device arguments (the C ABI receives bare
pointers, so the element type and the extent of a tensor are checked before
the pointer is passed): wrong dtype or too few elements raise ValueError
before any library call; None and raw integer addresses pass unchecked."""
import ctypes

import pytest

torch = pytest.importorskip("torch")
w = pytest.importorskip("paper_2101_07249_gb300")


def test_wrong_element_type_is_rejected():
    with pytest.raises(ValueError, match="expected torch.float64"):
        w._dev(torch.zeros(8, dtype=torch.float32), torch.float64, 8, "X")


def test_too_few_elements_are_rejected():
    with pytest.raises(ValueError, match="needs at least 9 elements"):
        w._dev(torch.zeros(8, dtype=torch.float64), torch.float64, 9, "X")


def test_checked_tensor_still_has_to_be_on_the_device():
    with pytest.raises(ValueError, match="CUDA tensor"):
        w._dev(torch.zeros(8, dtype=torch.float64), torch.float64, 8, "X")


def test_none_and_raw_addresses_pass():
    assert w._dev(None, torch.float64, 8, "X") is None
    p = w._dev(4096, torch.float64, 8, "X")
    assert isinstance(p, ctypes.c_void_p) and p.value == 4096


def test_precision_element_types():
    assert w._fdtype(w.FP64) is torch.float64
    assert w._fdtype(w.MIXED) is torch.float32
    assert w._fdtype(7) is None


def test_static_lmp_arguments_are_checked_before_the_call():
    """wc4d_lmp_apply_static passes bare pointers: FP64 and the extents
    k * nA (U), k (theta) and nA (v, y) are checked first."""
    k, nA = 3, 10
    f64 = torch.float64
    # the other arguments as raw addresses, which pass unchecked (every case
    # below raises before the library is called)
    ok = dict(U=4096, theta=8192, v=12288, y=16384)
    bad = [("U", torch.zeros(k * nA, dtype=torch.float32), "expected torch.float64"),
           ("U", torch.zeros(k * nA - 1, dtype=f64), "needs at least 30"),
           ("theta", torch.ones(k - 1, dtype=f64), "needs at least 3"),
           ("v", torch.zeros(nA - 1, dtype=f64), "needs at least 10"),
           ("y", torch.zeros(nA, dtype=torch.float32), "expected torch.float64")]
    for name, t, msg in bad:
        a = dict(ok)
        a[name] = t
        with pytest.raises(ValueError, match=msg):
            w.wc4d_lmp_apply_static(a["U"], a["theta"], k, nA, a["v"], a["y"])
