"""Host-side checks of the C ABI: the library builds for sm_103a, loads without
a GPU and exports every function include/nncandelinc.h declares; and the bit
rule the pass kernel uses to round TF32 remainders."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:[A-Za-z_][A-Za-z0-9_]*[\s*]+)+([a-z_][a-z0-9_]*)\s*\(",
                             text, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_1909_07570_gb300 import build as b
    path = b.build()
    return ctypes.CDLL(path)


def test_header_declares_the_four_calls():
    names = _declared_functions()
    for fn in ("ntd_fit", "nncp_core_fit", "nncp_core_fit_batched", "candelinc_lift",
               "recon_residual", "nnc_status_string"):
        assert fn in names


def test_library_exports_every_declared_symbol(lib):
    for fn in sorted(_declared_functions()):
        assert hasattr(lib, fn), fn


def test_binding_covers_every_declared_symbol():
    from paper_1909_07570_gb300 import native
    assert set(native.EXPORTED) == _declared_functions()


def test_status_strings_without_gpu(lib):
    lib.nnc_status_string.restype = ctypes.c_char_p
    assert lib.nnc_status_string(0) == b"ok"
    assert b"negative" in lib.nnc_status_string(-2)


def test_argument_checks_need_no_gpu(lib):
    # Invalid options are rejected before any CUDA call.
    from paper_1909_07570_gb300 import native
    native.load()
    opts = native.nnc_opts(-1, 0, 1e-12)
    dims = (ctypes.c_int64 * 3)(4, 4, 4)
    m = (ctypes.c_int * 3)(2, 2, 2)
    ptrs = (ctypes.c_void_p * 3)(1, 1, 1)
    st = native._lib.ntd_fit(ctypes.c_void_p(1), 3, dims, m, 1, ctypes.byref(opts), ptrs,
                             ctypes.c_void_p(1), None, None, None)
    assert st == -1
    opts = native.nnc_opts(3, 0, 1e-12)
    st = native._lib.ntd_fit(ctypes.c_void_p(1), 5, dims, m, 1, ctypes.byref(opts), ptrs,
                             ctypes.c_void_p(1), None, None, None)
    assert st == -1
    bad_m = (ctypes.c_int * 3)(2, 0, 2)
    st = native._lib.ntd_fit(ctypes.c_void_p(1), 3, dims, bad_m, 1, ctypes.byref(opts), ptrs,
                             ctypes.c_void_p(1), None, None, None)
    assert st == -1


def test_tf32_rounding_bit_rule():
    # The pass kernel rounds x to TF32 (its hi part), and the remainder x - x_hi
    # too, by adding half of the 13 dropped bits to the sign-magnitude pattern
    # and clearing them. Check
    # that rule against round-to-nearest, ties away from zero, on the TF32 grid
    # (10 stored mantissa bits), computed exactly in float64.
    rng = np.random.default_rng(7)
    x = (rng.standard_normal(20000) * np.exp2(rng.integers(-60, 60, 20000))).astype(np.float32)
    ties = (np.float32(1.0) + np.float32(2.0 ** -11) * np.arange(1, 64, 2)).astype(np.float32)
    x = np.concatenate([x, ties, -ties, np.float32([0.0, -0.0, 1.0, 2.0 ** -130, 3.0 * 2.0 ** -140])])
    bits = x.view(np.uint32)
    got = ((bits + np.uint32(0x1000)) & np.uint32(0xFFFFE000)).view(np.float32).astype(np.float64)
    xd = x.astype(np.float64)
    mant, expo = np.frexp(xd)                       # xd = mant * 2^expo, 0.5 <= |mant| < 1
    expo = np.maximum(expo, -125)                   # subnormal float32: fixed spacing 2^-136 (11 bits kept)
    spacing = np.exp2(expo - 11.0)
    q = xd / spacing
    ref = np.sign(q) * np.floor(np.abs(q) + 0.5) * spacing
    np.testing.assert_array_equal(got, ref)
    # The split x = x_hi + x_lo with both parts so rounded: the remainder of
    # x_hi is exact in float32 and takes both signs; x_hi + x_lo is within 2^-22
    # of x (relative) for normal x.
    xs = np.abs(x[np.abs(x) > 2.0 ** -100]).astype(np.float32)
    hi = ((xs.view(np.uint32) + np.uint32(0x1000)) & np.uint32(0xFFFFE000)).view(np.float32)
    rem = (xs - hi).astype(np.float32)
    np.testing.assert_array_equal(rem.astype(np.float64), xs.astype(np.float64) - hi.astype(np.float64))
    assert (rem > 0).any() and (rem < 0).any()
    lo = ((rem.view(np.uint32) + np.uint32(0x1000)) & np.uint32(0xFFFFE000)).view(np.float32)
    err = np.abs(hi.astype(np.float64) + lo.astype(np.float64) - xs.astype(np.float64))
    assert np.all(err <= 2.0 ** -22 * xs.astype(np.float64))
