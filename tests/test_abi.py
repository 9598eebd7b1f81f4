"""The C ABI without a GPU: the library loads, exports every function include/fbp.h
declares, and validates arguments on the host before touching CUDA."""
import ctypes

import numpy as np
import pytest


def test_every_declared_symbol_is_exported(fbp):
    names = fbp.header_functions()
    assert len(names) >= 14
    lib = fbp.load_library()
    for name in names:
        assert hasattr(lib, name), name


def test_status_strings(fbp):
    assert fbp.fbp_status_str(0) == "ok"
    assert "aligned" in fbp.fbp_status_str(3)
    assert fbp.fbp_status_str(99) == "unknown status"


def test_default_coefficients_come_from_the_committed_table(fbp, coeff_table):
    for e in coeff_table["entries"]:
        b, a = fbp.fbp_default_coeffs(e["N"], e["order"])
        np.testing.assert_array_equal(b, e["b"])
        np.testing.assert_array_equal(a, e["a"])
    b3, a3 = fbp.fbp_default_coeffs(256)
    assert len(b3) == 3 and len(a3) == 3
    with pytest.raises(fbp.FbpError):
        fbp.fbp_default_coeffs(3, 3)


def _plan_status(fbp, N, K, M, batch, coeffs, fuse_k=0):
    lib = fbp.load_library()
    h = ctypes.c_void_p()
    cs = None if coeffs is None else ctypes.byref(fbp.coeffs_struct(*coeffs))
    return lib.fbp_plan(ctypes.byref(h), N, K, M, batch, cs, fuse_k)


def test_plan_rejects_bad_arguments_before_cuda(fbp):
    good = ([0.12, -0.23, 0.11], list(np.poly([0.9, 0.5, -0.3])[1:]))
    assert _plan_status(fbp, 96, 8, 8, 1, good) == 2            # N not a power of two
    assert _plan_status(fbp, 8192, 8, 8, 1, good) == 2          # N too large
    assert _plan_status(fbp, 64, 1, 8, 1, good) == 1            # K < 2
    assert _plan_status(fbp, 64, 8, 8, 0, good) == 1            # batch < 1
    assert _plan_status(fbp, 64, 8, 8, 1, ([1.0], [-1.01])) == 1    # pole at 1.01
    repeated = ([0.1, -0.1, 0.0], list(np.poly([0.5, 0.5, 0.2])[1:]))
    assert _plan_status(fbp, 64, 8, 8, 1, repeated) == 2        # repeated pole
    assert _plan_status(fbp, 64, 8, 8, 1, good, fuse_k=7) == 2  # fuse_k out of range
    assert _plan_status(fbp, 4096, 8, 8, 1, good, fuse_k=5) == 2   # second pass > 6 stages
    assert _plan_status(fbp, 64, 8, 8, 1, good, fuse_k=1) == 2     # 2-row first-pass blocks


def test_null_pointers_are_rejected(fbp):
    lib = fbp.load_library()
    assert lib.fbp_plan(None, 64, 8, 8, 1, None, 0) == 1
    assert lib.fbp_reconstruct(None, None, None, None) == 1
    assert lib.fbp_filter_iir(None, None, None, None) == 1
    assert lib.fbp_workspace_bytes(None) == 0
    assert lib.fbp_set_chunk(None, 1) == 1
    assert lib.fbp_plan_destroy(None) == 0
    assert lib.fbp_default_coeffs(256, 3, None) == 1


def test_volume_arguments_are_checked_before_cuda(fbp):
    lib = fbp.load_library()
    h = ctypes.c_void_p()
    item = fbp.fbp_item(64, 96, 91, 16 * 1000, 16 * 2000)     # aligned, never dereferenced
    arr = (fbp.fbp_item * 1)(item)
    assert lib.fbp_volume_create(None, arr, 1, 0, 0) == 1
    assert lib.fbp_volume_create(ctypes.byref(h), None, 1, 0, 0) == 1
    assert lib.fbp_volume_create(ctypes.byref(h), arr, 0, 0, 0) == 1
    assert lib.fbp_volume_create(ctypes.byref(h), arr, 1, 0, 4) == 1         # unknown flag
    bad = (fbp.fbp_item * 1)(fbp.fbp_item(96, 96, 91, 16 * 1000, 16 * 2000))
    assert lib.fbp_volume_create(ctypes.byref(h), bad, 1, 0, 0) == 2         # N = 96
    bad = (fbp.fbp_item * 1)(fbp.fbp_item(64, 1, 91, 16 * 1000, 16 * 2000))
    assert lib.fbp_volume_create(ctypes.byref(h), bad, 1, 0, 0) == 1         # K = 1
    bad = (fbp.fbp_item * 1)(fbp.fbp_item(64, 96, 91, 16 * 1000 + 4, 16 * 2000))
    assert lib.fbp_volume_create(ctypes.byref(h), bad, 1, 0, 0) == 3         # misaligned
    bad = (fbp.fbp_item * 1)(fbp.fbp_item(64, 96, 91, None, 16 * 2000))
    assert lib.fbp_volume_create(ctypes.byref(h), bad, 1, 0, 0) == 1         # NULL buffer
    assert h.value is None
    assert lib.fbp_volume_run(None, None) == 1
    assert lib.fbp_volume_tune(None, None, None, None) == 1
    assert lib.fbp_volume_info(None, None, None) == 1
    assert lib.fbp_volume_group(None, 0, None, None, None, None, None, None) == 1
    assert lib.fbp_volume_destroy(None) == 0


def test_checked_library_exports_the_abi_and_its_test_hook(fbp):
    # the bounds-checked build: every function of include/fbp.h plus include/fbp_check.h;
    # the ordinary library does not export the test hook
    from paper_2007_06289_gb300 import build
    path = build.build(bounds_check=True)
    checked = ctypes.CDLL(path)
    hooks = fbp.header_functions(fbp.CHECK_HEADER)
    assert hooks == ["fbp_check_cnn_image_limit", "fbp_check_set_row_angle"]
    for name in fbp.header_functions() + hooks:
        assert hasattr(checked, name), name
    for name in hooks:
        assert not hasattr(fbp.load_library(), name), name
    # argument checks come before any CUDA call: FBP_ERR_INVALID_ARG without a GPU
    checked.fbp_check_cnn_image_limit.argtypes = [ctypes.c_int]
    checked.fbp_check_set_row_angle.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int]
    assert checked.fbp_check_cnn_image_limit(-1) == 1
    assert checked.fbp_check_set_row_angle(None, 0, 0, 0) == 1
