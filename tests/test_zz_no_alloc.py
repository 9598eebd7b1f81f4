"""The allocation-free Hough back projection (fbp_fht_backproject_static).

It serves callers that cannot allocate device memory, so it takes no plan and no
workspace and keeps its scratch in a fixed array inside the library.  This file is
collected last so that a run stopping at the first failure has run everything else; it
also passes on its own in a fresh process.  Each check calls the entry point twice in a
row (the second call sees the first call's leftovers in the shared scratch) and compares
with fbp_fht_backproject, bit for bit like every other Hough test.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("N", [2, 4, 8, 64, 256, 512])
def test_static_scratch_matches_planned_backprojection_twice(fbp, N):
    import torch
    lib = fbp.load_library()
    plan = fbp.fbp_plan(N, 8, 8, 2)
    rng = np.random.default_rng(N)
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        lin = torch.from_numpy(rng.normal(size=(2, 4, N, 2 * N)).astype(np.float32)).cuda()
        want = torch.empty((2, N, N), device="cuda")
        got = torch.full((2, N, N), float("nan"), device="cuda")
        fbp.fbp_fht_backproject(plan, lin, want)
        rc = lib.fbp_fht_backproject_static(N, 2, ctypes.c_void_p(lin.data_ptr()),
                                            ctypes.c_void_p(got.data_ptr()),
                                            ctypes.c_void_p(stream))
        assert rc == 0, fbp.fbp_status_str(rc)
        torch.cuda.synchronize()
        assert torch.equal(got, want), f"call {call}"


def test_static_scratch_rejects_sizes_beyond_its_limit(fbp):
    import torch
    lib = fbp.load_library()
    buf = torch.zeros(16, device="cuda")
    p = ctypes.c_void_p(buf.data_ptr())
    assert lib.fbp_fht_backproject_static(1024, 1, p, p, None) == 2     # N above the maximum
    assert lib.fbp_fht_backproject_static(48, 1, p, p, None) == 2       # not a power of two
    assert lib.fbp_fht_backproject_static(64, 0, p, p, None) == 1       # empty batch


def test_static_scratch_allocates_nothing(fbp):
    # After one warm-up call (which may make the driver back the fixed array and load the
    # kernels), further calls leave the device's free memory unchanged.
    import torch
    lib = fbp.load_library()
    N = 512
    lin = torch.zeros((3, 4, N, 2 * N), device="cuda")
    img = torch.empty((3, N, N), device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    args = (N, 3, ctypes.c_void_p(lin.data_ptr()), ctypes.c_void_p(img.data_ptr()),
            ctypes.c_void_p(stream))
    assert lib.fbp_fht_backproject_static(*args) == 0
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        assert lib.fbp_fht_backproject_static(*args) == 0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
