"""Thin ctypes binding of libfbp (include/fbp.h): same names, argument marshalling only.

Every step of the reconstruction runs in the library's CUDA kernels; this module checks
shapes, dtypes and devices of torch tensors, passes their device pointers and the current
CUDA stream, and turns status codes into exceptions.  There is no fallback: if the
library is missing or a call fails, an exception is raised.
"""
from __future__ import annotations

import ctypes
import os
import re

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfbp.so")
CHECKED_LIB_PATH = os.path.join(_HERE, "libfbp_checked.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "fbp.h")
CHECK_HEADER = os.path.join(os.path.dirname(_HERE), "include", "fbp_check.h")
MAX_ORDER = 8

_STATUS = {0: "FBP_OK", 1: "FBP_ERR_INVALID_ARG", 2: "FBP_ERR_UNSUPPORTED",
           3: "FBP_ERR_MISALIGNED", 4: "FBP_ERR_OOM", 5: "FBP_ERR_CUDA",
           6: "FBP_ERR_TIMEOUT", 7: "FBP_ERR_INTERNAL"}


class FbpError(RuntimeError):
    def __init__(self, fn, code):
        self.code = code
        super().__init__(f"{fn} failed: {_STATUS.get(code, code)} ({fbp_status_str(code)})")


class fbp_item(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("K", ctypes.c_int), ("M", ctypes.c_int),
                ("d_sino", ctypes.c_void_p), ("d_img", ctypes.c_void_p)]


FBP_VOLUME_GRAPH = 1


class fbp_iir_coeffs(ctypes.Structure):
    _fields_ = [("mb", ctypes.c_int), ("q", ctypes.c_int),
                ("b", ctypes.c_double * MAX_ORDER), ("a", ctypes.c_double * MAX_ORDER)]


_lib = None


def load_library(path: str | None = None) -> ctypes.CDLL:
    """Load libfbp.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    # FBP_LIBRARY names another build of the library (the bounds-checked one, in tests)
    path = path or os.environ.get("FBP_LIBRARY") or LIB_PATH
    if not os.path.exists(path):
        raise ImportError(f"libfbp.so not found at {path}; build it with "
                          "paper_2007_06289_gb300.build.build()")
    lib = ctypes.CDLL(path)
    P, I, F, V, S = ctypes.c_void_p, ctypes.c_int, ctypes.c_float, ctypes.c_void_p, ctypes.c_size_t
    sig = {
        "fbp_default_coeffs": (I, [I, I, ctypes.POINTER(fbp_iir_coeffs)]),
        "fbp_plan": (I, [ctypes.POINTER(P), I, I, I, I, ctypes.POINTER(fbp_iir_coeffs), I]),
        "fbp_plan_destroy": (I, [P]),
        "fbp_workspace_bytes": (S, [P]),
        "fbp_set_workspace": (I, [P, V, S]),
        "fbp_set_chunk": (I, [P, I]),
        "fbp_filter_iir": (I, [P, V, V, V]),
        "fbp_filter_fir": (I, [P, V, V, V]),
        "fbp_resample_st": (I, [P, V, V, V]),
        "fbp_fht_backproject": (I, [P, V, V, V]),
        "fbp_reconstruct": (I, [P, V, V, V]),
        "fbp_reconstruct_host": (I, [P, V, V, I, V]),
        "fbp_direct_reconstruct": (I, [P, V, V, V]),
        "fbp_fht_backproject_adjoint": (I, [P, V, V, V]),
        "fbp_hough_project": (I, [P, V, V, V]),
        "fbp_hough_data": (I, [P, V, V, V]),
        "fbp_radon": (I, [P, V, V, V]),
        "fbp_sirt": (I, [P, V, V, I, F, V]),
        "fbp_resample_st_adjoint": (I, [P, V, V, V]),
        "fbp_reconstruct_adjoint": (I, [P, V, V, V]),
        "fbp_fht_backproject_static": (I, [I, I, V, V, V]),
        "fbp_plan_info": (I, [P] + [ctypes.POINTER(I)] * 6),
        "fbp_profile_enable": (I, [P, I]),
        "fbp_profile_reset": (I, [P]),
        "fbp_profile_read": (I, [P, I, ctypes.POINTER(ctypes.c_double),
                                 ctypes.POINTER(ctypes.c_longlong)]),
        "fbp_status_str": (ctypes.c_char_p, [I]),
        "fbp_cnn_param_count": (S, []),
        "fbp_cnn_workspace_bytes": (S, [I, I, I]),
        "fbp_cnn_forward": (I, [V, V, V, V, S, I, I, I, V]),
        "fbp_cnn_backward": (I, [V, V, V, V, V, S, I, I, V]),
        "fbp_cnn_last_error": (I, []),
        "fbp_volume_create": (I, [ctypes.POINTER(P), ctypes.POINTER(fbp_item), I, I, I]),
        "fbp_volume_run": (I, [P, V]),
        "fbp_volume_tune": (I, [P, V, ctypes.POINTER(I), ctypes.POINTER(I)]),
        "fbp_volume_info": (I, [P, ctypes.POINTER(I), ctypes.POINTER(S)]),
        "fbp_volume_group": (I, [P, I] + [ctypes.POINTER(I)] * 6),
        "fbp_volume_destroy": (I, [P]),
        "fbp_last_device_error": (I, [P]),
    }
    if hasattr(lib, "fbp_check_set_row_angle"):           # bounds-checked build only
        sig["fbp_check_set_row_angle"] = (I, [P, I, I, I])
        sig["fbp_check_cnn_image_limit"] = (I, [I])
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    del F
    _lib = lib
    return lib


def header_functions(path: str = HEADER) -> list[str]:
    """Names of the functions that include/fbp.h declares."""
    text = open(path).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\*?\s+\**(fbp_\w+)\s*\(", text, flags=re.M)))


def _check(fn, code):
    if code != 0:
        raise FbpError(fn, code)


def fbp_status_str(code: int) -> str:
    return load_library().fbp_status_str(int(code)).decode()


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _dev_ptr(t, shape, name):
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name}: expected a torch tensor")
    if not t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous():
        raise ValueError(f"{name}: expected a contiguous float32 CUDA tensor")
    if t.numel() != _prod(shape):
        raise ValueError(f"{name}: expected {shape} elements, got shape {tuple(t.shape)}")
    return ctypes.c_void_p(t.data_ptr())


def _prod(shape):
    out = 1
    for v in shape:
        out *= v
    return out


def coeffs_struct(b, a) -> fbp_iir_coeffs:
    c = fbp_iir_coeffs()
    c.mb, c.q = len(b), len(a)
    if not (1 <= c.mb <= MAX_ORDER and 0 <= c.q <= MAX_ORDER):
        raise ValueError("filter order must be <= 8")
    for k, v in enumerate(b):
        c.b[k] = float(v)
    for k, v in enumerate(a):
        c.a[k] = float(v)
    return c


def fbp_default_coeffs(N: int, order: int = 0):
    """(b, a) lists of the built-in fitted filter for image size N (float64)."""
    c = fbp_iir_coeffs()
    _check("fbp_default_coeffs", load_library().fbp_default_coeffs(N, order, ctypes.byref(c)))
    return [c.b[k] for k in range(c.mb)], [c.a[k] for k in range(c.q)]


class Plan:
    """Owner of an fbp_plan_t handle (destroyed with the object)."""

    def __init__(self, N, K, M, batch, coeffs=None, fuse_k=0):
        lib = load_library()
        h = ctypes.c_void_p()
        cs = None if coeffs is None else ctypes.byref(coeffs_struct(*coeffs))
        _check("fbp_plan", lib.fbp_plan(ctypes.byref(h), N, K, M, batch, cs, fuse_k))
        self._h = h
        self.N, self.K, self.M, self.batch = N, K, M, batch
        self._refresh()
        self._ws = None

    def _refresh(self):
        vals = [ctypes.c_int() for _ in range(6)]
        _check("fbp_plan_info",
               load_library().fbp_plan_info(self._h, *[ctypes.byref(v) for v in vals]))
        self.fuse_k, self.chunk = vals[4].value, vals[5].value

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load_library().fbp_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # shapes
    @property
    def sino_shape(self):
        return (self.batch, self.K, self.M)

    @property
    def lin_shape(self):
        return (self.batch, 4, self.N, 2 * self.N)

    @property
    def img_shape(self):
        return (self.batch, self.N, self.N)


def fbp_plan(N: int, K: int, M: int, batch: int = 1, coeffs=None, fuse_k: int = 0) -> Plan:
    return Plan(N, K, M, batch, coeffs, fuse_k)


def fbp_plan_destroy(plan: Plan) -> None:
    plan.close()


def fbp_workspace_bytes(plan: Plan) -> int:
    return int(load_library().fbp_workspace_bytes(plan.handle))


def fbp_set_chunk(plan: Plan, chunk: int) -> None:
    """Slices per kernel sequence (0 = default); before the plan has a workspace."""
    _check("fbp_set_chunk", load_library().fbp_set_chunk(plan.handle, int(chunk)))
    plan._refresh()


def fbp_set_workspace(plan: Plan, ws) -> None:
    """Give the plan a caller-owned workspace (a CUDA uint8 tensor kept alive by the plan)."""
    lib = load_library()
    if ws is None:
        _check("fbp_set_workspace", lib.fbp_set_workspace(plan.handle, None, 0))
    else:
        _check("fbp_set_workspace",
               lib.fbp_set_workspace(plan.handle, ctypes.c_void_p(ws.data_ptr()),
                                     ws.numel() * ws.element_size()))
    plan._ws = ws


def fbp_plan_info(plan: Plan) -> dict:
    return dict(N=plan.N, K=plan.K, M=plan.M, batch=plan.batch, fuse_k=plan.fuse_k,
                chunk=plan.chunk)


def fbp_filter_iir(plan: Plan, sino, filt, stream=None) -> None:
    _check("fbp_filter_iir", load_library().fbp_filter_iir(
        plan.handle, _dev_ptr(sino, plan.sino_shape, "sino"),
        _dev_ptr(filt, plan.sino_shape, "filt"), _stream_ptr(stream)))


def fbp_filter_fir(plan: Plan, sino, filt, stream=None) -> None:
    _check("fbp_filter_fir", load_library().fbp_filter_fir(
        plan.handle, _dev_ptr(sino, plan.sino_shape, "sino"), _dev_ptr(filt, plan.sino_shape, "filt"),
        _stream_ptr(stream)))


def fbp_resample_st(plan: Plan, filt, lin, stream=None) -> None:
    _check("fbp_resample_st", load_library().fbp_resample_st(
        plan.handle, _dev_ptr(filt, plan.sino_shape, "filt"),
        _dev_ptr(lin, plan.lin_shape, "lin"), _stream_ptr(stream)))


def fbp_fht_backproject(plan: Plan, lin, img, stream=None) -> None:
    _check("fbp_fht_backproject", load_library().fbp_fht_backproject(
        plan.handle, _dev_ptr(lin, plan.lin_shape, "lin"),
        _dev_ptr(img, plan.img_shape, "img"), _stream_ptr(stream)))


def fbp_fht_backproject_static(N: int, lin, img, stream=None) -> None:
    """Hough back projection without a plan or workspace, for callers that cannot
    allocate device memory (scratch is a fixed array inside the library, N <= 512)."""
    count = lin.shape[0]
    _check("fbp_fht_backproject_static", load_library().fbp_fht_backproject_static(
        N, count, _dev_ptr(lin, (count, 4, N, 2 * N), "lin"),
        _dev_ptr(img, (count, N, N), "img"), _stream_ptr(stream)))


def fbp_reconstruct(plan: Plan, sino, img, stream=None) -> None:
    _check("fbp_reconstruct", load_library().fbp_reconstruct(
        plan.handle, _dev_ptr(sino, plan.sino_shape, "sino"),
        _dev_ptr(img, plan.img_shape, "img"), _stream_ptr(stream)))


def fbp_fht_backproject_adjoint(plan: Plan, img_grad, lin_grad, stream=None) -> None:
    _check("fbp_fht_backproject_adjoint", load_library().fbp_fht_backproject_adjoint(
        plan.handle, _dev_ptr(img_grad, plan.img_shape, "img_grad"),
        _dev_ptr(lin_grad, plan.lin_shape, "lin_grad"), _stream_ptr(stream)))


def fbp_hough_project(plan: Plan, img, lin, stream=None) -> None:
    _check("fbp_hough_project", load_library().fbp_hough_project(
        plan.handle, _dev_ptr(img, plan.img_shape, "img"),
        _dev_ptr(lin, plan.lin_shape, "lin"), _stream_ptr(stream)))


def fbp_hough_data(plan: Plan, sino, lin, stream=None) -> None:
    _check("fbp_hough_data", load_library().fbp_hough_data(
        plan.handle, _dev_ptr(sino, plan.sino_shape, "sino"),
        _dev_ptr(lin, plan.lin_shape, "lin"), _stream_ptr(stream)))


def fbp_radon(plan: Plan, img, sino, stream=None) -> None:
    _check("fbp_radon", load_library().fbp_radon(
        plan.handle, _dev_ptr(img, plan.img_shape, "img"),
        _dev_ptr(sino, plan.sino_shape, "sino"), _stream_ptr(stream)))


def fbp_sirt(plan: Plan, lin_data, img, iters: int, lam: float = 1.0, stream=None) -> None:
    """`iters` SIRT steps on img (in/out) for Hough-space data lin_data."""
    _check("fbp_sirt", load_library().fbp_sirt(
        plan.handle, _dev_ptr(lin_data, plan.lin_shape, "lin_data"),
        _dev_ptr(img, plan.img_shape, "img"), int(iters), float(lam), _stream_ptr(stream)))


def fbp_resample_st_adjoint(plan: Plan, lin_grad, filt_grad, stream=None) -> None:
    _check("fbp_resample_st_adjoint", load_library().fbp_resample_st_adjoint(
        plan.handle, _dev_ptr(lin_grad, plan.lin_shape, "lin_grad"),
        _dev_ptr(filt_grad, plan.sino_shape, "filt_grad"), _stream_ptr(stream)))


def fbp_reconstruct_adjoint(plan: Plan, img_grad, sino_grad, stream=None) -> None:
    _check("fbp_reconstruct_adjoint", load_library().fbp_reconstruct_adjoint(
        plan.handle, _dev_ptr(img_grad, plan.img_shape, "img_grad"),
        _dev_ptr(sino_grad, plan.sino_shape, "sino_grad"), _stream_ptr(stream)))


def fbp_direct_reconstruct(plan: Plan, sino, img, stream=None) -> None:
    _check("fbp_direct_reconstruct", load_library().fbp_direct_reconstruct(
        plan.handle, _dev_ptr(sino, plan.sino_shape, "sino"),
        _dev_ptr(img, plan.img_shape, "img"), _stream_ptr(stream)))


def fbp_reconstruct_host(plan: Plan, h_sino, h_img, count=None, stream=None) -> None:
    """Host (preferably pinned) float32 CPU tensors [count][K][M] -> [count][N][N]."""
    import torch
    for t, nm in ((h_sino, "h_sino"), (h_img, "h_img")):
        if not isinstance(t, torch.Tensor) or t.is_cuda or t.dtype != torch.float32 \
                or not t.is_contiguous():
            raise ValueError(f"{nm}: expected a contiguous float32 CPU tensor")
    count = count if count is not None else h_sino.shape[0]
    if h_sino.numel() < count * plan.K * plan.M or h_img.numel() < count * plan.N * plan.N:
        raise ValueError("host buffers too small for count slices")
    _check("fbp_reconstruct_host", load_library().fbp_reconstruct_host(
        plan.handle, ctypes.c_void_p(h_sino.data_ptr()), ctypes.c_void_p(h_img.data_ptr()),
        int(count), _stream_ptr(stream)))


KERNELS = ("iir", "resample", "pass1_resample", "pass1_linogram", "pass2", "fir", "direct_bp",
           "pass2_h")


def fbp_profile_enable(plan: Plan, enable: bool = True) -> None:
    _check("fbp_profile_enable", load_library().fbp_profile_enable(plan.handle, int(enable)))


def fbp_profile_reset(plan: Plan) -> None:
    _check("fbp_profile_reset", load_library().fbp_profile_reset(plan.handle))


def fbp_profile_read(plan: Plan) -> dict:
    """{kernel name: (event-timed ms, launches)} since the last reset."""
    lib = load_library()
    out = {}
    for k, name in enumerate(KERNELS):
        ms, n = ctypes.c_double(), ctypes.c_longlong()
        _check("fbp_profile_read", lib.fbp_profile_read(plan.handle, k, ctypes.byref(ms),
                                                        ctypes.byref(n)))
        out[name] = (ms.value, n.value)
    return out


def fbp_last_device_error(plan: Plan) -> int:
    return int(load_library().fbp_last_device_error(plan.handle))


# ----------------------------------------------------------------------------- ragged volumes
class Volume:
    """Owner of an fbp_volume_t over slices of mixed sizes: `items` is a list of
    (N, sino, img) with sino a [K][M] and img an [N][N] float32 CUDA tensor (kept alive by
    the volume)."""

    def __init__(self, items, order: int = 0, graph: bool = False):
        lib = load_library()
        arr = (fbp_item * len(items))()
        for i, (N, sino, img) in enumerate(items):
            if sino.dim() != 2 or tuple(img.shape) != (N, N):
                raise ValueError(f"item {i}: expected sino [K][M] and img [N][N]")
            K, M = sino.shape
            arr[i] = fbp_item(N, K, M, _dev_ptr(sino, (K, M), "sino"),
                              _dev_ptr(img, (N, N), "img"))
        h = ctypes.c_void_p()
        _check("fbp_volume_create",
               lib.fbp_volume_create(ctypes.byref(h), arr, len(items), int(order),
                                     FBP_VOLUME_GRAPH if graph else 0))
        self._h = h
        self._items = list(items)

    @property
    def handle(self):
        return self._h

    def run(self, stream=None) -> None:
        _check("fbp_volume_run", load_library().fbp_volume_run(self._h, _stream_ptr(stream)))

    def tune(self, stream=None) -> list[tuple[int, int]]:
        """Autotune every group; returns [(fuse_k, chunk)] per group."""
        n = self.info()["groups"]
        ks, cs = (ctypes.c_int * n)(), (ctypes.c_int * n)()
        _check("fbp_volume_tune",
               load_library().fbp_volume_tune(self._h, _stream_ptr(stream), ks, cs))
        return [(ks[i], cs[i]) for i in range(n)]

    def info(self) -> dict:
        g, ws = ctypes.c_int(), ctypes.c_size_t()
        _check("fbp_volume_info",
               load_library().fbp_volume_info(self._h, ctypes.byref(g), ctypes.byref(ws)))
        return {"groups": g.value, "workspace_bytes": ws.value}

    def group(self, i: int) -> dict:
        vals = [ctypes.c_int() for _ in range(6)]
        _check("fbp_volume_group", load_library().fbp_volume_group(
            self._h, int(i), *[ctypes.byref(v) for v in vals]))
        return dict(zip(("N", "K", "M", "items", "fuse_k", "chunk"), (v.value for v in vals)))

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load_library().fbp_volume_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fbp_volume_create(items, order: int = 0, graph: bool = False) -> Volume:
    return Volume(items, order, graph)


def fbp_volume_run(volume: Volume, stream=None) -> None:
    volume.run(stream)


def fbp_volume_tune(volume: Volume, stream=None):
    return volume.tune(stream)


def fbp_volume_info(volume: Volume) -> dict:
    return volume.info()


def fbp_volume_group(volume: Volume, i: int) -> dict:
    return volume.group(i)


def fbp_volume_destroy(volume: Volume) -> None:
    volume.close()


# ----------------------------------------------------------------------------- learned corrector
def fbp_cnn_param_count() -> int:
    return int(load_library().fbp_cnn_param_count())


def fbp_cnn_workspace_bytes(N: int, batch: int, train: bool) -> int:
    return int(load_library().fbp_cnn_workspace_bytes(int(N), int(batch), int(bool(train))))


def _ws_ptr(ws):
    import torch
    if not isinstance(ws, torch.Tensor) or not ws.is_cuda or not ws.is_contiguous():
        raise ValueError("ws: expected a contiguous CUDA tensor")
    return ctypes.c_void_p(ws.data_ptr()), ws.numel() * ws.element_size()


def fbp_cnn_forward(params, x, y, ws, train: bool = False, stream=None) -> None:
    """y = x + net(x) for x [batch][N][N] (float32 CUDA); ws from fbp_cnn_workspace_bytes."""
    B, N = x.shape[0], x.shape[-1]
    p, nb = _ws_ptr(ws)
    _check("fbp_cnn_forward", load_library().fbp_cnn_forward(
        _dev_ptr(params, (fbp_cnn_param_count(),), "params"), _dev_ptr(x, (B, N, N), "x"),
        _dev_ptr(y, (B, N, N), "y"), p, nb, N, B, int(bool(train)), _stream_ptr(stream)))


def fbp_cnn_backward(params, x, gy, gparams, ws, stream=None) -> None:
    B, N = x.shape[0], x.shape[-1]
    p, nb = _ws_ptr(ws)
    _check("fbp_cnn_backward", load_library().fbp_cnn_backward(
        _dev_ptr(params, (fbp_cnn_param_count(),), "params"), _dev_ptr(x, (B, N, N), "x"),
        _dev_ptr(gy, (B, N, N), "gy"), _dev_ptr(gparams, (fbp_cnn_param_count(),), "gparams"),
        p, nb, N, B, _stream_ptr(stream)))


def fbp_cnn_last_error() -> int:
    """Read and clear the corrector's device status word (synchronises the device)."""
    return int(load_library().fbp_cnn_last_error())


def fbp_check_set_row_angle(plan: Plan, q: int, i: int, k0: int) -> None:
    """Test hook of the bounds-checked library (include/fbp_check.h)."""
    _check("fbp_check_set_row_angle",
           load_library().fbp_check_set_row_angle(plan.handle, int(q), int(i), int(k0)))


def fbp_check_cnn_image_limit(images: int) -> None:
    """Test hook of the bounds-checked library (include/fbp_check.h)."""
    _check("fbp_check_cnn_image_limit", load_library().fbp_check_cnn_image_limit(int(images)))
