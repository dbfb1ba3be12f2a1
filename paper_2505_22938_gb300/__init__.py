"""Thin Python binding of libfim, the GB300 exact isotropic median filter.

Every function here marshals arguments into the C ABI declared in ``include/fim.h``
and calls it; all filtering happens in the library's CUDA kernels. Names follow the C ABI.
PyTorch is used only to hand over device pointers and streams (``tensor.data_ptr()``,
``torch.cuda.current_stream().cuda_stream``); the C signatures carry plain pointers.

The library is built in-tree (``paper_2505_22938_gb300/_build/libfim.so``). Importing
this module never falls back to any other implementation: if the library cannot be
loaded, ``lib()`` raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

FIM_U8, FIM_U16, FIM_F32 = 0, 1, 2
FIM_BORDER_CLAMP = 0
STATUS = {0: "FIM_OK", 1: "FIM_ERR_INVALID_ARG", 2: "FIM_ERR_UNSUPPORTED", 3: "FIM_ERR_OOM",
          4: "FIM_ERR_CUDA", 5: "FIM_ERR_TIMEOUT", 6: "FIM_ERR_INTERNAL"}
DTYPES = {"u8": FIM_U8, "u16": FIM_U16, "f32": FIM_F32}
ELEM_SIZE = {FIM_U8: 1, FIM_U16: 2, FIM_F32: 4}

# Every symbol include/fim.h declares, with (restype, argtypes).
_c = ctypes
_P = _c.c_void_p
_PP = _c.POINTER(_c.c_void_p)
SIGNATURES = {
    "fim_create_kernel_circle": (_c.c_int, [_c.c_int, _PP]),
    "fim_create_kernel_disk_limit": (_c.c_int, [_c.c_int64, _PP]),
    "fim_create_kernel_ellipse": (_c.c_int, [_c.c_int, _c.c_int, _PP]),
    "fim_create_kernel_polygon": (_c.c_int, [_P, _c.c_int, _PP]),
    "fim_create_kernel_spans": (_c.c_int, [_P, _P, _c.c_int, _c.c_int, _PP]),
    "fim_kernel_info": (_c.c_int, [_P, _P, _P, _P, _P, _P]),
    "fim_destroy_kernel": (None, [_P]),
    "fim_median": (_c.c_int, [_P, _P, _c.c_int, _c.c_int, _c.c_size_t, _c.c_int, _P, _c.c_int, _P]),
    "fim_percentile": (_c.c_int, [_P, _P, _c.c_int, _c.c_int, _c.c_size_t, _c.c_int, _P, _c.c_double,
                                  _c.c_int, _P]),
    "fim_percentiles": (_c.c_int, [_P, _P, _P, _c.c_int, _c.c_int, _c.c_int, _c.c_size_t, _c.c_int, _P,
                                   _c.c_int, _P]),
    "fim_percentile_map": (_c.c_int, [_P, _P, _P, _c.c_size_t, _c.c_int, _c.c_int, _c.c_size_t, _c.c_int, _P,
                                      _c.c_int, _P]),
    "fim_median_radii": (_c.c_int, [_P, _P, _P, _c.c_int, _c.c_int, _c.c_int, _c.c_size_t, _c.c_int, _c.c_int,
                                    _P]),
    "fim_median_host": (_c.c_int, [_P, _P, _c.c_int, _c.c_int, _c.c_size_t, _c.c_int, _P, _c.c_int, _P]),
    "fim_median_noalloc": (_c.c_int, [_P, _P, _c.c_int, _c.c_int, _c.c_size_t, _c.c_int, _P, _c.c_int, _P]),
    "fim_sync_status": (_c.c_int, [_P]),
    "fim_status_string": (_c.c_char_p, [_c.c_int]),
    "fim_version": (_c.c_char_p, []),
    "fim_debug_phase_clocks": (_c.c_int, [_P, _c.c_int]),
    "fim_plan_info": (_c.c_int, [_P, _c.c_int, _c.c_int, _c.c_int, _P, _P, _P, _P, _P]),
    "fim_release_workspace": (_c.c_int, []),
    "fim_autotune": (_c.c_int, [_P, _P, _c.c_int, _c.c_int, _c.c_size_t, _c.c_int, _P, _c.c_int, _P, _P, _P]),
    "fim_autotune_clear": (_c.c_int, []),
    "fim_batch_create": (_c.c_int, [_P, _c.c_int, _PP]),
    "fim_batch_run": (_c.c_int, [_P, _P]),
    "fim_batch_info": (_c.c_int, [_P, _P, _P, _P, _P]),
    "fim_batch_destroy": (None, [_P]),
    "fim_median_batch": (_c.c_int, [_P, _c.c_int, _P]),
    "fim_model_param_count": (_c.c_int, []),
    "fim_model_create": (_c.c_int, [_c.c_uint64, _PP]),
    "fim_model_destroy": (None, [_P]),
    "fim_model_get_params": (_c.c_int, [_P, _P, _P]),
    "fim_model_set_params": (_c.c_int, [_P, _P]),
    "fim_model_bracket_z": (_c.c_float, [_P]),
    "fim_model_forward": (_c.c_int, [_P, _P, _c.c_int, _c.c_int, _P, _P]),
    "fim_model_loss_grad": (_c.c_int, [_P, _P, _c.c_int, _c.c_int, _P, _c.c_int, _P, _P, _P]),
    "fim_model_train": (_c.c_int, [_P, _P, _c.c_int, _c.c_int, _c.c_int, _c.c_float, _P, _P]),
    "fim_model_calibrate": (_c.c_int, [_P, _P, _c.c_int, _c.c_double, _P, _P]),
    "fim_model_save": (_c.c_int, [_P, _c.c_char_p]),
    "fim_model_load": (_c.c_int, [_c.c_char_p, _PP]),
    "fim_collect_seed_samples": (_c.c_int, [_P, _P, _c.c_int, _c.c_int, _c.c_size_t, _c.c_int, _P, _P, _c.c_int,
                                            _P, _P]),
    "fim_median_learned": (_c.c_int, [_P, _P, _c.c_int, _c.c_int, _c.c_size_t, _c.c_int, _P, _P, _c.c_int, _P,
                                      _P]),
}

N_FEATURES = 41
ROW = N_FEATURES + 1


class fim_job(ctypes.Structure):
    """Mirror of the C struct fim_job."""
    _fields_ = [("in_ptr", ctypes.c_void_p), ("out_ptr", ctypes.c_void_p), ("w", ctypes.c_int),
                ("h", ctypes.c_int), ("pitch_bytes", ctypes.c_size_t), ("dtype", ctypes.c_int),
                ("kernel", ctypes.c_void_p), ("percentile", ctypes.c_double)]

_lock = threading.Lock()
_lib = None


class FimError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {STATUS.get(code, code)}")
        self.code = code


def lib_path() -> str:
    return _build.LIB_PATH


def lib(build_if_missing: bool = True) -> ctypes.CDLL:
    """Loads libfim (building it first if needed) and declares every exported signature."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build() if build_if_missing else _build.LIB_PATH
            if not os.path.exists(path):
                raise RuntimeError(f"libfim is not built ({path}); run paper_2505_22938_gb300.build.build()")
            handle = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(handle, name)
                fn.restype = res
                fn.argtypes = args
            _lib = handle
    return _lib


def _check(code: int, what: str) -> None:
    if code != 0:
        raise FimError(code, what)


class Kernel:
    """Owns a fim_kernel handle."""

    def __init__(self, handle: ctypes.c_void_p):
        self.handle = handle

    @property
    def info(self) -> dict:
        vals = [ctypes.c_int() for _ in range(5)]
        _check(lib().fim_kernel_info(self.handle, *[ctypes.byref(v) for v in vals]), "fim_kernel_info")
        n, xmin, xmax, ymin, ymax = (v.value for v in vals)
        return dict(ntaps=n, xmin=xmin, xmax=xmax, ymin=ymin, ymax=ymax)

    def close(self) -> None:
        if self.handle:
            lib().fim_destroy_kernel(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _new_kernel(fn_name: str, *args) -> Kernel:
    h = ctypes.c_void_p()
    _check(getattr(lib(), fn_name)(*args, ctypes.byref(h)), fn_name)
    return Kernel(h)


def fim_create_kernel_circle(radius: int) -> Kernel:
    return _new_kernel("fim_create_kernel_circle", int(radius))


def fim_create_kernel_disk_limit(limit: int) -> Kernel:
    return _new_kernel("fim_create_kernel_disk_limit", int(limit))


def fim_create_kernel_ellipse(a: int, b: int) -> Kernel:
    return _new_kernel("fim_create_kernel_ellipse", int(a), int(b))


def fim_create_kernel_polygon(xy) -> Kernel:
    flat = [float(v) for p in xy for v in p]
    arr = (ctypes.c_double * len(flat))(*flat)
    return _new_kernel("fim_create_kernel_polygon", ctypes.cast(arr, ctypes.c_void_p), len(flat) // 2)


def fim_create_kernel_spans(lo, hi, dy0: int) -> Kernel:
    lo = [int(v) for v in lo]
    hi = [int(v) for v in hi]
    a = (ctypes.c_int * len(lo))(*lo)
    b = (ctypes.c_int * len(hi))(*hi)
    return _new_kernel("fim_create_kernel_spans", ctypes.cast(a, ctypes.c_void_p), ctypes.cast(b, ctypes.c_void_p),
                       int(dy0), len(lo))


def fim_median(in_ptr: int, out_ptr: int, w: int, h: int, pitch_bytes: int, dtype: int, kernel: Kernel,
               stream: int = 0, border: int = FIM_BORDER_CLAMP) -> None:
    """Raw C-ABI call on device pointers (asynchronous on `stream`)."""
    _check(lib().fim_median(in_ptr, out_ptr, w, h, pitch_bytes, dtype, kernel.handle, border, stream or None),
           "fim_median")


def fim_median_noalloc(in_ptr: int, out_ptr: int, w: int, h: int, pitch_bytes: int, dtype: int, kernel: Kernel,
                       stream: int = 0, border: int = FIM_BORDER_CLAMP) -> None:
    """fim_median without any device allocation: uses the library's fixed device workspace."""
    _check(lib().fim_median_noalloc(in_ptr, out_ptr, w, h, pitch_bytes, dtype, kernel.handle, border,
                                    stream or None), "fim_median_noalloc")


def fim_percentile(in_ptr: int, out_ptr: int, w: int, h: int, pitch_bytes: int, dtype: int, kernel: Kernel,
                   percentile: float, stream: int = 0, border: int = FIM_BORDER_CLAMP) -> None:
    _check(lib().fim_percentile(in_ptr, out_ptr, w, h, pitch_bytes, dtype, kernel.handle, float(percentile),
                                border, stream or None), "fim_percentile")


def fim_percentiles(in_ptr: int, out_ptrs, percentiles, w: int, h: int, pitch_bytes: int, dtype: int,
                    kernel: Kernel, stream: int = 0, border: int = FIM_BORDER_CLAMP) -> None:
    """Several percentile filters of one image from one ordinal transform per tile."""
    count = len(out_ptrs)
    outs = (_c.c_void_p * max(count, 1))(*[_c.c_void_p(p) for p in out_ptrs])
    pcts = (_c.c_double * max(len(percentiles), 1))(*[float(x) for x in percentiles])
    _check(lib().fim_percentiles(in_ptr, outs, pcts, count, w, h, pitch_bytes, dtype, kernel.handle, border,
                                 stream or None), "fim_percentiles")


def fim_median_radii(in_ptr: int, out_ptrs, kernels, w: int, h: int, pitch_bytes: int, dtype: int,
                     stream: int = 0, border: int = FIM_BORDER_CLAMP) -> None:
    """Median filters with several disk kernels from one ordinal transform per tile."""
    count = len(out_ptrs)
    outs = (_c.c_void_p * max(count, 1))(*[_c.c_void_p(p) for p in out_ptrs])
    ks = (_c.c_void_p * max(len(kernels), 1))(*[k.handle for k in kernels])
    _check(lib().fim_median_radii(in_ptr, outs, ks, count, w, h, pitch_bytes, dtype, border, stream or None),
           "fim_median_radii")


def fim_percentile_map(in_ptr: int, out_ptr: int, pct_ptr: int, pct_pitch_bytes: int, w: int, h: int,
                       pitch_bytes: int, dtype: int, kernel: Kernel, stream: int = 0,
                       border: int = FIM_BORDER_CLAMP) -> None:
    """Rank-order filter with a percentile per output pixel (device float32 map)."""
    _check(lib().fim_percentile_map(in_ptr, out_ptr, pct_ptr, pct_pitch_bytes, w, h, pitch_bytes, dtype,
                                    kernel.handle, border, stream or None), "fim_percentile_map")


def fim_median_host(in_ptr: int, out_ptr: int, w: int, h: int, pitch_bytes: int, dtype: int, kernel: Kernel,
                    stream: int = 0, border: int = FIM_BORDER_CLAMP) -> None:
    """Raw C-ABI call on HOST pointers; returns once the result is in host memory."""
    _check(lib().fim_median_host(in_ptr, out_ptr, w, h, pitch_bytes, dtype, kernel.handle, border,
                                 stream or None), "fim_median_host")


def fim_sync_status(stream: int = 0) -> int:
    return int(lib().fim_sync_status(stream or None))


def fim_status_string(code: int) -> str:
    return lib().fim_status_string(int(code)).decode()


def fim_autotune(in_ptr: int, out_ptr: int, w: int, h: int, pitch_bytes: int, dtype: int, kernel: Kernel,
                 stream: int = 0, cta_threads: int = 0) -> tuple:
    tw, th = ctypes.c_int(), ctypes.c_int()
    _check(lib().fim_autotune(in_ptr, out_ptr, w, h, pitch_bytes, dtype, kernel.handle, int(cta_threads),
                              stream or None, ctypes.byref(tw), ctypes.byref(th)), "fim_autotune")
    return tw.value, th.value


def fim_autotune_clear() -> None:
    _check(lib().fim_autotune_clear(), "fim_autotune_clear")


class Batch:
    """Owns a fim_batch handle (and keeps its kernels alive)."""

    def __init__(self, jobs: list, kernels: list):
        arr = (fim_job * len(jobs))(*jobs)
        h = ctypes.c_void_p()
        _check(lib().fim_batch_create(ctypes.cast(arr, ctypes.c_void_p), len(jobs), ctypes.byref(h)),
               "fim_batch_create")
        self.handle = h
        self._kernels = kernels

    def run(self, stream: int = 0) -> None:
        _check(lib().fim_batch_run(self.handle, stream or None), "fim_batch_run")

    @property
    def info(self) -> dict:
        vals = [ctypes.c_int() for _ in range(4)]
        _check(lib().fim_batch_info(self.handle, *[ctypes.byref(v) for v in vals]), "fim_batch_info")
        return dict(zip(("total_tiles", "grid", "threads", "smem_bytes"), (v.value for v in vals)))

    def close(self) -> None:
        if self.handle:
            lib().fim_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def make_job(in_ptr: int, out_ptr: int, w: int, h: int, pitch_bytes: int, dtype: int, kernel: Kernel,
             percentile: float = -1.0) -> fim_job:
    return fim_job(in_ptr, out_ptr, w, h, pitch_bytes, dtype, kernel.handle, float(percentile))


def fim_batch_create(jobs: list, kernels: list) -> Batch:
    return Batch(jobs, kernels)


def fim_median_batch(jobs: list, stream: int = 0) -> None:
    arr = (fim_job * len(jobs))(*jobs)
    _check(lib().fim_median_batch(ctypes.cast(arr, ctypes.c_void_p), len(jobs), stream or None),
           "fim_median_batch")


class Model:
    """Owns a fim_model handle (the learned seed-bracket network)."""

    def __init__(self, handle):
        self.handle = handle

    @classmethod
    def create(cls, seed: int = 1) -> "Model":
        h = ctypes.c_void_p()
        _check(lib().fim_model_create(int(seed), ctypes.byref(h)), "fim_model_create")
        return cls(h)

    @classmethod
    def load(cls, path: str) -> "Model":
        h = ctypes.c_void_p()
        _check(lib().fim_model_load(path.encode(), ctypes.byref(h)), "fim_model_load")
        return cls(h)

    def save(self, path: str) -> None:
        _check(lib().fim_model_save(self.handle, path.encode()), "fim_model_save")

    @staticmethod
    def param_count() -> int:
        return int(lib().fim_model_param_count())

    def params(self):
        import numpy as np
        n = self.param_count()
        f = np.empty(n, np.float32)
        b = np.empty(n, np.uint16)
        _check(lib().fim_model_get_params(self.handle, f.ctypes.data, b.ctypes.data), "fim_model_get_params")
        return f, b

    def set_params(self, host_fp32) -> None:
        import numpy as np
        a = np.ascontiguousarray(host_fp32, dtype=np.float32)
        assert a.size == self.param_count()
        _check(lib().fim_model_set_params(self.handle, a.ctypes.data), "fim_model_set_params")

    @property
    def bracket_z(self) -> float:
        return float(lib().fim_model_bracket_z(self.handle))

    def forward(self, x_ptr: int, rows: int, row_stride: int, out_ptr: int, stream: int = 0) -> None:
        _check(lib().fim_model_forward(self.handle, x_ptr, rows, row_stride, out_ptr, stream or None),
               "fim_model_forward")

    def loss_grad(self, x_ptr: int, rows: int, row_stride: int, y_ptr: int, y_stride: int, grad_ptr: int,
                  stream: int = 0) -> float:
        loss = ctypes.c_float()
        _check(lib().fim_model_loss_grad(self.handle, x_ptr, rows, row_stride, y_ptr, y_stride, grad_ptr or None,
                                         ctypes.byref(loss), stream or None), "fim_model_loss_grad")
        return loss.value

    def train(self, rows_ptr: int, rows: int, epochs: int, batch: int, lr: float, stream: int = 0) -> float:
        loss = ctypes.c_float()
        _check(lib().fim_model_train(self.handle, rows_ptr, rows, epochs, batch, float(lr), stream or None,
                                     ctypes.byref(loss)), "fim_model_train")
        return loss.value

    def calibrate(self, rows_ptr: int, rows: int, coverage: float, stream: int = 0) -> float:
        z = ctypes.c_float()
        _check(lib().fim_model_calibrate(self.handle, rows_ptr, rows, float(coverage), stream or None,
                                         ctypes.byref(z)), "fim_model_calibrate")
        return z.value

    def close(self) -> None:
        if self.handle:
            lib().fim_model_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fim_collect_seed_samples(in_ptr: int, out_ptr: int, w: int, h: int, pitch_bytes: int, dtype: int, kernel: Kernel,
                             rows_ptr: int, capacity: int, count_ptr: int, stream: int = 0) -> None:
    _check(lib().fim_collect_seed_samples(in_ptr, out_ptr, w, h, pitch_bytes, dtype, kernel.handle, rows_ptr,
                                          capacity, count_ptr, stream or None), "fim_collect_seed_samples")


def fim_median_learned(in_ptr: int, out_ptr: int, w: int, h: int, pitch_bytes: int, dtype: int, kernel: Kernel,
                       model, stream: int = 0, stats_ptr: int = 0, border: int = FIM_BORDER_CLAMP) -> None:
    _check(lib().fim_median_learned(in_ptr, out_ptr, w, h, pitch_bytes, dtype, kernel.handle,
                                    model.handle if model is not None else None, border, stream or None,
                                    stats_ptr or None), "fim_median_learned")


def fim_release_workspace() -> None:
    _check(lib().fim_release_workspace(), "fim_release_workspace")


def fim_version() -> str:
    return lib().fim_version().decode()


def fim_plan_info(kernel: Kernel, dtype: int, w: int, h: int) -> dict:
    vals = [ctypes.c_int() for _ in range(5)]
    _check(lib().fim_plan_info(kernel.handle, dtype, w, h, *[ctypes.byref(v) for v in vals]), "fim_plan_info")
    return dict(zip(("tile_w", "tile_h", "footprint", "threads", "smem_bytes"), (v.value for v in vals)))


def fim_debug_phase_clocks(dev_ptr: int, tiles: int) -> None:
    _check(lib().fim_debug_phase_clocks(dev_ptr or None, int(tiles)), "fim_debug_phase_clocks")


# ---------------------------------------------------------------------------------------------
# torch conveniences (device memory and streams only)
# ---------------------------------------------------------------------------------------------

def _torch_dtype_code(t) -> int:
    import torch
    m = {torch.uint8: FIM_U8, torch.uint16: FIM_U16, torch.float32: FIM_F32}
    if t.dtype not in m:
        raise TypeError(f"unsupported dtype {t.dtype}")
    return m[t.dtype]


def _stream_handle(stream=None) -> int:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def median(img, kernel: Kernel, out=None, stream=None):
    """Median-filters a 2-D CUDA tensor (uint8, uint16 or float32) on the current stream."""
    import torch
    assert img.is_cuda and img.dim() == 2 and img.stride(1) == 1
    code = _torch_dtype_code(img)
    if out is None:
        out = torch.empty_like(img, memory_format=torch.contiguous_format)
    assert out.shape == img.shape and out.dtype == img.dtype and out.stride(0) == img.stride(0)
    pitch = img.stride(0) * img.element_size()
    h, w = img.shape
    fim_median(img.data_ptr(), out.data_ptr(), w, h, pitch, code, kernel, _stream_handle(stream))
    return out


def percentile(img, kernel: Kernel, pct: float, out=None, stream=None):
    import torch
    assert img.is_cuda and img.dim() == 2 and img.stride(1) == 1
    code = _torch_dtype_code(img)
    if out is None:
        out = torch.empty_like(img, memory_format=torch.contiguous_format)
    pitch = img.stride(0) * img.element_size()
    h, w = img.shape
    fim_percentile(img.data_ptr(), out.data_ptr(), w, h, pitch, code, kernel, pct, _stream_handle(stream))
    return out


def percentiles(img, kernel: Kernel, pcts, stream=None):
    """Returns one filtered image per percentile in `pcts` (at most 8), all from one launch."""
    import torch
    assert img.is_cuda and img.dim() == 2 and img.stride(1) == 1
    code = _torch_dtype_code(img)
    outs = [torch.empty_strided(img.shape, img.stride(), dtype=img.dtype, device=img.device) for _ in pcts]
    pitch = img.stride(0) * img.element_size()
    h, w = img.shape
    fim_percentiles(img.data_ptr(), [o.data_ptr() for o in outs], list(pcts), w, h, pitch, code, kernel,
                    _stream_handle(stream))
    return outs


def median_radii(img, kernels, stream=None):
    """Returns one median-filtered image per disk kernel in `kernels` (at most 8), all from one
    launch."""
    import torch
    assert img.is_cuda and img.dim() == 2 and img.stride(1) == 1
    code = _torch_dtype_code(img)
    outs = [torch.empty_strided(img.shape, img.stride(), dtype=img.dtype, device=img.device) for _ in kernels]
    pitch = img.stride(0) * img.element_size()
    h, w = img.shape
    fim_median_radii(img.data_ptr(), [o.data_ptr() for o in outs], list(kernels), w, h, pitch, code,
                     _stream_handle(stream))
    return outs


def percentile_map(img, kernel: Kernel, pct, out=None, stream=None):
    """Filters a 2-D CUDA tensor with a percentile per pixel: pct is a float32 CUDA tensor of
    the image's shape (values in [0, 100])."""
    import torch
    assert img.is_cuda and img.dim() == 2 and img.stride(1) == 1
    assert pct.is_cuda and pct.dtype == torch.float32 and pct.shape == img.shape and pct.stride(1) == 1
    code = _torch_dtype_code(img)
    if out is None:
        out = torch.empty_strided(img.shape, img.stride(), dtype=img.dtype, device=img.device)
    assert out.shape == img.shape and out.dtype == img.dtype and out.stride(0) == img.stride(0)
    pitch = img.stride(0) * img.element_size()
    h, w = img.shape
    fim_percentile_map(img.data_ptr(), out.data_ptr(), pct.data_ptr(), pct.stride(0) * 4, w, h, pitch, code,
                       kernel, _stream_handle(stream))
    return out


def median_host(arr, kernel: Kernel, out=None, stream=None):
    """Median-filters a 2-D host numpy array through fim_median_host (copies in and out)."""
    import numpy as np
    codes = {np.dtype(np.uint8): FIM_U8, np.dtype(np.uint16): FIM_U16, np.dtype(np.float32): FIM_F32}
    a = np.ascontiguousarray(arr)
    code = codes[a.dtype]
    if out is None:
        out = np.empty_like(a)
    h, w = a.shape
    fim_median_host(a.ctypes.data, out.ctypes.data, w, h, a.strides[0], code, kernel,
                    _stream_handle(stream) if stream is not None else 0)
    return out
