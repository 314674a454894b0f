"""Python binding of libdeconv.so, the GB300 partial-ADMM deconvolution library
(arXiv:1602.01410, "A Framework for Fast Image Deconvolution with Incomplete
Observations").

The functions below carry the names of the C entry points declared in
include/deconv.h and only marshal arguments (ints, doubles and raw pointers)
through ctypes; every step of the solve runs in the library's CUDA kernels.
`Plan` is a convenience wrapper that owns the device workspace as a torch
tensor and passes torch tensors' data pointers and the current CUDA stream.

The library must be built first (``paper_1602_01410_gb300.build.build()`` or
``__graft_entry__.build()``); importing the functions fails loudly when it is
missing.  There is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdeconv.so")

DECONV_OK, DECONV_EINVAL, DECONV_EUNSUPPORTED, DECONV_ENOMEM, DECONV_ECUDA, DECONV_ETIMEOUT, \
    DECONV_ENONFINITE = range(7)
DECONV_F32, DECONV_F64 = 0, 1

# Entry points declared in include/deconv.h (checked by the test suite).
EXPORTS = ("deconv_workspace_size", "deconv_plan_create", "deconv_solve", "deconv_solve_host",
           "deconv_profile_passes", "deconv_sync", "deconv_plan_destroy", "deconv_status_string",
           "deconv_solve_noalloc")


class DeconvError(RuntimeError):
    def __init__(self, status: int, where: str):
        super().__init__(f"{where}: {deconv_status_string(status)} (status {status})")
        self.status = status


class deconv_dims(ctypes.Structure):
    _fields_ = [("batch", ctypes.c_int32), ("channels", ctypes.c_int32),
                ("rows", ctypes.POINTER(ctypes.c_int32)), ("cols", ctypes.POINTER(ctypes.c_int32)),
                ("ksize", ctypes.c_int32), ("kernel_per_image", ctypes.c_int32),
                ("dtype", ctypes.c_int32), ("relax", ctypes.c_float)]


_lib = None


def load() -> ctypes.CDLL:
    """Load libdeconv.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_1602_01410_gb300.build.build()")
        lib = ctypes.CDLL(LIB_PATH)
        vp, i32, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_double
        lib.deconv_workspace_size.argtypes = [ctypes.POINTER(deconv_dims), ctypes.POINTER(ctypes.c_size_t)]
        lib.deconv_plan_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(deconv_dims), vp, vp, dbl, dbl,
                                           vp, ctypes.c_size_t, vp]
        lib.deconv_solve.argtypes = [vp, vp, vp, i32, i32, vp]
        lib.deconv_solve_host.argtypes = [vp, vp, vp, i32]
        lib.deconv_profile_passes.argtypes = [vp, i32, ctypes.POINTER(ctypes.c_float)]
        lib.deconv_sync.argtypes = [vp]
        lib.deconv_solve_noalloc.argtypes = [ctypes.POINTER(deconv_dims), vp, vp, vp, vp, dbl, dbl, i32, vp]
        lib.deconv_plan_destroy.argtypes = [vp]
        lib.deconv_status_string.argtypes = [ctypes.c_int]
        lib.deconv_status_string.restype = ctypes.c_char_p
        for name in EXPORTS:
            if name != "deconv_status_string":
                getattr(lib, name).restype = ctypes.c_int
        _lib = lib
    return _lib


def make_dims(rows: Sequence[int], cols: Sequence[int], ksize: int, channels: int = 1,
              dtype: int = DECONV_F32, relax: float = 2.0, kernel_per_image: int = 0):
    """Build a deconv_dims; returns (dims, keepalive) - keep both referenced."""
    r = (ctypes.c_int32 * len(rows))(*rows)
    c = (ctypes.c_int32 * len(cols))(*cols)
    d = deconv_dims(len(rows), channels, r, c, ksize, kernel_per_image, dtype, relax)
    return d, (r, c)


def _check(status: int, where: str) -> None:
    if status != DECONV_OK:
        raise DeconvError(status, where)


# ------------------------------------------------------------- C entry points


def deconv_status_string(status: int) -> str:
    return load().deconv_status_string(int(status)).decode()


def deconv_workspace_size(dims: deconv_dims) -> int:
    n = ctypes.c_size_t(0)
    _check(load().deconv_workspace_size(ctypes.byref(dims), ctypes.byref(n)), "deconv_workspace_size")
    return n.value


def deconv_plan_create(dims: deconv_dims, h_ptr: int, mask_ptr: int, lam: float, mu: float,
                       workspace_ptr: int, workspace_bytes: int, stream: int) -> int:
    plan = ctypes.c_void_p()
    _check(load().deconv_plan_create(ctypes.byref(plan), ctypes.byref(dims), h_ptr, mask_ptr, float(lam),
                                     float(mu), workspace_ptr, workspace_bytes, stream), "deconv_plan_create")
    return plan.value


def deconv_solve(plan: int, y_ptr: Optional[int], x_ptr: Optional[int], iters: int, warm: int = 0,
                 stats_ptr: Optional[int] = None) -> None:
    _check(load().deconv_solve(plan, y_ptr, x_ptr, int(iters), int(warm), stats_ptr), "deconv_solve")


def deconv_solve_host(plan: int, y_host_ptr: int, x_host_ptr: int, iters: int) -> None:
    _check(load().deconv_solve_host(plan, y_host_ptr, x_host_ptr, int(iters)), "deconv_solve_host")


def deconv_profile_passes(plan: int, iters: int):
    """Mean (column pass, row pass) kernel durations in ms over `iters` iterations."""
    out = (ctypes.c_float * 2)()
    _check(load().deconv_profile_passes(plan, int(iters), out), "deconv_profile_passes")
    return float(out[0]), float(out[1])


def deconv_sync(plan: int) -> int:
    """Returns the device-side status (DECONV_OK, DECONV_ENONFINITE, ...)."""
    return load().deconv_sync(plan)


def deconv_solve_noalloc(dims: deconv_dims, h_ptr: int, mask_ptr: int, y_ptr: int, x_ptr: int, lam: float,
                         mu: float, iters: int, stream: int) -> None:
    """Whole solve with the workspace in the library's static 32 MiB device
    array (no device allocation); synchronises `stream`."""
    _check(load().deconv_solve_noalloc(ctypes.byref(dims), h_ptr, mask_ptr, y_ptr, x_ptr, float(lam), float(mu),
                                       int(iters), stream), "deconv_solve_noalloc")


def deconv_plan_destroy(plan: int) -> None:
    _check(load().deconv_plan_destroy(plan), "deconv_plan_destroy")


# ------------------------------------------------------- torch convenience


class Plan:
    """A plan whose workspace is a torch CUDA tensor.

    shapes: list of (M, N) extended sizes; h: torch tensor (K, K) or (B, K, K)
    on the device; mask: uint8 tensor in the batch layout (flat or any shape
    with the right number of elements)."""

    def __init__(self, shapes, h, mask, lam: float, mu: float, channels: int = 1, relax: float = 2.0,
                 stream=None):
        import torch
        self._torch = torch
        self.dtype = h.dtype
        dt = DECONV_F32 if h.dtype == torch.float32 else DECONV_F64
        K = h.shape[-1]
        kpi = 1 if h.dim() == 3 else 0
        self.shapes = [tuple(s) for s in shapes]
        self.channels = channels
        self.dims, self._keep = make_dims([s[0] for s in shapes], [s[1] for s in shapes], K, channels, dt,
                                          relax, kpi)
        self.workspace_bytes = deconv_workspace_size(self.dims)
        dev = h.device
        self.workspace = torch.empty(self.workspace_bytes + 256, dtype=torch.uint8, device=dev)
        off = (-self.workspace.data_ptr()) % 256
        self._ws_ptr = self.workspace.data_ptr() + off
        self.stream = stream if stream is not None else torch.cuda.current_stream(dev)
        self._h = h.contiguous()
        self._mask = mask.contiguous()
        self.handle = deconv_plan_create(self.dims, self._h.data_ptr(), self._mask.data_ptr(), lam, mu,
                                         self._ws_ptr, self.workspace_bytes, self.stream.cuda_stream)
        self.numel = sum(channels * M * N for (M, N) in self.shapes)

    def solve(self, y, iters: int, x=None, warm: bool = False, stats=None):
        torch = self._torch
        if x is None:
            x = torch.empty(self.numel, dtype=self.dtype, device=self.workspace.device)
        deconv_solve(self.handle, None if warm else y.data_ptr(), x.data_ptr(), iters, int(warm),
                     None if stats is None else stats.data_ptr())
        return x

    def solve_host(self, y_host, x_host, iters: int) -> None:
        deconv_solve_host(self.handle, y_host.data_ptr(), x_host.data_ptr(), iters)

    def profile_passes(self, iters: int):
        return deconv_profile_passes(self.handle, iters)

    def sync(self) -> int:
        return deconv_sync(self.handle)

    def close(self) -> None:
        if getattr(self, "handle", None):
            deconv_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
