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

Typical use (device tensors; y and mask in the batch layout of deconv.h)::

    plan = Plan([(M, N)], h, mask, lam, mu)          # extended grid M x N, K x K kernel
    plan.set_options(bgs_passes=K // 2, tikh_iters=100, adapt_t=3.0)   # optional variants
    plan.autotune(y, cache="tunes.json")            # optional: launch shapes for this GPU, cached
    x = plan.solve(y, iters)                         # x^{iters}
    loss, dlam, dh = plan.grad(y, x_true, iters)     # gradient of the unrolled solve (defaults only)

For sizes with a prime factor above 5, ``deconv_fast_shape`` and ``enlarge``
give a supported grid with the added pixels unobserved.
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
           "deconv_solve_noalloc", "deconv_grad_workspace_size", "deconv_grad", "deconv_last_error",
           "deconv_state_bytes", "deconv_state_get", "deconv_state_set", "deconv_kernel_launches",
           "deconv_set_options", "deconv_get_mu", "deconv_fast_shape", "deconv_retune", "deconv_get_tune",
           "deconv_autotune", "deconv_set_profiling", "deconv_graph_pass_times", "deconv_vjp",
           "deconv_set_wait_limit")


class DeconvError(RuntimeError):
    def __init__(self, status: int, where: str):
        detail = f" [{deconv_last_error()}]" if status == DECONV_ECUDA else ""
        super().__init__(f"{where}: {deconv_status_string(status)} (status {status}){detail}")
        self.status = status


class deconv_dims(ctypes.Structure):
    _fields_ = [("batch", ctypes.c_int32), ("channels", ctypes.c_int32),
                ("rows", ctypes.POINTER(ctypes.c_int32)), ("cols", ctypes.POINTER(ctypes.c_int32)),
                ("ksize", ctypes.c_int32), ("kernel_per_image", ctypes.c_int32),
                ("dtype", ctypes.c_int32), ("relax", ctypes.c_float),
                ("ksizes", ctypes.POINTER(ctypes.c_int32))]


class deconv_options(ctypes.Structure):
    _fields_ = [("bgs_passes", ctypes.c_int32), ("tikh_iters", ctypes.c_int32),
                ("tikh_tau", ctypes.c_double), ("adapt_t", ctypes.c_double)]


class deconv_tune(ctypes.Structure):
    _fields_ = [("row_ctas", ctypes.c_int32), ("col_ctas", ctypes.c_int32), ("row_stage", ctypes.c_int32),
                ("fft_values", ctypes.c_int32), ("col_fft_values", ctypes.c_int32),
                ("l2_group_mb", ctypes.c_int32), ("generic", ctypes.c_int32), ("fused_rows", ctypes.c_int32),
                ("chains", ctypes.c_int32)]


TUNE_FIELDS = tuple(name for name, _ in deconv_tune._fields_)


def _tune_dict(t: "deconv_tune") -> dict:
    return {name: int(getattr(t, name)) for name in TUNE_FIELDS}


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
        lib.deconv_set_profiling.argtypes = [vp, i32]
        lib.deconv_set_wait_limit.argtypes = [vp, ctypes.c_int64]
        lib.deconv_graph_pass_times.argtypes = [vp, ctypes.POINTER(ctypes.c_float)]
        lib.deconv_sync.argtypes = [vp]
        lib.deconv_solve_noalloc.argtypes = [ctypes.POINTER(deconv_dims), vp, vp, vp, vp, dbl, dbl, i32, vp]
        lib.deconv_grad_workspace_size.argtypes = [vp, i32, i32, ctypes.POINTER(ctypes.c_size_t)]
        lib.deconv_grad.argtypes = [vp, vp, vp, i32, i32, vp, ctypes.c_size_t, ctypes.POINTER(dbl),
                                    ctypes.POINTER(dbl), vp, vp]
        lib.deconv_vjp.argtypes = [vp, vp, vp, i32, i32, vp, ctypes.c_size_t, ctypes.POINTER(dbl), vp, vp]
        lib.deconv_plan_destroy.argtypes = [vp]
        lib.deconv_status_string.argtypes = [ctypes.c_int]
        lib.deconv_status_string.restype = ctypes.c_char_p
        lib.deconv_state_bytes.argtypes = [vp, ctypes.POINTER(ctypes.c_size_t)]
        lib.deconv_kernel_launches.argtypes = [vp, i32, i32, i32, ctypes.POINTER(ctypes.c_int64)]
        lib.deconv_state_get.argtypes = [vp, vp]
        lib.deconv_state_set.argtypes = [vp, vp]
        lib.deconv_last_error.argtypes = []
        lib.deconv_set_options.argtypes = [vp, ctypes.POINTER(deconv_options)]
        lib.deconv_get_mu.argtypes = [vp, ctypes.POINTER(dbl)]
        lib.deconv_retune.argtypes = [vp, ctypes.POINTER(deconv_tune)]
        lib.deconv_get_tune.argtypes = [vp, ctypes.POINTER(deconv_tune)]
        lib.deconv_autotune.argtypes = [vp, vp, i32, ctypes.POINTER(deconv_tune), ctypes.POINTER(ctypes.c_float)]
        lib.deconv_fast_shape.argtypes = [i32, i32, i32, i32, i32, ctypes.POINTER(i32), ctypes.POINTER(i32)]
        lib.deconv_last_error.restype = ctypes.c_char_p
        for name in EXPORTS:
            if name not in ("deconv_status_string", "deconv_last_error"):
                getattr(lib, name).restype = ctypes.c_int
        _lib = lib
    return _lib


def make_dims(rows: Sequence[int], cols: Sequence[int], ksize: int, channels: int = 1,
              dtype: int = DECONV_F32, relax: float = 2.0, kernel_per_image: int = 0,
              ksizes: Optional[Sequence[int]] = None):
    """Build a deconv_dims; returns (dims, keepalive) - keep both referenced.
    ksizes: per-image kernel supports (uneven supports in one batch)."""
    r = (ctypes.c_int32 * len(rows))(*rows)
    c = (ctypes.c_int32 * len(cols))(*cols)
    k = (ctypes.c_int32 * len(ksizes))(*ksizes) if ksizes is not None else None
    d = deconv_dims(len(rows), channels, r, c, ksize, kernel_per_image, dtype, relax,
                    k if k is not None else ctypes.POINTER(ctypes.c_int32)())
    return d, (r, c, k)


def _check(status: int, where: str) -> None:
    if status != DECONV_OK:
        raise DeconvError(status, where)


# ------------------------------------------------------------- C entry points


def deconv_status_string(status: int) -> str:
    return load().deconv_status_string(int(status)).decode()


def deconv_last_error() -> str:
    return load().deconv_last_error().decode()


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


def deconv_set_wait_limit(plan: int, ns: int) -> None:
    _check(load().deconv_set_wait_limit(plan, int(ns)), "deconv_set_wait_limit")


def deconv_set_profiling(plan: int, on: bool) -> None:
    _check(load().deconv_set_profiling(plan, 1 if on else 0), "deconv_set_profiling")


def deconv_graph_pass_times(plan: int):
    """Mean (column passes, row passes, whole iteration) in ms per iteration,
    from the CUDA events of the last replay of the profiled captured loop."""
    out = (ctypes.c_float * 3)()
    _check(load().deconv_graph_pass_times(plan, out), "deconv_graph_pass_times")
    return float(out[0]), float(out[1]), float(out[2])


def deconv_sync(plan: int) -> int:
    """Returns the device-side status (DECONV_OK, DECONV_ENONFINITE, ...)."""
    return load().deconv_sync(plan)


def deconv_solve_noalloc(dims: deconv_dims, h_ptr: int, mask_ptr: int, y_ptr: int, x_ptr: int, lam: float,
                         mu: float, iters: int, stream: int) -> None:
    """Whole solve with the workspace in the library's static 32 MiB device
    array (no device allocation); synchronises `stream`."""
    _check(load().deconv_solve_noalloc(ctypes.byref(dims), h_ptr, mask_ptr, y_ptr, x_ptr, float(lam), float(mu),
                                       int(iters), stream), "deconv_solve_noalloc")


def deconv_grad_workspace_size(plan: int, iters: int, ckpt_every: int) -> int:
    n = ctypes.c_size_t(0)
    _check(load().deconv_grad_workspace_size(plan, int(iters), int(ckpt_every), ctypes.byref(n)),
           "deconv_grad_workspace_size")
    return n.value


def deconv_grad(plan: int, y_ptr: int, xtrue_ptr: int, iters: int, ckpt_every: int, gws_ptr: int, gws_bytes: int,
                dh_ptr: int, x_out_ptr: Optional[int] = None):
    """Returns (loss, dL/dlambda); dL/dh is written to dh_ptr (device)."""
    loss, dlam = ctypes.c_double(0), ctypes.c_double(0)
    _check(load().deconv_grad(plan, y_ptr, xtrue_ptr, int(iters), int(ckpt_every), gws_ptr, gws_bytes,
                              ctypes.byref(loss), ctypes.byref(dlam), dh_ptr, x_out_ptr), "deconv_grad")
    return loss.value, dlam.value


def deconv_vjp(plan: int, y_ptr: int, xbar_ptr: int, iters: int, ckpt_every: int, gws_ptr: int, gws_bytes: int,
               dh_ptr: int, x_out_ptr: Optional[int] = None) -> float:
    """dL/dlambda for dL/dx^iters = xbar; dL/dh is written to dh_ptr (device)."""
    dlam = ctypes.c_double(0)
    _check(load().deconv_vjp(plan, y_ptr, xbar_ptr, int(iters), int(ckpt_every), gws_ptr, gws_bytes,
                             ctypes.byref(dlam), dh_ptr, x_out_ptr), "deconv_vjp")
    return dlam.value


def deconv_kernel_launches(plan: int, iters: int, mode: int = 0, ckpt_every: int = 10) -> int:
    n = ctypes.c_int64(0)
    _check(load().deconv_kernel_launches(plan, int(iters), int(mode), int(ckpt_every), ctypes.byref(n)),
           "deconv_kernel_launches")
    return n.value


def deconv_state_bytes(plan: int) -> int:
    n = ctypes.c_size_t(0)
    _check(load().deconv_state_bytes(plan, ctypes.byref(n)), "deconv_state_bytes")
    return n.value


def deconv_state_get(plan: int, blob_ptr: int) -> None:
    _check(load().deconv_state_get(plan, blob_ptr), "deconv_state_get")


def deconv_state_set(plan: int, blob_ptr: int) -> None:
    _check(load().deconv_state_set(plan, blob_ptr), "deconv_state_set")


def deconv_set_options(plan: int, bgs_passes: int = 1, tikh_iters: int = 0, tikh_tau: float = 1e-3,
                       adapt_t: float = 0.0) -> None:
    o = deconv_options(int(bgs_passes), int(tikh_iters), float(tikh_tau), float(adapt_t))
    _check(load().deconv_set_options(plan, ctypes.byref(o)), "deconv_set_options")


def deconv_get_mu(plan: int, nimg: int):
    out = (ctypes.c_double * nimg)()
    _check(load().deconv_get_mu(plan, out), "deconv_get_mu")
    return [float(v) for v in out]


def deconv_retune(plan: int, row_ctas: int = 0, col_ctas: int = 0, row_stage: int = -1, fft_values: int = 0,
                  col_fft_values: int = 0, l2_group_mb: int = 0, generic: int = 0, fused_rows: int = 0,
                  chains: int = 0) -> None:
    t = deconv_tune(int(row_ctas), int(col_ctas), int(row_stage), int(fft_values), int(col_fft_values),
                    int(l2_group_mb), int(generic), int(fused_rows), int(chains))
    _check(load().deconv_retune(plan, ctypes.byref(t)), "deconv_retune")


def deconv_get_tune(plan: int) -> dict:
    t = deconv_tune()
    _check(load().deconv_get_tune(plan, ctypes.byref(t)), "deconv_get_tune")
    return _tune_dict(t)


def deconv_autotune(plan: int, y_ptr: int, trial_iters: int = 20):
    """Returns (best tuning as a dict, its ms per iteration)."""
    t, ms = deconv_tune(), ctypes.c_float(0.0)
    _check(load().deconv_autotune(plan, y_ptr, trial_iters, ctypes.byref(t), ctypes.byref(ms)), "deconv_autotune")
    return _tune_dict(t), float(ms.value)


def deconv_fast_shape(M: int, N: int, channels: int = 1, ksize: int = 3, dtype: int = DECONV_F32):
    """Smallest supported extended grid >= M x N (see deconv.h)."""
    mo, no = ctypes.c_int32(0), ctypes.c_int32(0)
    _check(load().deconv_fast_shape(M, N, channels, ksize, dtype, ctypes.byref(mo), ctypes.byref(no)),
           "deconv_fast_shape")
    return int(mo.value), int(no.value)


def enlarge(y, mask, shape):
    """Embed (C, M, N) arrays y and mask (numpy or torch) at the top-left of a
    (C, M2, N2) grid; the added pixels are unobserved (mask 0, y 0)."""
    M2, N2 = shape
    C, M, N = y.shape
    if M2 < M or N2 < N:
        raise ValueError("the enlarged grid must contain the original one")
    if hasattr(y, "new_zeros"):  # torch
        y2, m2 = y.new_zeros((C, M2, N2)), mask.new_zeros((C, M2, N2))
    else:
        import numpy as np
        y2, m2 = np.zeros((C, M2, N2), y.dtype), np.zeros((C, M2, N2), mask.dtype)
    y2[:, :M, :N] = y
    m2[:, :M, :N] = mask
    return y2, m2


def crop(x, shape):
    """The (C, M, N) window of an enlarged (C, M2, N2) result."""
    M, N = shape
    return x[:, :M, :N]


def deconv_plan_destroy(plan: int) -> None:
    _check(load().deconv_plan_destroy(plan), "deconv_plan_destroy")


# ------------------------------------------------------- torch convenience


def _source_digest() -> str:
    """Digest of the library's source (CUDA, C++ and the C header): a cached
    tuning is reused only by the build it was measured on."""
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(_HERE, "csrc")
    for name in sorted(os.listdir(csrc)):
        if not name.endswith((".cu", ".cuh", ".h")):
            continue
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(name.encode() + b"\0" + f.read())
    with open(os.path.join(os.path.dirname(_HERE), "include", "deconv.h"), "rb") as f:
        h.update(f.read())
    return h.hexdigest()[:16]


def tune_key(shapes, channels: int, ksize: int, dtype: int, relax: float, kernel_per_image: int, ksizes,
             options, device: str) -> str:
    """Key of a cached launch tuning: everything that changes which tuning is
    fastest (the batch geometry, element type, iteration variant and GPU)
    plus the library source it was measured with."""
    import json
    return json.dumps({"shapes": [list(map(int, s)) for s in shapes], "channels": int(channels),
                       "ksize": int(ksize), "dtype": int(dtype), "relax": float(relax),
                       "kernel_per_image": int(kernel_per_image),
                       "ksizes": None if ksizes is None else [int(k) for k in ksizes],
                       "options": [float(v) for v in options], "device": device,
                       "source": _source_digest()}, sort_keys=True)


class TuneCache:
    """Launch tunings chosen by deconv_autotune, kept in a JSON file so that
    later plans of the same key skip the timing runs.  A missing or
    unreadable file reads as empty; writes replace the file atomically."""

    def __init__(self, path: str):
        self.path = path

    def _read(self) -> dict:
        import json
        try:
            with open(self.path) as f:
                data = json.load(f)
            return data if isinstance(data, dict) else {}
        except (OSError, ValueError):
            return {}

    def get(self, key: str):
        hit = self._read().get(key)
        if not isinstance(hit, dict) or "tune" not in hit:
            return None
        return hit

    def put(self, key: str, tune: dict, ms_per_iter: float) -> None:
        import json
        import tempfile
        data = self._read()
        data[key] = {"tune": dict(tune), "ms_per_iter": float(ms_per_iter)}
        d = os.path.dirname(os.path.abspath(self.path))
        fd, tmp = tempfile.mkstemp(dir=d, prefix=".tune_cache")
        with os.fdopen(fd, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)
        os.replace(tmp, self.path)


class Plan:
    """A plan whose workspace is a torch CUDA tensor.

    shapes: list of (M, N) extended sizes; h: torch tensor (K, K) or (B, K, K)
    on the device; mask: uint8 tensor in the batch layout (flat or any shape
    with the right number of elements)."""

    def __init__(self, shapes, h, mask, lam: float, mu: float, channels: int = 1, relax: float = 2.0,
                 stream=None, ksizes=None):
        import torch
        self._torch = torch
        self.dtype = h.dtype
        dt = DECONV_F32 if h.dtype == torch.float32 else DECONV_F64
        K = h.shape[-1]
        kpi = 1 if h.dim() == 3 else 0
        self.shapes = [tuple(s) for s in shapes]
        self.channels = channels
        self.ksize, self.kernel_per_image, self.relax, self._dt = K, kpi, float(relax), dt
        self.ksizes = None if ksizes is None else [int(k) for k in ksizes]
        self.options = (1, 0, 1e-3, 0.0)
        self.dims, self._keep = make_dims([s[0] for s in shapes], [s[1] for s in shapes], K, channels, dt,
                                          relax, kpi, ksizes)
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

    def grad(self, y, x_true, iters: int, ckpt_every: int = 10, x_out=None):
        """Loss mean((x^iters - x_true)^2), dL/dlambda and dL/dh (tensor shaped like h)."""
        torch = self._torch
        n = deconv_grad_workspace_size(self.handle, iters, ckpt_every)
        gws = torch.empty(n + 256, dtype=torch.uint8, device=self.workspace.device)
        gptr = gws.data_ptr() + (-gws.data_ptr()) % 256
        dh = torch.empty_like(self._h)
        loss, dlam = deconv_grad(self.handle, y.data_ptr(), x_true.data_ptr(), iters, ckpt_every, gptr, n,
                                 dh.data_ptr(), None if x_out is None else x_out.data_ptr())
        return loss, dlam, dh

    def vjp(self, y, xbar, iters: int, ckpt_every: int = 10, x_out=None):
        """(dL/dlambda, dL/dh) for a loss L with dL/dx^iters = xbar."""
        torch = self._torch
        n = deconv_grad_workspace_size(self.handle, iters, ckpt_every)
        gws = torch.empty(n + 256, dtype=torch.uint8, device=self.workspace.device)
        gptr = gws.data_ptr() + (-gws.data_ptr()) % 256
        dh = torch.empty_like(self._h)
        dlam = deconv_vjp(self.handle, y.data_ptr(), xbar.data_ptr(), iters, ckpt_every, gptr, n, dh.data_ptr(),
                          None if x_out is None else x_out.data_ptr())
        return dlam, dh

    def set_options(self, bgs_passes: int = 1, tikh_iters: int = 0, tikh_tau: float = 1e-3,
                    adapt_t: float = 0.0) -> None:
        """BGS passes per iteration, Tikhonov warm start, penalty adaptation (see deconv.h)."""
        deconv_set_options(self.handle, bgs_passes, tikh_iters, tikh_tau, adapt_t)
        self.options = (bgs_passes, tikh_iters, tikh_tau, adapt_t)

    def autotune(self, y, trial_iters: int = 20, cache: Optional[str] = None):
        """Pick the fastest launch tuning for this plan (see deconv_autotune).
        With `cache` (a JSON file path), a tuning stored for the same key
        (`tune_key`) is applied with deconv_retune instead of timing the
        candidates again, and a new choice is stored.  Either way the plan is
        left with no iteration state.  Returns (tuning, ms per iteration)."""
        if cache is None:
            return deconv_autotune(self.handle, y.data_ptr(), trial_iters)
        torch = self._torch
        dev = self.workspace.device
        props = torch.cuda.get_device_properties(dev)
        key = tune_key(self.shapes, self.channels, self.ksize, self._dt, self.relax, self.kernel_per_image,
                       self.ksizes, self.options, f"{props.name} / {props.multi_processor_count} SMs")
        store = TuneCache(cache)
        hit = store.get(key)
        if hit is not None:
            self.retune(**hit["tune"])
            return dict(hit["tune"]), float(hit["ms_per_iter"])
        best, ms = deconv_autotune(self.handle, y.data_ptr(), trial_iters)
        store.put(key, best, ms)
        return best, ms

    def retune(self, row_ctas: int = 0, col_ctas: int = 0, row_stage: int = -1, fft_values: int = 0,
               col_fft_values: int = 0, l2_group_mb: int = 0, generic: int = 0, fused_rows: int = 0,
               chains: int = 0) -> None:
        deconv_retune(self.handle, row_ctas, col_ctas, row_stage, fft_values, col_fft_values, l2_group_mb, generic,
                      fused_rows, chains)

    def set_wait_limit(self, ns: int) -> None:
        deconv_set_wait_limit(self.handle, ns)

    def get_mu(self):
        """Per-image penalty of the next iteration (list of floats)."""
        return deconv_get_mu(self.handle, len(self.shapes))

    def solve_host(self, y_host, x_host, iters: int) -> None:
        deconv_solve_host(self.handle, y_host.data_ptr(), x_host.data_ptr(), iters)

    def profile_passes(self, iters: int):
        return deconv_profile_passes(self.handle, iters)

    def set_profiling(self, on: bool) -> None:
        deconv_set_profiling(self.handle, on)

    def graph_pass_times(self):
        return deconv_graph_pass_times(self.handle)

    def state_get(self):
        """Opaque device checkpoint of the iteration state (uint8 tensor)."""
        blob = self._torch.empty(deconv_state_bytes(self.handle), dtype=self._torch.uint8,
                                 device=self.workspace.device)
        deconv_state_get(self.handle, blob.data_ptr())
        return blob

    def state_set(self, blob) -> None:
        deconv_state_set(self.handle, blob.data_ptr())

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


class DeconvLoss:
    """torch.autograd.Function: L = mean((x^iters - x_true)^2) of the unrolled
    partial ADMM as a differentiable function of lambda (0-dim tensor) and
    the blur kernel h; the forward call runs deconv_grad, which returns the
    loss and both gradients together, and backward scales them by the
    incoming gradient.  y, mask and x_true are data (no gradient)."""

    @staticmethod
    def apply(lam, h, y, mask, x_true, shapes, mu: float, iters: int, channels: int = 1, ckpt_every: int = 10,
              relax: float = 2.0):
        return _deconv_loss_fn().apply(lam, h, y, mask, x_true, tuple(map(tuple, shapes)), mu, iters, channels,
                                       ckpt_every, relax)


_LOSS_FN = None


def _deconv_loss_fn():
    global _LOSS_FN
    if _LOSS_FN is None:
        import torch

        class _Fn(torch.autograd.Function):
            @staticmethod
            def forward(ctx, lam, h, y, mask, x_true, shapes, mu, iters, channels, ckpt_every, relax):
                plan = Plan(list(shapes), h.detach(), mask, float(lam), mu, channels=channels, relax=relax)
                try:
                    loss, dlam, dh = plan.grad(y.detach(), x_true, iters, ckpt_every)
                finally:
                    plan.close()
                ctx.save_for_backward(torch.tensor(dlam, dtype=h.dtype, device=h.device), dh)
                return torch.tensor(loss, dtype=h.dtype, device=h.device)

            @staticmethod
            def backward(ctx, g):
                dlam, dh = ctx.saved_tensors
                return (g * dlam, g * dh) + (None,) * 9

        _LOSS_FN = _Fn
    return _LOSS_FN


class DeconvSolve:
    """torch.autograd.Function: x^iters of the unrolled partial ADMM as a
    differentiable function of lambda (0-dim tensor) and the blur kernel h,
    for any downstream loss.  forward runs the solve; backward runs
    deconv_vjp with the incoming gradient on x (it recomputes the forward
    from checkpoints every ckpt_every iterations) and returns dL/dlambda and
    dL/dh.  y and mask are data (no gradient)."""

    @staticmethod
    def apply(lam, h, y, mask, shapes, mu: float, iters: int, channels: int = 1, ckpt_every: int = 10,
              relax: float = 2.0):
        return _deconv_solve_fn().apply(lam, h, y, mask, tuple(map(tuple, shapes)), mu, iters, channels,
                                        ckpt_every, relax)


_SOLVE_FN = None


def _deconv_solve_fn():
    global _SOLVE_FN
    if _SOLVE_FN is None:
        import torch

        class _Fn(torch.autograd.Function):
            @staticmethod
            def forward(ctx, lam, h, y, mask, shapes, mu, iters, channels, ckpt_every, relax):
                plan = Plan(list(shapes), h.detach(), mask, float(lam), mu, channels=channels, relax=relax)
                try:
                    x = plan.solve(y.detach(), iters)
                    if plan.sync() != DECONV_OK:
                        raise DeconvError(plan.sync(), "DeconvSolve.forward")
                    x = x.clone()
                finally:
                    plan.close()
                ctx.save_for_backward(lam.detach(), h.detach(), y.detach(), mask)
                ctx.cfg = (shapes, mu, iters, channels, ckpt_every, relax)
                return x

            @staticmethod
            def backward(ctx, gx):
                lam, h, y, mask = ctx.saved_tensors
                shapes, mu, iters, channels, ckpt_every, relax = ctx.cfg
                plan = Plan(list(shapes), h, mask, float(lam), mu, channels=channels, relax=relax)
                try:
                    dlam, dh = plan.vjp(y, gx.contiguous().to(h.dtype), iters, ckpt_every)
                finally:
                    plan.close()
                return (torch.tensor(dlam, dtype=h.dtype, device=h.device), dh) + (None,) * 8

        _SOLVE_FN = _Fn
    return _SOLVE_FN
