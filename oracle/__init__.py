"""FP64 CPU oracle for the partial-ADMM deconvolution (arXiv:1602.01410).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only callers.  The product path (the CUDA
library and its Python binding) never imports this package.

The arithmetic lives in ``oracle.c`` (plain C, FP64, OpenMP over rows); this
module compiles it with gcc and wraps it with ctypes.  Every wrapper takes and
returns float64 numpy arrays in the layouts documented in ``oracle.c``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Optional, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_SO = os.path.join(_HERE, "liboracle.so")
_lib = None

_D = ctypes.POINTER(ctypes.c_double)
_U8 = ctypes.POINTER(ctypes.c_uint8)


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so next to it (gcc, -O2, OpenMP)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=gnu11",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_SO)
        i, d = ctypes.c_int, ctypes.c_double
        lib.or_fft1d.argtypes = [_D, i, i]
        lib.or_fft2d.argtypes = [_D, i, i, i]
        for f in (lib.or_conv_circ, lib.or_conv_circ_adj, lib.or_conv_valid):
            f.argtypes = [_D, i, i, _D, i, _D]
        lib.or_diff_fwd.argtypes = [_D, i, i, _D, _D]
        lib.or_diff_adj.argtypes = [_D, _D, i, i, _D]
        lib.or_vsoft.argtypes = [_D, i, i, d, _D]
        lib.or_solve_x.argtypes = [_D, i, i, _D, i, d, _D]
        lib.or_init_ytilde.argtypes = [_D, _U8, i, i, i, i, _D]
        lib.or_admm.argtypes = [i, i, i, i, _D, _D, _U8, d, d, d, i, i, i, _D, _D, _D, _D, _D]
        lib.or_admm.restype = i
        lib.or_admm_ex.argtypes = [i, i, i, i, _D, _D, _U8, d, _D, d, i, i, i, i, d, i, d, _D, _D, _D, _D, _D, _D]
        lib.or_admm_ex.restype = i
        lib.or_tikhonov.argtypes = [i, i, i, _D, _U8, i, d, _D, _D]
        lib.or_admm_grad.argtypes = [i, i, i, i, _D, _D, _U8, d, d, d, i, i, _D, _D, _D, _D, _D]
        lib.or_admm_grad.restype = i
        _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(_D)


def _c(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def set_threads(n: int) -> None:
    """OpenMP thread count for subsequent calls (must precede the first call
    in a process to take effect through OMP_NUM_THREADS)."""
    os.environ["OMP_NUM_THREADS"] = str(int(n))


# ------------------------------------------------------------ primitives ---


def fft(x: np.ndarray, sign: int = -1) -> np.ndarray:
    """Unnormalised 1-D DFT, X[k] = sum_n x[n] exp(sign 2 pi i n k / L)."""
    a = np.ascontiguousarray(np.asarray(x, np.complex128))
    buf = a.view(np.float64).copy()
    _load().or_fft1d(_p(buf), a.size, sign)
    return buf.view(np.complex128)


def fft2(x: np.ndarray, sign: int = -1) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(x, np.complex128))
    buf = a.view(np.float64).copy()
    _load().or_fft2d(_p(buf), a.shape[0], a.shape[1], sign)
    return buf.view(np.complex128).reshape(a.shape)


def conv_circ(x: np.ndarray, h: np.ndarray) -> np.ndarray:
    """T~ x: circular convolution on the M x N grid (Eq. (4))."""
    x, h = _c(x), _c(h)
    out = np.empty_like(x)
    _load().or_conv_circ(_p(x), x.shape[0], x.shape[1], _p(h), h.shape[0], _p(out))
    return out


def conv_circ_adj(y: np.ndarray, h: np.ndarray) -> np.ndarray:
    """T~^T y: circular correlation."""
    y, h = _c(y), _c(h)
    out = np.empty_like(y)
    _load().or_conv_circ_adj(_p(y), y.shape[0], y.shape[1], _p(h), h.shape[0], _p(out))
    return out


def conv_valid(x: np.ndarray, h: np.ndarray) -> np.ndarray:
    """T x: linear convolution restricted to the valid region (Eq. (1))."""
    x, h = _c(x), _c(h)
    K = h.shape[0]
    out = np.empty((x.shape[0] - K + 1, x.shape[1] - K + 1))
    _load().or_conv_valid(_p(x), x.shape[0], x.shape[1], _p(h), K, _p(out))
    return out


def diff_fwd(x: np.ndarray) -> Tuple[np.ndarray, np.ndarray]:
    """(D_h x, D_v x): periodic forward first differences."""
    x = _c(x)
    dh, dv = np.empty_like(x), np.empty_like(x)
    _load().or_diff_fwd(_p(x), x.shape[0], x.shape[1], _p(dh), _p(dv))
    return dh, dv


def diff_adj(uh: np.ndarray, uv: np.ndarray) -> np.ndarray:
    """D^T [u_h; u_v]."""
    uh, uv = _c(uh), _c(uv)
    out = np.empty_like(uh)
    _load().or_diff_adj(_p(uh), _p(uv), uh.shape[0], uh.shape[1], _p(out))
    return out


def vsoft(a: np.ndarray, tau: float) -> np.ndarray:
    """Vector soft-threshold over axis 0 of a (dim, n) array."""
    a = _c(a)
    dim = a.shape[0]
    flat = a.reshape(dim, -1)
    out = np.empty_like(flat)
    _load().or_vsoft(_p(flat), flat.shape[1], dim, float(tau), _p(out))
    return out.reshape(a.shape)


def solve_x(rhs: np.ndarray, h: np.ndarray, mu: float) -> np.ndarray:
    """(T~^T T~ + mu D^T D)^{-1} rhs via the DFT of the operator's first column."""
    rhs, h = _c(rhs), _c(h)
    out = np.empty_like(rhs)
    _load().or_solve_x(_p(rhs), rhs.shape[0], rhs.shape[1], _p(h), h.shape[0], float(mu), _p(out))
    return out


def init_ytilde(y: np.ndarray, mask: np.ndarray, K: int, round_f32: bool = True) -> np.ndarray:
    """Initial extended observation y~0 (border padding, mean fill)."""
    y = _c(y)
    m = np.ascontiguousarray(mask, np.uint8)
    out = np.empty_like(y)
    _load().or_init_ytilde(_p(y), m.ctypes.data_as(_U8), y.shape[0], y.shape[1], K,
                           int(round_f32), _p(out))
    return out


# ---------------------------------------------------------- partial ADMM ---


class State:
    """Partial-ADMM state for C channels: yt (C,M,N), d and v (C,2,M,N), and
    the penalty mu the next iteration uses (None: the caller's mu)."""

    def __init__(self, yt: np.ndarray, d: np.ndarray, v: np.ndarray, mu: Optional[float] = None):
        self.yt, self.d, self.v, self.mu = yt, d, v, mu

    def copy(self) -> "State":
        return State(self.yt.copy(), self.d.copy(), self.v.copy(), self.mu)


def tikhonov(yt: np.ndarray, mask: np.ndarray, h: np.ndarray, iters: int, tau: float = 1e-3):
    """Eqs. (ini_x)-(ini_z) on one channel plane from z^0 = the unobserved
    entries of yt.  Returns (y~ with z^{iters}, x^{iters})."""
    yt = _c(yt).copy()
    M, N = yt.shape
    m = np.ascontiguousarray(mask, np.uint8).reshape(M, N)
    h = _c(h)
    x = np.zeros((M, N))
    _load().or_tikhonov(M, N, h.shape[0], _p(h), m.ctypes.data_as(_U8), int(iters), float(tau), _p(yt), _p(x))
    return yt, x


def passes_ad(K: int) -> int:
    """BGS passes of the paper's Proposed-AD for a K x K = (2b+1) x (2b+1) blur: b."""
    return max(1, K // 2)


def admm(y: np.ndarray, mask: np.ndarray, h: np.ndarray, lam: float, mu: float, iters: int,
         relax: float = 2.0, state: Optional[State] = None, round_f32: bool = True,
         stats: bool = False, passes: int = 1, adapt_t: float = 0.0, tikh_iters: int = 0,
         tikh_tau: float = 1e-3, mu_hist: bool = False):
    """Run `iters` partial-ADMM iterations on one image of C channels.

    y, mask: (C, M, N).  passes: BGS passes per iteration; adapt_t > 0: the
    penalty adaptation of Eq. (varying_penalty) with threshold t; tikh_iters
    > 0 (fresh start only): Tikhonov warm start of z with tau = tikh_tau.
    Returns (x, state, stats) where x is (C, M, N) = x^{iters} (x^0 of the
    initial state for a fresh start with iters = 0), state the
    final State and stats an (iters, 4) array of [||dd||^2, ||dz||^2,
    mu ||dv||^2, J] (or None); with mu_hist=True a fourth item, the (iters,)
    penalties the iterations used."""
    y = _c(y)
    if y.ndim == 2:
        y = y[None]
    C, M, N = y.shape
    m = np.ascontiguousarray(mask, np.uint8).reshape(C, M, N)
    h = _c(h)
    init = state is None
    st = State(np.zeros((C, M, N)), np.zeros((C, 2, M, N)), np.zeros((C, 2, M, N))) if init else state.copy()
    muv = np.array([float(mu if st.mu is None else st.mu)])
    x = np.zeros((C, M, N))
    s = np.zeros((max(iters, 1), 4)) if stats else None
    mh = np.zeros(max(iters, 1))
    rc = _load().or_admm_ex(C, M, N, h.shape[0], _p(h), _p(y), m.ctypes.data_as(_U8), float(lam), _p(muv),
                            float(relax), int(iters), int(init), int(round_f32), int(passes), float(adapt_t),
                            int(tikh_iters), float(tikh_tau), _p(st.yt), _p(st.d), _p(st.v), _p(x),
                            _p(s) if stats else None, _p(mh))
    if rc != 0:
        raise RuntimeError(f"or_admm_ex failed: {rc}")
    st.mu = float(muv[0])
    out = (x, st, (s[:iters] if stats else None))
    return out + (mh[:iters],) if mu_hist else out


def admm_grad(y: np.ndarray, mask: np.ndarray, h: np.ndarray, lam: float, mu: float, iters: int,
              x_true: np.ndarray, relax: float = 2.0, round_f32: bool = True):
    """Loss L = mean((x^{iters} - x_true)^2) over the C x M x N image and its
    gradients: returns (L, dL/dlambda, dL/dh (K x K), x^{iters})."""
    y = _c(y)
    if y.ndim == 2:
        y = y[None]
    C, M, N = y.shape
    m = np.ascontiguousarray(mask, np.uint8).reshape(C, M, N)
    h = _c(h)
    xt = _c(x_true).reshape(C, M, N)
    loss = np.zeros(1)
    dlam = np.zeros(1)
    dh = np.zeros_like(h)
    x = np.zeros((C, M, N))
    rc = _load().or_admm_grad(C, M, N, h.shape[0], _p(h), _p(y), m.ctypes.data_as(_U8), float(lam), float(mu),
                              float(relax), int(iters), int(round_f32), _p(xt), _p(loss), _p(dlam), _p(dh), _p(x))
    if rc != 0:
        raise RuntimeError(f"or_admm_grad failed: {rc}")
    return float(loss[0]), float(dlam[0]), dh, x


def loss_only(y, mask, h, lam, mu, iters, x_true, relax=2.0, round_f32=True) -> float:
    """L = mean((x^{iters} - x_true)^2) from the forward oracle (for finite differences)."""
    x, _, _ = admm(y, mask, h, lam, mu, iters, relax=relax, round_f32=round_f32)
    return float(np.mean((x - np.asarray(x_true).reshape(x.shape)) ** 2))
