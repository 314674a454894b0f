"""Seeded synthetic inputs for the partial-ADMM deconvolution workloads.

This module is the only code shared by the CUDA path's tests, the benchmark
and the FP64 oracle's tests.  It makes scenes, point spread functions,
observation masks and noisy observations; it holds none of the solver's
arithmetic (no DFT solve, no TV prox, no dual update).  The blur used to
synthesise an observation is the paper's data protocol (Sec. III: circular
convolution cropped to the part that equals the linear convolution, then
i.i.d. Gaussian noise at a given BSNR) and is done here with a library
routine (scipy.signal.fftconvolve, 'valid' mode).

Conventions (shared with the solver's plan):
  * The unknown image x lives on the extended grid M x N = (m+2b) x (n+2b)
    (Sec. I-A, the paragraph before Eq. (1)).
  * The kernel h is (2b+1) x (2b+1), row-major, with its origin at h[b][b];
    the blur is a true convolution, (Tx)[i][j] = sum_{p,q} h[p+b][q+b]
    x[i-p][j-q] (Eq. (1)).
  * The observation y is returned on the full M x N grid with the blurred,
    noisy value at observed pixels and 0 elsewhere; mask[i][j] = 1 marks an
    observed pixel.  The boundary band of width b is never observed (Eq. (4)).
"""
from __future__ import annotations

import dataclasses
from typing import List, Sequence, Tuple

import numpy as np
from scipy.signal import fftconvolve

# ---------------------------------------------------------------- scenes ---


def _rng(seed: int, j: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, j])))


def scene_shapes(rng: np.random.Generator, M: int, N: int) -> np.ndarray:
    """Uniform [0,1] background, 8-16 axis-aligned rectangles and 4-8 disks
    painted in random order, each with a uniform [0,1] value."""
    img = np.full((M, N), rng.uniform(0.0, 1.0))
    n_rect = int(rng.integers(8, 17))
    n_disk = int(rng.integers(4, 9))
    kinds = ["r"] * n_rect + ["d"] * n_disk
    order = rng.permutation(len(kinds))
    ii, jj = np.mgrid[0:M, 0:N]
    for k in order:
        val = rng.uniform(0.0, 1.0)
        if kinds[k] == "r":
            i0, i1 = np.sort(rng.integers(0, M + 1, size=2))
            j0, j1 = np.sort(rng.integers(0, N + 1, size=2))
            img[i0:i1, j0:j1] = val
        else:
            ci, cj = rng.uniform(0, M), rng.uniform(0, N)
            rad = rng.uniform(min(M, N) / 16, min(M, N) / 5)
            img[(ii - ci) ** 2 + (jj - cj) ** 2 <= rad * rad] = val
    return img


def _rect_geometry(rng: np.random.Generator, M: int, N: int, count: int):
    geo = []
    for _ in range(count):
        i0, i1 = np.sort(rng.integers(0, M + 1, size=2))
        j0, j1 = np.sort(rng.integers(0, N + 1, size=2))
        geo.append((int(i0), int(i1), int(j0), int(j1)))
    return geo


def grf_texture(rng: np.random.Generator, M: int, N: int, sigma_f: float = 0.02) -> np.ndarray:
    """Gaussian random field: white noise shaped by a Gaussian spectral
    envelope exp(-f^2 / (2 sigma_f^2)), f the radial frequency in cycles/px."""
    w = rng.standard_normal((M, N))
    fi = np.fft.fftfreq(M)[:, None]
    fj = np.fft.fftfreq(N)[None, :]
    env = np.exp(-(fi * fi + fj * fj) / (2.0 * sigma_f * sigma_f))
    return np.real(np.fft.ifft2(np.fft.fft2(w) * env))


def _minmax(a: np.ndarray) -> np.ndarray:
    lo, hi = a.min(), a.max()
    return (a - lo) / (hi - lo) if hi > lo else np.zeros_like(a)


def scene_piecewise_smooth(rng: np.random.Generator, M: int, N: int, n_rect: int = 40) -> np.ndarray:
    """Random rectangles (random values) mixed 0.7/0.3 with a low-frequency
    GRF texture, min-max scaled to [0,1]."""
    rect = np.full((M, N), rng.uniform(0.0, 1.0))
    for (i0, i1, j0, j1) in _rect_geometry(rng, M, N, n_rect):
        rect[i0:i1, j0:j1] = rng.uniform(0.0, 1.0)
    tex = _minmax(grf_texture(rng, M, N))
    return _minmax(0.7 * rect + 0.3 * tex)


def scene_rgb(rng: np.random.Generator, M: int, N: int, n_rect: int = 30) -> np.ndarray:
    """Three channels: independent GRF per channel plus rectangles with shared
    geometry and per-channel values.  Shape (3, M, N), each channel in [0,1]."""
    geo = _rect_geometry(rng, M, N, n_rect)
    out = np.empty((3, M, N))
    for c in range(3):
        rect = np.full((M, N), rng.uniform(0.0, 1.0))
        for (i0, i1, j0, j1) in geo:
            rect[i0:i1, j0:j1] = rng.uniform(0.0, 1.0)
        tex = _minmax(grf_texture(rng, M, N))
        out[c] = _minmax(0.6 * rect + 0.4 * tex)
    return out


# ------------------------------------------------------------------ PSFs ---


def psf_uniform(K: int) -> np.ndarray:
    return np.full((K, K), 1.0 / (K * K))


def psf_gaussian(K: int, sigma: float) -> np.ndarray:
    b = K // 2
    p = np.arange(-b, b + 1)
    g = np.exp(-(p[:, None] ** 2 + p[None, :] ** 2) / (2.0 * sigma * sigma))
    return g / g.sum()


def psf_motion(rng: np.random.Generator, K: int, steps: int = 200) -> np.ndarray:
    """Random-walk motion blur: `steps` unit moves in x or y from the centre,
    clamped to the support, visit counts normalised to sum 1."""
    b = K // 2
    h = np.zeros((K, K))
    i = j = b
    h[i, j] += 1
    moves = np.array([(0, 1), (0, -1), (1, 0), (-1, 0)])
    for s in rng.integers(0, 4, size=steps):
        di, dj = moves[s]
        i = min(max(i + di, 0), K - 1)
        j = min(max(j + dj, 0), K - 1)
        h[i, j] += 1
    return h / h.sum()


# ----------------------------------------------------------------- masks ---


def mask_crop(M: int, N: int, b: int) -> np.ndarray:
    """Unknown boundaries: only the valid (M-2b) x (N-2b) region is observed."""
    m = np.zeros((M, N), np.uint8)
    m[b:M - b, b:N - b] = 1
    return m


def mask_random_missing(rng: np.random.Generator, M: int, N: int, b: int, frac: float) -> np.ndarray:
    """Valid crop with exactly round(frac*k0) of its k0 pixels removed,
    chosen by a seeded permutation."""
    m = mask_crop(M, N, b)
    idx = np.flatnonzero(m.ravel())
    drop = rng.permutation(idx.size)[: int(round(frac * idx.size))]
    flat = m.ravel()
    flat[idx[drop]] = 0
    return m


def mask_decimation(M: int, N: int, b: int, factor: int) -> np.ndarray:
    """Superresolution lattice: valid pixels with (i-b) % f == 0 and (j-b) % f == 0."""
    m = np.zeros((M, N), np.uint8)
    m[b:M - b:factor, b:N - b:factor] = 1
    return m


def mask_bayer_rggb(M: int, N: int, b: int) -> np.ndarray:
    """Per-channel RGGB masks (3, M, N) relative to the valid crop origin:
    R at (even, even), G at (even, odd) and (odd, even), B at (odd, odd)."""
    m = np.zeros((3, M, N), np.uint8)
    crop = mask_crop(M, N, b).astype(bool)
    ii, jj = np.mgrid[0:M, 0:N]
    pi, pj = (ii - b) % 2, (jj - b) % 2
    m[0] = crop & (pi == 0) & (pj == 0)
    m[1] = crop & (pi != pj)
    m[2] = crop & (pi == 1) & (pj == 1)
    return m


# ----------------------------------------------------------- observation ---


def blur_valid(x: np.ndarray, h: np.ndarray) -> np.ndarray:
    """Linear 'valid' convolution (library routine), (M-2b) x (N-2b)."""
    return fftconvolve(x, h, mode="valid")


def observe(rng: np.random.Generator, x: np.ndarray, h: np.ndarray, mask: np.ndarray,
            bsnr_db: float) -> np.ndarray:
    """Blur, add i.i.d. Gaussian noise with sigma^2 = var(blurred valid region)
    / 10^(BSNR/10), keep observed pixels, zero elsewhere; full M x N grid."""
    M, N = x.shape
    b = h.shape[0] // 2
    bv = blur_valid(x, h)
    sigma = np.sqrt(np.var(bv) / 10.0 ** (bsnr_db / 10.0))
    y = np.zeros((M, N))
    y[b:M - b, b:N - b] = bv + sigma * rng.standard_normal(bv.shape)
    return np.where(mask != 0, y, 0.0)


# ------------------------------------------------------------- workloads ---


@dataclasses.dataclass
class Problem:
    """One batch of images ready for the solver.

    x_true, y: lists of (C, M, N) float64 arrays (y already rounded to the
    working precision's values when `dtype` is float32); mask: list of
    (C, M, N) uint8; h: (K, K) float64 (or list of per-image kernels)."""
    name: str
    x_true: List[np.ndarray]
    y: List[np.ndarray]
    mask: List[np.ndarray]
    h: np.ndarray
    lam: float
    mu: float
    iters: int
    channels: int
    dtype: str
    relax: float = 2.0

    @property
    def shapes(self) -> List[Tuple[int, int]]:
        return [a.shape[-2:] for a in self.y]

    @property
    def ksize(self) -> int:
        return self.h.shape[-1]

    def pixels(self) -> int:
        return sum(M * N for (M, N) in self.shapes) * self.channels


def _round(a: np.ndarray, dtype: str) -> np.ndarray:
    return a.astype(np.float32).astype(np.float64) if dtype == "f32" else a


def make_single(name: str, seed: int, M: int, N: int, h: np.ndarray, mask_kind: str,
                bsnr: float, lam: float, mu: float, iters: int, dtype: str,
                frac: float = 0.0, scene: str = "smooth") -> Problem:
    rng = _rng(seed, 0)
    b = h.shape[0] // 2
    x = scene_shapes(rng, M, N) if scene == "shapes" else scene_piecewise_smooth(rng, M, N)
    if mask_kind == "crop":
        m = mask_crop(M, N, b)
    elif mask_kind == "random":
        m = mask_random_missing(rng, M, N, b, frac)
    elif mask_kind == "full":
        m = np.ones((M, N), np.uint8)
    else:
        raise ValueError(mask_kind)
    h = _round(h, dtype)
    y = _round(observe(rng, x, h, m, bsnr), dtype)
    return Problem(name, [x[None]], [y[None]], [m[None]], h, lam, mu, iters, 1, dtype)


def config_c1(dtype: str = "f64", iters: int = 300) -> Problem:
    """64x64 shapes scene, 9x9 uniform blur, 56x56 valid crop, BSNR 50 dB,
    lambda 2e-5, mu 1e-3."""
    return make_single("c1-64x64-uniform9-crop", 1001, 64, 64, psf_uniform(9), "crop",
                       50.0, 2e-5, 1e-3, iters, dtype, scene="shapes")


def config_c2(iters: int = 500, size: int = 1024) -> Problem:
    """1024x1024 piecewise-smooth scene, 21x21 random-walk motion blur,
    1004x1004 valid crop with 40% of its pixels missing, BSNR 40 dB,
    lambda 2e-6, mu 1e-3."""
    rng = _rng(1002, 1000)
    h = psf_motion(rng, 21)
    return make_single(f"c2-{size}x{size}-motion21-missing40", 1002, size, size, h, "random",
                       40.0, 2e-6, 1e-3, iters, "f32", frac=0.4)


def make_batch(name: str, seed: int, sizes: Sequence[Tuple[int, int]], h: np.ndarray,
               mask_kind: str, bsnr: float, lam: float, mu: float, iters: int,
               channels: int = 1, frac: float = 0.0, dtype: str = "f32") -> Problem:
    b = h.shape[0] // 2
    h = _round(h, dtype)
    xs, ys, ms = [], [], []
    for j, (M, N) in enumerate(sizes):
        rng = _rng(seed, j)
        if channels == 3:
            x = scene_rgb(rng, M, N)
        else:
            x = scene_piecewise_smooth(rng, M, N)[None]
        if mask_kind == "decim4":
            m = np.repeat(mask_decimation(M, N, b, 4)[None], channels, 0)
        elif mask_kind == "bayer":
            m = mask_bayer_rggb(M, N, b)
        elif mask_kind == "random":
            m = np.repeat(mask_random_missing(rng, M, N, b, frac)[None], channels, 0)
        elif mask_kind == "crop":
            m = np.repeat(mask_crop(M, N, b)[None], channels, 0)
        else:
            raise ValueError(mask_kind)
        y = np.stack([_round(observe(rng, x[c], h, m[c], bsnr), dtype) for c in range(channels)])
        xs.append(x)
        ys.append(y)
        ms.append(m)
    return Problem(name, xs, ys, ms, h, lam, mu, iters, channels, dtype)


def config_c3(iters: int = 300, sides: Sequence[int] = (256, 384, 512, 768, 1024),
              count: int = 16) -> Problem:
    """16 square images with sides drawn from {256,...,1024}, 9x9 Gaussian
    (sigma 2), x4 decimation lattice, BSNR 40 dB, lambda 2e-4, mu 1e-3."""
    rng = _rng(1003, 1000)
    s = [int(v) for v in rng.choice(np.asarray(sides), size=count)]
    return make_batch("c3-16xSR4-gauss9", 1003, [(v, v) for v in s], psf_gaussian(9, 2.0),
                      "decim4", 40.0, 2e-4, 1e-3, iters)


def config_c4(iters: int = 400, sides: Sequence[int] = (512, 768, 1024, 1280, 1536),
              count: int = 32) -> Problem:
    """32 RGB frames with sides from {512,...,1536}, 13x13 Gaussian (sigma
    2.5), RGGB Bayer mask, vectorial TV, BSNR 45 dB, lambda 1e-5, mu 1e-3."""
    rng = _rng(1004, 1000)
    s = [int(v) for v in rng.choice(np.asarray(sides), size=count)]
    return make_batch("c4-32xRGB-bayer-gauss13", 1004, [(v, v) for v in s],
                      psf_gaussian(13, 2.5), "bayer", 45.0, 1e-5, 1e-3, iters, channels=3)


def config_c5(iters: int = 100, count: int = 8, size: int = 512) -> Problem:
    """8 images of 512x512, 15x15 Gaussian (sigma sqrt(15)), valid crop with
    20% random missing pixels, BSNR 40 dB, lambda 5e-6, mu 1e-3."""
    return make_batch("c5-8x512-gauss15-missing20", 1005, [(size, size)] * count,
                      psf_gaussian(15, float(np.sqrt(15.0))), "random", 40.0, 5e-6, 1e-3,
                      iters, frac=0.2)


def random_problem(seed: int, sizes: Sequence[Tuple[int, int]], K: int, mask_kind: str = "random",
                   frac: float = 0.3, channels: int = 1, lam: float = 1e-4, mu: float = 1e-2,
                   iters: int = 5, dtype: str = "f32", psf: str = "gauss", bsnr: float = 40.0) -> Problem:
    """Small seeded problems for parity tests (several tiles and ragged tails)."""
    rng = _rng(seed, 999)
    if psf == "gauss":
        h = psf_gaussian(K, max(0.5, K / 4.0))
    elif psf == "motion":
        h = psf_motion(rng, K, steps=4 * K)
    else:
        h = psf_uniform(K)
    return make_batch(f"rand-{seed}", seed, sizes, h, mask_kind, bsnr, lam, mu, iters,
                      channels=channels, frac=frac, dtype=dtype)
