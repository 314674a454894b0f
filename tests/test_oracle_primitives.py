"""Pins of the FP64 oracle's primitives against definitions and library
routines (no GPU).

* DFT: the textbook O(L^2) sum and numpy.fft, Parseval, round trip.
* Blurs: scipy's linear 'valid' convolution equals the circular one on the
  valid region (Sec. III: circular convolution cropped to the part that
  coincides with the linear one), a brute-force loop, and the BCCB
  diagonalisation by the DFT (Sec. II-B, the paragraph after the z-update).
* Adjoints: <Ax, y> = <x, A^T y> for T~ and D.
* Vector soft-threshold (Sec. III-B): brute-force minimisation of
  tau ||v|| + 1/2 ||v - a||^2.
* Initialisation (Sec. III-B, border padding): a brute-force loop.
"""
import numpy as np
import pytest
from scipy.optimize import minimize
from scipy.signal import convolve2d

import oracle
from paper_1602_01410_gb300 import inputs


def naive_dft(x, sign=-1):
    L = x.size
    n = np.arange(L)
    W = np.exp(sign * 2j * np.pi * np.outer(n, n) / L)
    return W @ x


@pytest.mark.parametrize("L", list(range(1, 17)) + [25, 27, 60, 64, 90, 384])
def test_fft_matches_naive_dft(L):
    rng = np.random.default_rng(L)
    x = rng.standard_normal(L) + 1j * rng.standard_normal(L)
    for sign in (-1, 1):
        got = oracle.fft(x, sign)
        ref = naive_dft(x, sign)
        assert np.max(np.abs(got - ref)) <= 1e-12 * max(1.0, np.max(np.abs(ref)))


@pytest.mark.parametrize("L", [7, 128, 384, 768, 1280, 1536])
def test_fft_matches_numpy_parseval_roundtrip(L):
    rng = np.random.default_rng(100 + L)
    x = rng.standard_normal(L) + 1j * rng.standard_normal(L)
    X = oracle.fft(x, -1)
    assert np.allclose(X, np.fft.fft(x), rtol=0, atol=1e-11 * np.sqrt(L))
    assert np.isclose(np.sum(np.abs(X) ** 2) / L, np.sum(np.abs(x) ** 2), rtol=1e-12)
    back = oracle.fft(X, +1) / L
    assert np.max(np.abs(back - x)) < 1e-12


@pytest.mark.parametrize("shape", [(6, 10), (64, 48), (60, 90)])
def test_fft2_matches_numpy(shape):
    rng = np.random.default_rng(7)
    x = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    assert np.allclose(oracle.fft2(x, -1), np.fft.fft2(x), rtol=0, atol=1e-10)
    assert np.allclose(oracle.fft2(x, +1), np.fft.ifft2(x) * x.size, rtol=0, atol=1e-10)


def centred_kernel_grid(h, M, N):
    """h~ on the M x N grid with h[b][b] at index (0, 0)."""
    K = h.shape[0]
    b = K // 2
    g = np.zeros((M, N))
    for p in range(-b, b + 1):
        for q in range(-b, b + 1):
            g[p % M, q % N] += h[p + b, q + b]
    return g


@pytest.mark.parametrize("M,N,K", [(12, 15, 3), (20, 16, 5), (33, 40, 9)])
def test_circular_equals_linear_on_valid_region(M, N, K):
    rng = np.random.default_rng(M * N + K)
    x = rng.standard_normal((M, N))
    h = rng.standard_normal((K, K))  # deliberately asymmetric
    b = K // 2
    lin = convolve2d(x, h, mode="valid")
    circ = oracle.conv_circ(x, h)
    assert np.max(np.abs(circ[b:M - b, b:N - b] - lin)) < 1e-12
    assert np.max(np.abs(oracle.conv_valid(x, h) - lin)) < 1e-12


def test_circular_conv_brute_force_and_bccb_diagonalisation():
    rng = np.random.default_rng(3)
    M, N, K = 7, 9, 5
    b = K // 2
    x = rng.standard_normal((M, N))
    h = rng.standard_normal((K, K))
    ref = np.zeros((M, N))
    for i in range(M):
        for j in range(N):
            for p in range(-b, b + 1):
                for q in range(-b, b + 1):
                    ref[i, j] += h[p + b, q + b] * x[(i - p) % M, (j - q) % N]
    got = oracle.conv_circ(x, h)
    assert np.max(np.abs(got - ref)) < 1e-12
    # T~ is diagonalised by the 2-D DFT: DFT(T~x) = DFT(h~) DFT(x).
    H = np.fft.fft2(centred_kernel_grid(h, M, N))
    assert np.max(np.abs(np.fft.fft2(got) - H * np.fft.fft2(x))) < 1e-11
    # and T~^T by the conjugate spectrum.
    assert np.max(np.abs(np.fft.fft2(oracle.conv_circ_adj(x, h)) - np.conj(H) * np.fft.fft2(x))) < 1e-11


@pytest.mark.parametrize("M,N,K", [(8, 8, 3), (17, 23, 7), (40, 36, 11)])
def test_adjoint_identities(M, N, K):
    rng = np.random.default_rng(11 + M)
    x, yv = rng.standard_normal((M, N)), rng.standard_normal((M, N))
    h = rng.standard_normal((K, K))
    lhs = np.vdot(oracle.conv_circ(x, h), yv)
    rhs = np.vdot(x, oracle.conv_circ_adj(yv, h))
    assert abs(lhs - rhs) <= 1e-13 * M * N * K * K
    uh, uv = rng.standard_normal((M, N)), rng.standard_normal((M, N))
    dh, dv = oracle.diff_fwd(x)
    lhs = np.vdot(dh, uh) + np.vdot(dv, uv)
    rhs = np.vdot(x, oracle.diff_adj(uh, uv))
    assert abs(lhs - rhs) <= 1e-13 * M * N


def test_differences_definition_and_spectrum():
    rng = np.random.default_rng(5)
    M, N = 6, 9
    x = rng.standard_normal((M, N))
    dh, dv = oracle.diff_fwd(x)
    assert np.array_equal(dh, np.roll(x, -1, axis=1) - x)
    assert np.array_equal(dv, np.roll(x, -1, axis=0) - x)
    # D^T D is BCCB with eigenvalues 4 sin^2(pi k1/M) + 4 sin^2(pi k2/N).
    e = np.zeros((M, N))
    e[0, 0] = 1
    col = oracle.diff_adj(*oracle.diff_fwd(e))
    k1 = np.arange(M)[:, None]
    k2 = np.arange(N)[None, :]
    lam = 4 * np.sin(np.pi * k1 / M) ** 2 + 4 * np.sin(np.pi * k2 / N) ** 2
    assert np.max(np.abs(np.fft.fft2(col) - lam)) < 1e-12


@pytest.mark.parametrize("dim", [2, 6])
def test_vector_soft_threshold_is_the_prox(dim):
    rng = np.random.default_rng(dim)
    tau = 0.7
    for trial in range(12):
        a = rng.standard_normal(dim) * rng.choice([0.2, 1.0, 3.0])
        got = oracle.vsoft(a[:, None], tau)[:, 0]
        obj = lambda v: tau * np.sqrt(np.sum(v * v) + 1e-30) + 0.5 * np.sum((v - a) ** 2)
        best = min((minimize(obj, x0, method="Powell", options={"xtol": 1e-12, "ftol": 1e-15, "maxiter": 20000})
                    for x0 in (a, np.zeros(dim) + 1e-3, a * 0.5)), key=lambda r: r.fun)
        assert obj(got) <= best.fun + 1e-9
        if np.linalg.norm(a) <= tau:
            assert np.all(got == 0)
        else:
            assert np.allclose(np.linalg.norm(got), np.linalg.norm(a) - tau, atol=1e-14)


def test_vector_soft_threshold_edge_cases():
    a = np.zeros((2, 3))
    a[:, 1] = [0.3, 0.4]  # norm 0.5 == tau
    a[:, 2] = [3.0, 4.0]
    v = oracle.vsoft(a, 0.5)
    assert np.all(v[:, 0] == 0) and np.all(v[:, 1] == 0)
    assert np.allclose(v[:, 2], [2.7, 3.6], atol=1e-15)


def brute_force_fill(y, mask, K):
    M, N = y.shape
    b = K // 2
    mean = y[mask != 0].mean()
    out = np.empty_like(y)
    for i in range(M):
        for j in range(N):
            ic, jc = min(max(i, b), M - b - 1), min(max(j, b), N - b - 1)
            inband = not (b <= i < M - b and b <= j < N - b)
            out[i, j] = y[i, j] if mask[i, j] else (y[ic, jc] if (inband and mask[ic, jc]) else mean)
    return out


def test_initial_state_of_every_channel_plane():
    # Three channels with their own Bayer planes: zero iterations return
    # x^0 = y~^0, each plane filled from its own mask and mean (Sec. III-B,
    # Sec. III-C).
    rng = np.random.default_rng(19)
    M, N, K = 12, 14, 3
    m = inputs.mask_bayer_rggb(M, N, K // 2)
    y = np.where(m, rng.random((3, M, N)), 0.0)
    x, _, _ = oracle.admm(y, m, np.full((K, K), 1.0 / K ** 2), 1e-3, 1e-2, 0, round_f32=False)
    for c in range(3):
        assert np.allclose(x[c], brute_force_fill(y[c], m[c], K), rtol=0, atol=1e-15), c


def test_init_ytilde_brute_force():
    rng = np.random.default_rng(9)
    M, N, K = 14, 17, 5
    b = K // 2
    y = rng.standard_normal((M, N))
    mask = np.zeros((M, N), np.uint8)
    mask[b:M - b, b:N - b] = rng.random((M - 2 * b, N - 2 * b)) > 0.35
    y = np.where(mask, y, 0.0)
    got = oracle.init_ytilde(y, mask, K, round_f32=False)
    assert np.allclose(got, brute_force_fill(y, mask, K), rtol=0, atol=1e-15)
    mean = y[mask != 0].mean()
    for i in range(M):
        for j in range(N):
            if mask[i, j]:
                assert got[i, j] == y[i, j]
                continue
            ic, jc = min(max(i, b), M - b - 1), min(max(j, b), N - b - 1)
            inband = not (b <= i < M - b and b <= j < N - b)
            want = y[ic, jc] if (inband and mask[ic, jc]) else mean
            assert np.isclose(got[i, j], want, rtol=0, atol=1e-15)
