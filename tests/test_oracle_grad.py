"""Pins of the oracle's reverse pass (the gradient of the unrolled partial
ADMM) against central finite differences of the oracle's forward pass, for
lambda and every kernel tap and along random directions of (lambda, h), one
and three channels, relax 1 and 2 (no GPU)."""
import numpy as np
import pytest

import oracle
from paper_1602_01410_gb300 import inputs


def problem(C, seed, M=12, N=14, K=5, frac=0.3):
    rng = np.random.default_rng(seed)
    b = K // 2
    h = inputs.psf_gaussian(K, 1.0) + 0.01 * rng.random((K, K))  # asymmetric
    h /= h.sum()
    if C == 1:
        x = inputs.scene_shapes(rng, M, N)[None]
        m = inputs.mask_random_missing(rng, M, N, b, frac)[None]
    else:
        x = inputs.scene_rgb(rng, M, N)
        m = inputs.mask_bayer_rggb(M, N, b)
    y = np.stack([inputs.observe(rng, x[c], h, m[c], 35.0) for c in range(C)])
    return y, m, h, x


@pytest.mark.parametrize("C", [1, 3])
def test_gradient_matches_central_differences(C):
    y, m, h, xt = problem(C, 40 + C)
    lam, mu, iters = 3e-3, 2e-2, 6
    L, dlam, dh, _ = oracle.admm_grad(y, m, h, lam, mu, iters, xt, round_f32=False)
    assert np.isclose(L, oracle.loss_only(y, m, h, lam, mu, iters, xt, round_f32=False), rtol=1e-13)
    eps = 1e-7
    fd = (oracle.loss_only(y, m, h, lam + eps, mu, iters, xt, round_f32=False) -
          oracle.loss_only(y, m, h, lam - eps, mu, iters, xt, round_f32=False)) / (2 * eps)
    assert abs(fd - dlam) <= 1e-6 * abs(dlam) + 1e-12
    K = h.shape[0]
    fdh = np.zeros_like(h)
    for t in range(K * K):
        e = np.zeros(K * K)
        e[t] = eps
        e = e.reshape(K, K)
        fdh.flat[t] = (oracle.loss_only(y, m, h + e, lam, mu, iters, xt, round_f32=False) -
                       oracle.loss_only(y, m, h - e, lam, mu, iters, xt, round_f32=False)) / (2 * eps)
    assert np.max(np.abs(fdh - dh)) <= 1e-6 * np.max(np.abs(dh))


def test_gradient_zero_iterations_and_lambda_zero():
    y, m, h, xt = problem(1, 7)
    L, dlam, dh, x = oracle.admm_grad(y, m, h, 0.0, 2e-2, 0, xt, round_f32=False)
    assert dlam == 0.0 and np.all(dh == 0.0)      # x^0 = y~0 depends on neither parameter
    L, dlam, dh, x = oracle.admm_grad(y, m, h, 0.0, 2e-2, 4, xt, round_f32=False)
    eps = 1e-7
    fd = (oracle.loss_only(y, m, h, eps, 2e-2, 4, xt, round_f32=False) - L) / eps  # one-sided at the lambda >= 0 edge
    assert abs(fd - dlam) <= 1e-4 * abs(dlam) + 1e-10


@pytest.mark.parametrize("C,relax", [(1, 2.0), (3, 1.0)])
def test_gradient_along_random_directions(C, relax):
    # <grad L, (u_lambda, U_h)> against the central difference of L along
    # random directions of (lambda, h), over a longer unrolled run.
    y, m, h, xt = problem(C, 60 + C)
    lam, mu, iters = 2e-3, 3e-2, 15
    L, dlam, dh, _ = oracle.admm_grad(y, m, h, lam, mu, iters, xt, relax=relax, round_f32=False)
    rng = np.random.default_rng(9)
    for _ in range(3):
        ul = rng.standard_normal() * lam
        uh = rng.standard_normal(h.shape) * h.std()
        eps = 1e-6
        fp = oracle.loss_only(y, m, h + eps * uh, lam + eps * ul, mu, iters, xt, relax=relax, round_f32=False)
        fm = oracle.loss_only(y, m, h - eps * uh, lam - eps * ul, mu, iters, xt, relax=relax, round_f32=False)
        fd = (fp - fm) / (2 * eps)
        an = dlam * ul + float(np.sum(dh * uh))
        assert abs(fd - an) <= 1e-6 * abs(an) + 1e-14, (fd, an)
