"""Synthetic-input generator checks (no GPU): mask patterns are exactly the
stated lattices, the boundary band is never observed (Eq. (4)), and the
noise level matches the requested BSNR."""
import numpy as np

from paper_1602_01410_gb300 import inputs


def test_crop_mask():
    m = inputs.mask_crop(20, 24, 3)
    assert m.sum() == 14 * 18
    assert m[3:17, 3:21].all()


def test_random_missing_exact_count_and_band():
    rng = np.random.default_rng(0)
    M, N, b = 64, 80, 4
    m = inputs.mask_random_missing(rng, M, N, b, 0.4)
    k0 = (M - 2 * b) * (N - 2 * b)
    assert m.sum() == k0 - int(round(0.4 * k0))
    band = np.ones((M, N), bool)
    band[b:M - b, b:N - b] = False
    assert not m[band].any()


def test_decimation_lattice():
    M, N, b = 40, 44, 4
    m = inputs.mask_decimation(M, N, b, 4)
    ii, jj = np.nonzero(m)
    assert np.all((ii - b) % 4 == 0) and np.all((jj - b) % 4 == 0)
    assert ii.min() == b and jj.min() == b and ii.max() < M - b and jj.max() < N - b
    assert m.sum() == len(range(b, M - b, 4)) * len(range(b, N - b, 4))


def test_bayer_partition():
    M, N, b = 30, 34, 6
    m = inputs.mask_bayer_rggb(M, N, b)
    s = m.astype(int).sum(0)
    crop = inputs.mask_crop(M, N, b)
    assert np.array_equal(s, crop.astype(int))
    assert m[0, b, b] == 1 and m[1, b, b + 1] == 1 and m[1, b + 1, b] == 1 and m[2, b + 1, b + 1] == 1
    assert m[0].sum() == 9 * 11 and m[2].sum() == 9 * 11 and m[1].sum() == 2 * 9 * 11


def test_bsnr_and_observation():
    rng = np.random.default_rng(1)
    M = N = 512
    h = inputs.psf_gaussian(9, 2.0)
    x = inputs.scene_piecewise_smooth(rng, M, N)
    m = inputs.mask_crop(M, N, 4)
    y = inputs.observe(np.random.default_rng(2), x, h, m, 40.0)
    bv = inputs.blur_valid(x, h)
    noise = y[4:-4, 4:-4] - bv
    bsnr = 10 * np.log10(np.var(bv) / np.var(noise))
    assert abs(bsnr - 40.0) < 0.05
    assert np.all(y[m == 0] == 0)


def test_psfs_normalised_and_odd():
    rng = np.random.default_rng(3)
    for h in (inputs.psf_uniform(9), inputs.psf_gaussian(13, 2.5), inputs.psf_motion(rng, 21)):
        assert h.shape[0] == h.shape[1] and h.shape[0] % 2 == 1
        assert np.isclose(h.sum(), 1.0) and np.all(h >= 0)


def test_scene_ranges():
    rng = np.random.default_rng(4)
    assert 0 <= inputs.scene_shapes(rng, 32, 32).min() and inputs.scene_shapes(rng, 32, 32).max() <= 1
    s = inputs.scene_rgb(rng, 48, 40)
    assert s.shape == (3, 48, 40) and s.min() >= 0 and s.max() <= 1


def test_configs_are_seeded():
    a = inputs.config_c1()
    b = inputs.config_c1()
    assert np.array_equal(a.y[0], b.y[0]) and np.array_equal(a.mask[0], b.mask[0])
    assert a.shapes == [(64, 64)] and a.ksize == 9
    assert a.mask[0].sum() == 56 * 56
