"""Arbitrary sizes (host logic, no GPU): deconv_fast_shape returns the
smallest-area 2-3-5-smooth grid the library runs (checked by brute force on
small sides), the identity on sizes that run as they are, and the
enlarge/crop helpers embed an image with the added pixels unobserved."""
import numpy as np
import pytest

import paper_1602_01410_gb300 as pkg


@pytest.fixture(scope="module", autouse=True)
def lib():
    from paper_1602_01410_gb300 import build
    build.build()


def smooth(n):
    for p in (2, 3, 5):
        while n % p == 0:
            n //= p
    return n == 1


def test_identity_on_supported_sizes():
    for M, N in [(64, 64), (1024, 1024), (384, 1280), (96, 160), (45, 75), (1000, 1125)]:
        assert pkg.deconv_fast_shape(M, N, 1, 5) == (M, N)


def test_smallest_smooth_sides():
    for M in list(range(9, 200, 7)) + [1009, 1111, 2039]:
        N = M + 4
        M2, N2 = pkg.deconv_fast_shape(M, N, 1, 9)
        assert smooth(M2) and smooth(N2) and M2 >= M and N2 >= N
        # every smaller-area pair of smooth sides is absent (small sides all run)
        cm = min(v for v in range(M, 4 * M) if smooth(v))
        cn = min(v for v in range(N, 4 * N) if smooth(v))
        assert (M2, N2) == (cm, cn)


def test_prime_sides_rgb_fp64():
    M2, N2 = pkg.deconv_fast_shape(1009, 757, 3, 13, pkg.DECONV_F64)
    assert smooth(M2) and smooth(N2) and M2 >= 1009 and N2 >= 757


def test_invalid_arguments():
    with pytest.raises(pkg.DeconvError):
        pkg.deconv_fast_shape(0, 10)
    with pytest.raises(pkg.DeconvError):
        pkg.deconv_fast_shape(10, 10, 2, 3)
    with pytest.raises(pkg.DeconvError):
        pkg.deconv_fast_shape(10, 10, 1, 4)


def test_enlarge_and_crop():
    rng = np.random.default_rng(0)
    y = rng.random((3, 13, 17))
    m = (rng.random((3, 13, 17)) > 0.5).astype(np.uint8)
    y2, m2 = pkg.enlarge(y, m, (15, 18))
    assert y2.shape == (3, 15, 18) and m2.shape == (3, 15, 18)
    assert np.array_equal(pkg.crop(y2, (13, 17)), y) and np.array_equal(pkg.crop(m2, (13, 17)), m)
    assert not m2[:, 13:, :].any() and not m2[:, :, 17:].any()
    assert not y2[:, 13:, :].any() and not y2[:, :, 17:].any()


def test_uneven_kernel_supports_validated():
    ok, _ = pkg.make_dims([32, 40], [32, 48], 9, kernel_per_image=1, ksizes=[9, 5])
    assert pkg.deconv_workspace_size(ok) > 0
    for kpi, ks in ((1, [9, 4]), (1, [11, 5]), (0, [9, 5]), (1, [9, 0])):
        d, _ = pkg.make_dims([32, 40], [32, 48], 9, kernel_per_image=kpi, ksizes=ks)
        with pytest.raises(pkg.DeconvError) as e:
            pkg.deconv_workspace_size(d)
        assert e.value.status == pkg.DECONV_EINVAL
