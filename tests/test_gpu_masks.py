"""Masks and indexing, bit for bit, on every observation pattern the paper
uses (Sec. III-B: unknown boundaries, border padding of the initial
estimate; Sec. III-C: inpainting, ×4 decimation for super-resolution, the
RGGB Bayer pattern for demosaicing).

Two exact checks per pattern, through the C ABI:

* zero iterations return the initial fill y~0 of every channel plane
  (observed pixels copied, boundary-band pixels clamped to the nearest
  valid-region index when that pixel is observed, every other unobserved
  pixel the FP64 mean of the observed ones rounded once), compared with the
  oracle's fill bit for bit, on small ragged grids and on the full
  16-image super-resolution and 32-frame demosaicing batches;
* after several iterations the observed entries of y~ = [y; z] still hold y
  exactly (the z-update touches unobserved pixels only), and the unobserved
  entries follow the oracle's z within the FP32 tolerance.
"""
import numpy as np
import pytest

import oracle
from paper_1602_01410_gb300 import inputs

from gpu_helpers import gpu_solve, split

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


CASES = [
    # (mask kind, channels, K, sizes): ragged tiles, odd sides, several row
    # blocks (2-3-5-smooth sides, the sizes the library runs as they are)
    ("crop", 1, 7, [(45, 75), (64, 96)]),
    ("decim4", 1, 9, [(96, 96), (60, 54), (128, 80)]),
    ("bayer", 3, 5, [(64, 80), (45, 50)]),
    ("random", 1, 5, [(96, 160), (30, 40)]),
]


def fill_of(prob, j):
    return np.stack([oracle.init_ytilde(prob.y[j][c], prob.mask[j][c], prob.ksize, round_f32=True)
                     .astype(np.float32).astype(np.float64) for c in range(prob.channels)])


@pytest.mark.parametrize("kind,channels,K,sizes", CASES)
def test_initial_fill_bit_exact(kind, channels, K, sizes):
    prob = inputs.random_problem(81, sizes, K, mask_kind=kind, channels=channels, frac=0.4, iters=0)
    xg, _, _ = gpu_solve(prob, iters=0)
    for j in range(len(sizes)):
        assert np.array_equal(xg[j], fill_of(prob, j)), (kind, j)


def test_initial_fill_bit_exact_uneven_kernel_supports():
    # one plan over images with their own kernel supports: each image's
    # boundary band (and so its border padding) follows its own kernel
    import torch
    import paper_1602_01410_gb300 as pkg
    parts = [inputs.random_problem(82 + i, [s], K, mask_kind=kind, frac=0.3, iters=0)
             for i, (s, K, kind) in enumerate([((64, 64), 9, "crop"), ((48, 80), 5, "decim4"),
                                                ((96, 64), 3, "random"), ((40, 40), 7, "crop")])]
    Kmax = max(p.ksize for p in parts)
    hs = []
    for p in parts:
        pad = (Kmax - p.ksize) // 2
        hs.append(np.pad(p.h, pad))
    dev = torch.device("cuda:0")
    h = torch.tensor(np.stack(hs), dtype=torch.float32, device=dev)
    mask = torch.tensor(np.concatenate([p.mask[0].ravel() for p in parts]), dtype=torch.uint8, device=dev)
    y = torch.tensor(np.concatenate([p.y[0].ravel() for p in parts]), dtype=torch.float32, device=dev)
    shapes = [p.shapes[0] for p in parts]
    plan = pkg.Plan(shapes, h, mask, parts[0].lam, parts[0].mu, ksizes=[p.ksize for p in parts])
    x = plan.solve(y, 0)
    assert plan.sync() == 0
    flat = x.double().cpu().numpy()
    o = 0
    for p in parts:
        M, N = p.shapes[0]
        got = flat[o:o + M * N].reshape(1, M, N)
        o += M * N
        assert np.array_equal(got, fill_of(p, 0))
    plan.close()


@pytest.mark.parametrize("kind,channels,K,sizes", CASES)
def test_observed_pixels_stay_exact_and_z_follows_the_oracle(kind, channels, K, sizes):
    iters = 3
    prob = inputs.random_problem(83, sizes, K, mask_kind=kind, channels=channels, frac=0.4, iters=iters)
    _, _, plan = gpu_solve(prob)
    blob = plan.state_get()
    total = sum(channels * M * N for (M, N) in prob.shapes)
    yt = blob[:4 * total].view(dtype=__import__("torch").float32).double().cpu().numpy()
    ytj = split(yt, prob)
    for j in range(len(sizes)):
        m = prob.mask[j] != 0
        y32 = prob.y[j].astype(np.float32).astype(np.float64)
        assert np.array_equal(ytj[j][m], y32[m]), (kind, j)
        _, st, _ = oracle.admm(prob.y[j], prob.mask[j], prob.h, prob.lam, prob.mu, iters, relax=prob.relax)
        z_gpu, z_or = ytj[j][~m], st.yt[~m]
        assert np.linalg.norm(z_gpu - z_or) <= 1e-4 * np.linalg.norm(z_or), (kind, j)
    plan.close()


@pytest.mark.parametrize("name", ["c3", "c4"])
def test_full_batch_initial_fill_bit_exact(name):
    # every image and plane of the 16-image super-resolution batch (x4
    # decimation) and of the 32-frame RGGB demosaicing batch, in one plan
    prob = {"c3": inputs.config_c3, "c4": inputs.config_c4}[name]()
    xg, _, _ = gpu_solve(prob, iters=0)
    for j in range(len(prob.shapes)):
        assert np.array_equal(xg[j], fill_of(prob, j)), (name, j, prob.shapes[j])
