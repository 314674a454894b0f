"""Pins of the oracle against worked examples derived by hand from the
paper's definitions (`tests/golden/*.txt`, each file citing the equation or
section it follows).  None of the stored values comes from the oracle or the
CUDA path; fractions are written exactly and parsed with `fractions`."""
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load(name):
    """Blocks of a fixture: {block name: list of rows of floats}."""
    blocks, cur = {}, None
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line.startswith("@"):
                cur = blocks.setdefault(line[1:], [])
                continue
            cur.append([float(Fraction(tok)) for tok in line.split()])
    return blocks


def mat(rows):
    return np.array(rows, dtype=np.float64)


def test_fixtures_present_and_cited():
    names = sorted(os.listdir(GOLDEN))
    assert len(names) >= 6
    for n in names:
        head = open(os.path.join(GOLDEN, n)).read().split("@", 1)[0]
        assert "Eq." in head or "Sec." in head, n


@pytest.mark.parametrize("case", sorted(load("vsoft_worked.txt")))
def test_vector_soft_threshold_worked(case):
    tau, a, v = load("vsoft_worked.txt")[case]
    got = oracle.vsoft(np.array(a).reshape(-1, 1), tau[0]).ravel()
    assert np.allclose(got, v, rtol=0, atol=1e-15), (got, v)


def test_circular_convolution_and_adjoint_of_an_impulse():
    g = load("conv_impulse_4x5.txt")
    h, x = mat(g["h"]), mat(g["x"])
    assert np.array_equal(oracle.conv_circ(x, h), mat(g["conv"]))
    assert np.array_equal(oracle.conv_circ_adj(x, h), mat(g["corr"]))


def test_valid_convolution_worked():
    g = load("conv_valid_4x4.txt")
    assert np.array_equal(oracle.conv_valid(mat(g["x"]), mat(g["h"])), mat(g["valid"]))


def test_periodic_differences_and_dtd_worked():
    g = load("diff_3x4.txt")
    x = mat(g["x"])
    dh, dv = oracle.diff_fwd(x)
    assert np.array_equal(dh, mat(g["dh"]))
    assert np.array_equal(dv, mat(g["dv"]))
    assert np.array_equal(oracle.diff_adj(dh, dv), mat(g["dtd"]))


def test_x_step_closed_form_on_a_3x3_grid():
    g = load("xstep_3x3_uniform.txt")
    x = oracle.solve_x(mat(g["rhs"]), mat(g["h"]), g["mu"][0][0])
    assert np.allclose(x, mat(g["x"]), rtol=0, atol=1e-14), x


@pytest.mark.parametrize("case", ["1", "2"])
def test_initial_fill_worked(case):
    g = load("init_fill_5x5.txt")
    y, m = mat(g["y" + case]), mat(g["mask" + case]).astype(np.uint8)
    yt = oracle.init_ytilde(y, m, 3, round_f32=False)
    assert np.allclose(yt, mat(g["yt" + case]), rtol=0, atol=1e-15), yt


@pytest.mark.parametrize("relax", [2, 1])
def test_one_iteration_worked_on_a_2x2_grid(relax):
    g = load("admm_one_iteration_2x2.txt")
    mu, lam = g["mu_lambda"][0]
    y, m = mat(g["y"]), mat(g["mask"]).astype(np.uint8)
    st = oracle.State(mat(g["yt0"])[None].copy(), np.zeros((1, 2, 2, 2)), np.zeros((1, 2, 2, 2)))
    x, st1, s = oracle.admm(y[None], m[None], np.ones((1, 1)), lam, mu, 1, relax=float(relax), state=st,
                            stats=True)
    tol = dict(rtol=0, atol=1e-14)
    assert np.allclose(x[0], mat(g["x1"]), **tol), x
    assert np.allclose(st1.yt[0], mat(g[f"yt1_relax{relax}"]), **tol), st1.yt
    assert np.allclose(st1.v[0], np.stack([mat(g["v1_h"]), mat(g["v1_v"])]), **tol), st1.v
    assert np.allclose(st1.d[0], np.stack([mat(g["d1_h"]), mat(g["d1_v"])]), **tol), st1.d
    assert np.allclose(s[0], g[f"stats_relax{relax}"][0], rtol=1e-14, atol=0), s


def test_penalty_adaptation_worked_on_a_2x2_grid():
    g = load("admm_one_iteration_2x2.txt")
    mu, lam = g["mu_lambda"][0]
    y, m = mat(g["y"]), mat(g["mask"]).astype(np.uint8)
    d1 = np.stack([mat(g["d1_h"]), mat(g["d1_v"])])
    for t, mu_after, scale in g["adapt"]:
        st = oracle.State(mat(g["yt0"])[None].copy(), np.zeros((1, 2, 2, 2)), np.zeros((1, 2, 2, 2)))
        st.mu = mu
        x, st1, _ = oracle.admm(y[None], m[None], np.ones((1, 1)), lam, mu, 1, state=st, adapt_t=t)
        assert st1.mu == mu_after, (t, st1.mu)
        assert np.allclose(st1.d[0], scale * d1, rtol=0, atol=1e-14), (t, st1.d)
        assert np.allclose(x[0], mat(g["x1"]), rtol=0, atol=1e-14)


def test_tikhonov_warm_start_worked_on_a_2x2_grid():
    g = load("admm_one_iteration_2x2.txt")
    mu, lam = g["mu_lambda"][0]
    tau, steps = g["tikh_tau_steps"][0]
    y, m = mat(g["y"]), mat(g["mask"]).astype(np.uint8)
    x, st, _ = oracle.admm(y[None], m[None], np.ones((1, 1)), lam, mu, 0, tikh_iters=int(steps), tikh_tau=tau,
                           round_f32=False)
    tol = dict(rtol=0, atol=1e-14)
    assert np.allclose(x[0], mat(g["tikh_x0"]), **tol), x
    assert np.allclose(st.yt[0], mat(g["tikh_yt0"]), **tol), st.yt
    assert np.allclose(st.v[0], np.stack([mat(g["tikh_v0_h"]), mat(g["tikh_v0_v"])]), **tol), st.v
    assert np.all(st.d == 0.0)


def test_two_bgs_passes_worked_on_a_2x2_grid():
    g = load("admm_one_iteration_2x2.txt")
    mu, lam = g["mu_lambda"][0]
    y, m = mat(g["y"]), mat(g["mask"]).astype(np.uint8)
    st = oracle.State(mat(g["yt0"])[None].copy(), np.zeros((1, 2, 2, 2)), np.zeros((1, 2, 2, 2)))
    x, st1, s = oracle.admm(y[None], m[None], np.ones((1, 1)), lam, mu, 1, state=st, passes=2, stats=True)
    assert np.allclose(x[0], mat(g["bgs2_x"]), rtol=0, atol=1e-14), x
    assert np.allclose(st1.yt[0], mat(g["bgs2_yt"]), rtol=0, atol=1e-14), st1.yt
    assert np.isclose(s[0, 1], g["bgs2_dz2"][0][0], rtol=1e-13, atol=0), s


def test_observation_masks_drawn_by_hand():
    from paper_1602_01410_gb300 import inputs
    g = load("masks_7x8.txt")
    M, N, b = 7, 8, 1
    assert np.array_equal(inputs.mask_crop(M, N, b), mat(g["crop"]))
    assert np.array_equal(inputs.mask_decimation(M, N, b, 2), mat(g["decimation2"]))
    bayer = inputs.mask_bayer_rggb(M, N, b)
    for c, name in enumerate(("bayer_r", "bayer_g", "bayer_b")):
        assert np.array_equal(bayer[c], mat(g[name])), name
