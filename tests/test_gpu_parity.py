"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on
the same seeded inputs.

Tolerances: relative L2 <= 1e-5 after one iteration (FP32), <= 1e-3 and
|dPSNR| <= 0.01 dB after a full run (FP32); the FP64 instantiation must stay
within 1e-10.  Masks and indexing are exact (the zero-iteration output is the
initial fill, compared bit for bit)."""
import numpy as np
import pytest

from paper_1602_01410_gb300 import inputs

from gpu_helpers import gpu_solve, oracle_solve, psnr, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def test_one_iteration_uneven_batch_random_mask():
    # several row blocks and column tiles per image, ragged last tiles, odd N
    prob = inputs.random_problem(11, [(96, 160), (120, 90), (45, 75), (64, 64)], 7, mask_kind="random",
                                 frac=0.4, iters=1)
    xg, _, _ = gpu_solve(prob)
    xo, _ = oracle_solve(prob)
    for a, b in zip(xg, xo):
        assert rel_l2([a], [b]) <= 1e-5


def test_one_iteration_vectorial_tv_bayer():
    prob = inputs.random_problem(12, [(64, 80), (60, 48)], 5, mask_kind="bayer", channels=3, iters=1)
    xg, _, _ = gpu_solve(prob)
    xo, _ = oracle_solve(prob)
    for a, b in zip(xg, xo):
        assert rel_l2([a], [b]) <= 1e-5


def test_one_iteration_decimation_and_crop():
    p1 = inputs.random_problem(13, [(96, 96), (48, 72)], 9, mask_kind="decim4", iters=1, lam=2e-4, mu=1e-3)
    p2 = inputs.random_problem(14, [(40, 50)], 3, mask_kind="crop", iters=1, psf="uniform")
    for prob in (p1, p2):
        xg, _, _ = gpu_solve(prob)
        xo, _ = oracle_solve(prob)
        assert rel_l2(xg, xo) <= 1e-5


def test_twenty_iterations_motion_blur():
    prob = inputs.random_problem(15, [(80, 120)], 9, mask_kind="random", frac=0.4, iters=20, psf="motion")
    xg, _, _ = gpu_solve(prob)
    xo, _ = oracle_solve(prob)
    assert rel_l2(xg, xo) <= 1e-4


def test_zero_iterations_is_the_initial_fill_bit_exact():
    import oracle
    prob = inputs.random_problem(16, [(48, 60), (30, 40)], 5, mask_kind="random", frac=0.5, iters=0)
    xg, _, _ = gpu_solve(prob, iters=0)
    for j in range(2):
        want = oracle.init_ytilde(prob.y[j][0], prob.mask[j][0], prob.ksize, round_f32=True)
        assert np.array_equal(xg[j][0], want.astype(np.float32).astype(np.float64))


def test_c1_fp64_full_run():
    prob = inputs.config_c1("f64")
    xg, _, _ = gpu_solve(prob)
    xo, _ = oracle_solve(prob)
    assert rel_l2(xg, xo) <= 1e-10


def test_c1_fp32_full_run():
    prob = inputs.config_c1("f32")
    xg, _, _ = gpu_solve(prob)
    xo, _ = oracle_solve(prob)
    assert rel_l2(xg, xo) <= 1e-3
    xt = prob.x_true[0]
    assert abs(psnr(xg[0], xt) - psnr(xo[0], xt)) <= 0.01


def test_stats_match_oracle():
    prob = inputs.random_problem(17, [(64, 96), (48, 48)], 5, mask_kind="random", frac=0.3, iters=8)
    xg, sg, _ = gpu_solve(prob, stats=True)
    _, so = oracle_solve(prob, stats=True)
    for j in range(2):
        o = so[j]
        # columns: ||dd||^2, ||dz||^2, J  (oracle: dd, dz, mu dv, J); every
        # iteration, the first included (d^0 = 0 on both sides)
        assert np.allclose(sg[j][:, 2], o[:, 3], rtol=1e-4)
        assert np.allclose(sg[j][:, 0], o[:, 0], rtol=2e-3, atol=1e-12), (sg[j][:, 0], o[:, 0])
        assert np.allclose(sg[j][:, 1], o[:, 1], rtol=2e-3, atol=1e-12)


def test_relax_one_matches_oracle():
    prob = inputs.random_problem(18, [(60, 64)], 5, mask_kind="random", frac=0.3, iters=10)
    xg, _, _ = gpu_solve(prob, relax=1.0)
    xo, _ = oracle_solve(prob, relax=1.0)
    assert rel_l2(xg, xo) <= 1e-4


def test_graph_replay_equals_direct_launches_and_is_deterministic():
    prob = inputs.random_problem(19, [(64, 80)], 5, mask_kind="random", frac=0.3, iters=45)
    a, _, _ = gpu_solve(prob)                 # graph replays
    b, _, _ = gpu_solve(prob, stats=True)     # direct launches
    c, _, _ = gpu_solve(prob)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[0], c[0])


def test_warm_continuation():
    import torch
    prob = inputs.random_problem(20, [(48, 64)], 5, mask_kind="random", frac=0.3, iters=7)
    full, _, _ = gpu_solve(prob)
    _, _, plan = gpu_solve(prob, iters=4)
    x = plan.solve(None, 3, warm=True)
    assert plan.sync() == 0
    assert np.array_equal(x.double().cpu().numpy().reshape(full[0].shape), full[0])


def test_solve_host_matches_device():
    import torch
    prob = inputs.random_problem(21, [(48, 64), (40, 40)], 5, mask_kind="random", frac=0.3, iters=6)
    xd, _, plan = gpu_solve(prob)
    y = torch.tensor(np.concatenate([a.ravel() for a in prob.y]), dtype=torch.float32).pin_memory()
    xh = torch.empty_like(y).pin_memory()
    plan.solve_host(y, xh, prob.iters)
    assert np.array_equal(xh.double().numpy(), np.concatenate([a.ravel() for a in xd]))


def test_nonfinite_input_reported():
    import paper_1602_01410_gb300 as pkg
    import torch
    prob = inputs.random_problem(22, [(32, 40)], 3, mask_kind="crop", iters=2)
    dev = torch.device("cuda:0")
    y = torch.tensor(prob.y[0], dtype=torch.float32, device=dev).reshape(-1)
    y[20 * 40 + 20] = float("nan")
    plan = pkg.Plan(prob.shapes, torch.tensor(prob.h, dtype=torch.float32, device=dev),
                    torch.tensor(prob.mask[0], dtype=torch.uint8, device=dev), prob.lam, prob.mu)
    plan.solve(y, 2)
    assert plan.sync() == pkg.DECONV_ENONFINITE
    plan.solve(torch.tensor(prob.y[0], dtype=torch.float32, device=dev).reshape(-1), 2)
    assert plan.sync() == pkg.DECONV_OK


def test_zero_dc_gain_rejected():
    import paper_1602_01410_gb300 as pkg
    import torch
    dev = torch.device("cuda:0")
    h = torch.zeros((3, 3), dtype=torch.float32, device=dev)
    h[0, 0], h[2, 2] = 1.0, -1.0
    mask = torch.ones(32 * 32, dtype=torch.uint8, device=dev)
    with pytest.raises(pkg.DeconvError) as e:
        pkg.Plan([(32, 32)], h, mask, 1e-3, 1e-2)
    assert e.value.status == pkg.DECONV_EINVAL


def test_pow2_passes_every_group_size():
    # rows and columns of 64 .. 1024: every threads-per-transform variant
    prob = inputs.random_problem(23, [(64, 1024), (128, 512), (256, 256), (512, 128), (1024, 64)], 5,
                                 mask_kind="random", frac=0.3, iters=1)
    xg, _, _ = gpu_solve(prob)
    xo, _ = oracle_solve(prob)
    for a, b in zip(xg, xo):
        assert rel_l2([a], [b]) <= 1e-5


def test_pow2_passes_vectorial_tv_and_stats():
    prob = inputs.random_problem(24, [(64, 64), (128, 256)], 5, mask_kind="bayer", channels=3, iters=3)
    xg, sg, _ = gpu_solve(prob, stats=True)
    xo, so = oracle_solve(prob, stats=True)
    for j in range(2):
        assert rel_l2([xg[j]], [xo[j]]) <= 3e-5
        assert np.allclose(sg[j][:, 2], so[j][:, 3], rtol=1e-4)
        # ||dd||^2 (the forward half's pixel-major step, summed over the
        # three channels) and ||dz||^2, every iteration
        assert np.allclose(sg[j][:, 0], so[j][:, 0], rtol=2e-3, atol=1e-12)
        assert np.allclose(sg[j][:, 1], so[j][:, 1], rtol=2e-3, atol=1e-12)


def test_generic_passes_on_pow2_sizes():
    # the shared-memory Stockham passes, forced through the tuning on sizes
    # that would otherwise take the register transforms
    prob = inputs.random_problem(25, [(128, 256), (64, 64)], 7, mask_kind="random", frac=0.4, iters=1)
    xg, _, _ = gpu_solve(prob, tune={"generic": 1})
    xo, _ = oracle_solve(prob)
    assert rel_l2(xg, xo) <= 1e-5


def test_image_groups_and_chains_of_the_captured_loop_change_nothing():
    # images are independent problems: running each image's 20-iteration
    # loops before the next image's (groups of one image), or every kernel
    # class's loop on a stream of its own (chains, here including a class of
    # the generic passes), gives the same bits as every pass over the whole
    # batch (one group)
    prob = inputs.random_problem(29, [(128, 256), (384, 384), (96, 160), (64, 64)], 7, mask_kind="random",
                                 frac=0.3, iters=45)
    one, _, _ = gpu_solve(prob, tune={"l2_group_mb": -1})
    each, _, _ = gpu_solve(prob, tune={"l2_group_mb": 1})
    chains, _, _ = gpu_solve(prob, tune={"chains": 1})
    for a, b, c in zip(one, each, chains):
        assert np.array_equal(a, b)
        assert np.array_equal(a, c)
    xo, _ = oracle_solve(prob)
    assert rel_l2(each, xo) <= 1e-4


def test_checkpoint_resume_in_another_plan():
    import paper_1602_01410_gb300 as pkg
    import torch
    prob = inputs.random_problem(26, [(64, 64), (48, 60)], 5, mask_kind="random", frac=0.3, iters=9)
    full, _, _ = gpu_solve(prob)
    _, _, plan = gpu_solve(prob, iters=5)
    blob = plan.state_get()
    dev = torch.device("cuda:0")
    plan2 = pkg.Plan(prob.shapes, torch.tensor(prob.h, dtype=torch.float32, device=dev),
                     torch.tensor(np.concatenate([m.ravel() for m in prob.mask]), dtype=torch.uint8, device=dev),
                     prob.lam, prob.mu)
    plan2.state_set(blob)
    x = plan2.solve(None, 4, warm=True)
    assert plan2.sync() == 0
    flat = np.concatenate([a.ravel() for a in full])
    assert np.array_equal(x.double().cpu().numpy(), flat)


def test_mixed_radix_passes_every_length():
    # lengths 3 * 2^k and 5 * 2^k (k = 7..9) through the radix-3/5 register
    # transforms, beside generic (96, 160) and power-of-two (64) lengths
    prob = inputs.random_problem(27, [(384, 640), (640, 384), (768, 96), (96, 1280), (1536, 160), (160, 2560),
                                      (1280, 64)], 7, mask_kind="random", frac=0.3, iters=1)
    xg, _, _ = gpu_solve(prob)
    xo, _ = oracle_solve(prob)
    for a, b in zip(xg, xo):
        assert rel_l2([a], [b]) <= 1e-5


def test_mixed_radix_vectorial_tv_and_stats():
    prob = inputs.random_problem(28, [(384, 384), (640, 768)], 5, mask_kind="bayer", channels=3, iters=3)
    xg, sg, _ = gpu_solve(prob, stats=True)
    xo, so = oracle_solve(prob, stats=True)
    for j in range(2):
        assert rel_l2([xg[j]], [xo[j]]) <= 3e-5
        assert np.allclose(sg[j][:, 2], so[j][:, 3], rtol=1e-4)
        # ||dd||^2 (the forward half's pixel-major step, summed over the
        # three channels) and ||dz||^2, every iteration
        assert np.allclose(sg[j][:, 0], so[j][:, 0], rtol=2e-3, atol=1e-12)
        assert np.allclose(sg[j][:, 1], so[j][:, 1], rtol=2e-3, atol=1e-12)


def test_mixed_radix_twenty_iterations():
    prob = inputs.random_problem(29, [(384, 640)], 9, mask_kind="random", frac=0.4, iters=20, psf="motion")
    xg, _, _ = gpu_solve(prob)
    xo, _ = oracle_solve(prob)
    assert rel_l2(xg, xo) <= 1e-4


def test_mixed_radix_fp64():
    prob = inputs.random_problem(30, [(384, 640), (768, 1280)], 5, mask_kind="random", frac=0.3, iters=2,
                                 dtype="f64")
    xg, _, _ = gpu_solve(prob)
    xo, _ = oracle_solve(prob)
    assert rel_l2(xg, xo) <= 1e-10


def test_vectorial_tv_register_passes_without_stats():
    # three channels, every register-FFT radix, statistics off (the channel
    # groups of a row share their squared norms through shared memory)
    prob = inputs.random_problem(31, [(64, 64), (128, 256), (384, 384), (640, 768), (512, 1280)], 7,
                                 mask_kind="bayer", channels=3, iters=3)
    xg, _, _ = gpu_solve(prob)
    xo, _ = oracle_solve(prob)
    for a, b in zip(xg, xo):
        assert rel_l2([a], [b]) <= 3e-5


@pytest.mark.parametrize("C,kind,sizes", [
    (1, "random", [(90, 75), (1024, 1024), (768, 768)]),
    (3, "bayer", [(90, 75), (768, 768), (512, 512)]),
])
def test_forward_row_prefetch_on_rows_off_16_byte_boundaries(C, kind, sizes):
    # A workspace above the plan's 64 MiB threshold turns on the forward
    # half's L2 prefetch of its input rows; the 90 x 75 first image (6,750
    # pixels per channel) puts every row of the images after it off a
    # 16-byte boundary, so each prefetch span must be widened to whole
    # granules inside its buffer.
    import paper_1602_01410_gb300 as pkg
    d, _keep = pkg.make_dims([m for m, n in sizes], [n for m, n in sizes], 7, channels=C)
    assert pkg.deconv_workspace_size(d) > 64 << 20
    prob = inputs.random_problem(61 + C, sizes, 7, mask_kind=kind, channels=C, frac=0.3, iters=2)
    xg, _, _ = gpu_solve(prob)
    xo, _ = oracle_solve(prob)
    assert rel_l2(xg, xo) <= 2e-5  # two FP32 iterations (one: <= 1e-5 in the tests above)
