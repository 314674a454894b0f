"""GPU parity of the iteration's variants against the FP64 oracle:
block-Gauss-Seidel passes (Sec. II-C, Proposed-AD) and the Tikhonov warm
start (Eqs. (ini_x)-(ini_z)), on register-FFT lengths (powers of two,
3 * 2^k), generic lengths and both channel counts.

Tolerances: FP32 relative L2 <= 1e-5 for one iteration, <= 1e-4 for a few;
the warm start with tau = 1e-3 divides by |H|^2 + 1e-3, which amplifies FP32
rounding where |H| is small (<= 1e-3 after 20 steps); FP64 <= 1e-10."""
import numpy as np
import pytest

from paper_1602_01410_gb300 import inputs

from gpu_helpers import gpu_solve, oracle_solve, rel_l2, torch_dev

pytestmark = pytest.mark.gpu

SIZES = [(96, 160), (128, 128), (384, 256), (45, 75), (256, 384)]


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def check(prob, tol, **opts):
    xg, _, _ = gpu_solve(prob, **opts)
    xo, _ = oracle_solve(prob, **opts)
    for a, b in zip(xg, xo):
        assert rel_l2([a], [b]) <= tol


def test_bgs_passes_one_iteration():
    check(inputs.random_problem(41, SIZES, 7, mask_kind="random", frac=0.4, iters=1), 1e-5, bgs_passes=3)


def test_bgs_passes_proposed_ad_ten_iterations():
    prob = inputs.random_problem(42, [(128, 256), (96, 160)], 9, mask_kind="random", frac=0.3, iters=10,
                                 psf="motion")
    check(prob, 1e-4, bgs_passes=4)


def test_bgs_passes_vectorial_tv():
    prob = inputs.random_problem(43, [(128, 128), (60, 48), (384, 384)], 5, mask_kind="bayer", channels=3, iters=3)
    check(prob, 3e-5, bgs_passes=2)


def test_bgs_passes_fp64():
    prob = inputs.random_problem(44, [(64, 64), (48, 60)], 5, mask_kind="random", frac=0.3, iters=4, dtype="f64")
    check(prob, 1e-10, bgs_passes=3)


def test_bgs_graph_replay_equals_direct_launches():
    prob = inputs.random_problem(45, [(64, 80), (128, 128)], 5, mask_kind="random", frac=0.3, iters=45)
    a, _, _ = gpu_solve(prob, bgs_passes=2)
    b, _, _ = gpu_solve(prob, stats=True, bgs_passes=2)
    for u, v in zip(a, b):
        assert np.array_equal(u, v)


def test_tikhonov_warm_start_alone():
    prob = inputs.random_problem(46, SIZES, 7, mask_kind="random", frac=0.4, iters=0)
    check(prob, 1e-5, tikh_iters=20, tikh_tau=0.1)
    check(prob, 1e-3, tikh_iters=20, tikh_tau=1e-3)


def test_tikhonov_then_admm():
    prob = inputs.random_problem(47, [(128, 256), (96, 160)], 9, mask_kind="crop", iters=5, psf="uniform")
    check(prob, 1e-4, tikh_iters=10, tikh_tau=0.05)


def test_tikhonov_vectorial_fp64():
    prob = inputs.random_problem(48, [(64, 64), (48, 60)], 5, mask_kind="bayer", channels=3, iters=3, dtype="f64")
    check(prob, 1e-10, tikh_iters=15, tikh_tau=1e-3, bgs_passes=2)


def test_options_validated():
    import paper_1602_01410_gb300 as pkg
    prob = inputs.random_problem(49, [(32, 32)], 3, iters=1)
    _, _, plan = gpu_solve(prob)
    for bad in ({"bgs_passes": 0}, {"bgs_passes": 65}, {"tikh_iters": -1}, {"tikh_tau": 0.0}, {"adapt_t": 0.5}):
        with pytest.raises(pkg.DeconvError) as e:
            plan.set_options(**bad)
        assert e.value.status == pkg.DECONV_EINVAL


# ------------------------------------------------- penalty adaptation ---

def check_adaptive(prob, tol, **opts):
    from gpu_helpers import oracle_final_mu
    xg, _, plan = gpu_solve(prob, **opts)
    xo, _ = oracle_solve(prob, **opts)
    mo = oracle_final_mu(prob, **opts)
    mg = plan.get_mu()
    print("final mu gpu", mg, "oracle", mo)
    assert mg == mo
    assert len(set(mo)) > 1 or mo[0] != prob.mu  # the rule fired
    for a, b in zip(xg, xo):
        assert rel_l2([a], [b]) <= tol


def test_adaptive_mu_from_a_large_penalty():
    prob = inputs.random_problem(51, SIZES, 7, mask_kind="random", frac=0.4, iters=12, mu=1.0)
    check_adaptive(prob, 1e-4, adapt_t=3.0)


def test_adaptive_mu_from_a_small_penalty():
    prob = inputs.random_problem(52, [(128, 256), (96, 160), (384, 384)], 9, mask_kind="crop", iters=12,
                                 mu=1e-5, lam=1e-4)
    check_adaptive(prob, 1e-4, adapt_t=3.0)


def test_adaptive_mu_vectorial_fp64_with_passes_and_warm_start():
    prob = inputs.random_problem(53, [(64, 64), (48, 60)], 5, mask_kind="bayer", channels=3, iters=10,
                                 dtype="f64", mu=1.0)
    check_adaptive(prob, 1e-10, adapt_t=3.0, bgs_passes=2, tikh_iters=5, tikh_tau=1e-2)


def test_adaptive_graph_replay_equals_direct_launches():
    prob = inputs.random_problem(54, [(64, 80), (128, 128)], 5, mask_kind="random", frac=0.3, iters=45, mu=1.0)
    a, _, pa = gpu_solve(prob, adapt_t=3.0)
    b, _, pb = gpu_solve(prob, stats=True, adapt_t=3.0)
    for u, v in zip(a, b):
        assert np.array_equal(u, v)
    assert pa.get_mu() == pb.get_mu()


def test_adaptive_warm_continuation_needs_a_fresh_solve():
    import paper_1602_01410_gb300 as pkg
    prob = inputs.random_problem(55, [(48, 64)], 5, mask_kind="random", frac=0.3, iters=7, mu=1.0)
    full, _, _ = gpu_solve(prob, adapt_t=3.0)
    _, _, plan = gpu_solve(prob, iters=4, adapt_t=3.0)
    x = plan.solve(None, 3, warm=True)
    assert plan.sync() == 0
    assert np.array_equal(x.double().cpu().numpy().reshape(full[0].shape), full[0])
    _, _, plan2 = gpu_solve(prob, iters=4)
    plan2.set_options(adapt_t=3.0)
    with pytest.raises(pkg.DeconvError) as e:
        plan2.solve(None, 3, warm=True)
    assert e.value.status == pkg.DECONV_EINVAL


def test_adaptive_checkpoint_resumes_in_another_plan():
    # The blob carries each image's penalties and v: a fresh plan continues
    # the adapted run bit for bit; a blob saved without adaptation is refused.
    import paper_1602_01410_gb300 as pkg
    torch, dev = torch_dev()
    prob = inputs.random_problem(56, [(64, 64), (48, 60)], 5, mask_kind="random", frac=0.3, iters=9, mu=1.0)
    full, _, pf = gpu_solve(prob, adapt_t=3.0)
    _, _, plan = gpu_solve(prob, iters=5, adapt_t=3.0)
    blob = plan.state_get()
    h = torch.tensor(prob.h, dtype=torch.float32, device=dev)
    mask = torch.tensor(np.concatenate([m.ravel() for m in prob.mask]), dtype=torch.uint8, device=dev)
    plan2 = pkg.Plan(prob.shapes, h, mask, prob.lam, prob.mu)
    plan2.set_options(adapt_t=3.0)
    plan2.state_set(blob)
    assert plan2.get_mu() == plan.get_mu()
    x = plan2.solve(None, 4, warm=True)
    assert plan2.sync() == 0
    assert np.array_equal(x.double().cpu().numpy(), np.concatenate([a.ravel() for a in full]))
    assert plan2.get_mu() == pf.get_mu()
    _, _, plain = gpu_solve(prob, iters=5)
    plan3 = pkg.Plan(prob.shapes, h, mask, prob.lam, prob.mu)
    plan3.set_options(adapt_t=3.0)
    plan3.state_set(plain.state_get())
    with pytest.raises(pkg.DeconvError) as e:
        plan3.solve(None, 2, warm=True)
    assert e.value.status == pkg.DECONV_EINVAL


# ------------------------------------------------------- arbitrary sizes ---

def enlarged(prob):
    import dataclasses
    import paper_1602_01410_gb300 as pkg
    ys, ms, xs = [], [], []
    for y, m, x in zip(prob.y, prob.mask, prob.x_true):
        shape = pkg.deconv_fast_shape(y.shape[1], y.shape[2], prob.channels, prob.ksize,
                                      pkg.DECONV_F32 if prob.dtype == "f32" else pkg.DECONV_F64)
        y2, m2 = pkg.enlarge(y, m, shape)
        x2, _ = pkg.enlarge(x, m, shape)
        ys.append(y2)
        ms.append(m2)
        xs.append(x2)
    return dataclasses.replace(prob, y=ys, mask=ms, x_true=xs)


def test_enlarged_prime_sizes():
    import paper_1602_01410_gb300 as pkg
    prob = inputs.random_problem(61, [(67, 131), (101, 97), (257, 263)], 7, mask_kind="crop", iters=1)
    big = enlarged(prob)
    assert big.shapes == [(72, 135), (108, 100), (270, 270)]
    check(big, 1e-5)
    big.iters = 15
    check(big, 1e-4)
    xg, _, _ = gpu_solve(big)
    for x, (M, N) in zip(xg, prob.shapes):
        assert pkg.crop(x, (M, N)).shape == (prob.channels, M, N)


def test_enlarged_rgb_with_all_variants():
    prob = inputs.random_problem(62, [(61, 59)], 5, mask_kind="bayer", channels=3, iters=6, mu=1.0)
    check_adaptive(enlarged(prob), 1e-4, adapt_t=3.0, bgs_passes=2, tikh_iters=4, tikh_tau=1e-2)


# ------------------------------------------------------------- autotuner ---

def test_every_tuning_keeps_parity():
    prob = inputs.random_problem(71, [(128, 256), (384, 384), (96, 160), (64, 1024)], 7, mask_kind="random",
                                 frac=0.3, iters=3)
    xo, _ = oracle_solve(prob)
    _, _, plan = gpu_solve(prob)
    import torch
    dev = torch.device("cuda:0")
    y = torch.tensor(np.concatenate([a.ravel() for a in prob.y]), dtype=torch.float32, device=dev)
    from gpu_helpers import split
    for t in [(152, 76, 0, 32, 32), (608, 608, 1, 32, 16), (304, 152, 1, 16, 32), (152, 608, 0, 16, 16),
              (0, 0, -1, 0, 0)]:
        plan.retune(*t)
        x = plan.solve(y, prob.iters)
        assert plan.sync() == 0
        for a, b in zip(split(x.double().cpu().numpy(), prob), xo):
            assert rel_l2([a], [b]) <= 3e-5


def test_autotune_picks_a_candidate_and_keeps_parity():
    import paper_1602_01410_gb300 as pkg
    prob = inputs.random_problem(72, [(256, 256), (384, 384)], 5, mask_kind="random", frac=0.3, iters=4)
    xo, _ = oracle_solve(prob)
    _, _, plan = gpu_solve(prob)
    import torch
    y = torch.tensor(np.concatenate([a.ravel() for a in prob.y]), dtype=torch.float32, device=torch.device("cuda:0"))
    best, ms = plan.autotune(y, 10)
    assert ms > 0 and best == pkg.deconv_get_tune(plan.handle)
    with pytest.raises(pkg.DeconvError):
        plan.solve(None, 2, warm=True)  # retuning discards the iteration state
    x = plan.solve(y, prob.iters)
    assert plan.sync() == 0
    from gpu_helpers import split
    for a, b in zip(split(x.double().cpu().numpy(), prob), xo):
        assert rel_l2([a], [b]) <= 3e-5


# ------------------------------------------------- uneven kernel supports ---

def test_uneven_kernel_supports_in_one_batch():
    # images blurred by 3x3, 7x7 and 11x11 kernels in one plan: the kernels
    # are zero-padded to 11x11, each image keeps its own boundary band
    import dataclasses
    import torch
    import paper_1602_01410_gb300 as pkg
    from gpu_helpers import split
    import oracle
    parts = [inputs.random_problem(81 + k, [s], k, mask_kind="random", frac=0.3, iters=1)
             for k, s in ((3, (96, 128)), (7, (128, 256)), (11, (384, 384)))]
    K = 11
    hs = []
    for pr in parts:
        k = pr.ksize
        pad = (K - k) // 2
        hs.append(np.pad(pr.h, pad))
    dev = torch.device("cuda:0")
    shapes = [pr.shapes[0] for pr in parts]
    h = torch.tensor(np.stack(hs), dtype=torch.float32, device=dev)
    mask = torch.tensor(np.concatenate([pr.mask[0].ravel() for pr in parts]), dtype=torch.uint8, device=dev)
    y = torch.tensor(np.concatenate([pr.y[0].ravel() for pr in parts]), dtype=torch.float32, device=dev)
    plan = pkg.Plan(shapes, h, mask, parts[0].lam, parts[0].mu, ksizes=[pr.ksize for pr in parts])
    merged = dataclasses.replace(parts[0], y=[pr.y[0] for pr in parts], mask=[pr.mask[0] for pr in parts],
                                 x_true=[pr.x_true[0] for pr in parts])
    for iters, tol in ((0, 0.0), (1, 1e-5), (10, 1e-4)):
        x = plan.solve(y, iters)
        assert plan.sync() == 0
        xg = split(x.double().cpu().numpy(), merged)
        for j, pr in enumerate(parts):
            if iters == 0:
                want = oracle.init_ytilde(pr.y[0][0], pr.mask[0][0], pr.ksize, round_f32=True)
                assert np.array_equal(xg[j][0], want.astype(np.float32).astype(np.float64))
            else:
                xo, _, _ = oracle.admm(pr.y[0], pr.mask[0], pr.h, pr.lam, pr.mu, iters, relax=pr.relax)
                assert rel_l2([xg[j]], [xo]) <= tol
