"""GPU reverse pass (deconv_grad) against the FP64 oracle's reverse pass on
the same seeded inputs: loss, dL/dlambda and dL/dh (every tap), for one and
three channels, power-of-two and 3 * 2^k / 5 * 2^k lengths, batches sharing
one kernel, and several checkpoint intervals (every step stored included);
the autograd wrappers and the vector-Jacobian product; and the full-size
differentiation workload (512 x 512, 15 x 15 Gaussian, 20% missing, 100
iterations, checkpoints every 10) on two images."""
import numpy as np
import pytest

import oracle
from paper_1602_01410_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def gpu_grad(prob, iters, ckpt):
    import torch
    import paper_1602_01410_gb300 as pkg
    dev = torch.device("cuda:0")
    dt = torch.float32 if prob.dtype == "f32" else torch.float64
    h = torch.tensor(prob.h, dtype=dt, device=dev)
    mask = torch.tensor(np.concatenate([m.ravel() for m in prob.mask]), dtype=torch.uint8, device=dev)
    y = torch.tensor(np.concatenate([a.ravel() for a in prob.y]), dtype=dt, device=dev)
    xt = torch.tensor(np.concatenate([a.ravel() for a in prob.x_true]), dtype=dt, device=dev)
    plan = pkg.Plan(prob.shapes, h, mask, prob.lam, prob.mu, channels=prob.channels)
    loss, dlam, dh = plan.grad(y, xt, iters, ckpt)
    assert plan.sync() == 0
    plan.close()
    return loss, dlam, dh.double().cpu().numpy()


def oracle_grad(prob, iters):
    n = [a.size for a in prob.x_true]
    tot = float(sum(n))
    L = dl = 0.0
    dh = np.zeros_like(prob.h)
    for j in range(len(prob.shapes)):
        l, a, g, _ = oracle.admm_grad(prob.y[j], prob.mask[j], prob.h, prob.lam, prob.mu, iters, prob.x_true[j],
                                      round_f32=prob.dtype == "f32")
        w = n[j] / tot
        L += w * l
        dl += w * a
        dh += w * g
    return L, dl, dh


def check(prob, iters, ckpt, rtol, ltol=1e-5):
    """ltol: loss tolerance (1e-5 for a few iterations; the full-run FP32
    tolerance 1e-3 after 100 iterations).  rtol: gradient tolerance relative
    to |dL/dlambda| and to max |dL/dh|."""
    L, dl, dh = gpu_grad(prob, iters, ckpt)
    Lo, dlo, dho = oracle_grad(prob, iters)
    el, edl, edh = abs(L - Lo) / abs(Lo), abs(dl - dlo) / abs(dlo), np.max(np.abs(dh - dho)) / np.max(np.abs(dho))
    print(f"{prob.name} iters {iters}: loss rel {el:.2e}, dlambda rel {edl:.2e}, dh rel {edh:.2e}")
    assert el <= ltol
    assert edl <= rtol
    assert edh <= rtol
    return L, dl, dh


def test_grad_small_one_channel_partial_segment():
    prob = inputs.random_problem(51, [(64, 64)], 5, mask_kind="random", frac=0.3, iters=7, lam=2e-3, mu=2e-2)
    check(prob, 7, 3, 2e-3)


def test_grad_batch_shared_kernel_and_checkpoint_invariance():
    prob = inputs.random_problem(52, [(64, 128), (128, 64)], 7, mask_kind="random", frac=0.2, iters=6,
                                 lam=1e-3, mu=2e-2)
    a = check(prob, 6, 2, 2e-3)
    for ck in (1, 4, 6):  # 6 = iters: every step stored in the forward run; 4: a short last segment
        b = gpu_grad(prob, 6, ck)
        assert np.isclose(a[0], b[0], rtol=1e-6) and np.isclose(a[1], b[1], rtol=1e-4)
        assert np.max(np.abs(a[2] - b[2])) <= 1e-4 * np.max(np.abs(a[2]))


def test_grad_radix_3_and_5_lengths():
    # 384 = 3 * 128 and 640 = 5 * 128: the reverse row kernels with the
    # radix-3 and radix-5 combine, as rows and as columns, one and three
    # channels, a checkpoint segment boundary inside the run
    prob = inputs.random_problem(58, [(384, 640), (640, 384)], 5, mask_kind="random", frac=0.3, iters=4, lam=2e-3,
                                 mu=2e-2)
    check(prob, 4, 3, 2e-3)
    prob3 = inputs.random_problem(59, [(384, 384)], 5, mask_kind="bayer", channels=3, iters=3, lam=2e-3, mu=2e-2)
    check(prob3, 3, 2, 2e-3)


def test_grad_vectorial_tv():
    prob = inputs.random_problem(53, [(64, 64)], 5, mask_kind="bayer", channels=3, iters=5, lam=2e-3, mu=2e-2)
    check(prob, 5, 5, 2e-3)


def test_autograd_function():
    import torch
    import paper_1602_01410_gb300 as pkg
    prob = inputs.random_problem(54, [(64, 64)], 5, mask_kind="random", frac=0.3, iters=4, lam=2e-3, mu=2e-2)
    dev = torch.device("cuda:0")
    lam = torch.tensor(prob.lam, dtype=torch.float32, device=dev, requires_grad=True)
    h = torch.tensor(prob.h, dtype=torch.float32, device=dev, requires_grad=True)
    mask = torch.tensor(prob.mask[0].ravel(), dtype=torch.uint8, device=dev)
    y = torch.tensor(prob.y[0].ravel(), dtype=torch.float32, device=dev)
    xt = torch.tensor(prob.x_true[0].ravel(), dtype=torch.float32, device=dev)
    loss = pkg.DeconvLoss.apply(lam, h, y, mask, xt, prob.shapes, prob.mu, 4)
    (3.0 * loss).backward()
    Lo, dlo, dho = oracle_grad(prob, 4)
    assert abs(float(loss.detach()) - Lo) <= 1e-5 * Lo
    assert abs(float(lam.grad) - 3 * dlo) <= 2e-3 * abs(3 * dlo)
    assert np.max(np.abs(h.grad.double().cpu().numpy() - 3 * dho)) <= 2e-3 * np.max(np.abs(3 * dho))


def test_grad_fullsize_differentiation_workload():
    # measured: loss 6e-5, dlambda 7e-5, dh 4e-4 relative to the FP64 oracle
    prob = inputs.config_c5(count=2)
    check(prob, prob.iters, 10, 2e-3, ltol=1e-3)


# ------------------------------------------- vector-Jacobian product ---

def _tensors(prob):
    import torch
    dev = torch.device("cuda:0")
    h = torch.tensor(prob.h, dtype=torch.float32, device=dev)
    mask = torch.tensor(np.concatenate([m.ravel() for m in prob.mask]), dtype=torch.uint8, device=dev)
    y = torch.tensor(np.concatenate([a.ravel() for a in prob.y]), dtype=torch.float32, device=dev)
    return h, mask, y


def test_vjp_against_central_differences_of_the_oracle():
    # L(lambda, h) = <w, x^iters> for a random w: dL/dx = w.  The GPU reverse
    # pass seeded with w against central differences of the FP64 oracle's
    # forward pass, in lambda and along a random direction of h.
    import torch
    import paper_1602_01410_gb300 as pkg
    prob = inputs.random_problem(55, [(64, 64), (64, 128)], 5, mask_kind="random", frac=0.3, iters=5, lam=2e-3,
                                 mu=2e-2)
    iters = 5
    rng = np.random.default_rng(55)
    ws = [rng.standard_normal(a.shape).astype(np.float32).astype(np.float64) for a in prob.y]

    def L(lam, h):
        return sum(float(np.sum(w * oracle.admm(prob.y[j], prob.mask[j], h, lam, prob.mu, iters, relax=prob.relax)[0]))
                   for j, w in enumerate(ws))

    h, mask, y = _tensors(prob)
    plan = pkg.Plan(prob.shapes, h, mask, prob.lam, prob.mu)
    wflat = torch.tensor(np.concatenate([w.ravel() for w in ws]), dtype=torch.float32, device=y.device)
    dlam, dh = plan.vjp(y, wflat, iters, 2)
    assert plan.sync() == 0
    plan.close()
    dh = dh.double().cpu().numpy()
    eps = 1e-7
    fd_lam = (L(prob.lam + eps, prob.h) - L(prob.lam - eps, prob.h)) / (2 * eps)
    U = rng.standard_normal(prob.h.shape)
    fd_h = (L(prob.lam, prob.h + eps * U) - L(prob.lam, prob.h - eps * U)) / (2 * eps)
    print(f"vjp: dlambda {dlam:.6e} vs FD {fd_lam:.6e}; <dh, U> {np.sum(dh * U):.6e} vs FD {fd_h:.6e}")
    assert abs(dlam - fd_lam) <= 2e-3 * abs(fd_lam)
    assert abs(np.sum(dh * U) - fd_h) <= 2e-3 * np.sum(np.abs(dh * U))


def test_vjp_with_the_squared_error_seed_equals_deconv_grad():
    import torch
    import paper_1602_01410_gb300 as pkg
    prob = inputs.random_problem(56, [(64, 128)], 7, mask_kind="random", frac=0.2, iters=6, lam=1e-3, mu=2e-2)
    h, mask, y = _tensors(prob)
    xt = torch.tensor(np.concatenate([a.ravel() for a in prob.x_true]), dtype=torch.float32, device=y.device)
    plan = pkg.Plan(prob.shapes, h, mask, prob.lam, prob.mu)
    x = torch.empty_like(y)
    loss, dlam_g, dh_g = plan.grad(y, xt, 6, 3, x_out=x)
    seed = (x - xt) * np.float32(2.0 / x.numel())
    dlam_v, dh_v = plan.vjp(y, seed, 6, 3)
    assert plan.sync() == 0
    plan.close()
    assert abs(dlam_v - dlam_g) <= 1e-5 * abs(dlam_g)
    assert torch.max(torch.abs(dh_v - dh_g)) <= 1e-5 * torch.max(torch.abs(dh_g))


def test_deconv_solve_autograd_under_another_loss():
    # a loss the library does not compute itself (weighted L1 of x): the
    # autograd function's gradients equal the VJP with that loss's dL/dx
    import torch
    import paper_1602_01410_gb300 as pkg
    prob = inputs.random_problem(57, [(64, 64)], 5, mask_kind="random", frac=0.3, iters=4, lam=2e-3, mu=2e-2)
    h, mask, y = _tensors(prob)
    lam = torch.tensor(prob.lam, dtype=torch.float32, device=y.device, requires_grad=True)
    hp = h.clone().requires_grad_(True)
    wt = torch.linspace(0.5, 1.5, y.numel(), device=y.device)
    x = pkg.DeconvSolve.apply(lam, hp, y, mask, prob.shapes, prob.mu, 4)
    loss = (wt * torch.abs(x - 0.5)).sum()
    loss.backward()
    plan = pkg.Plan(prob.shapes, h, mask, prob.lam, prob.mu)
    dlam, dh = plan.vjp(y, (wt * torch.sign(x.detach() - 0.5)).contiguous(), 4, 10)
    plan.close()
    assert abs(float(lam.grad) - dlam) <= 1e-5 * abs(dlam)
    assert torch.max(torch.abs(hp.grad - dh)) <= 1e-5 * torch.max(torch.abs(dh))
