"""The fused row pass (inverse and forward halves of a plain iteration in one
kernel, row blocks taken from a work queue in order, each waiting for the x
rows of the blocks above it) against the two-kernel row pass and the FP64
oracle, and its bounded waits.

* one channel and three channels (vectorial TV), batches of uneven sizes
  (several kernel classes running side by side), one row per work item
  (the first and last items of an image then reach across the periodic
  boundary and two items up) and many rows per item, over 45 iterations
  (two replays of the captured 20-iteration loop);
* a wait limit of 0 (no waiting allowed): every item that depends on
  another gives up at once (fused row pass), or every inverse row half
  gives up on the bulk copies of its row spectra (two-kernel row pass); the
  call reports DECONV_ETIMEOUT, and the plan works again once the limit is
  restored.

Waits in these tests are bounded at 50 ms."""
import numpy as np
import pytest

from paper_1602_01410_gb300 import inputs

from gpu_helpers import oracle_solve, rel_l2, split

pytestmark = pytest.mark.gpu

WAIT_NS = 50_000_000


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def run(prob, iters, **tune):
    import torch
    import paper_1602_01410_gb300 as pkg
    dev = torch.device("cuda:0")
    h = torch.tensor(prob.h, dtype=torch.float32, device=dev)
    mask = torch.tensor(np.concatenate([m.ravel() for m in prob.mask]), dtype=torch.uint8, device=dev)
    y = torch.tensor(np.concatenate([a.ravel() for a in prob.y]), dtype=torch.float32, device=dev)
    plan = pkg.Plan(prob.shapes, h, mask, prob.lam, prob.mu, channels=prob.channels)
    plan.set_wait_limit(WAIT_NS)
    if tune:
        plan.retune(**tune)
    x = plan.solve(y, iters)
    status = plan.sync()
    out = split(x.double().cpu().numpy(), prob)
    plan.close()
    return status, out


CASES = [
    # (channels, mask, sizes, K): uneven batches, ragged last row blocks
    (1, "random", [(96, 160), (128, 128), (60, 64)], 5),
    (3, "bayer", [(64, 80), (96, 96)], 5),
]


@pytest.mark.parametrize("C,kind,sizes,K", CASES)
@pytest.mark.parametrize("row_ctas", [608, 16])  # one row per item / many rows per item
def test_fused_row_pass_matches_the_two_kernels_and_the_oracle(C, kind, sizes, K, row_ctas):
    import paper_1602_01410_gb300 as pkg
    iters = 45
    prob = inputs.random_problem(91 + C, sizes, K, mask_kind=kind, channels=C, frac=0.3, iters=iters)
    st_f, fused = run(prob, iters, row_ctas=row_ctas, fused_rows=1)
    st_s, two = run(prob, iters, row_ctas=row_ctas, fused_rows=0)
    assert st_f == pkg.DECONV_OK and st_s == pkg.DECONV_OK
    for a, b in zip(fused, two):
        assert rel_l2([a], [b]) <= 1e-6
    xo, _ = oracle_solve(prob)
    for a, b in zip(fused, xo):
        assert rel_l2([a], [b]) <= 1e-4


@pytest.mark.parametrize("fused", [1, 0])  # the fused items' flags / the inverse half's bulk copies
def test_wait_limit_zero_reports_a_timeout_and_the_plan_recovers(fused):
    import torch
    import paper_1602_01410_gb300 as pkg
    prob = inputs.random_problem(95, [(128, 128), (96, 160)], 5, mask_kind="random", frac=0.3, iters=3)
    dev = torch.device("cuda:0")
    h = torch.tensor(prob.h, dtype=torch.float32, device=dev)
    mask = torch.tensor(np.concatenate([m.ravel() for m in prob.mask]), dtype=torch.uint8, device=dev)
    y = torch.tensor(np.concatenate([a.ravel() for a in prob.y]), dtype=torch.float32, device=dev)
    plan = pkg.Plan(prob.shapes, h, mask, prob.lam, prob.mu)
    plan.retune(row_ctas=608, fused_rows=fused)  # several row blocks per image: items wait on one another
    plan.set_wait_limit(0)
    plan.solve(y, 3)
    assert plan.sync() == pkg.DECONV_ETIMEOUT
    plan.set_wait_limit(WAIT_NS)
    x = plan.solve(y, 3)
    assert plan.sync() == pkg.DECONV_OK
    xo, _ = oracle_solve(prob)
    assert rel_l2(split(x.double().cpu().numpy(), prob), xo) <= 1e-4
    with pytest.raises(pkg.DeconvError):
        plan.set_wait_limit(-1)
    plan.close()
