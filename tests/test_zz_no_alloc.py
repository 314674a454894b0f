"""The allocation-free entry point (deconv_solve_noalloc) against the
workspace-based one.

deconv_solve_noalloc serves callers that may not allocate device memory: it
keeps its scratch in a static device array that every call on a device
shares.  This file is named to be collected last.  It checks two calls in a
row (two different problems, so the second call must not see the first
call's state) against Plan.solve on the same inputs, and that a problem too
large for the array is refused before any launch."""
import numpy as np
import pytest

from paper_1602_01410_gb300 import inputs

from gpu_helpers import gpu_solve, rel_l2, split

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def noalloc_solve(prob):
    import torch
    import paper_1602_01410_gb300 as pkg
    dev = torch.device("cuda:0")
    h = torch.tensor(prob.h, dtype=torch.float32, device=dev)
    mask = torch.tensor(np.concatenate([m.ravel() for m in prob.mask]), dtype=torch.uint8, device=dev)
    y = torch.tensor(np.concatenate([a.ravel() for a in prob.y]), dtype=torch.float32, device=dev)
    x = torch.full_like(y, float("nan"))
    dims, keep = pkg.make_dims([s[0] for s in prob.shapes], [s[1] for s in prob.shapes], prob.ksize,
                               prob.channels)
    stream = torch.cuda.current_stream(dev)
    pkg.deconv_solve_noalloc(dims, h.data_ptr(), mask.data_ptr(), y.data_ptr(), x.data_ptr(), prob.lam, prob.mu,
                             prob.iters, stream.cuda_stream)
    return split(x.double().cpu().numpy(), prob)


def test_two_calls_in_a_row_match_the_workspace_entry_point():
    a = inputs.random_problem(31, [(96, 120), (60, 64)], 7, mask_kind="random", frac=0.4, iters=30)
    b = inputs.random_problem(32, [(128, 128)], 5, mask_kind="decim4", iters=25)
    for prob in (a, b):
        got = noalloc_solve(prob)
        want, _, _ = gpu_solve(prob)
        assert rel_l2(got, want) <= 1e-5


def test_too_large_is_refused():
    import torch
    import paper_1602_01410_gb300 as pkg
    dims, keep = pkg.make_dims([1024], [1024], 21, 1)
    assert pkg.deconv_workspace_size(dims) > (32 << 20)
    with pytest.raises(pkg.DeconvError) as e:
        pkg.deconv_solve_noalloc(dims, 256, 256, 256, 256, 1e-3, 1e-3, 1, torch.cuda.current_stream().cuda_stream)
    assert e.value.status == pkg.DECONV_ENOMEM
