"""The plain comparison path in bench.py computes the same iteration as the
FP64 oracle (so timing it against the fused path compares equal work), and
its autograd gradient matches the oracle's reverse pass.  Runs on CPU."""
import numpy as np
import torch

import bench
import oracle
from paper_1602_01410_gb300 import inputs


def test_plain_solve_matches_oracle():
    prob = inputs.random_problem(61, [(32, 48), (40, 40)], 5, mask_kind="random", frac=0.3, iters=6, dtype="f64")
    xs = bench.plain_solve(prob, 6, torch.device("cpu"), torch.float64)
    for j, x in enumerate(xs):
        xo, _, _ = oracle.admm(prob.y[j], prob.mask[j], prob.h, prob.lam, prob.mu, 6, round_f32=False)
        assert np.max(np.abs(x.numpy() - xo)) < 1e-10


def test_plain_grad_matches_oracle():
    prob = inputs.random_problem(62, [(32, 32)], 5, mask_kind="random", frac=0.3, iters=4, dtype="f64",
                                 lam=2e-3, mu=2e-2)
    L, dl, dh = bench.plain_grad(prob, 4, torch.device("cpu"), torch.float64)
    Lo, dlo, dho, _ = oracle.admm_grad(prob.y[0], prob.mask[0], prob.h, prob.lam, prob.mu, 4, prob.x_true[0],
                                       round_f32=False)
    assert abs(L - Lo) < 1e-12 and abs(dl - dlo) < 1e-9 * abs(dlo)
    assert np.max(np.abs(dh.numpy() - dho)) < 1e-9 * np.max(np.abs(dho))
