"""Shared helpers for the GPU tests: run a Problem through the C ABI and
through the FP64 oracle on the same seeded inputs."""
from __future__ import annotations

import numpy as np

import oracle
from paper_1602_01410_gb300 import inputs


def torch_dev():
    import torch
    return torch, torch.device("cuda:0")


def gpu_solve(prob: inputs.Problem, iters=None, stats=False, dtype=None, relax=None, tune=None, **opts):
    """Returns (list of (C, M, N) float64 arrays, stats array or None, plan).
    tune: None or deconv_retune keywords; opts: deconv_set_options keywords
    (bgs_passes, tikh_iters, tikh_tau, adapt_t)."""
    import paper_1602_01410_gb300 as pkg
    torch, dev = torch_dev()
    dt = dtype or (torch.float32 if prob.dtype == "f32" else torch.float64)
    iters = prob.iters if iters is None else iters
    h = torch.tensor(prob.h, dtype=dt, device=dev)
    mask = torch.tensor(np.concatenate([m.ravel() for m in prob.mask]), dtype=torch.uint8, device=dev)
    y = torch.tensor(np.concatenate([a.ravel() for a in prob.y]), dtype=dt, device=dev)
    plan = pkg.Plan(prob.shapes, h, mask, prob.lam, prob.mu, channels=prob.channels,
                    relax=prob.relax if relax is None else relax)
    if tune:
        plan.retune(**tune)
    if opts:
        plan.set_options(**opts)
    st = torch.zeros((len(prob.shapes), max(iters, 1), 3), dtype=torch.float64, device=dev) if stats else None
    x = plan.solve(y, iters, stats=st)
    status = plan.sync()
    assert status == pkg.DECONV_OK, pkg.deconv_status_string(status)
    xs = split(x.double().cpu().numpy(), prob)
    return xs, (st.cpu().numpy() if stats else None), plan


def split(flat: np.ndarray, prob: inputs.Problem):
    out, o = [], 0
    for (M, N) in prob.shapes:
        n = prob.channels * M * N
        out.append(flat[o:o + n].reshape(prob.channels, M, N))
        o += n
    return out


def oracle_solve(prob: inputs.Problem, iters=None, stats=False, relax=None, bgs_passes=1, tikh_iters=0,
                 tikh_tau=1e-3, adapt_t=0.0):
    iters = prob.iters if iters is None else iters
    xs, ss = [], []
    for j in range(len(prob.shapes)):
        x, _, s = oracle.admm(prob.y[j], prob.mask[j], prob.h, prob.lam, prob.mu, iters,
                              relax=prob.relax if relax is None else relax,
                              round_f32=prob.dtype == "f32", stats=stats, passes=bgs_passes,
                              tikh_iters=tikh_iters, tikh_tau=tikh_tau, adapt_t=adapt_t)
        xs.append(x)
        ss.append(s)
    return xs, ss


def oracle_final_mu(prob: inputs.Problem, iters=None, **opts):
    """Final per-image penalty of the oracle run (penalty adaptation)."""
    iters = prob.iters if iters is None else iters
    out = []
    for j in range(len(prob.shapes)):
        _, st, _ = oracle.admm(prob.y[j], prob.mask[j], prob.h, prob.lam, prob.mu, iters, relax=prob.relax,
                               round_f32=prob.dtype == "f32", passes=opts.get("bgs_passes", 1),
                               tikh_iters=opts.get("tikh_iters", 0), tikh_tau=opts.get("tikh_tau", 1e-3),
                               adapt_t=opts.get("adapt_t", 0.0))
        out.append(st.mu)
    return out


def rel_l2(a, b) -> float:
    a = np.concatenate([v.ravel() for v in a])
    b = np.concatenate([v.ravel() for v in b])
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def psnr(x, ref) -> float:
    mse = np.mean((x - ref) ** 2)
    return float(10 * np.log10(1.0 / mse))
