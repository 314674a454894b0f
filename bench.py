#!/usr/bin/env python3
"""Benchmark of the partial-ADMM deconvolution hot path on GB300.

Metric: Mpixel * ADMM-iterations / s (channel-pixels of the extended grid
times iterations, per second of device time), whole job over all ranks.

A step is one deconv_solve call of the workload: the initial fill (border
padding) and the workload's full iteration count, inputs resident in HBM.
Default workload (N = 1), the largest: 32 RGB FP32 frames with sides from
{512, ..., 1536} (113 M channel-pixels), 13 x 13 Gaussian blur (sigma 2.5),
RGGB Bayer mask, vectorial TV, BSNR 45 dB, 400 iterations.  Batches shard by
image across ranks (strong scaling, no data-path collective); single-image
work does not shard: under torchrun every rank solves its own replica (weak
scaling).

Timing: W untimed warm-up steps, then K steps, each preceded by an L2 flush
(a 512 MB device write, outside the timed events) and bracketed by CUDA
events on the plan's stream; a barrier and a device synchronise on both
sides; the max over ranks.  `e2e` times the same step from host buffers:
deconv_solve_host (pinned host y in, host x out, copies included), or for
the gradient workload pinned y and x_true copied in, deconv_grad, and the
loss and gradients read back.
`roofline` is the whole iteration against the HBM roofline: the method's
own bytes per channel-pixel and iteration (y~ read, z written, d read and
written, H^ read, mask bits) times the measured rate, over the measured
copy bandwidth.  Its `passes` split one iteration into column and row
passes with CUDA events captured between the passes of the CUDA graph, in
one profiled replay right after the timed steps (same plan, stream and
tuning).  `plain` times the unfused per-image cuFFT path with CUDA events
over the same iteration count (torch.autograd for the gradient workload).
`cpu_baseline` times the FP64 oracle on the host cores on a bounded sample.
`--impl reference` times the oracle itself as the reference arm.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

WORKLOADS = {
    "c2": "1024x1024 FP32, 21x21 random-walk motion blur, 1004x1004 valid crop with 40% missing, "
          "BSNR 40 dB, lambda 2e-6, mu 1e-3, 500 iterations",
    "c1": "64x64 FP64, 9x9 uniform blur, 56x56 valid crop, BSNR 50 dB, lambda 2e-5, mu 1e-3, 300 iterations",
    "c3": "16 FP32 images with sides from {256..1024}, 9x9 Gaussian (sigma 2), x4 decimation, "
          "BSNR 40 dB, lambda 2e-4, mu 1e-3, 300 iterations",
    "c4": "32 RGB FP32 frames with sides from {512..1536}, 13x13 Gaussian (sigma 2.5), RGGB Bayer, "
          "vectorial TV, BSNR 45 dB, lambda 1e-5, mu 1e-3, 400 iterations",
    "c5": "8 FP32 512x512 images, 15x15 Gaussian, 20% missing, BSNR 40 dB, lambda 5e-6, mu 1e-3, "
          "100 iterations",
}


def make_problem(name: str):
    from paper_1602_01410_gb300 import inputs
    return {"c1": lambda: inputs.config_c1("f64"), "c2": inputs.config_c2, "c3": inputs.config_c3,
            "c4": inputs.config_c4, "c5": inputs.config_c5}[name]()


# The method's own bytes per channel-pixel and iteration (FP32; FP64
# doubles the values): what one iteration must read and write whatever the
# design.  Row pass: y~ read 4, z written 4f (f = unobserved fraction),
# d = (d_h, d_v) read 8 and written 8, mask bits 1/8.  Column pass: the
# H^ half-spectrum 4.  The row-spectral intermediates the two-pass design
# writes and reads (about 8 B each way per pass) are design traffic, not
# counted here.
def algorithmic_bytes(f_unobs: float, esz: int = 4):
    s = esz / 4.0
    row = (20.0 + 4.0 * f_unobs) * s + 0.125
    col = 4.0 * s
    return {"row": row, "col": col, "iter": row + col}


def algorithmic_bytes_per_px(f_unobs: float, esz: int = 4) -> float:
    return algorithmic_bytes(f_unobs, esz)["iter"]


class ClockSampler:
    """nvidia-smi sampling during the timed region."""
    FIELDS = ["clocks.sm", "clocks.max.sm", "clocks_event_reasons.hw_slowdown",
              "clocks_event_reasons.hw_thermal_slowdown", "clocks_event_reasons.sw_thermal_slowdown",
              "clocks_event_reasons.sw_power_cap"]

    def __init__(self, index: int):
        self.index = index
        self.samples = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + ",".join(self.FIELDS),
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=subprocess.PIPE,
                stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == len(self.FIELDS):
                self.samples.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        reasons = set()
        for s in self.samples:
            for name, v in zip(["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"], s[2:]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.samples)}


# ----------------------------------------------------------------- plain ---
# The plain comparison path: one image at a time, cuFFT (torch.fft) for every
# transform and separate torch elementwise/stencil ops for every step of the
# iteration (no fusion, no packing of real transforms).  Used only as a timed
# comparison; the library never calls it.


def plain_setup(prob, j, dev, dt):
    import torch
    M, N = prob.shapes[j]
    K = prob.ksize
    b = K // 2
    hg = torch.zeros((M, N), dtype=dt, device=dev)
    hk = torch.tensor(prob.h, dtype=dt, device=dev)
    for p in range(-b, b + 1):
        for q in range(-b, b + 1):
            hg[p % M, q % N] += hk[p + b, q + b]
    H = torch.fft.rfft2(hg)
    k1 = torch.arange(M, device=dev, dtype=dt)[:, None]
    k2 = torch.arange(N // 2 + 1, device=dev, dtype=dt)[None, :]
    D2 = 4 * torch.sin(torch.pi * k1 / M) ** 2 + 4 * torch.sin(torch.pi * k2 / N) ** 2
    den = H.real ** 2 + H.imag ** 2 + prob.mu * D2
    return H, den


def plain_init(y, m, K):
    """Initial fill (border padding, mean of the observed values elsewhere)."""
    import torch
    C, M, N = y.shape
    b = K // 2
    obs = m != 0
    mean = (y * obs).sum(dim=(1, 2), keepdim=True) / obs.sum(dim=(1, 2), keepdim=True).clamp(min=1)
    ii = torch.arange(M, device=y.device).clamp(b, M - b - 1)
    jj = torch.arange(N, device=y.device).clamp(b, N - b - 1)
    yc, oc = y[:, ii][:, :, jj], obs[:, ii][:, :, jj]
    band = torch.ones((M, N), dtype=torch.bool, device=y.device)
    band[b:M - b, b:N - b] = False
    fill = torch.where(band[None] & oc, yc, mean.expand_as(y))
    return torch.where(obs, y, fill)


def plain_iterate(yt, d, v, y, m, H, den, lam, mu, relax, iters):
    import torch
    obs = m != 0
    tau = lam / mu
    x = None
    for _ in range(iters):
        u = v - d
        dtu = (torch.roll(u[:, 0], 1, 2) - u[:, 0]) + (torch.roll(u[:, 1], 1, 1) - u[:, 1])
        rhs = torch.fft.irfft2(torch.conj(H) * torch.fft.rfft2(yt), s=yt.shape[-2:]) + mu * dtu
        x = torch.fft.irfft2(torch.fft.rfft2(rhs) / den, s=yt.shape[-2:])
        t = torch.fft.irfft2(H * torch.fft.rfft2(x), s=yt.shape[-2:])
        yt = torch.where(obs, yt, relax * t - (relax - 1) * yt)
        dx = torch.stack([torch.roll(x, -1, 2) - x, torch.roll(x, -1, 1) - x], 1)
        a = dx + d
        nrm = torch.sqrt((a * a).sum(dim=(0, 1), keepdim=True))
        v = a * torch.clamp(1 - tau / torch.clamp(nrm, min=1e-30), min=0)
        d = a - v
    return x, yt, d, v


def plain_prepare(prob, dev, dt):
    """Per-image device inputs and spectra of the plain path (set-up, not timed)."""
    import torch
    out = []
    for j in range(len(prob.shapes)):
        H, den = plain_setup(prob, j, dev, dt)
        y = torch.tensor(prob.y[j], dtype=dt, device=dev)
        m = torch.tensor(prob.mask[j], device=dev)
        out.append((H, den, y, m))
    return out


def plain_solve(prob, iters, dev, dt, prepared=None):
    import torch
    prepared = prepared or plain_prepare(prob, dev, dt)
    out = []
    for (H, den, y, m) in prepared:
        yt = plain_init(y, m, prob.ksize)
        v = torch.stack([torch.roll(yt, -1, 2) - yt, torch.roll(yt, -1, 1) - yt], 1)
        d = torch.zeros_like(v)
        x, _, _, _ = plain_iterate(yt, d, v, y, m, H, den, prob.lam, prob.mu, prob.relax, iters)
        out.append(x)
    return out


def plain_grad(prob, iters, dev, dt):
    """torch.autograd through the unrolled plain iteration: loss and gradients."""
    import torch
    lam = torch.tensor(prob.lam, dtype=dt, device=dev, requires_grad=True)
    hk = torch.tensor(prob.h, dtype=dt, device=dev, requires_grad=True)
    n_all = float(sum(a.size for a in prob.x_true))
    loss = 0.0
    for j in range(len(prob.shapes)):
        M, N = prob.shapes[j]
        K = prob.ksize
        b = K // 2
        idx_i = torch.tensor([p % M for p in range(-b, b + 1)], device=dev)
        idx_j = torch.tensor([q % N for q in range(-b, b + 1)], device=dev)
        hg = torch.zeros((M, N), dtype=dt, device=dev).index_put((idx_i[:, None], idx_j[None, :]), hk)
        H = torch.fft.rfft2(hg)
        k1 = torch.arange(M, device=dev, dtype=dt)[:, None]
        k2 = torch.arange(N // 2 + 1, device=dev, dtype=dt)[None, :]
        den = H.real ** 2 + H.imag ** 2 + prob.mu * (4 * torch.sin(torch.pi * k1 / M) ** 2 +
                                                     4 * torch.sin(torch.pi * k2 / N) ** 2)
        y = torch.tensor(prob.y[j], dtype=dt, device=dev)
        m = torch.tensor(prob.mask[j], device=dev)
        yt = plain_init(y, m, K)
        v = torch.stack([torch.roll(yt, -1, 2) - yt, torch.roll(yt, -1, 1) - yt], 1)
        d = torch.zeros_like(v)
        x, _, _, _ = plain_iterate(yt, d, v, y, m, H, den, lam, prob.mu, prob.relax, iters)
        xt = torch.tensor(prob.x_true[j], dtype=dt, device=dev)
        loss = loss + ((x - xt) ** 2).sum() / n_all
    loss.backward()
    return float(loss.detach()), float(lam.grad), hk.grad.detach()


def subset_problem(prob, idx):
    """The images `idx` of a batch, as a Problem of their own."""
    import copy
    sub = copy.copy(prob)
    sub.x_true = [prob.x_true[j] for j in idx]
    sub.y = [prob.y[j] for j in idx]
    sub.mask = [prob.mask[j] for j in idx]
    return sub


# DRAM bytes (read + write) per channel-pixel and iteration, all kernels of
# one iteration, from an ncu capture of the kernels as they stand (file
# named beside each figure; the capture's per-pixel figure is scaled to the
# workload's pixels).  A workload without a capture of the current kernels
# reports traffic null.
ITER_TRAFFIC_BYTES_PER_PX = {
    "c4": (63.85, "profiles/traffic_c4_1536_rgb_ncu.md: ncu dram__bytes_read.sum + dram__bytes_write.sum of the "
                  "three kernels of one iteration on the four 1536x1536 RGB frames (cold cache), per channel-pixel, "
                  "times the pixels of one iteration"),
}


def l2_copy_peak_gbs(dev, mb: int = 32, reps: int = 40) -> float:
    """Read + write bandwidth of device copies between two buffers that stay
    in L2 (2 x 32 MB; L2 is 126 MB), replayed as one CUDA graph so that the
    short copies are not separated by launch gaps; CUDA events, best of three
    replays."""
    import torch
    n = mb * 1024 * 1024 // 4
    a = torch.rand(n, device=dev)
    b = torch.empty_like(a)
    side = torch.cuda.Stream(device=dev)
    side.wait_stream(torch.cuda.current_stream(dev))
    with torch.cuda.stream(side):
        for _ in range(3):
            b.copy_(a)
    torch.cuda.current_stream(dev).wait_stream(side)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        for _ in range(reps):
            b.copy_(a)
    g.replay()
    torch.cuda.synchronize(dev)
    best = 0.0
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        g.replay()
        e1.record()
        torch.cuda.synchronize(dev)
        best = max(best, 2.0 * n * 4 * reps / (e0.elapsed_time(e1) / 1e3) / 1e9)
    return best


def measured_peak_hbm():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def host_cores() -> int:
    """Cores the oracle's OpenMP threads may use: the affinity mask, capped by
    OMP_NUM_THREADS when that is set."""
    try:
        n = len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        n = os.cpu_count() or 1
    omp = os.environ.get("OMP_NUM_THREADS", "")
    if omp.isdigit() and int(omp) > 0:
        n = min(n, int(omp))
    return n


def cpu_baseline(name: str, budget_s: float = 20.0, options=(1, 0, 1e-3, 0.0)):
    """FP64 oracle on the host cores: a bounded sample of the workload (with
    the same iteration options: BGS passes, Tikhonov steps and tau, adaptation)."""
    import oracle
    prob = make_problem(name)
    j = 0
    y, m = prob.y[j], prob.mask[j]
    px = prob.channels * y.shape[-2] * y.shape[-1]
    opts = dict(passes=options[0], tikh_iters=options[1], tikh_tau=options[2], adapt_t=options[3])
    t0 = time.perf_counter()
    oracle.admm(y, m, prob.h, prob.lam, prob.mu, 1, **opts)
    t1 = time.perf_counter()
    per_iter = max(t1 - t0, 1e-3)
    n = max(2, min(prob.iters, int(budget_s / per_iter)))
    t0 = time.perf_counter()
    oracle.admm(y, m, prob.h, prob.lam, prob.mu, n, **opts)
    dt = time.perf_counter() - t0
    cores = host_cores()
    return {"value": px * n / dt / 1e6, "unit": "Mpx*iter/s", "cores": cores, "kind": "oracle",
            "sample": f"image 0 of the workload ({y.shape[-2]}x{y.shape[-1]}x{prob.channels}), {n} iterations "
                      f"incl. setup, FP64 C+OpenMP, {dt:.1f} s"}


def run_reference(args, rank: int, world: int):
    if rank != 0:
        return
    import oracle
    prob = make_problem(args.config)
    y, m = prob.y[0], prob.mask[0]
    px = prob.channels * y.shape[-2] * y.shape[-1]
    sample_iters = max(1, min(prob.iters, args.ref_iters))
    opts = dict(passes=args.bgs_passes, tikh_iters=args.tikh_iters, tikh_tau=args.tikh_tau, adapt_t=args.adapt_t)
    for _ in range(args.warmup):
        oracle.admm(y, m, prob.h, prob.lam, prob.mu, 1, **opts)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.admm(y, m, prob.h, prob.lam, prob.mu, sample_iters, **opts)
    dt = time.perf_counter() - t0
    value = px * sample_iters * args.steps / dt / 1e6
    cores = host_cores()
    out = {"impl": "reference", "metric": "Mpx*iter/s", "value": value, "unit": "Mpx*iter/s", "n_gpus": 0,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic (seeded generator)",
           "config": {"workload": f"{args.config}: {WORKLOADS[args.config]}",
                      "sample": f"image 0, {sample_iters} iterations per step",
                      "options": {"bgs_passes": args.bgs_passes, "tikh_iters": args.tikh_iters,
                                  "tikh_tau": args.tikh_tau, "adapt_t": args.adapt_t}},
           "cpu_baseline": {"value": value, "unit": "Mpx*iter/s", "cores": cores, "kind": "oracle",
                            "sample": f"image 0 of the workload, {sample_iters} iterations per step, "
                                      f"{args.steps} steps"},
           "e2e": {"value": value, "unit": "Mpx*iter/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="c4", choices=sorted(WORKLOADS))
    ap.add_argument("--ref-iters", type=int, default=10)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true",
                    help="skip the plain per-image cuFFT comparison (torch.autograd for c5)")
    ap.add_argument("--plain-iters", type=int, default=0,
                    help="iterations of the plain comparison (0: the workload's own count)")
    ap.add_argument("--e2e-steps", type=int, default=5, help="steps of the end-to-end (host buffer) leg")
    ap.add_argument("--iters", type=int, default=0,
                    help="override the workload's iteration count (profiling runs; recorded in config)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default launch tuning (the autotuner runs at plan set-up, outside the timing)")
    ap.add_argument("--tune-iters", type=int, default=30)
    ap.add_argument("--tune", type=str, default="",
                    help="a launch tuning as JSON (deconv_retune keywords) instead of the autotuner (profiling runs)")
    ap.add_argument("--images", type=str, default="",
                    help="comma-separated image indices of the batch to keep (small profiling cases)")
    ap.add_argument("--timed-only", action="store_true",
                    help="skip the e2e, per-pass and CPU-baseline legs (profiling runs)")
    ap.add_argument("--bgs-passes", type=int, default=1,
                    help="BGS passes per iteration (Proposed-AD: (K - 1) / 2 for a K x K blur)")
    ap.add_argument("--adapt-t", type=float, default=0.0, help="penalty adaptation threshold t (0: fixed mu)")
    ap.add_argument("--tikh-iters", type=int, default=0, help="Tikhonov warm-start steps per solve")
    ap.add_argument("--tikh-tau", type=float, default=1e-3)
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch
    import torch.distributed as dist

    import paper_1602_01410_gb300 as pkg
    from paper_1602_01410_gb300 import build as pkg_build

    pkg_build.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if world > 1:
            dist.barrier()

    prob = make_problem(args.config)
    if args.iters > 0:
        prob.iters = args.iters
    if args.images:
        prob = subset_problem(prob, [int(v) for v in args.images.split(",")])
    total_px_all = prob.pixels()
    sharded = world > 1 and len(prob.shapes) > 1
    if sharded:
        # Independent images: each rank solves its share (no data-path collective).
        from paper_1602_01410_gb300 import shard
        mine = shard.partition([prob.channels * M * N for (M, N) in prob.shapes], world)[rank]
        prob = subset_problem(prob, mine)
    dt = torch.float64 if prob.dtype == "f64" else torch.float32
    esz = 8 if prob.dtype == "f64" else 4
    h = torch.tensor(prob.h, dtype=dt, device=dev)
    mask_np = np.concatenate([m.ravel() for m in prob.mask])
    y_np = np.concatenate([a.ravel() for a in prob.y])
    mask = torch.tensor(mask_np, dtype=torch.uint8, device=dev)
    y = torch.tensor(y_np, dtype=dt, device=dev)
    stream = torch.cuda.Stream(device=dev)
    pkg.Plan(prob.shapes, h, mask, prob.lam, prob.mu, channels=prob.channels, stream=stream).close()  # warm-up
    torch.cuda.synchronize(dev)
    t_plan = time.perf_counter()
    plan = pkg.Plan(prob.shapes, h, mask, prob.lam, prob.mu, channels=prob.channels, stream=stream)
    torch.cuda.synchronize(dev)
    plan_ms = (time.perf_counter() - t_plan) * 1e3
    x = torch.empty_like(y)
    px = prob.pixels()
    f_unobs = float(1.0 - mask_np.mean())
    alg = algorithmic_bytes(f_unobs, esz)
    peak, peak_kind = measured_peak_hbm()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    grad_mode = args.config == "c5"
    options = (args.bgs_passes, args.tikh_iters, args.tikh_tau, args.adapt_t)
    variant = options != (1, 0, 1e-3, 0.0)
    if variant:
        if grad_mode:
            raise SystemExit("the gradient workload runs the default iteration only")
        plan.set_options(*options)
    tune = None
    if args.tune:
        tune = json.loads(args.tune)
        plan.retune(**tune)
    elif not args.no_autotune:  # timed on the forward iteration (the gradient step reuses its passes)
        with torch.cuda.stream(stream):
            tune, _ = plan.autotune(y, args.tune_iters)
    if grad_mode:
        x_true = torch.tensor(np.concatenate([a.ravel() for a in prob.x_true]), dtype=dt, device=dev)
        gws_n = pkg.deconv_grad_workspace_size(plan.handle, prob.iters, 10)
        gws = torch.empty(gws_n + 256, dtype=torch.uint8, device=dev)
        gptr = gws.data_ptr() + (-gws.data_ptr()) % 256
        dh = torch.empty_like(h)

    def step():
        if grad_mode:
            loss, dlam = pkg.deconv_grad(plan.handle, y.data_ptr(), x_true.data_ptr(), prob.iters, 10, gptr, gws_n,
                                         dh.data_ptr(), x.data_ptr())
            if sharded:
                from paper_1602_01410_gb300 import shard
                shard.combine_grad(loss, dlam, dh, prob.pixels(), total_px_all)
        else:
            plan.solve(y, prob.iters, x=x)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
    torch.cuda.synchronize(dev)
    status = plan.sync()
    if status != pkg.DECONV_OK:
        raise SystemExit(f"solve failed: {pkg.deconv_status_string(status)}")

    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    torch.cuda.synchronize(dev)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    with torch.cuda.stream(stream):
        for k in range(args.steps):
            flush.fill_(float(k))
            starts[k].record(stream)
            step()
            ends[k].record(stream)
    torch.cuda.synchronize(dev)
    barrier()
    clk = clocks.stop()
    t_ms = sum(s.elapsed_time(e) for s, e in zip(starts, ends))
    if plan.sync() != pkg.DECONV_OK:
        raise SystemExit("solve reported a device error")
    t = torch.tensor([t_ms], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    t_ms = float(t.item())
    units = (total_px_all if sharded else px * world) * prob.iters * args.steps
    value = units / (t_ms / 1e3) / 1e6
    if args.timed_only:
        if rank == 0:
            print(json.dumps({"metric": "Mpx*iter/s", "value": value, "unit": "Mpx*iter/s", "n_gpus": world,
                              "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_ms / args.steps,
                              "config": {"workload": args.config, "iterations": prob.iters,
                                         "tune": tune if tune is not None else "default launch tuning"},
                              "clocks": clk, "timed_only": True}))
        plan.close()
        if world > 1:
            dist.destroy_process_group()
        return

    # End to end through the public API, host buffers in and out.
    y_host = torch.tensor(y_np, dtype=dt).pin_memory()
    if grad_mode:
        # the gradient step: pinned y and x_true copied in on the plan's stream,
        # deconv_grad (returns loss and dL/dlambda on the host), dL/dh read back
        xt_host = x_true.cpu().pin_memory()
        dh_host = torch.empty(tuple(dh.shape), dtype=dt).pin_memory()
        y_dev, xt_dev = torch.empty_like(y), torch.empty_like(x_true)
        e2e_in = (y_host.numel() + xt_host.numel()) * esz
        e2e_out = dh_host.numel() * esz + 16

        def e2e_step():
            with torch.cuda.stream(stream):
                y_dev.copy_(y_host, non_blocking=True)
                xt_dev.copy_(xt_host, non_blocking=True)
                loss, dlam = pkg.deconv_grad(plan.handle, y_dev.data_ptr(), xt_dev.data_ptr(), prob.iters, 10,
                                             gptr, gws_n, dh.data_ptr(), x.data_ptr())
                if sharded:
                    from paper_1602_01410_gb300 import shard
                    shard.combine_grad(loss, dlam, dh, prob.pixels(), total_px_all)
                dh_host.copy_(dh, non_blocking=True)
            stream.synchronize()
    else:
        # the forward solve through deconv_solve_host (copies inside the call)
        x_host = torch.empty_like(y_host).pin_memory()
        e2e_in = e2e_out = int(y_np.size * esz)

        def e2e_step():
            plan.solve_host(y_host, x_host, prob.iters)
    e2e_step()
    barrier()
    e2e_ms = 0.0
    e2e_steps = max(1, min(args.steps, args.e2e_steps))
    for k in range(e2e_steps):
        flush.fill_(float(k))
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        e2e_step()
        e2e_ms += (time.perf_counter() - t0) * 1e3
    e = torch.tensor([e2e_ms], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(e, op=dist.ReduceOp.MAX)
    e2e_units = (total_px_all if sharded else px * world) * prob.iters * e2e_steps
    e2e_value = e2e_units / (float(e.item()) / 1e3) / 1e6

    # Split of one iteration into its passes: one profiled replay of the
    # captured loop (CUDA events between the passes), same plan and stream.
    passes = None
    if not grad_mode and prob.iters > 20:
        plan.set_profiling(True)
        with torch.cuda.stream(stream):
            flush.fill_(0.0)
            plan.solve(y, min(prob.iters, 41), x=x)
        ms_col, ms_row, ms_it = plan.graph_pass_times()
        plan.set_profiling(False)
        passes = {}
        for name, ms in (("col", ms_col), ("row", ms_row)) if ms_col >= 0 else ():
            b_px = alg[name]
            gbs = b_px * px / (ms / 1e3) / 1e9 / world if ms > 0 else None
            passes[name] = {"ms_per_iter": ms, "algorithmic_bytes_per_px": b_px, "achieved_gbs": gbs,
                            "frac": (gbs / peak) if gbs else None}
        passes["iteration_ms"] = ms_it
        if ms_col >= 0:
            passes["dominant"] = "row" if ms_row >= ms_col else "col"
        else:
            passes["note"] = ("the kernel classes run as independent chains, so their passes overlap: "
                              "only the whole iteration is timed")
        passes["how"] = ("CUDA events captured between the passes of the CUDA graph (20-iteration loop), "
                         "one replay after the timed steps; the events replace the overlap of each pass's "
                         "launch with the previous pass's tail")
    launches_per_step = pkg.deconv_kernel_launches(plan.handle, prob.iters, 1 if grad_mode else 0, 10)
    step_gbs = value * 1e6 * alg["iter"] / 1e9 / world
    traffic_px = ITER_TRAFFIC_BYTES_PER_PX.get(args.config) if not (args.images or variant) else None

    out = {
        "metric": "Mpx*iter/s", "value": value, "unit": "Mpx*iter/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_ms / args.steps, "higher_is_better": True,
        "scaling": "strong" if sharded else "weak",
        "vs_baseline": None, "dtype": "f64" if esz == 8 else "f32", "data": "synthetic (seeded generator)",
        "config": {"workload": f"{args.config}: {WORKLOADS[args.config]}",
                   "pixels_per_iter": px, "iterations": prob.iters,
                   "plan_create_ms": plan_ms,
                   "l2": "flushed before every timed step (512 MB write); the plan's "
                         f"{plan.workspace_bytes / 2**20:.0f} MB workspace is reused across the step's iterations",
                   "parallelism": ("images sharded across ranks" if sharded else "replicas") if world > 1
                   else "single GPU",
                   "tune": tune if tune is not None else "default launch tuning",
                   "options": {"bgs_passes": args.bgs_passes, "tikh_iters": args.tikh_iters,
                               "tikh_tau": args.tikh_tau, "adapt_t": args.adapt_t}},
        "e2e": {"value": e2e_value, "unit": "Mpx*iter/s", "h2d_bytes_per_step": int(e2e_in),
                "d2h_bytes_per_step": int(e2e_out), "steps": e2e_steps},
        # Whole iteration against HBM: the method's bytes per channel-pixel
        # and iteration at the timed rate (counted for one BGS pass at fixed
        # mu: not reported for the variants, nor for the gradient step).
        "roofline": {"bound": "hbm", "kernel": "one iteration (column pass + row pass)",
                     "achieved": None if (variant or grad_mode) else step_gbs, "peak": peak, "unit": "GB/s",
                     "frac": None if (variant or grad_mode) else step_gbs / peak, "peak_kind": peak_kind,
                     "algorithmic_bytes_per_px_iter": alg["iter"],
                     "traffic": (traffic_px[0] * px if traffic_px else None),
                     "traffic_source": (traffic_px[1] if traffic_px else None),
                     "passes": passes},
        "clocks": clk,
        "gpu_launches": launches_per_step * args.steps,
    }
    if args.config == "c2" and not variant:
        # The single 1024^2 image's 52 MB state stays in L2: its binding roof is
        # L2 bandwidth, against which the design's own traffic is compared
        # (the method's bytes, plus the two row-spectral intermediates written
        # and read, 32 B, plus x written and read back and y~ read twice, 12 B).
        l2_peak = l2_copy_peak_gbs(dev)
        design = alg["iter"] + 32.0 * esz / 4 + 12.0 * esz / 4
        l2_gbs = value * 1e6 * design / 1e9 / world
        out["roofline"]["l2"] = {"peak_gbs": l2_peak, "peak_kind": "measured here: L2-resident device copies, "
                                 "2 x 32 MB, one CUDA graph", "design_bytes_per_px_iter": design, "achieved_gbs": l2_gbs,
                                 "frac": l2_gbs / l2_peak}
    if grad_mode:
        out["config"]["step"] = ("deconv_grad: forward with checkpoints every 10 iterations, loss, reverse pass "
                                 "(dL/dlambda, dL/dh); value counts forward iterations")
        out["e2e"]["note"] = ("e2e times the gradient step: pinned y and x_true in, deconv_grad, loss, "
                              "dL/dlambda and dL/dh out")
    if not args.no_plain and not variant:
        n_it = prob.iters if args.plain_iters <= 0 else min(prob.iters, args.plain_iters)
        prepared = None if grad_mode else plain_prepare(prob, dev, dt)
        for _ in range(2):
            (plain_grad(prob, 2, dev, dt) if grad_mode else plain_solve(prob, 2, dev, dt, prepared))
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        flush.fill_(1.0)
        e0.record()
        if grad_mode:
            plain_grad(prob, n_it, dev, dt)
        else:
            plain_solve(prob, n_it, dev, dt, prepared)
        e1.record()
        torch.cuda.synchronize(dev)
        pt = e0.elapsed_time(e1) / 1e3
        pv = px * n_it / pt / 1e6
        out["plain"] = {"value": pv, "unit": "Mpx*iter/s", "iterations": n_it, "speedup": value / pv,
                        "timing": "CUDA events on the current stream, one run of the full iteration count "
                                  "(per-image spectra and inputs prepared before the timed region)",
                        "what": ("torch.autograd through the unrolled per-image torch.fft iteration" if grad_mode
                                 else "per-image torch.fft (cuFFT) transforms and unfused torch ops")}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args.config, options=options)
    if rank == 0:
        print(json.dumps(out))
    plan.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
