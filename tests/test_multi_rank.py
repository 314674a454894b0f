"""Multi-rank host logic on CPU (gloo, world size 2): the image partition
covers every image once and balances pixels; per-rank gradients of the
differentiation workload, combined with one all-reduce, equal the
full-batch gradient (FP64 oracle)."""
import os
import socket

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1602_01410_gb300 import shard


def test_partition_covers_and_balances():
    sizes = [256 * 256, 1024 * 1024, 512 * 512, 384 * 384, 768 * 768, 1024 * 1024, 256 * 256]
    for world in (1, 2, 3, 4, 8):
        parts = shard.partition(sizes, world)
        assert sorted(j for p in parts for j in p) == list(range(len(sizes)))
        loads = [sum(sizes[j] for j in p) for p in parts]
        assert max(loads) - min(loads) <= max(sizes)
    assert shard.partition([5, 5], 2) == [[0], [1]]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import oracle
    from paper_1602_01410_gb300 import inputs
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    prob = inputs.random_problem(71, [(16, 16), (20, 24), (24, 16)], 3, mask_kind="random", frac=0.3, iters=3,
                                 dtype="f64", lam=2e-3, mu=2e-2)
    px = [a.size for a in prob.x_true]
    mine = shard.partition(px, world)[rank]
    local_px = sum(px[j] for j in mine)
    L = dl = 0.0
    dh = np.zeros_like(prob.h)
    for j in mine:
        l, a, g, _ = oracle.admm_grad(prob.y[j], prob.mask[j], prob.h, prob.lam, prob.mu, 3, prob.x_true[j],
                                      round_f32=False)
        L += l * px[j] / local_px
        dl += a * px[j] / local_px
        dh += g * px[j] / local_px
    Lc, dlc, dhc = shard.combine_grad(L, dl, torch.tensor(dh), local_px, sum(px))
    if rank == 0:
        out.put((Lc, dlc, dhc.numpy()))
    dist.barrier()
    dist.destroy_process_group()


def test_sharded_gradient_equals_full_batch():
    import oracle
    from paper_1602_01410_gb300 import inputs
    prob = inputs.random_problem(71, [(16, 16), (20, 24), (24, 16)], 3, mask_kind="random", frac=0.3, iters=3,
                                 dtype="f64", lam=2e-3, mu=2e-2)
    px = [a.size for a in prob.x_true]
    L = dl = 0.0
    dh = np.zeros_like(prob.h)
    for j in range(3):
        l, a, g, _ = oracle.admm_grad(prob.y[j], prob.mask[j], prob.h, prob.lam, prob.mu, 3, prob.x_true[j],
                                      round_f32=False)
        w = px[j] / sum(px)
        L, dl, dh = L + w * l, dl + w * a, dh + w * g
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    Lc, dlc, dhc = q.get(timeout=120)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert abs(Lc - L) < 1e-14 and abs(dlc - dl) < 1e-12 * abs(dl)
    assert np.max(np.abs(dhc - dh)) < 1e-12 * np.max(np.abs(dh))


def _gather_worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    pixels = [3 * 16 * 16, 20 * 24, 64 * 64, 8 * 8, 3 * 32 * 48]
    full = torch.arange(sum(pixels), dtype=torch.float64)
    begin = np.concatenate([[0], np.cumsum(pixels)])
    mine = shard.partition(pixels, world)[rank]
    local = torch.cat([full[begin[j]:begin[j + 1]] for j in mine])
    got = shard.gather_batch(local, pixels)
    out.put((rank, bool(torch.equal(got, full))))
    dist.barrier()
    dist.destroy_process_group()


def test_gather_batch_reassembles_the_sharded_batch():
    assert shard.gather_batch(torch.ones(3), [3]).tolist() == [1.0, 1.0, 1.0]  # no process group
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_gather_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert res == {0: True, 1: True}
