"""Multi-GPU work split for batches of independent images.

Images of a batch are independent problems, so a batch shards across ranks
by image with no exchange during the iterations: `partition` assigns images
greedily, longest first, to the least-loaded rank (load = pixels, so the
per-iteration time, which is proportional to the pixel count, balances).
A single image does not shard (a distributed 2-D DFT would need two
all-to-all transposes per iteration); those workloads run as replicas.

For the differentiation workload each rank returns the loss and gradients
of the mean over ITS pixels; `combine_grad` re-weights them by the pixel
share and sums them across ranks (one all-reduce of 2 + K*K numbers).
After a sharded solve `gather_batch` reassembles the whole batch of x on
every rank (one all-gather, outside the iterations).
"""
from __future__ import annotations

from typing import List, Sequence, Tuple


def partition(pixels: Sequence[int], world: int) -> List[List[int]]:
    """Image indices per rank; every image on exactly one rank."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(pixels)), key=lambda j: (-pixels[j], j))
    loads = [0] * world
    parts: List[List[int]] = [[] for _ in range(world)]
    for j in order:
        r = min(range(world), key=lambda k: (loads[k], k))
        parts[r].append(j)
        loads[r] += pixels[j]
    return [sorted(p) for p in parts]


def combine_grad(loss: float, dlam: float, dh, local_px: int, total_px: int, group=None) -> Tuple[float, float, object]:
    """All-reduce the pixel-weighted loss and gradients of every rank (torch
    tensors on the rank's device; dh is a tensor shaped like h)."""
    import torch
    import torch.distributed as dist
    w = float(local_px) / float(total_px)
    buf = torch.cat([torch.tensor([loss * w, dlam * w], dtype=dh.dtype, device=dh.device), dh.reshape(-1) * w])
    if dist.is_available() and dist.is_initialized():
        dist.all_reduce(buf, op=dist.ReduceOp.SUM, group=group)
    return float(buf[0]), float(buf[1]), buf[2:].reshape(dh.shape)


def gather_batch(x_local, pixels: Sequence[int], group=None):
    """Reassemble a sharded batch on every rank.

    x_local: the rank's images (those `partition(pixels, world)` gave it, in
    increasing index order) concatenated in the batch layout, a 1-D torch
    tensor; pixels[j]: elements of image j (channels x rows x cols).  Returns
    the whole batch in the original image order, on x_local's device.  One
    all-gather of equal-length (zero-padded) buffers; with no process group
    initialised it returns x_local unchanged (one rank holds everything)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return x_local
    world = dist.get_world_size(group)
    parts = partition(pixels, world)
    longest = max(sum(pixels[j] for j in p) for p in parts)
    buf = torch.zeros(longest, dtype=x_local.dtype, device=x_local.device)
    buf[:x_local.numel()] = x_local.reshape(-1)
    bufs = [torch.empty_like(buf) for _ in range(world)]
    dist.all_gather(bufs, buf, group=group)
    begin = [0]
    for n in pixels:
        begin.append(begin[-1] + n)
    out = torch.empty(begin[-1], dtype=x_local.dtype, device=x_local.device)
    for r, p in enumerate(parts):
        o = 0
        for j in p:
            out[begin[j]:begin[j + 1]] = bufs[r][o:o + pixels[j]]
            o += pixels[j]
    return out
