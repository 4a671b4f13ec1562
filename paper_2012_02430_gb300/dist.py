"""Multi-GPU sharding of one amplitude's slices (one process per GPU).

Slices are independent contractions (Eq. 2); the paper gives every MPI rank its
own slices and ends with one reduce-sum of the slice results (Alg. 1). Here rank
r of W contracts a contiguous block of slice ids and the ranks exchange their
FP64 partial sums with an all-gather, which every rank adds in rank order, so
the total is the same on every rank and from run to run. With torch.distributed
the exchange runs over NCCL on GPUs (gloo in the CPU tests).
"""

from __future__ import annotations


def slice_range(nslices: int, rank: int, world: int):
    """Contiguous block of slice ids [lo, hi) of `rank`; blocks differ by at most one."""
    if world < 1 or not 0 <= rank < world or nslices < 0:
        raise ValueError("bad rank/world/nslices")
    base, extra = divmod(nslices, world)
    lo = rank * base + min(rank, extra)
    hi = lo + base + (1 if rank < extra else 0)
    return lo, hi


def sharded_sum(partial, nslices: int, rank: int, world: int, group=None, device="cpu"):
    """Sum over all slices of partial(lo, count) (a complex), computed on each rank's
    block and combined across ranks in rank order."""
    import torch
    import torch.distributed as dist
    lo, hi = slice_range(nslices, rank, world)
    mine = partial(lo, hi - lo) if hi > lo else 0j
    if world == 1:
        return complex(mine)
    t = torch.tensor([mine.real, mine.imag], dtype=torch.float64, device=device)
    parts = [torch.zeros(2, dtype=torch.float64, device=device) for _ in range(world)]
    dist.all_gather(parts, t, group=group)
    re = im = 0.0
    for p in parts:  # rank order
        re += float(p[0])
        im += float(p[1])
    return complex(re, im)


def gpu_partial(net, out):
    """partial(lo, count) for sharded_sum: the library's device-resident run of a block
    of slices of a prepared, uploaded Network (qtensor.Network); `out` is a float64
    CUDA tensor of 2 elements."""
    def f(lo, count):
        net.run(lo, count, out)
        return complex(out[0].item(), out[1].item())
    return f
