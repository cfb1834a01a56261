"""Multi-GPU sharding of the contraction (one process per GPU).

The slices of a sliced contraction path (Sec. 3.1) are independent
sub-networks whose results add up to the amplitude, and so are bitstring
batches and trajectories.  Two ways to use several GPUs:

  * bitstring sharding: every rank contracts its own batches; no collective
    on the data path (the benchmark's weak-scaling mode);
  * slice sharding: every rank contracts one contiguous block of the slices
    of the same batch (tnq_amplitudes_slices) and one FP64 all-reduce adds
    the partial amplitudes.

The helpers below hold the partition and the reduction; the contraction
itself is libtnq's.
"""
from __future__ import annotations

import numpy as np


def block_range(rank: int, world: int, n: int):
    """Contiguous block [begin, begin + count) of n units for `rank` (sizes differ by at most 1)."""
    if not (0 <= rank < world):
        raise ValueError("rank outside [0, world)")
    q, r = divmod(n, world)
    begin = rank * q + min(rank, r)
    return begin, q + (1 if rank < r else 0)


def allreduce_partials(partial: np.ndarray, group=None) -> np.ndarray:
    """Sum FP64 partial results over the ranks of `group` (torch.distributed)."""
    import torch
    import torch.distributed as dist
    t = torch.from_numpy(np.ascontiguousarray(partial, dtype=np.float64))
    backend = dist.get_backend(group)
    if backend == "nccl":
        t = t.cuda()
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t.cpu().numpy()


def amplitudes_slice_sharded(ctx, plan, bits, group=None) -> np.ndarray:
    """Complex amplitudes of `bits`, each rank contracting its block of slices."""
    import torch.distributed as dist
    from . import tnq
    rank, world = dist.get_rank(group), dist.get_world_size(group)
    n_slices = 2 ** plan.info["n_sliced"]
    begin, count = block_range(rank, world, n_slices)
    b = np.ascontiguousarray(bits, dtype=np.int8)
    out = np.zeros((b.shape[0], 2), dtype=np.float64)
    if count > 0:
        tnq.tnq_amplitudes_slices(ctx.h, plan.h, b, begin, count, out)
    total = allreduce_partials(out, group)
    return total[:, 0] + 1j * total[:, 1]
