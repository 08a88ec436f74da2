"""Data-parallel force-matching training over the configurations of a batch.

Each rank evaluates a contiguous shard of the configurations (balanced by atom
count).  The loss terms of a shard are normalised by the whole batch (number of
configurations B, total atoms sum N), so the loss is the sum of the shard losses
and the full-batch parameter gradient is the sum of the shard gradients: one
all_reduce (sum) of the parameter gradient per step, the only exchange of a
training step.  Every rank then holds the same gradient and applies the same
update.

    lo, hi = shard_by_atoms(n_atoms, rank, world)
    ... E, F of configurations lo..hi-1 ...
    loss = shard_loss(E, F, E_ref, F_ref, n_atoms[lo:hi], n_configs_total, n_atoms_total)
    loss.backward()
    allreduce_grad(weights.grad)
"""
from __future__ import annotations

import numpy as np


def shard_by_atoms(n_atoms, rank, world):
    """[lo, hi): the contiguous range of configurations of rank `rank` among
    `world` ranks, cut where the running atom count crosses k/world of the total
    (every configuration lands in exactly one shard; a shard may be empty when
    there are fewer configurations than ranks)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank must be in [0, world)")
    c = np.concatenate([[0], np.cumsum(np.asarray(n_atoms, np.int64))])
    total = c[-1]
    cuts = [0] + [int(np.searchsorted(c[1:], total * k / world, side="left")) + 1 for k in range(1, world)] \
        + [len(c) - 1]
    cuts = np.maximum.accumulate(np.minimum(cuts, len(c) - 1))
    return int(cuts[rank]), int(cuts[rank + 1])


def shard_loss(E, F, E_ref, F_ref, n_atoms, n_configs_total, n_atoms_total, w_force=10.0):
    """The shard's part of (1/B) sum_b ((E_b - E_ref_b)/N_b)^2 +
    w_force/(3 sum N) sum (F - F_ref)^2, with B and sum N of the whole batch."""
    le = (((E - E_ref) / n_atoms) ** 2).sum() / float(n_configs_total)
    lf = ((F.double() - F_ref.double()) ** 2).sum() / (3.0 * float(n_atoms_total))
    return le + w_force * lf


def allreduce_grad(grad):
    """Sum of the ranks' gradients, in place (no-op without an initialised
    process group of more than one rank)."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(grad, op=dist.ReduceOp.SUM)
    return grad
