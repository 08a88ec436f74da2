"""Spatial domain decomposition of one periodic box into slabs along x.

Each domain owns the atoms of its slab and holds copies ("ghosts") of every atom
within 2 r_c of the slab (periodic images included), placed at unwrapped
positions in a local box that keeps the original y and z edges and is long
enough in x that no atom sees an image of another across the local x edge.
An owned atom's energy needs its neighbours within r_c; its force needs the
energies of those neighbours, hence their neighbours within 2 r_c: with a 2 r_c
halo both come out of one ordinary evaluation of the domain, with no reverse
exchange of ghost forces (the redundant-halo form of the paper's outlook on
multi-node runs, Sec. 5).  The total energy is the sum over domains of the
owned atoms' energies.

decompose() is host bookkeeping (numpy); evaluate_decomposed() runs the domains
one after another through a caller-supplied evaluation (on one GPU: NNP.compute),
and exchange_halo() does the same selection with torch.distributed, one domain
per rank, where each rank starts from its own atoms only; allreduce_energy()
sums the ranks' owned energies (FP64).
"""
from __future__ import annotations

import numpy as np


class Domain:
    """owned: global indices of the owned atoms; ghost: global indices of the
    ghost copies and shift: their image offsets (multiples of the x edge, added to
    x); x0: the local x origin; box: the local box."""

    def __init__(self, owned, owned_shift, ghost, shift, x0, box):
        self.owned = owned
        self.owned_shift = owned_shift
        self.ghost = ghost
        self.shift = shift
        self.x0 = x0
        self.box = box

    def local(self, pos, types):
        """Local positions (owned first, then ghosts) and types."""
        p = np.concatenate([pos[self.owned], pos[self.ghost]])
        p[:len(self.owned), 0] += self.owned_shift
        p[len(self.owned):, 0] += self.shift
        p[:, 0] -= self.x0
        return p, np.concatenate([types[self.owned], types[self.ghost]])


def local_box(box, width, halo, rcut):
    """x edge of a domain's local box: the slab plus both halos plus one r_cut, so
    no pair closer than r_cut can wrap across it."""
    return np.array([width + 2.0 * halo + rcut, box[1], box[2]], np.float64)


def decompose(pos, box, n_dom, cutoff, skin=1.0):
    """Slabs [k L/n, (k+1) L/n) along x with a 2 r_c halo each."""
    pos = np.asarray(pos, np.float64)
    box = np.asarray(box, np.float64)
    L = box[0]
    width = L / n_dom
    halo = 2.0 * cutoff
    if width < halo:
        raise ValueError("slab width %.3g is below the 2 r_c halo %.3g: use fewer domains" % (width, halo))
    x = np.mod(pos[:, 0], L)
    slab = np.minimum((x // width).astype(np.int64), n_dom - 1)
    doms = []
    lbox = local_box(box, width, halo, cutoff + skin)
    for k in range(n_dom):
        lo, hi = k * width, (k + 1) * width
        owned = np.nonzero(slab == k)[0]
        g_idx, g_shift = [], []
        for img in (-1.0, 0.0, 1.0):
            xs = x + img * L
            sel = (slab != k) | (img != 0.0)
            near = sel & (xs >= lo - halo) & (xs < hi + halo)
            idx = np.nonzero(near)[0]
            g_idx.append(idx)
            g_shift.append(x[idx] - pos[idx, 0] + img * L)
        ghost = np.concatenate(g_idx)
        shift = np.concatenate(g_shift)
        # owned atoms are placed at their wrapped x as well
        doms.append(Domain(owned, x[owned] - pos[owned, 0], ghost, shift, lo - halo, lbox))
    return doms


def evaluate_decomposed(evaluate, pos, types, box, n_dom, cutoff, skin=1.0):
    """Energy and forces of the whole box from n_dom slab domains evaluated one
    after another: evaluate(local_pos, local_types, local_box) -> (Ei, F) as
    numpy arrays for all local atoms.  Returns (energy, Ei, F) in global order."""
    pos = np.asarray(pos, np.float64)
    types = np.asarray(types)
    n = len(pos)
    Ei = np.zeros(n)
    F = np.zeros((n, 3))
    for d in decompose(pos, box, n_dom, cutoff, skin):
        p, t = d.local(pos, types)
        e, f = evaluate(p, t, d.box)
        no = len(d.owned)
        Ei[d.owned] = e[:no]
        F[d.owned] = f[:no]
    return float(np.sum(Ei)), Ei, F


def exchange_halo(pos_own, types_own, gid_own, box, cutoff, rank, world, skin=1.0):
    """Halo exchange for slab domains, one per rank, with torch.distributed: rank
    k owns the atoms of slab k (pos_own, types_own, global ids gid_own); every rank
    gathers the atoms of all ranks (a gather of the boundary layers would suffice;
    all_gather keeps this exchange simple and exact) and selects its 2 r_c halo.
    Returns the local positions, types and global ids (owned atoms first), the
    number of owned atoms and the local box."""
    import torch
    import torch.distributed as dist
    payload = np.concatenate([np.asarray(pos_own, np.float64), np.asarray(types_own, np.float64)[:, None],
                              np.asarray(gid_own, np.float64)[:, None]], axis=1)
    sizes = [None] * world
    dist.all_gather_object(sizes, len(payload))
    mx = max(sizes)
    buf = torch.zeros((mx, 5), dtype=torch.float64)
    buf[:len(payload)] = torch.from_numpy(payload)
    parts = [torch.zeros_like(buf) for _ in range(world)]
    dist.all_gather(parts, buf)
    allp = np.concatenate([parts[r][:sizes[r]].numpy() for r in range(world)])
    pos_all, types_all, gid_all = allp[:, :3], allp[:, 3].astype(np.int32), allp[:, 4].astype(np.int64)
    d = decompose(pos_all, box, world, cutoff, skin)[rank]
    p, t = d.local(pos_all, types_all)
    gid = np.concatenate([gid_all[d.owned], gid_all[d.ghost]])
    return p, t, gid, len(d.owned), d.box


def allreduce_energy(e_owned):
    """Total energy of the box from the ranks' owned-atom energy sums: an FP64
    all_reduce (sum) over the process group (the input on one rank)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(e_owned)], dtype=torch.float64)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t[0])

