"""Spatial domain decomposition of one periodic box into slabs along x (the
paper's outlook on multi-node runs, Sec. 5).

Each domain owns the atoms of its slab [k W, (k+1) W), W = L / n, and holds
copies ("ghosts") of every atom within 2 r_c of the slab (periodic images
included), placed at unwrapped positions in a local box that keeps the original
y and z edges and is long enough in x that no atom sees an image of another
across the local x edge.  An owned atom's energy needs its neighbours within
r_c; its force needs the energies of those neighbours, hence their neighbours
within 2 r_c: with a 2 r_c halo both come out of one ordinary evaluation of the
domain, with no reverse exchange of ghost forces.  The box's energy is the sum
over domains of the owned atoms' energies, and its virial the sum over domains
of the pair virial of the owned atoms' energies (nnp_compute_domain).

Since W >= 2 r_c, a slab's halo lies inside its two neighbouring slabs: the
exchange is point to point, each rank sending the 2 r_c layer at each of its
slab's faces to the neighbour on that side (exchange_halo), then one FP64
all_reduce of the energy and the virial (allreduce_energy_virial).  decompose()
does the same selection on one host from all positions (the one-process
emulation of evaluate_decomposed(), which runs the domains one after another).
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


def _check_width(L, n_dom, cutoff):
    width = L / n_dom
    halo = 2.0 * cutoff
    if width < halo:
        raise ValueError("slab width %.3g is below the 2 r_c halo %.3g: use fewer domains" % (width, halo))
    return width, halo


def decompose(pos, box, n_dom, cutoff, skin=1.0):
    """Slabs [k L/n, (k+1) L/n) along x with a 2 r_c halo each (from all positions)."""
    pos = np.asarray(pos, np.float64)
    box = np.asarray(box, np.float64)
    L = box[0]
    width, halo = _check_width(L, n_dom, cutoff)
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
    """Energy, forces and virial of the whole box from n_dom slab domains
    evaluated one after another: evaluate(local_pos, local_types, local_box,
    n_owned) -> (Ei, F, W) with Ei, F for all local atoms and W the virial of the
    owned atoms' energies (numpy).  Returns (energy, Ei, F, W) in global order."""
    pos = np.asarray(pos, np.float64)
    types = np.asarray(types)
    n = len(pos)
    Ei = np.zeros(n)
    F = np.zeros((n, 3))
    W = np.zeros((3, 3))
    for d in decompose(pos, box, n_dom, cutoff, skin):
        p, t = d.local(pos, types)
        no = len(d.owned)
        e, f, w = evaluate(p, t, d.box, no)
        Ei[d.owned] = e[:no]
        F[d.owned] = f[:no]
        W += np.asarray(w).reshape(3, 3)
    return float(np.sum(Ei)), Ei, F, W


def boundary_layers(pos_own, box, cutoff, rank, world):
    """The owned atoms (wrapped x) in the 2 r_c layers at the slab's two faces:
    (indices of the left layer, indices of the right layer)."""
    L = float(box[0])
    width, halo = _check_width(L, world, cutoff)
    x = np.mod(np.asarray(pos_own, np.float64)[:, 0], L)
    lo, hi = rank * width, (rank + 1) * width
    left = np.nonzero(x < lo + halo)[0]
    right = np.nonzero(x >= hi - halo)[0]
    return left, right


def exchange_halo(pos_own, types_own, gid_own, box, cutoff, rank, world, skin=1.0, device="cpu"):
    """Point-to-point halo exchange for slab domains, one per rank, over
    torch.distributed (gloo on CPU tensors; NCCL with device tensors).  Rank k
    owns the atoms of slab k (pos_own, types_own, global ids gid_own; any x
    image).  It sends its left 2 r_c layer to rank k - 1 and its right layer to
    rank k + 1 (periodic), and receives the matching layers from them; the
    received atoms, shifted by the box edge across the periodic seam, are its
    ghosts.  Two messages per direction (size, then payload), nothing else.
    Returns the local positions, types and global ids (owned atoms first), the
    number of owned atoms, the local box and the bytes sent."""
    import torch
    import torch.distributed as dist
    box = np.asarray(box, np.float64)
    L = float(box[0])
    width, halo = _check_width(L, world, cutoff)
    pos_own = np.asarray(pos_own, np.float64).copy()
    pos_own[:, 0] = np.mod(pos_own[:, 0], L)
    left, right = boundary_layers(pos_own, box, cutoff, rank, world)
    rows = np.concatenate([pos_own, np.asarray(types_own, np.float64)[:, None],
                           np.asarray(gid_own, np.float64)[:, None]], axis=1)
    to_left = torch.from_numpy(np.ascontiguousarray(rows[left])).to(device)
    to_right = torch.from_numpy(np.ascontiguousarray(rows[right])).to(device)
    lnb, rnb = (rank - 1) % world, (rank + 1) % world
    # tags: 0 = a left layer (travels to the left neighbour), 1 = a right layer
    n_out = [torch.tensor([len(left)], dtype=torch.int64, device=device),
             torch.tensor([len(right)], dtype=torch.int64, device=device)]
    n_in = [torch.zeros(1, dtype=torch.int64, device=device), torch.zeros(1, dtype=torch.int64, device=device)]
    reqs = [dist.isend(n_out[0], lnb, tag=0), dist.isend(n_out[1], rnb, tag=1),
            dist.irecv(n_in[0], rnb, tag=0), dist.irecv(n_in[1], lnb, tag=1)]
    for r in reqs:
        r.wait()
    from_right = torch.zeros((int(n_in[0].item()), 5), dtype=torch.float64, device=device)
    from_left = torch.zeros((int(n_in[1].item()), 5), dtype=torch.float64, device=device)
    reqs = []
    if len(left):
        reqs.append(dist.isend(to_left, lnb, tag=2))
    if len(right):
        reqs.append(dist.isend(to_right, rnb, tag=3))
    if len(from_right):
        reqs.append(dist.irecv(from_right, rnb, tag=2))
    if len(from_left):
        reqs.append(dist.irecv(from_left, lnb, tag=3))
    for r in reqs:
        r.wait()
    fr = from_right.cpu().numpy()
    fl = from_left.cpu().numpy()
    # the right neighbour's left layer sits above this slab; across the seam
    # (this is the last slab) it is an image at +L; likewise the left layer at -L
    if rank == world - 1:
        fr[:, 0] += L
    if rank == 0:
        fl[:, 0] -= L
    ghosts = np.concatenate([fr, fl])
    x0 = rank * width - halo
    loc = np.concatenate([rows, ghosts])
    p = loc[:, :3].copy()
    p[:, 0] -= x0
    t = loc[:, 3].astype(np.int32)
    gid = loc[:, 4].astype(np.int64)
    sent = (len(left) + len(right)) * 5 * 8 + 2 * 8
    return p, t, gid, len(rows), local_box(box, width, halo, cutoff + skin), sent


def allreduce_energy_virial(e_owned, w_owned):
    """The box's energy and virial from the ranks' owned-atom sums: one FP64
    all_reduce (sum) of ten numbers over the process group."""
    import torch
    import torch.distributed as dist
    t = torch.tensor(np.r_[float(e_owned), np.asarray(w_owned, np.float64).reshape(9)], dtype=torch.float64)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
    v = t.numpy()
    return float(v[0]), v[1:].reshape(3, 3)
