"""Algorithmic operation counts of the hot path, per unit of work.

The counts are those of the method's formulas (not of any particular kernel):
an FMA counts 2 flops, an add or multiply 1, and each transcendental or
reciprocal/square root counts one special-function op (MUFU) and no flops.
Units are read from the library's work counters:

  list entries   neighbour-list entries within cutoff + skin (displacement + r^2: 8 flops)
  neighbours     entries within the cutoff
  pairs          neighbour pairs j < k examined by the angular loop
  triplets       pairs that contribute (narrow: r_jk < r_c; wide: all pairs)

Descriptor pass (Fig. 1b step 1, angular loop of Sec. 3.1):
  per neighbour: sqrt (1 MUFU); cutoff: argument FMA 2 + sin, cos (2 MUFU) + square 1;
                 per angular eta: exp argument FMA 2 + exp (1 MUFU) + times f_c 1
  per (neighbour, matching radial function): r - r_s 1, square 1, argument FMA 2,
                 exp (1 MUFU), times f_c 1, accumulate 1 = 6 flops
  per examined pair (narrow only): r_jk vector 3 + r_jk^2 5 = 8 flops
  per triplet: dot 5, cos = dot / (r_j r_k) 2 + 1 MUFU, bases 1 +- cos 2,
               squarings to the largest zeta per lambda (1 flop each);
               narrow: sqrt (1 MUFU), cutoff 3 flops + 2 MUFU, per eta exp 3 flops
               + 1 MUFU and the product R = P_j P_k P_jk f 3; wide: per eta R = P_j P_k 1;
               per descriptor term one FMA (2)
Force pass (Fig. 1b step 3, recompute of dG/dr):
  per neighbour: as the descriptor pass + f_c' 2 + per angular eta P' 4;
                 per matching radial function: value 6 + derivative 4 + accumulate 2
                 = 12 flops, 1 MUFU; per neighbour g = (sum) d / r: 1 MUFU + 3
  per examined pair (narrow only): 8 flops
  per triplet: dot 5, cos 2 + 1 MUFU, bases 2, per squaring level 2 (value and
               derivative powers), per descriptor term 2 FMA (4 flops); narrow: sqrt,
               cutoff 3 flops + 2 MUFU, 1/r_jk 1 MUFU, per eta 3 + 1 MUFU (exp) + 5 (P_jk, P'_jk);
               per eta the three or four products into dPhi/dc, dPhi/dr_j, dPhi/dr_k,
               dPhi/dr_jk: 11 (wide) / 14 (narrow); coefficients 10, the two
               gradient vectors 30, accumulation 6
Network (Fig. 1b step 2): forward 2 (n_in n_out + n_out) per layer plus the
  activation; backward 2 n_in n_out per layer; per atom.
"""
from __future__ import annotations

import math


def _structure(model):
    sf = model["sf"][0]
    n_rad = sum(1 for d in sf if d["type"] == "radial")
    rad_elems = {d.get("e1", -1) for d in sf if d["type"] == "radial"}
    n_elem = len(model["sf"])
    rad_match = n_rad if rad_elems == {-1} else n_rad / max(1, n_elem)
    ang = [d for d in sf if d["type"] != "radial"]
    kind = ang[0]["type"] if ang else None
    etas = sorted({d["eta"] for d in ang})
    lev = {}
    for d in ang:
        lam = d["lambda"]
        lev[lam] = max(lev.get(lam, 0), int(round(math.log2(d["zeta"]))))
    return n_rad, rad_match, kind, len(etas), len(ang), sum(lev.values())


def descriptor_ops(model, list_entries, neighbours, pairs, triplets):
    """(flops, mufu) of the descriptor pass."""
    n_rad, rad_match, kind, n_eta, n_terms, levels = _structure(model)
    fl = 8 * list_entries
    mu = 0
    fl += neighbours * (3 + 4 * n_eta + 6 * rad_match)
    mu += neighbours * (3 + n_eta + rad_match)
    if kind == "narrow":
        fl += 8 * pairs
        fl += triplets * (5 + 2 + 2 + levels + 3 + n_eta * (3 + 3) + 2 * n_terms)
        mu += triplets * (1 + 1 + 2 + n_eta)
    elif kind == "wide":
        fl += triplets * (5 + 2 + 2 + levels + n_eta + 2 * n_terms)
        mu += triplets * 1
    return fl, mu


def force_ops(model, list_entries, neighbours, pairs, triplets):
    """(flops, mufu) of the force pass."""
    n_rad, rad_match, kind, n_eta, n_terms, levels = _structure(model)
    fl = 8 * list_entries
    mu = 0
    fl += neighbours * (3 + 2 + 8 * n_eta + 12 * rad_match + 3)
    mu += neighbours * (3 + n_eta + rad_match + 1)
    common = 5 + 2 + 2 + 2 * levels + 4 * n_terms + 10 + 30 + 6
    if kind == "narrow":
        fl += 8 * pairs
        fl += triplets * (common + 3 + n_eta * (3 + 5 + 14))
        mu += triplets * (1 + 1 + 2 + 1 + n_eta)
    elif kind == "wide":
        fl += triplets * (common + n_eta * 11)
        mu += triplets * 1
    return fl, mu


def network_ops(model, n_atoms):
    w = model["widths"]
    fl = 0
    for l in range(len(w) - 1):
        fl += 2 * (w[l] * w[l + 1] + w[l + 1]) + 2 * w[l] * w[l + 1]
    mu = sum(w[1:-1])
    return fl * n_atoms, mu * n_atoms
