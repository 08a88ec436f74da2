"""Writes the descriptor scaling constants (mu, s) of the synthetic models.

The paper uses trained n2p2 models whose input scaling is part of the model
files (Sec. 3.3); those are not available.  The stand-in models scale each
descriptor as G~ = (G - mu) / s with, per (element, descriptor),
mu = mean over the calibration atoms of that element and
s = max(std, 1e-3 |mu|, 1e-12), so that tanh layers are not saturated.

Calibration configurations: the 192-atom random water box (water model), and for
the FCC model nine 4,000-atom FCC boxes covering the variation a fitting set
holds: Gaussian displacements sigma in {0.05, 0.1, 0.2} A times lattice
constants {3.45, 3.52, 3.59} A (+-2 %).  (A single sigma = 0.05 A crystal varies
its radial descriptors by < 1 %, which gives |mu/s| ~ 150: a model whose FP32
evaluation error is dominated by the 1e-7 rounding of G amplified 150 times.)
Only the oracle is called.  Run from the repository root:
python -m oracle.calibrate_scaling
"""
from __future__ import annotations

import json
import os
import sys

import numpy as np

_ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if _ROOT not in sys.path:
    sys.path.insert(0, _ROOT)

import oracle  # noqa: E402
import workloads  # noqa: E402


def _stats(G, types, n_elem, n_sf):
    mu, s = [], []
    for e in range(n_elem):
        g = G[types == e, :n_sf[e]]
        m = g.mean(0)
        sd = g.std(0)
        mu.append(m.tolist())
        s.append(np.maximum.reduce([sd, 1e-3 * np.abs(m), np.full_like(m, 1e-12)]).tolist())
    return mu, s


def main():
    out_dir = os.path.join(_ROOT, "workloads", "data")
    os.makedirs(out_dir, exist_ok=True)
    fcc_set = [workloads.fcc((10, 10, 10), a=a, sigma=sg, seed=100 + k)
               for k, (sg, a) in enumerate((sg, a) for sg in (0.05, 0.1, 0.2) for a in (3.45, 3.52, 3.59))]
    jobs = [
        ("water", workloads.water_model, [workloads.water_random()]),
        ("water_resolved", lambda: workloads.water_model(resolved=True), [workloads.water_random()]),
        ("fcc", workloads.fcc_model, fcc_set),
    ]
    for name, mk, configs in jobs:
        model = mk()
        model["sf_mu"] = [np.zeros(len(r)) for r in model["sf"]]
        model["sf_s"] = [np.ones(len(r)) for r in model["sf"]]
        Gs, Ts = [], []
        for pos, types, box in configs:
            Gs.append(oracle.compute(model, pos, types, box)["G"])
            Ts.append(types)
        mu, s = _stats(np.concatenate(Gs), np.concatenate(Ts), len(model["sf"]), [len(r) for r in model["sf"]])
        path = os.path.join(out_dir, "sf_scaling_%s.json" % name)
        with open(path, "w") as f:
            json.dump({"written_by": "oracle/calibrate_scaling.py", "model": name, "mu": mu, "s": s}, f, indent=1)
        print("wrote", path)


if __name__ == "__main__":
    main()
