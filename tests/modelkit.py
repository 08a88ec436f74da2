"""Small hand-made model descriptions for the tests (identity scaling, random weights)."""
import numpy as np

import workloads


def model_from_rows(rows_per_elem, cutoff, hidden=(4,), seed=0, masses=None):
    n_elem = len(rows_per_elem)
    n_g = len(rows_per_elem[0])
    widths = [n_g, *hidden, 1]
    return {
        "name": "test",
        "elements": ["X%d" % e for e in range(n_elem)],
        "masses": list(masses) if masses is not None else [1.0] * n_elem,
        "cutoff": float(cutoff),
        "sf": rows_per_elem,
        "sf_mu": [np.zeros(len(r)) for r in rows_per_elem],
        "sf_s": [np.ones(len(r)) for r in rows_per_elem],
        "widths": widths,
        "weights": workloads.random_weights(widths, n_elem, seed),
    }


def radial(eta, rs=0.0, e1=-1):
    return {"type": "radial", "e1": e1, "e2": -1, "eta": float(eta), "rs": float(rs)}


def angular(kind, eta, zeta, lam, e1=-1, e2=-1):
    return {"type": kind, "e1": e1, "e2": e2, "eta": float(eta), "zeta": float(zeta), "lambda": float(lam)}
