"""Descriptor sets outside the two specialised instantiations (water: narrow,
2 eta; FCC: wide, 3 eta) run the generic kernel instantiations: narrow with 1,
3 or 4 eta (4: the angular sums packed over two eta pairs; 3: stored queues
without staged neighbours), wide with 2 eta, and radial functions only.
Energies, forces and virial against the FP64 oracle on the 192-atom water-like
box, with the same tolerances as the other parity tests."""
import numpy as np
import pytest

import oracle
import workloads
from tests.gpuhelp import check, f32, to_dev
from tests.modelkit import angular, model_from_rows, radial

pytestmark = pytest.mark.gpu

RC = 6.0


def _rows(kind, etas):
    rows = [radial(eta) for eta in (0.002, 0.02, 0.1, 0.3)]
    rows += [radial(0.05, rs=1.0, e1=0), radial(0.05, rs=1.0, e1=1)]
    for eta in etas:
        for z in (1.0, 2.0, 4.0, 16.0):
            rows.append(angular(kind, eta, z, 1.0))
        for z in (1.0, 4.0):
            rows.append(angular(kind, eta, z, -1.0))
    return rows


@pytest.mark.parametrize("kind,etas", [
    ("narrow", (0.004,)),
    ("narrow", (0.001, 0.01, 0.03)),
    ("narrow", (0.001, 0.004, 0.01, 0.03)),
    ("wide", (0.002, 0.02)),
    ("radial", ()),
])
def test_generic_term_sets(kind, etas):
    from paper_2002_00054_b300 import NNP
    rows = _rows(kind, etas)
    model = model_from_rows([rows, rows], RC, hidden=(8, 6), seed=11, masses=[15.999, 1.008])
    pos, types, box = workloads.water_random(seed=21)
    pos, box = f32(pos), f32(box)
    ref = oracle.compute(model, pos, types, box)
    nnp = NNP(model)
    p, t = to_dev(pos, types)
    for _ in range(2):   # the second call runs with the capacity re-tuned from the first
        out = nnp.compute(p, t, box)
        check(out, ref, what="%s, %d eta" % (kind, len(etas)))
    assert np.isfinite(out["energy"].item())
