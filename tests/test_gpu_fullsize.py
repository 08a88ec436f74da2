"""The benchmark workloads at full size, in the launch configuration bench.py
times: outputs on sampled atoms (random ones and atoms next to the box faces,
whose pairs cross the periodic boundary) against the oracle, which evaluates
exactly those atoms and their neighbours."""
import numpy as np
import pytest
import torch

import oracle
import workloads
from tests.gpuhelp import F_ABS, E_REL, f32

pytestmark = pytest.mark.gpu


def _sample(pos, box, n_random=24, seed=0):
    rng = np.random.default_rng(seed)
    idx = set(rng.choice(len(pos), n_random, replace=False).tolist())
    for a in range(3):   # atoms within 1 A of each face
        for near in (pos[:, a] < 1.0, pos[:, a] > box[a] - 1.0):
            cand = np.nonzero(near)[0]
            idx.update(rng.choice(cand, 2, replace=False).tolist())
    return np.array(sorted(idx))


def _check_sampled(out, ref, idx, f_abs=F_ABS):
    Ei = out["Ei"].double().cpu().numpy()[idx]
    F = out["F"].double().cpu().numpy()[idx]
    # the scale floor is the sampled atoms' rms energy (the full box's is not known here)
    scale = np.maximum(np.abs(ref["Ei"]), np.sqrt(np.mean(ref["Ei"] ** 2)))
    tol = E_REL * scale
    assert np.all(np.abs(Ei - ref["Ei"]) <= tol), np.max(np.abs(Ei - ref["Ei"]) / tol)
    assert np.abs(F - ref["F"]).max() <= f_abs, np.abs(F - ref["F"]).max()


@pytest.mark.parametrize("name", ["water_2m", "fcc_1m"])
def test_full_size_sampled_parity(name):
    from paper_2002_00054_b300 import NNP
    if name == "water_2m":
        pos, types, box = workloads.water_lattice((16, 24, 28))
        m, max_nb = workloads.water_model(), 200
    else:
        pos, types, box = workloads.fcc((64, 64, 64))
        m, max_nb = workloads.fcc_model(), 160
    pos, box = f32(pos), f32(box)
    nnp = NNP(m, max_neighbors=max_nb)
    p = torch.tensor(pos, dtype=torch.float32, device="cuda")
    t = torch.tensor(types, dtype=torch.int32, device="cuda")
    out = nnp.compute(p, t, box)
    idx = _sample(pos, box)
    ref = oracle.compute_subset(m, pos, types, box, idx)
    _check_sampled(out, ref, idx)
    # the BF16 network on the same sampled atoms: force RMS error <= 5e-3 eV/A
    bf = NNP(m, max_neighbors=max_nb, precision="bf16").compute(p, t, box)
    dF = bf["F"].double().cpu().numpy()[idx] - ref["F"]
    assert np.sqrt(np.mean(dF ** 2)) <= 5e-3
