"""velocity-Verlet NVE on the GPU against the oracle's trajectory (Sec. 4.2)."""
import numpy as np
import pytest
import torch

import oracle
import workloads
from tests.gpuhelp import f32, to_dev

pytestmark = pytest.mark.gpu


def test_nve_10_steps_matches_oracle():
    from paper_2002_00054_b300 import NNP
    m = workloads.water_model()
    pos, types, box = workloads.water_random()
    pos, box = f32(pos), f32(box)
    vel = f32(workloads.maxwell_boltzmann(types, m["masses"]))
    p_ref, v_ref, log_ref = oracle.md(m, pos, vel, types, box, 0.5, 10)
    nnp = NNP(m)
    p, t = to_dev(pos, types)
    v = torch.tensor(vel, dtype=torch.float32, device="cuda")
    log = nnp.step(p, v, t, box, 0.5, 10).cpu().numpy()
    assert np.abs(p.double().cpu().numpy() - p_ref).max() < 1e-4
    assert np.abs(v.double().cpu().numpy() - v_ref).max() < 1e-4
    np.testing.assert_allclose(log[:, 0], log_ref[:, 0], rtol=0, atol=1e-5 * np.abs(log_ref[:, 0]).max() + 1e-4)
    np.testing.assert_allclose(log[:, 1], log_ref[:, 1], rtol=1e-4, atol=1e-4)


def test_nve_drift_small():
    """Conserved energy of the GPU trajectory: 200 steps of 0.25 fs."""
    from paper_2002_00054_b300 import NNP
    m = workloads.water_model()
    pos, types, box = workloads.water_lattice((2, 2, 2), seed=9)
    vel = workloads.maxwell_boltzmann(types, m["masses"], seed=3)
    nnp = NNP(m)
    p, t = to_dev(f32(pos), types)
    v = torch.tensor(vel, dtype=torch.float32, device="cuda")
    log = nnp.step(p, v, t, f32(box), 0.25, 200).cpu().numpy()
    etot = log.sum(1)
    assert np.abs(etot - etot[0]).max() / len(pos) < 2e-4
    assert nnp.stats()["rebuilds"] >= 1
