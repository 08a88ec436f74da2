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


def test_step_continuation_is_bitwise_identical():
    """step(4) then step(6) on the same buffers equals step(10): the second call
    reuses the first call's final forces instead of recomputing them."""
    from paper_2002_00054_b300 import NNP
    m = workloads.water_model()
    pos, types, box = workloads.water_random()
    vel = workloads.maxwell_boltzmann(types, m["masses"])
    nnp = NNP(m)
    p1, t = to_dev(f32(pos), types)
    v1 = torch.tensor(vel, dtype=torch.float32, device="cuda")
    p2, v2 = p1.clone(), v1.clone()
    la = nnp.step(p1, v1, t, f32(box), 0.5, 4)
    n_first = nnp.stats()["kernel_launches"]
    lb = nnp.step(p1, v1, t, f32(box), 0.5, 6)
    assert nnp.stats()["kernel_launches"] < n_first * 6 / 4 + 2   # no extra force evaluation
    ref = NNP(m)
    lc = ref.step(p2, v2, t, f32(box), 0.5, 10)
    assert torch.equal(p1, p2) and torch.equal(v1, v2)
    assert torch.equal(torch.cat([la, lb[1:]]), lc)
    # a modified position forces a fresh evaluation (not the cached forces); the
    # fresh handle builds its list in another slot order, so compare to rounding
    p1[0, 0] += 0.01
    nnp.step(p1, v1, t, f32(box), 0.5, 1)
    p2[0, 0] += 0.01
    ref2 = NNP(m)
    ref2.step(p2, v2, t, f32(box), 0.5, 1)
    assert torch.allclose(p1, p2, rtol=0, atol=1e-6) and torch.allclose(v1, v2, rtol=0, atol=1e-6)


def test_kernel_group_timing():
    from paper_2002_00054_b300 import NNP
    m = workloads.water_model()
    pos, types, box = workloads.water_lattice((2, 2, 2))
    nnp = NNP(m)
    p, t = to_dev(f32(pos), types)
    v = torch.zeros_like(p)
    nnp.profile(True)
    nnp.step(p, v, t, f32(box), 0.5, 3)
    kt = nnp.kernel_times()
    assert kt["force"][1] == 4 and kt["descriptors"][1] == 4 and kt["force"][0] > 0
    assert kt["integrate"][1] == 1 + 3 * 2
