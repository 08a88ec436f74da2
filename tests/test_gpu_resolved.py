"""Angular descriptors resolved by neighbour-element pair (the water model with
14 narrow angular functions for each of the pairs (O,O), (O,H), (H,H); n_G = 58)
on the GPU against the oracle: descriptors, energies, forces, virial, the
parameter gradient (descriptor tangents by class) and the BF16 network."""
import numpy as np
import pytest
import torch

import oracle
import workloads
from tests.gpuhelp import check, f32, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def model():
    return workloads.water_model(resolved=True)


def test_resolved_descriptors(model):
    from paper_2002_00054_b300 import NNP
    nnp = NNP(model)
    pos, types, box = workloads.water_random()
    pos, box = f32(pos), f32(box)
    ref = oracle.compute(model, pos, types, box)
    p, t = to_dev(pos, types)
    G, dEdG = nnp.descriptors(p, t, box)
    G = G.double().cpu().numpy()
    gref = ref["G"][:, :58]
    gerr = np.abs(G - gref) / np.maximum(np.abs(gref).max(0), 1e-30)
    assert gerr.max() < 2e-6, gerr.max()
    dref = ref["dEdG"][:, :58]
    assert (np.abs(dEdG.double().cpu().numpy() - dref) / np.abs(dref).max()).max() < 2e-5


@pytest.mark.parametrize("case", ["random", "lattice"])
def test_resolved_energy_forces(model, case):
    from paper_2002_00054_b300 import NNP
    nnp = NNP(model)
    if case == "random":
        pos, types, box = workloads.water_random()
    else:
        pos, types, box = workloads.water_lattice((2, 2, 2), seed=11)   # cell-list path
    pos, box = f32(pos), f32(box)
    ref = oracle.compute(model, pos, types, box)
    p, t = to_dev(pos, types)
    out = nnp.compute(p, t, box)
    check(out, ref, what="resolved water %s" % case)


def test_resolved_param_grad(model):
    from paper_2002_00054_b300 import NNP
    nnp = NNP(model)
    pos, types, box = workloads.water_random(seed=31)
    pos, box = f32(pos), f32(box)
    rng = np.random.default_rng(8)
    u = f32(rng.normal(size=pos.shape) * 0.1)
    p, t = to_dev(pos, types)
    g = nnp.param_grad(p, t, [0, len(p)], box[None, :], torch.tensor([0.3], dtype=torch.float64, device="cuda"),
                       torch.tensor(u, dtype=torch.float32, device="cuda"))
    ref = oracle.param_grad(model, pos, types, box, 0.3, u)
    err = np.abs(g.double().cpu().numpy() - ref).max() / np.abs(ref).max()
    assert err <= 2e-4, err


def test_resolved_bf16_network(model):
    from paper_2002_00054_b300 import NNP
    pos, types, box = workloads.water_lattice((2, 2, 2), seed=12)
    pos, box = f32(pos), f32(box)
    ref = oracle.compute(model, pos, types, box)
    p, t = to_dev(pos, types)
    out = NNP(model, precision="bf16").compute(p, t, box)
    dF = out["F"].double().cpu().numpy() - ref["F"]
    assert np.sqrt(np.mean(dF ** 2)) <= 5e-3
