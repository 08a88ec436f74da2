"""Differentiation form: batched energies/forces and the force-matching parameter
gradient (energy term and double backward) against the FP64 oracle's analytic
gradient, which tests/test_oracle_pins.py pins to finite differences of the loss.
Inputs and weights are float32-representable and identical on both sides."""
import numpy as np
import pytest
import torch

import oracle
import workloads
from tests.gpuhelp import check, f32

pytestmark = pytest.mark.gpu


def _model():
    m = workloads.water_model()
    m["weights"] = [f32(w) for w in m["weights"]]
    return m


def _batch(n_mols=(8, 22, 37, 64), seed=0):
    systems = []
    for k, nm in enumerate(n_mols):
        L = (3 * nm / workloads.WATER_DENSITY_ATOMS) ** (1 / 3)
        p, t, b = workloads.water_random(nm, L, seed=300 + 7 * k + seed)
        systems.append((f32(p), t, f32(b)))
    starts = np.cumsum([0] + [len(p) for p, _, _ in systems]).astype(np.int32)
    pos = np.concatenate([p for p, _, _ in systems])
    types = np.concatenate([t for _, t, _ in systems]).astype(np.int32)
    boxes = np.stack([b for _, _, b in systems])
    return systems, starts, pos, types, boxes


def _dev(pos, types):
    return (torch.tensor(pos, dtype=torch.float32, device="cuda"), torch.tensor(types, dtype=torch.int32, device="cuda"))


def test_compute_batch_matches_oracle():
    from paper_2002_00054_b300 import NNP
    m = _model()
    systems, starts, pos, types, boxes = _batch()
    nnp = NNP(m)
    p, t = _dev(pos, types)
    out = nnp.compute_batch(p, t, starts, boxes, atom_energy=True)
    for b, (pb, tb, bb) in enumerate(systems):
        ref = oracle.compute(m, pb, tb, bb)
        sl = slice(starts[b], starts[b + 1])
        sub = {"Ei": out["Ei"][sl], "F": out["F"][sl], "energy": out["energy"][b:b + 1]}
        check(sub, ref, what="system %d" % b)


def _oracle_grad(m, systems, dLdE, u):
    g = 0.0
    for b, (pb, tb, bb) in enumerate(systems):
        ub = None if u is None else u[b]
        g = g + oracle.param_grad(m, pb, tb, bb, 0.0 if dLdE is None else float(dLdE[b]), ub)
    return g


def _close(g, ref, rel=2e-4):
    err = np.abs(g - ref).max() / np.abs(ref).max()
    assert err <= rel, "max error %.3g of max |g|" % err
    return err


@pytest.mark.parametrize("terms", ["energy", "force", "both"])
def test_param_grad_matches_oracle(terms):
    from paper_2002_00054_b300 import NNP
    m = _model()
    systems, starts, pos, types, boxes = _batch()
    rng = np.random.default_rng(5)
    dLdE = rng.normal(size=len(systems)) if terms != "force" else None
    u = f32(rng.normal(size=pos.shape) * 0.1) if terms != "energy" else None
    nnp = NNP(m)
    p, t = _dev(pos, types)
    g = nnp.param_grad(p, t, starts, boxes,
                       None if dLdE is None else torch.tensor(dLdE, dtype=torch.float64, device="cuda"),
                       None if u is None else torch.tensor(u, dtype=torch.float32, device="cuda"))
    ub = None if u is None else [u[starts[b]:starts[b + 1]] for b in range(len(systems))]
    ref = _oracle_grad(m, systems, dLdE, ub)
    _close(g.double().cpu().numpy(), ref)


def _loss_grad_oracle(m, systems, starts, Eref, Fref, wF):
    B = len(systems)
    n_tot = sum(len(p) for p, _, _ in systems)
    dLdE, us = [], []
    for b, (pb, tb, bb) in enumerate(systems):
        r = oracle.compute(m, pb, tb, bb)
        dLdE.append(2.0 * (r["energy"] - Eref[b]) / len(pb) ** 2 / B)
        us.append(2.0 * wF * (r["F"] - Fref[starts[b]:starts[b + 1]]) / (3 * n_tot))
    return _oracle_grad(m, systems, np.array(dLdE), us)


@pytest.mark.parametrize("form", ["double_backward", "energy_forces"])
def test_autograd_force_matching_gradient(form):
    from paper_2002_00054_b300 import NNP
    from paper_2002_00054_b300.autograd import EnergyForces, NNPEnergy, TrainingBatch, force_matching_loss
    m = _model()
    teacher = workloads.water_model(seed=workloads.SEED_TEACHER_MODEL)
    systems, starts, pos, types, boxes = _batch(seed=1)
    rng = np.random.default_rng(2)
    Eref = np.array([oracle.compute(teacher, p, t, b)["energy"] for p, t, b in systems])
    Fref = np.concatenate([oracle.compute(teacher, p, t, b)["F"] for p, t, b in systems])
    Fref = Fref + rng.normal(0, 0.01, Fref.shape)
    nnp = NNP(m)
    p, t = _dev(pos, types)
    batch = TrainingBatch(nnp, t, starts, boxes)
    w = torch.tensor(np.concatenate(m["weights"]), dtype=torch.float32, device="cuda", requires_grad=True)
    n_atoms = torch.tensor(np.diff(starts), dtype=torch.float64, device="cuda")
    Er = torch.tensor(Eref, device="cuda")
    Fr = torch.tensor(Fref, device="cuda")
    if form == "double_backward":
        x = p.clone().requires_grad_(True)
        E = NNPEnergy.apply(x, w, batch)
        F = -torch.autograd.grad(E.sum(), x, create_graph=True)[0]
    else:
        E, F = EnergyForces.apply(p, w, batch)
    loss = force_matching_loss(E, F, Er, Fr, n_atoms, 10.0)
    loss.backward()
    ref = _loss_grad_oracle(m, systems, starts, Eref, Fref, 10.0)
    _close(w.grad.double().cpu().numpy(), ref)
