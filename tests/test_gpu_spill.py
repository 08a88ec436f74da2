"""The wide-capacity pass.  The main descriptor, force and tangent launches stage
at most C neighbours inside the cutoff per atom in shared memory; atoms with
more are evaluated by a second launch whose capacity is the list stride.  C is
re-tuned after every call from the counts seen, so a low-density system first
shrinks it below the counts of a liquid-density one, which then has atoms on
both sides of it.  Everything is compared with the oracle, and with the same
system evaluated by a fresh handle whose C no atom exceeds."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import workloads
from tests.gpuhelp import F_ABS, check, f32, to_dev

pytestmark = pytest.mark.gpu

RC = 6.0


def _counts(pos, box):
    """Neighbours inside the cutoff per atom (minimum image; box edges > 2 rc)."""
    d = pos[:, None, :] - pos[None, :, :]
    d -= np.round(d / box) * box
    r2 = (d ** 2).sum(-1)
    np.fill_diagonal(r2, np.inf)
    return (r2 < RC * RC).sum(1)


def _systems():
    m = workloads.water_model()
    L_low = workloads.WATER_CELL / 0.75 ** (1 / 3)       # 0.75 of liquid density
    low = workloads.water_random(box=L_low, seed=77)
    liquid = workloads.water_random(seed=78)
    return m, [(f32(p), t, f32(b)) for p, t, b in (low, liquid)]


def _shrink(nnp, low):
    p, t = to_dev(low[0], low[1])
    nnp.compute(p, t, low[2])
    return nnp.stats()["rc_capacity"]


def test_spilled_atoms_match_oracle_and_fresh_handle():
    from paper_2002_00054_b300 import NNP
    m, (low, liq) = _systems()
    nnp = NNP(m)
    c0 = nnp.stats()["rc_capacity"]
    C = _shrink(nnp, low)
    assert C < c0 and C >= _counts(*low[::2]).max()
    cnt = _counts(liq[0], liq[2])
    assert 0 < (cnt > C).sum() < len(cnt), "the liquid system must straddle the capacity"
    p, t = to_dev(liq[0], liq[1])
    out = nnp.compute(p, t, liq[2])
    s = nnp.stats()
    assert abs(s["spilled_atoms"] - int((cnt > C).sum())) <= 2
    assert s["max_cutoff_row"] == cnt.max()
    ref = oracle.compute(m, *liq)
    check(out, ref, what="liquid water with spilled atoms")
    # the same numbers as a handle whose capacity covers every atom
    fresh = NNP(m)
    o2 = fresh.compute(p, t, liq[2])
    assert fresh.stats()["spilled_atoms"] == 0
    assert torch.equal(out["Ei"], o2["Ei"])
    assert torch.equal(out["F"], o2["F"])   # integer force accumulators: order-independent sums
    # descriptors through the same two passes
    _shrink(nnp, low)
    G, _ = nnp.descriptors(p, t, liq[2])
    G2, _ = fresh.descriptors(p, t, liq[2])
    assert nnp.stats()["spilled_atoms"] > 0
    assert torch.equal(G, G2)


def test_spilled_atoms_in_step_and_param_grad():
    from paper_2002_00054_b300 import NNP
    m, (low, liq) = _systems()
    nnp = NNP(m)
    p, t = to_dev(liq[0], liq[1])
    rng = np.random.default_rng(3)
    u = f32(rng.normal(size=liq[0].shape) * 0.1)
    _shrink(nnp, low)
    g = nnp.param_grad(p, t, [0, len(p)], liq[2][None, :], torch.tensor([0.7], dtype=torch.float64, device="cuda"),
                       torch.tensor(u, dtype=torch.float32, device="cuda"))
    assert nnp.stats()["spilled_atoms"] > 0
    ref = oracle.param_grad(m, *liq, 0.7, u)
    err = np.abs(g.double().cpu().numpy() - ref).max() / np.abs(ref).max()
    assert err <= 2e-4, err
    # ten velocity-Verlet steps with spilled atoms against the oracle
    _shrink(nnp, low)
    v0 = f32(workloads.maxwell_boltzmann(liq[1], m["masses"]))
    x = p.clone()
    v = torch.tensor(v0, dtype=torch.float32, device="cuda")
    lg = nnp.step(x, v, t, liq[2], 0.5, 10).cpu().numpy()
    assert nnp.stats()["spilled_atoms"] > 0
    pr, vr, lr = oracle.md(m, liq[0], v0, liq[1], liq[2], 0.5, 10)
    assert np.abs(x.double().cpu().numpy() - pr).max() < 1e-4
    assert np.abs(v.double().cpu().numpy() - vr).max() < 1e-4
    np.testing.assert_allclose(lg[:, 0], lr[:, 0], rtol=0, atol=1e-5 * np.abs(lr[:, 0]).max() + 1e-4)


def test_spilled_atoms_in_static_entry():
    from paper_2002_00054_b300 import NNP
    m, (low, liq) = _systems()
    nnp = NNP(m)
    _shrink(nnp, low)
    p, t = to_dev(liq[0], liq[1])
    n = len(p)
    e = torch.zeros(1, dtype=torch.float64, device="cuda")
    ei = torch.zeros(n, dtype=torch.float32, device="cuda")
    f = torch.zeros((n, 3), dtype=torch.float32, device="cuda")
    b = np.ascontiguousarray(liq[2], np.float64)
    buf = ctypes.create_string_buffer(256)
    rc = nnp._lib.nnp_compute_static(nnp.h, n, ctypes.c_void_p(p.data_ptr()), ctypes.c_void_p(t.data_ptr()),
                                     b.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.c_void_p(e.data_ptr()),
                                     ctypes.c_void_p(ei.data_ptr()), ctypes.c_void_p(f.data_ptr()), buf, 256,
                                     ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, buf.value
    ref = oracle.compute(m, *liq)
    check({"Ei": ei, "F": f, "energy": e}, ref, what="static entry with spilled atoms")
    assert np.abs(f.double().cpu().numpy() - ref["F"]).max() <= F_ABS


def test_large_forces_take_the_exact_range_test():
    """Output-layer weights x 3000 (forces up to ~8000 eV/A): for about a third
    of the atoms the per-atom bound on the triplet contributions exceeds half the
    fixed-point range, so the force kernel tests each contribution; the bound
    itself stays below the range, so no contribution fails the test, and the
    forces of both kinds of atoms match the oracle (tolerances x 3000)."""
    from paper_2002_00054_b300 import NNP
    scale = 3000.0
    m = workloads.water_model()
    w = [x.copy() for x in m["weights"]]
    for x in w:
        x[-26:-1] *= scale
    big = dict(m, weights=w)
    pos, types, box = workloads.water_random()
    p, t = to_dev(f32(pos), types)
    out = NNP(big).compute(p, t, f32(box))
    ref = oracle.compute(big, f32(pos), types, f32(box))
    dF = np.abs(out["F"].double().cpu().numpy() - ref["F"]).max()
    assert dF <= scale * F_ABS, dF
    dE = np.abs(out["Ei"].double().cpu().numpy() - ref["Ei"]).max()
    assert dE <= 1e-5 * np.abs(ref["Ei"]).max(), dE


def test_force_contribution_out_of_range_is_an_error():
    """Force contributions are summed in fixed point (|v| < 32000 eV/A per
    contribution); a model whose forces exceed that range fails the call with
    NNP_ENONFINITE instead of returning wrapped sums."""
    from paper_2002_00054_b300 import NNP
    from paper_2002_00054_b300._capi import NNPError
    m = workloads.water_model()
    w = [x.copy() for x in m["weights"]]
    for x in w:
        x[-26:-1] *= 1e7   # output-layer weights (25 of them, then the bias)
    big = dict(m, weights=w)
    nnp = NNP(big)
    pos, types, box = workloads.water_random()
    p, t = to_dev(f32(pos), types)
    with pytest.raises(NNPError, match="exceeds"):
        nnp.compute(p, t, f32(box))
    # the handle stays usable: the same system with the unscaled model's weights
    nnp.set_weights(torch.tensor(np.concatenate(m["weights"]), dtype=torch.float32, device="cuda"))
    out = nnp.compute(p, t, f32(box))
    check(out, oracle.compute(m, f32(pos), types, f32(box)), what="after a range error")
