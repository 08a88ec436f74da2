"""nnp_step replays one step's launch sequence as a CUDA graph.  The replayed
trajectory must be bitwise the one of launching every kernel directly
(NNP_STEP_GRAPH=0): rebuild decisions, wide-capacity atoms and the energy-log
entry are all taken on the device, so every step runs the same launches.  Also:
errors raised at any step of a call are reported by the call."""
import numpy as np
import pytest
import torch

import workloads
from tests.gpuhelp import f32, to_dev

pytestmark = pytest.mark.gpu


def _run(model, pos, types, box, vel, dt, n_steps, env, monkeypatch, calls=1, **kw):
    from paper_2002_00054_b300 import NNP
    if env is not None:
        monkeypatch.setenv("NNP_STEP_GRAPH", env)
    else:
        monkeypatch.delenv("NNP_STEP_GRAPH", raising=False)
    nnp = NNP(model, **kw)
    monkeypatch.delenv("NNP_STEP_GRAPH", raising=False)
    p, t = to_dev(f32(pos), types)
    v = torch.tensor(vel, dtype=torch.float32, device="cuda")
    logs = []
    for c in range(calls):
        lg = nnp.step(p, v, t, f32(box), dt, n_steps)
        logs.append(lg if c == 0 else lg[1:])
    s = nnp.stats()
    nnp.close()
    return p, v, torch.cat(logs), s


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_graph_replay_is_bitwise_eager(precision, monkeypatch):
    m = workloads.water_model()
    pos, types, box = workloads.water_lattice((2, 2, 2), seed=9)
    vel = workloads.maxwell_boltzmann(types, m["masses"], seed=3, T=600.0)
    kw = {"precision": precision}
    pg, vg, lg, sg = _run(m, pos, types, box, vel, 0.5, 60, None, monkeypatch, **kw)
    pe, ve, le, se = _run(m, pos, types, box, vel, 0.5, 60, "0", monkeypatch, **kw)
    assert torch.equal(pg, pe) and torch.equal(vg, ve)
    assert torch.equal(lg, le)
    assert sg["rebuilds"] == se["rebuilds"] >= 1          # rebuilds happened inside the replays
    assert sg["kernel_launches"] == se["kernel_launches"]
    assert np.isfinite(lg.cpu().numpy()).all()


def test_graph_replay_continuing_calls(monkeypatch):
    """Three calls of 7 steps on one handle (the executable graph is updated in
    place) against one eager call of 21 steps."""
    m = workloads.water_model()
    pos, types, box = workloads.water_random(seed=5)
    vel = workloads.maxwell_boltzmann(types, m["masses"], seed=4)
    pg, vg, lg, _ = _run(m, pos, types, box, vel, 0.5, 7, None, monkeypatch, calls=3)
    pe, ve, le, _ = _run(m, pos, types, box, vel, 0.5, 21, "0", monkeypatch)
    assert torch.equal(pg, pe) and torch.equal(vg, ve)
    assert torch.equal(lg, le)


def test_graph_replay_across_system_sizes(monkeypatch):
    """One handle steps systems of different sizes one after another (a new
    capture each call; the cached executable is updated or re-instantiated)."""
    from paper_2002_00054_b300 import NNP
    m = workloads.water_model()
    nnp = NNP(m)
    monkeypatch.setenv("NNP_STEP_GRAPH", "0")
    ref = NNP(m)
    monkeypatch.delenv("NNP_STEP_GRAPH")
    for cells in [(2, 2, 2), (1, 1, 1), (3, 2, 2)]:
        pos, types, box = workloads.water_lattice(cells, seed=2)
        vel = workloads.maxwell_boltzmann(types, m["masses"], seed=6)
        p1, t = to_dev(f32(pos), types)
        v1 = torch.tensor(vel, dtype=torch.float32, device="cuda")
        p2, v2 = p1.clone(), v1.clone()
        la = nnp.step(p1, v1, t, f32(box), 0.5, 5)
        lb = ref.step(p2, v2, t, f32(box), 0.5, 5)
        assert torch.equal(p1, p2) and torch.equal(v1, v2) and torch.equal(la, lb)


def test_error_at_first_step_is_kept(monkeypatch):
    """Two atoms closer than 1e-4 A at the start: the first evaluation raises the
    error, later steps (the pair has moved apart) are clean; the call must still
    report the error of its first evaluation."""
    from paper_2002_00054_b300 import NNP, NNPError
    m = workloads.water_model()
    pos, types, box = workloads.water_random(seed=5)
    pos = f32(pos)
    pos[1] = pos[0] + np.array([8e-5, 0.0, 0.0], np.float32)
    vel = np.zeros_like(pos)
    vel[1, 0] = 0.02
    p, t = to_dev(pos, types)
    v = torch.tensor(vel, dtype=torch.float32, device="cuda")
    nnp = NNP(m)
    with pytest.raises(NNPError) as e:
        nnp.step(p, v, t, f32(box), 0.5, 5)
    assert e.value.status == 4
    # the state after the call evaluates cleanly: the error came from an earlier step
    fresh = NNP(m)
    out = fresh.compute(p, t, f32(box))
    assert np.isfinite(out["energy"].item())
