"""Slab domain decomposition with a 2 r_c halo (paper_2002_00054_b300/domain.py;
the paper's outlook on multi-node runs, Sec. 5): owned energies and forces of
every domain, evaluated on its own, and the sum over domains of the owned
atoms' energy and virial reproduce the undivided periodic box.  CPU: the oracle
as the local evaluation, in one process and on gloo ranks that exchange only
their 2 r_c boundary layers point to point; GPU: nnp_compute_domain, domains one
after another on one device, against the oracle."""
import os
import socket

import numpy as np
import pytest

import oracle
import workloads
from paper_2002_00054_b300 import domain
from tests.gpuhelp import F_ABS, check, f32


def _oracle_eval(model):
    def ev(p, t, b, n_own):
        r = oracle.compute_owned(model, p, t, b, n_own)
        return r["Ei"], r["F"], r["virial"]
    return ev


def _case(reps=(3, 2, 2)):
    m = workloads.water_model()
    pos, types, box = workloads.water_lattice(reps, seed=21)
    return m, f32(pos), types, f32(box)


@pytest.mark.parametrize("n_dom", [2, 3])
def test_decomposed_oracle_matches_undivided(n_dom):
    m, pos, types, box = _case()
    ref = oracle.compute(m, pos, types, box)
    E, Ei, F, W = domain.evaluate_decomposed(_oracle_eval(m), pos, types, box, n_dom, m["cutoff"])
    assert abs(E - ref["energy"]) <= 1e-9 * abs(ref["energy"])
    np.testing.assert_allclose(Ei, ref["Ei"], rtol=0, atol=1e-10)
    np.testing.assert_allclose(F, ref["F"], rtol=0, atol=1e-9)
    np.testing.assert_allclose(W, ref["virial"], rtol=0, atol=1e-8)


def test_decompose_rejects_thin_slabs():
    m, pos, types, box = _case()
    with pytest.raises(ValueError, match="halo"):
        domain.decompose(pos, box, 4, m["cutoff"])   # 9.3 A slabs < 12 A halo


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    m, pos, types, box = _case((6, 2, 2))
    # each rank starts from the atoms of its own slab only
    x = np.mod(pos[:, 0], box[0])
    mine = np.nonzero(np.minimum((x // (box[0] / world)).astype(int), world - 1) == rank)[0]
    p, t, gid, n_own, lbox, sent = domain.exchange_halo(pos[mine], types[mine], mine, box, m["cutoff"], rank, world)
    r = oracle.compute_owned(m, p, t, lbox, n_own)
    E, W = domain.allreduce_energy_virial(r["energy"], r["virial"])
    np.save(os.path.join(out, "r%d.npy" % rank),
            np.concatenate([gid[:n_own, None].astype(float), r["Ei"][:n_own, None], r["F"][:n_own]], axis=1))
    np.save(os.path.join(out, "e%d.npy" % rank), np.r_[E, W.reshape(9), sent, n_own, len(p)])
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_ranks_exchange_boundary_layers_and_match_undivided(tmp_path, world):
    import torch.multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    mp.start_processes(_rank, args=(world, port, str(tmp_path)), nprocs=world, start_method="spawn", join=True)
    m, pos, types, box = _case((6, 2, 2))
    ref = oracle.compute(m, pos, types, box)
    rows = np.concatenate([np.load(os.path.join(tmp_path, "r%d.npy" % r)) for r in range(world)])
    gid = rows[:, 0].astype(int)
    assert sorted(gid.tolist()) == list(range(len(pos)))
    np.testing.assert_allclose(rows[:, 1], ref["Ei"][gid], rtol=0, atol=1e-10)
    np.testing.assert_allclose(rows[:, 2:], ref["F"][gid], rtol=0, atol=1e-9)
    for r in range(world):   # every rank holds the box's energy and virial after the all_reduce
        e = np.load(os.path.join(tmp_path, "e%d.npy" % r))
        assert abs(e[0] - ref["energy"]) <= 1e-9 * abs(ref["energy"])
        np.testing.assert_allclose(e[1:10].reshape(3, 3), ref["virial"], rtol=0, atol=1e-8)
        # exactly the atoms of the slab's two 2 r_c boundary layers travel, and a
        # rank's ghosts are its neighbours' facing layers (counted from positions)
        x = np.mod(pos[:, 0], box[0])
        rc = m["cutoff"]
        assert (e[10] - 16) / 40 == _layer(x, box[0], world, r, "left", rc) + _layer(x, box[0], world, r, "right", rc)
        ghosts = _layer(x, box[0], world, (r + 1) % world, "left", rc) + \
            _layer(x, box[0], world, (r - 1) % world, "right", rc)
        assert e[12] - e[11] == ghosts
    if world == 2:   # the wider slabs send about 2 x 2 r_c / width of their atoms
        assert (np.load(os.path.join(tmp_path, "e0.npy"))[10] - 16) / 40 < 0.75 * len(pos) / 2


def _layer(x, L, world, q, side, rc):
    """Atoms of slab q within 2 r_c of its left or right face."""
    w = L / world
    xq = x[np.minimum((x // w).astype(int), world - 1) == q]
    return int(np.sum(xq < q * w + 2 * rc) if side == "left" else np.sum(xq >= (q + 1) * w - 2 * rc))


@pytest.mark.gpu
@pytest.mark.parametrize("n_dom", [2, 4])
def test_decomposed_gpu_matches_oracle(n_dom):
    import torch
    from paper_2002_00054_b300 import NNP
    m = workloads.water_model()
    pos, types, box = workloads.water_lattice((6, 3, 3), seed=22)
    pos, box = f32(pos), f32(box)
    nnp = NNP(m)
    ref = oracle.compute(m, pos, types, box)

    def ev(lp, lt, lb, n_own):
        o = nnp.compute_domain(torch.tensor(lp, dtype=torch.float32, device="cuda"),
                               torch.tensor(lt, dtype=torch.int32, device="cuda"), lb, n_own)
        assert abs(o["energy"].item() - o["Ei"][:n_own].double().sum().item()) <= 1e-6 * n_own
        return o["Ei"].double().cpu().numpy(), o["F"].double().cpu().numpy(), o["virial"].cpu().numpy()

    E, Ei, F, W = domain.evaluate_decomposed(ev, pos, types, box, n_dom, m["cutoff"])
    out = {"Ei": torch.tensor(Ei), "F": torch.tensor(F), "energy": torch.tensor([E]),
           "virial": torch.tensor(W)}
    check(out, ref, what="%d domains" % n_dom)
    assert np.abs(F - ref["F"]).max() <= F_ABS
