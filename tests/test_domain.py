"""Slab domain decomposition with a 2 r_c halo (paper_2002_00054_b300/domain.py):
owned energies and forces of every domain, evaluated on its own, reproduce the
undivided periodic box.  CPU: with the oracle as the local evaluation, one
process and two gloo ranks; GPU: with the CUDA path, domains run one after
another on one device."""
import os
import socket

import numpy as np
import pytest

import oracle
import workloads
from paper_2002_00054_b300 import domain
from tests.gpuhelp import f32


def _oracle_eval(model):
    def ev(p, t, b):
        r = oracle.compute(model, p, t, b)
        return r["Ei"], r["F"]
    return ev


def _case():
    m = workloads.water_model()
    pos, types, box = workloads.water_lattice((3, 2, 2), seed=21)
    return m, f32(pos), types, f32(box)


@pytest.mark.parametrize("n_dom", [2, 3])
def test_decomposed_oracle_matches_undivided(n_dom):
    m, pos, types, box = _case()
    ref = oracle.compute(m, pos, types, box)
    E, Ei, F = domain.evaluate_decomposed(_oracle_eval(m), pos, types, box, n_dom, m["cutoff"])
    assert abs(E - ref["energy"]) <= 1e-9 * abs(ref["energy"])
    np.testing.assert_allclose(Ei, ref["Ei"], rtol=0, atol=1e-10)
    np.testing.assert_allclose(F, ref["F"], rtol=0, atol=1e-9)


def test_decompose_rejects_thin_slabs():
    m, pos, types, box = _case()
    with pytest.raises(ValueError, match="halo"):
        domain.decompose(pos, box, 4, m["cutoff"])   # 9.3 A slabs < 12 A halo


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    m, pos, types, box = _case()
    # each rank starts from the atoms of its own slab only
    x = np.mod(pos[:, 0], box[0])
    mine = np.nonzero(np.minimum((x // (box[0] / world)).astype(int), world - 1) == rank)[0]
    p, t, gid, n_own, lbox = domain.exchange_halo(pos[mine], types[mine], mine, box, m["cutoff"], rank, world)
    r = oracle.compute(m, p, t, lbox)
    np.save(os.path.join(out, "r%d.npy" % rank),
            np.concatenate([gid[:n_own, None].astype(float), r["Ei"][:n_own, None], r["F"][:n_own]], axis=1))
    np.save(os.path.join(out, "e%d.npy" % rank), np.array([domain.allreduce_energy(r["Ei"][:n_own].sum())]))
    dist.destroy_process_group()


def test_two_gloo_ranks_match_undivided(tmp_path):
    import torch.multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    mp.start_processes(_rank, args=(2, port, str(tmp_path)), nprocs=2, start_method="spawn", join=True)
    m, pos, types, box = _case()
    ref = oracle.compute(m, pos, types, box)
    rows = np.concatenate([np.load(os.path.join(tmp_path, "r%d.npy" % r)) for r in range(2)])
    gid = rows[:, 0].astype(int)
    assert sorted(gid.tolist()) == list(range(len(pos)))
    np.testing.assert_allclose(rows[:, 1], ref["Ei"][gid], rtol=0, atol=1e-10)
    np.testing.assert_allclose(rows[:, 2:], ref["F"][gid], rtol=0, atol=1e-9)
    assert abs(rows[:, 1].sum() - ref["energy"]) <= 1e-9 * abs(ref["energy"])
    for r in range(2):   # every rank holds the total energy after the all_reduce
        assert abs(np.load(os.path.join(tmp_path, "e%d.npy" % r))[0] - ref["energy"]) <= 1e-9 * abs(ref["energy"])


@pytest.mark.gpu
@pytest.mark.parametrize("n_dom", [2, 4])
def test_decomposed_gpu_matches_undivided(n_dom):
    import torch
    from paper_2002_00054_b300 import NNP
    m = workloads.water_model()
    pos, types, box = workloads.water_lattice((6, 3, 3), seed=22)
    pos, box = f32(pos), f32(box)
    nnp = NNP(m)
    p = torch.tensor(pos, dtype=torch.float32, device="cuda")
    t = torch.tensor(types, dtype=torch.int32, device="cuda")
    full = nnp.compute(p, t, box)

    def ev(lp, lt, lb):
        o = nnp.compute(torch.tensor(lp, dtype=torch.float32, device="cuda"),
                        torch.tensor(lt, dtype=torch.int32, device="cuda"), lb)
        return o["Ei"].double().cpu().numpy(), o["F"].double().cpu().numpy()

    E, Ei, F = domain.evaluate_decomposed(ev, pos, types, box, n_dom, m["cutoff"])
    Ef = full["Ei"].double().cpu().numpy()
    assert np.abs(Ei - Ef).max() <= 1e-5 * np.abs(Ef).max()
    assert np.abs(F - full["F"].double().cpu().numpy()).max() <= 1e-4
    assert abs(E - full["energy"].item()) <= 1e-5 * np.abs(Ef).sum()
