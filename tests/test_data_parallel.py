"""Data-parallel force-matching training over configurations.  CPU: the shards
partition the batch; two gloo ranks, each with its own shard's gradient of the
loss (normalised by the whole batch) from the FP64 oracle, all_reduce to the
full-batch gradient.  GPU: the library's shard gradients sum to its full-batch
gradient."""
import os
import socket

import numpy as np
import pytest

import oracle
import workloads
from paper_2002_00054_b300.data_parallel import allreduce_grad, shard_by_atoms, shard_loss

W_FORCE = 10.0


def _batch(n_configs=4):
    systems = workloads.train_batch()[:n_configs]
    m = workloads.water_model()
    teacher = workloads.water_model(seed=workloads.SEED_TEACHER_MODEL)
    rng = np.random.default_rng(17)
    Eref, Fref = [], []
    for pos, types, box in systems:
        r = oracle.compute(teacher, pos, types, box)
        Eref.append(r["energy"])
        Fref.append(r["F"] + 0.01 * rng.normal(size=r["F"].shape))
    return m, systems, np.array(Eref), Fref


def _oracle_grad(m, systems, Eref, Fref, lo, hi, B, n_tot):
    """Gradient of the loss terms of configurations lo..hi-1 (whole-batch
    normalisers): dL/dE_b dE_b/dtheta + sum_m dL/dF_m . dF_m/dtheta."""
    g = np.zeros(len(np.concatenate(m["weights"])))
    for b in range(lo, hi):
        pos, types, box = systems[b]
        r = oracle.compute(m, pos, types, box)
        n = len(pos)
        dLdE = 2.0 * (r["energy"] - Eref[b]) / n ** 2 / B
        u = 2.0 * W_FORCE * (r["F"] - Fref[b]) / (3.0 * n_tot)
        g += oracle.param_grad(m, pos, types, box, dLdE, u)
    return g


def test_shards_partition_and_balance():
    rng = np.random.default_rng(1)
    for _ in range(200):
        n = rng.integers(1, 600, size=rng.integers(1, 12))
        world = int(rng.integers(1, 7))
        sh = [shard_by_atoms(n, r, world) for r in range(world)]
        assert sh[0][0] == 0 and sh[-1][1] == len(n)
        assert all(a[1] == b[0] for a, b in zip(sh, sh[1:]))
        assert all(n[lo:hi].sum() <= n.sum() / world + n.max() for lo, hi in sh)
    with pytest.raises(ValueError):
        shard_by_atoms([1, 2], 2, 2)


def test_shard_losses_sum_to_the_batch_loss():
    import torch
    from paper_2002_00054_b300.autograd import force_matching_loss
    rng = np.random.default_rng(2)
    n = np.array([66, 120, 510, 300, 90])
    E, Er = torch.tensor(rng.normal(size=5)), torch.tensor(rng.normal(size=5))
    F, Fr = torch.tensor(rng.normal(size=(n.sum(), 3))), torch.tensor(rng.normal(size=(n.sum(), 3)))
    na = torch.tensor(n, dtype=torch.float64)
    full = force_matching_loss(E, F, Er, Fr, na, W_FORCE)
    starts = np.concatenate([[0], np.cumsum(n)])
    parts = 0.0
    for r in range(3):
        lo, hi = shard_by_atoms(n, r, 3)
        a, b = starts[lo], starts[hi]
        parts = parts + shard_loss(E[lo:hi], F[a:b], Er[lo:hi], Fr[a:b], na[lo:hi], len(n), n.sum(), W_FORCE)
    assert abs(float(parts) - float(full)) <= 1e-12 * abs(float(full))


def _rank(rank, world, port, out):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    m, systems, Eref, Fref = _batch()
    n = [len(p) for p, _, _ in systems]
    lo, hi = shard_by_atoms(n, rank, world)
    g = torch.from_numpy(_oracle_grad(m, systems, Eref, Fref, lo, hi, len(systems), sum(n)))
    allreduce_grad(g)
    np.save(os.path.join(out, "g%d.npy" % rank), g.numpy())
    dist.destroy_process_group()


def test_two_gloo_ranks_sum_to_the_batch_gradient(tmp_path):
    import torch.multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    mp.start_processes(_rank, args=(2, port, str(tmp_path)), nprocs=2, start_method="spawn", join=True)
    m, systems, Eref, Fref = _batch()
    n = [len(p) for p, _, _ in systems]
    full = _oracle_grad(m, systems, Eref, Fref, 0, len(systems), len(systems), sum(n))
    for r in range(2):
        g = np.load(os.path.join(tmp_path, "g%d.npy" % r))
        np.testing.assert_allclose(g, full, rtol=1e-9, atol=1e-12 * np.abs(full).max())


@pytest.mark.gpu
def test_gpu_shard_gradients_sum_to_the_batch_gradient():
    import torch
    from paper_2002_00054_b300 import NNP
    from paper_2002_00054_b300.autograd import EnergyForces, TrainingBatch, force_matching_loss
    systems = workloads.train_batch()[:12]
    m = workloads.water_model()
    teacher = NNP(workloads.water_model(seed=workloads.SEED_TEACHER_MODEL))
    nnp = NNP(m)
    n = np.array([len(p) for p, _, _ in systems])
    starts = np.concatenate([[0], np.cumsum(n)]).astype(np.int32)
    pos = torch.tensor(np.concatenate([p for p, _, _ in systems]), dtype=torch.float32, device="cuda")
    types = torch.tensor(np.concatenate([t for _, t, _ in systems]), dtype=torch.int32, device="cuda")
    boxes = np.stack([b for _, _, b in systems]).astype(np.float32).astype(np.float64)
    lab = teacher.compute_batch(pos, types, starts, boxes)
    Eref, Fref = lab["energy"], lab["F"].double()
    na = torch.tensor(n, dtype=torch.float64, device="cuda")

    def grad(lo, hi, whole):
        a, b = int(starts[lo]), int(starts[hi])
        w = torch.tensor(np.concatenate(m["weights"]), dtype=torch.float32, device="cuda", requires_grad=True)
        batch = TrainingBatch(nnp, types[a:b], starts[lo:hi + 1] - starts[lo], boxes[lo:hi])
        E, F = EnergyForces.apply(pos[a:b], w, batch)
        if whole:
            loss = force_matching_loss(E, F, Eref, Fref, na, W_FORCE)
        else:
            loss = shard_loss(E, F, Eref[lo:hi], Fref[a:b], na[lo:hi], len(n), int(n.sum()), W_FORCE)
        loss.backward()
        return w.grad.double().cpu().numpy()

    full = grad(0, len(n), True)
    parts = sum(grad(*shard_by_atoms(n, r, 2), False) for r in range(2))
    assert np.abs(parts - full).max() <= 2e-4 * np.abs(full).max()
