"""nnp_compute_static: the allocation-free entry point for callers that cannot
allocate device memory when they need forces (codes that reserve all device
memory up front, or time loops that must not pay for cudaMalloc's implicit
synchronisation).  Called through the C ABI and checked against nnp_compute on
the same inputs, twice in a row (the second call runs on the scratch the first
one left behind).  This file is collected last."""
import ctypes

import numpy as np
import pytest
import torch

import workloads
import oracle
from tests.gpuhelp import E_REL, F_ABS, check, energy_err, f32, to_dev

pytestmark = pytest.mark.gpu


def _static(nnp, p, t, box):
    lib = nnp._lib
    n = p.shape[0]
    e = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    ei = torch.full((n,), float("nan"), dtype=torch.float32, device="cuda")
    f = torch.full((n, 3), float("nan"), dtype=torch.float32, device="cuda")
    b = np.ascontiguousarray(box, np.float64)
    buf = ctypes.create_string_buffer(512)
    rc = lib.nnp_compute_static(nnp.h, n, ctypes.c_void_p(p.data_ptr()), ctypes.c_void_p(t.data_ptr()),
                                b.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.c_void_p(e.data_ptr()),
                                ctypes.c_void_p(ei.data_ptr()), ctypes.c_void_p(f.data_ptr()), buf, 512,
                                ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return rc, buf.value.decode(), e, ei, f


def _cluster(n=150, radius=5.4, min_sep=1.3, box=40.0, seed=77):
    """A dense isolated ball: atoms near its centre have more neighbours inside
    the cutoff than the handle's shared-memory capacity, so the call's
    wide-capacity pass runs; every neighbour-list row stays below 192."""
    rng = np.random.default_rng(seed)
    c = np.full(3, box / 2)
    pts = []
    while len(pts) < n:
        x = c + rng.uniform(-radius, radius, 3)
        if np.linalg.norm(x - c) > radius:
            continue
        if all(np.linalg.norm(x - q) >= min_sep for q in pts):
            pts.append(x)
    return np.array(pts), np.zeros(n, np.int32), np.array([box, box, box])


def _cases():
    L = (3 * 21 / workloads.WATER_DENSITY_ATOMS) ** (1 / 3)
    return [("water", workloads.water_model, workloads.water_random()),
            ("water", workloads.water_model, workloads.water_random(21, L, seed=121)),
            ("fcc", workloads.fcc_model, workloads.fcc((2, 2, 2), sigma=0.1, seed=4)),
            # exactly NNP_STATIC_MAX_ATOMS atoms at the default max_neighbors
            ("fcc", workloads.fcc_model, workloads.fcc((4, 8, 8), sigma=0.1, seed=5)),
            ("fcc", workloads.fcc_model, _cluster())]


def test_static_matches_compute_on_two_calls_in_a_row():
    from paper_2002_00054_b300 import NNP
    handles = {}
    for ci, (name, mk, (pos, types, box)) in enumerate(_cases()):
        ref_nnp = handles.setdefault(name, NNP(mk()))
        nnp = NNP(mk())   # fresh handle: its capacity has not been re-tuned by a call
        pos, box = f32(pos), f32(box)
        p, t = to_dev(pos, types)
        ref = ref_nnp.compute(p, t, box)
        if len(pos) == 150:
            # the cluster sends atoms through the wide-capacity pass: some atom has
            # more neighbours inside the cutoff than the capacity the static call uses
            C = nnp.stats()["rc_capacity"]
            d = pos[:, None, :] - pos[None, :, :]
            cnt = ((d ** 2).sum(-1) < nnp.cutoff ** 2).sum(1) - 1
            assert cnt.max() > C, (cnt.max(), C)
        Ei_ref = ref["Ei"].double().cpu().numpy()
        first = None
        for call in range(2):
            rc, msg, e, ei, f = _static(nnp, p, t, box)
            assert rc == 0, msg
            Ei = ei.double().cpu().numpy()
            assert energy_err(Ei, Ei_ref) <= E_REL
            assert np.abs(f.double().cpu().numpy() - ref["F"].double().cpu().numpy()).max() <= F_ABS
            assert abs(e.item() - ref["energy"].item()) <= E_REL * np.abs(Ei_ref).sum()
            if first is None:
                first = (e.clone(), ei.clone(), f.clone())
                if ci in (0, 3):
                    # the 192-atom water box and the 1,024-atom FCC box against the oracle too
                    check({"energy": e, "Ei": ei, "F": f}, oracle.compute(mk(), pos.astype(np.float64), types,
                                                                         box.astype(np.float64)),
                          what="static %s %d" % (name, len(pos)))
            else:
                assert torch.equal(first[0], e) and torch.equal(first[1], ei) and torch.equal(first[2], f)


def test_static_rejects_sizes_beyond_its_limit():
    from paper_2002_00054_b300 import NNP
    nnp = NNP(workloads.water_model())
    pos, types, box = workloads.water_lattice((2, 2, 2))   # 1,536 atoms > 1,024
    p, t = to_dev(f32(pos), types)
    rc, msg, *_ = _static(nnp, p, t, f32(box))
    assert rc == 1 and "1024" in msg
    big = NNP(workloads.water_model(), max_neighbors=1024)   # 1,024 atoms x 1,024 slots exceed the array
    pos, types, box = workloads.water_random()
    p, t = to_dev(f32(pos), types)
    rc, msg, *_ = _static(big, p, t, f32(box))
    assert rc == 0, msg
    pos, types, box = workloads.water_lattice((2, 2, 2))
    p, t = to_dev(f32(pos)[:1000], types[:1000])
    rc, msg, *_ = _static(big, p, t, f32(box))
    assert rc == 1 and "bytes" in msg
