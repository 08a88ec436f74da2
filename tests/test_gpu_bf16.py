"""Precision form: the per-element networks in BF16 on the tensor cores (FP32
accumulation), descriptors and forces in FP32.  Errors against the FP64 oracle are
stated for every case; the force RMS error must stay <= 5e-3 eV/A."""
import numpy as np
import pytest
import torch

import oracle
import workloads
from tests.gpuhelp import f32, to_dev

pytestmark = pytest.mark.gpu

F_RMS_BF16 = 5e-3


def _cases():
    return [("water 192", workloads.water_model, workloads.water_random()),
            ("water 1536", workloads.water_model, workloads.water_lattice((2, 2, 2), seed=5)),
            ("fcc 4000", workloads.fcc_model, workloads.fcc((10, 10, 10))),
            ("fcc 32", workloads.fcc_model, workloads.fcc((2, 2, 2), sigma=0.1, seed=4))]


@pytest.mark.parametrize("idx", range(4))
def test_bf16_network_force_error(idx):
    from paper_2002_00054_b300 import NNP
    name, mk, (pos, types, box) = _cases()[idx]
    m = mk()
    pos, box = f32(pos), f32(box)
    ref = oracle.compute(m, pos, types, box)
    p, t = to_dev(pos, types)
    bf = NNP(m, precision="bf16").compute(p, t, box)
    fp = NNP(m).compute(p, t, box)
    F = bf["F"].double().cpu().numpy()
    f_rms = np.sqrt(np.mean((F - ref["F"]) ** 2))
    f_max = np.abs(F - ref["F"]).max()
    e_err = np.abs(bf["Ei"].double().cpu().numpy() - ref["Ei"])
    e_scale = np.sqrt(np.mean(ref["Ei"] ** 2))
    fp_rms = np.sqrt(np.mean((fp["F"].double().cpu().numpy() - F) ** 2))
    print("%s BF16: force RMS err %.2e, max %.2e eV/A; per-atom energy RMS err %.2e eV (%.1e of rms E_i); "
          "force RMS vs FP32 path %.2e" % (name, f_rms, f_max, np.sqrt(np.mean(e_err ** 2)),
                                             np.sqrt(np.mean(e_err ** 2)) / e_scale, fp_rms))
    assert f_rms <= F_RMS_BF16
    # energies: BF16 rounding of the network inputs and activations (2^-9 relative)
    assert np.sqrt(np.mean(e_err ** 2)) <= 2e-2 * e_scale
    # the rounded weights make the per-atom errors correlated: bound the mean per-atom error
    assert abs(bf["energy"].item() - ref["energy"]) / len(pos) <= 2e-2 * e_scale


def test_bf16_input_gradient_close_to_fp32():
    """dE/dG of the tensor-core network against the FP32 network on the same descriptors."""
    from paper_2002_00054_b300 import NNP
    m = workloads.water_model()
    pos, types, box = workloads.water_lattice((2, 2, 2), seed=5)
    p, t = to_dev(f32(pos), types)
    g_bf, d_bf = NNP(m, precision="bf16").descriptors(p, t, f32(box))
    g_fp, d_fp = NNP(m).descriptors(p, t, f32(box))
    assert torch.equal(g_bf, g_fp)   # descriptors are FP32 in both
    rel = (d_bf - d_fp).abs().max() / d_fp.abs().max()
    assert rel < 2e-2, rel.item()


def test_bf16_ragged_element_tiles():
    """Element tiles of 128 atoms with ragged tails: 63-atom and 111-atom systems."""
    from paper_2002_00054_b300 import NNP
    m = workloads.water_model()
    bf, fp = NNP(m, precision="bf16"), NNP(m)
    for n_mol in (21, 37):
        L = (3 * n_mol / workloads.WATER_DENSITY_ATOMS) ** (1 / 3)
        pos, types, box = workloads.water_random(n_mol, L, seed=100 + n_mol)
        p, t = to_dev(f32(pos), types)
        a, b = bf.compute(p, t, f32(box)), fp.compute(p, t, f32(box))
        assert torch.isfinite(a["F"]).all()
        assert (a["F"] - b["F"]).pow(2).mean().sqrt().item() <= F_RMS_BF16


def test_static_entry_rejects_bf16():
    import ctypes
    from paper_2002_00054_b300 import NNP
    nnp = NNP(workloads.water_model(), precision="bf16")
    pos, types, box = workloads.water_random()
    p, t = to_dev(f32(pos), types)
    b = np.ascontiguousarray(f32(box))
    buf = ctypes.create_string_buffer(256)
    rc = nnp._lib.nnp_compute_static(nnp.h, len(pos), ctypes.c_void_p(p.data_ptr()), ctypes.c_void_p(t.data_ptr()),
                                     b.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), None, None, None, buf, 256,
                                     None)
    assert rc == 7 and b"FP32" in buf.value
