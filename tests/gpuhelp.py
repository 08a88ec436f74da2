"""Shared helpers of the GPU parity tests: run the CUDA path and the oracle on the
same float32-representable inputs and compare with the stated tolerances."""
import numpy as np
import torch

import oracle

# FP32 path tolerances against the FP64 oracle, as stated for the method:
#   forces: <= 1e-4 eV/A max-abs;
#   per-atom energy: |dE_i| <= 1e-5 * max(|E_i|, rms(E)) (the "1e-5 relative" bound,
#   with the rms as the floor of the scale so that near-zero E_i are not divided by).
E_REL = 1e-5
F_ABS = 1e-4


def f32(x):
    """The float32 value of x, as float64 (both sides get exactly these inputs)."""
    return np.asarray(x, np.float32).astype(np.float64)


def to_dev(pos, types):
    return (torch.tensor(np.asarray(pos, np.float32), device="cuda"),
            torch.tensor(np.asarray(types, np.int32), device="cuda"))


def energy_err(Ei, ref_Ei):
    scale = np.maximum(np.abs(ref_Ei), np.sqrt(np.mean(ref_Ei ** 2)))
    return np.max(np.abs(Ei - ref_Ei) / scale)


def energy_tol(ref, e_rel=E_REL):
    """Per-atom energy tolerance: e_rel * max(|E_i|, rms E)."""
    Ei = ref["Ei"]
    return e_rel * np.maximum(np.abs(Ei), np.sqrt(np.mean(Ei ** 2)))


def check(out, ref, e_rel=E_REL, f_abs=F_ABS, what=""):
    Ei = out["Ei"].double().cpu().numpy()
    F = out["F"].double().cpu().numpy()
    ee = energy_err(Ei, ref["Ei"])
    fe = np.abs(F - ref["F"]).max() if len(F) else 0.0
    tol = energy_tol(ref, e_rel)
    worst = np.max(np.abs(Ei - ref["Ei"]) / tol) if len(Ei) else 0.0
    assert worst <= 1.0, "%s per-atom energy err %.3g of tolerance (rel err %.3g)" % (what, worst, ee)
    assert fe <= f_abs, "%s force max-abs err %.3g" % (what, fe)
    E = out["energy"].item()
    tol_e = tol.sum() + 1e-12
    assert abs(E - ref["energy"]) <= tol_e, "%s total energy %r vs %r" % (what, E, ref["energy"])
    if out.get("virial") is not None and "virial" in ref:
        W = out["virial"].cpu().numpy()
        tol_w = 1e-5 * max(1.0, np.abs(ref["virial"]).max()) * max(1.0, np.sqrt(len(Ei)))
        assert np.abs(W - ref["virial"]).max() <= tol_w, "%s virial" % what
    return ee, fe
