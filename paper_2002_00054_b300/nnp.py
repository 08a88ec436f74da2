"""Python handle over the C ABI: marshals a model description and torch CUDA
tensors into libnnp.so calls.  Every step of the computation runs in the CUDA
kernels of that library; this module only checks arguments and passes pointers."""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _capi

_TYPE_CODE = {"radial": _capi.NNP_SF_RADIAL, "narrow": _capi.NNP_SF_ANG_NARROW, "wide": _capi.NNP_SF_ANG_WIDE}


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _need(t, dtype, shape, name, device):
    if not isinstance(t, torch.Tensor):
        raise TypeError("%s must be a torch tensor" % name)
    if t.device.type != "cuda" or t.device.index != device:
        raise ValueError("%s must be on cuda:%d" % (name, device))
    if t.dtype != dtype or not t.is_contiguous() or tuple(t.shape) != tuple(shape):
        raise ValueError("%s must be a contiguous %s tensor of shape %s (got %s %s)"
                         % (name, dtype, tuple(shape), t.dtype, tuple(t.shape)))
    return t


class NNP:
    """One model on one CUDA device (a C-ABI handle)."""

    def __init__(self, model: dict, device: int = 0, precision: str = "fp32", skin: float = 1.0,
                 max_neighbors: int = 192):
        self._lib = _capi.load()
        sf = model["sf"]
        ne = len(sf)
        rows = [d for e in range(ne) for d in sf[e]]
        self._sf = (_capi.SfDesc * len(rows))()
        for k, d in enumerate(rows):
            self._sf[k] = _capi.SfDesc(_TYPE_CODE[d["type"]], int(d.get("e1", -1)), int(d.get("e2", -1)),
                                       float(d["eta"]), float(d.get("rs", 0.0)), float(d.get("zeta", 1.0)),
                                       float(d.get("lambda", 1.0)))
        self._masses = np.ascontiguousarray(model["masses"], np.float64)
        self._nsf = np.ascontiguousarray([len(r) for r in sf], np.int32)
        self._mu = np.ascontiguousarray(np.concatenate([np.asarray(m, np.float64) for m in model["sf_mu"]]))
        self._s = np.ascontiguousarray(np.concatenate([np.asarray(m, np.float64) for m in model["sf_s"]]))
        self._widths = np.ascontiguousarray(model["widths"], np.int32)
        self._w = np.ascontiguousarray(np.concatenate([np.asarray(w, np.float64) for w in model["weights"]]))
        p = _capi.Params()
        p.n_elements = ne
        p.masses_amu = self._masses.ctypes.data_as(_capi.c_double_p)
        p.cutoff = float(model["cutoff"])
        p.skin = float(skin)
        p.n_sf = self._nsf.ctypes.data_as(_capi.c_int_p)
        p.sf = self._sf
        p.sf_shift = self._mu.ctypes.data_as(_capi.c_double_p)
        p.sf_scale = self._s.ctypes.data_as(_capi.c_double_p)
        p.n_layers = len(self._widths) - 1
        p.widths = self._widths.ctypes.data_as(_capi.c_int_p)
        p.weights = self._w.ctypes.data_as(_capi.c_double_p)
        p.mlp_precision = {"fp32": _capi.NNP_FP32, "bf16": _capi.NNP_BF16}[precision]
        p.max_neighbors = int(max_neighbors)
        self.params = p
        h = ctypes.c_void_p()
        rc = self._lib.nnp_create(ctypes.byref(p), int(device), ctypes.byref(h))
        if rc != 0:
            raise _capi.NNPError(rc, self._lib.nnp_last_error(None).decode())
        self.h = h
        self.device = int(device)
        self.n_g = int(self._widths[0])
        self.cutoff = float(model["cutoff"])
        self.n_elements = ne

    # ------------------------------------------------------------------ utils
    def _check(self, rc):
        if rc != 0:
            raise _capi.NNPError(rc, self._lib.nnp_last_error(self.h).decode())

    def _box(self, box):
        b = np.ascontiguousarray(np.asarray(box, np.float64).reshape(3))
        return b, b.ctypes.data_as(_capi.c_double_p)

    def close(self):
        if getattr(self, "h", None):
            self._lib.nnp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def num_params(self):
        return int(self._lib.nnp_num_params(self.h))

    # ------------------------------------------------------------------- calls
    def compute(self, pos, types, box, forces=True, atom_energy=True, virial=True, stream=None):
        """Energy (fp64), per-atom energies, forces and virial of one system."""
        n = int(pos.shape[0]) if pos.dim() == 2 else 0
        dev = torch.device("cuda", self.device)
        _need(pos, torch.float32, (n, 3), "pos", self.device)
        _need(types, torch.int32, (n,), "types", self.device)
        out = {"energy": torch.empty(1, dtype=torch.float64, device=dev)}
        out["Ei"] = torch.empty(n, dtype=torch.float32, device=dev) if atom_energy else None
        out["F"] = torch.empty((n, 3), dtype=torch.float32, device=dev) if forces else None
        out["virial"] = torch.empty(9, dtype=torch.float64, device=dev) if virial else None
        b, bp = self._box(box)
        rc = self._lib.nnp_compute(self.h, n, _ptr(pos), _ptr(types), bp, 0.0, _ptr(out["energy"]),
                                   _ptr(out["Ei"]), _ptr(out["F"]), _ptr(out["virial"]), _stream(stream))
        self._check(rc)
        if out["virial"] is not None:
            out["virial"] = out["virial"].view(3, 3)
        return out

    def compute_domain(self, pos, types, box, n_owned, stream=None):
        """One spatial domain (owned atoms first, then its 2 r_c halo): energy and
        virial of the owned atoms' energies (fp64), Ei and F of every local atom."""
        n = int(pos.shape[0]) if pos.dim() == 2 else 0
        dev = torch.device("cuda", self.device)
        _need(pos, torch.float32, (n, 3), "pos", self.device)
        _need(types, torch.int32, (n,), "types", self.device)
        out = {"energy": torch.empty(1, dtype=torch.float64, device=dev),
               "Ei": torch.empty(n, dtype=torch.float32, device=dev),
               "F": torch.empty((n, 3), dtype=torch.float32, device=dev),
               "virial": torch.empty(9, dtype=torch.float64, device=dev)}
        b, bp = self._box(box)
        rc = self._lib.nnp_compute_domain(self.h, n, int(n_owned), _ptr(pos), _ptr(types), bp, _ptr(out["energy"]),
                                          _ptr(out["Ei"]), _ptr(out["F"]), _ptr(out["virial"]), _stream(stream))
        self._check(rc)
        out["virial"] = out["virial"].view(3, 3)
        return out

    def compute_into(self, pos, types, box, energy, Ei=None, F=None, virial=None, stream=None):
        """nnp_compute into caller-provided device tensors (no allocation)."""
        b, bp = self._box(box)
        rc = self._lib.nnp_compute(self.h, int(pos.shape[0]), _ptr(pos), _ptr(types), bp, 0.0, _ptr(energy),
                                   _ptr(Ei), _ptr(F), _ptr(virial), _stream(stream))
        self._check(rc)

    def descriptors(self, pos, types, box, dEdG=True, stream=None):
        n = int(pos.shape[0])
        dev = torch.device("cuda", self.device)
        _need(pos, torch.float32, (n, 3), "pos", self.device)
        _need(types, torch.int32, (n,), "types", self.device)
        G = torch.empty((n, self.n_g), dtype=torch.float32, device=dev)
        dG = torch.empty((n, self.n_g), dtype=torch.float32, device=dev) if dEdG else None
        b, bp = self._box(box)
        self._check(self._lib.nnp_descriptors(self.h, n, _ptr(pos), _ptr(types), bp, _ptr(G), _ptr(dG),
                                              _stream(stream)))
        return G, dG

    def descriptors_flat(self, pos, types, box, stream=None):
        """Raw descriptors G with one thread per atom (the parallelism ablation)."""
        n = int(pos.shape[0])
        _need(pos, torch.float32, (n, 3), "pos", self.device)
        _need(types, torch.int32, (n,), "types", self.device)
        G = torch.empty((n, self.n_g), dtype=torch.float32, device=torch.device("cuda", self.device))
        b, bp = self._box(box)
        self._check(self._lib.nnp_descriptors_flat(self.h, n, _ptr(pos), _ptr(types), bp, _ptr(G), _stream(stream)))
        return G

    def descriptors_pair(self, pos, types, box, stream=None):
        """Raw descriptors G with one thread per (atom, neighbour), atomic updates
        of G_i (the hierarchical level of the parallelism ablation)."""
        n = int(pos.shape[0])
        _need(pos, torch.float32, (n, 3), "pos", self.device)
        _need(types, torch.int32, (n,), "types", self.device)
        G = torch.empty((n, self.n_g), dtype=torch.float32, device=torch.device("cuda", self.device))
        b, bp = self._box(box)
        self._check(self._lib.nnp_descriptors_pair(self.h, n, _ptr(pos), _ptr(types), bp, _ptr(G), _stream(stream)))
        return G

    def descriptors_cell(self, pos, types, box, stream=None):
        """Raw descriptors G with one CTA per cell, neighbours found in a shared
        copy of the cell's stencil (the CTA-per-cell level of the ablation)."""
        n = int(pos.shape[0])
        _need(pos, torch.float32, (n, 3), "pos", self.device)
        _need(types, torch.int32, (n,), "types", self.device)
        G = torch.empty((n, self.n_g), dtype=torch.float32, device=torch.device("cuda", self.device))
        b, bp = self._box(box)
        self._check(self._lib.nnp_descriptors_cell(self.h, n, _ptr(pos), _ptr(types), bp, _ptr(G), _stream(stream)))
        return G

    def step(self, pos, vel, types, box, dt, n_steps, log=True, stream=None):
        """n_steps velocity-Verlet steps in place; returns the (PE, KE) log [n_steps+1, 2] (fp64)."""
        n = int(pos.shape[0])
        _need(pos, torch.float32, (n, 3), "pos", self.device)
        _need(vel, torch.float32, (n, 3), "vel", self.device)
        _need(types, torch.int32, (n,), "types", self.device)
        lg = torch.empty((n_steps + 1, 2), dtype=torch.float64, device=pos.device) if log else None
        b, bp = self._box(box)
        self._check(self._lib.nnp_step(self.h, n, _ptr(pos), _ptr(vel), _ptr(types), bp, float(dt), int(n_steps),
                                       _ptr(lg), _stream(stream)))
        return lg

    # --------------------------------------------------------------- batches
    @staticmethod
    def _layout(starts, boxes):
        st = np.ascontiguousarray(np.asarray(starts, np.int32).reshape(-1))
        bx = np.ascontiguousarray(np.asarray(boxes, np.float64).reshape(-1, 3))
        if st.size != bx.shape[0] + 1:
            raise ValueError("starts must have n_systems + 1 entries")
        return st, bx

    def compute_batch(self, pos, types, starts, boxes, forces=True, atom_energy=False, stream=None):
        """Energies [B] (fp64), forces and per-atom energies of a batch of systems."""
        st, bx = self._layout(starts, boxes)
        n = int(st[-1])
        _need(pos, torch.float32, (n, 3), "pos", self.device)
        _need(types, torch.int32, (n,), "types", self.device)
        dev = pos.device
        out = {"energy": torch.empty(len(bx), dtype=torch.float64, device=dev),
               "F": torch.empty((n, 3), dtype=torch.float32, device=dev) if forces else None,
               "Ei": torch.empty(n, dtype=torch.float32, device=dev) if atom_energy else None}
        self._check(self._lib.nnp_compute_batch(
            self.h, len(bx), st.ctypes.data_as(_capi.c_int_p), bx.ctypes.data_as(_capi.c_double_p), _ptr(pos),
            _ptr(types), _ptr(out["energy"]), _ptr(out["Ei"]), _ptr(out["F"]), _stream(stream)))
        return out

    def param_grad(self, pos, types, starts, boxes, dLdE=None, dLdF=None, stream=None):
        """sum_b dLdE_b dE_b/dtheta + sum_m dLdF_m . dF_m/dtheta  (float32 [num_params])."""
        st, bx = self._layout(starts, boxes)
        n = int(st[-1])
        _need(pos, torch.float32, (n, 3), "pos", self.device)
        _need(types, torch.int32, (n,), "types", self.device)
        if dLdE is not None:
            _need(dLdE, torch.float64, (len(bx),), "dLdE", self.device)
        if dLdF is not None:
            _need(dLdF, torch.float32, (n, 3), "dLdF", self.device)
        g = torch.empty(self.num_params, dtype=torch.float32, device=pos.device)
        self._check(self._lib.nnp_param_grad(
            self.h, len(bx), st.ctypes.data_as(_capi.c_int_p), bx.ctypes.data_as(_capi.c_double_p), _ptr(pos),
            _ptr(types), _ptr(dLdE), _ptr(dLdF), _ptr(g), _stream(stream)))
        return g

    def set_weights(self, w, stream=None):
        _need(w, torch.float32, (self.num_params,), "weights", self.device)
        self._check(self._lib.nnp_set_weights(self.h, _ptr(w), _stream(stream)))

    def profile(self, enable=True):
        """Start (clearing totals) or stop per-kernel-group device timing."""
        self._check(self._lib.nnp_profile(self.h, 1 if enable else 0))

    def kernel_times(self):
        """{group name: (total ms, launches)} since profile(True)."""
        k = self._lib.nnp_num_kernel_groups()
        ms = (ctypes.c_double * k)()
        n = (ctypes.c_longlong * k)()
        m = self._lib.nnp_kernel_times(self.h, k, ms, n)
        if m < 0:
            self._check(m)
        return {self._lib.nnp_kernel_group_name(i).decode(): (ms[i], n[i]) for i in range(m)}

    def stats(self):
        s = _capi.Stats()
        self._check(self._lib.nnp_get_stats(self.h, ctypes.byref(s)))
        return {k: (float(getattr(s, k)) if t is ctypes.c_double else int(getattr(s, k)))
                for k, t in _capi.Stats._fields_}
