"""FP64 CPU oracle for the Behler-Parrinello NNP hot path (arXiv 2002.00054).

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package; the product path never
does.  It shares no code with the CUDA library: the C source ``nnp_oracle.c`` is
compiled on its own into ``liboracle.so`` and loaded through ctypes here.

Functions and the paper passages they follow:
  neighbors()      -- per-atom neighbour entries within r_c, periodic images
                      included (brute force or cell list; Sec. 3.2 uses a
                      Cabana neighbour list, construction not described).
  compute()        -- descriptors G (Fig. 1b step 1, the radial formula; the
                      angular "extra loop over neighbours of neighbours" of
                      Sec. 3.1), network energies E_i (step 2), total energy
                      (E_system += E_i), forces by the chain rule of step 3 and
                      the pair virial.
  compute_subset() -- the same outputs for a chosen set of atoms only.
  compute_owned()  -- energy and virial of the first n_own atoms' energies
                      (a spatial domain's owned atoms; Sec. 5's multi-node
                      outlook), Ei and F of every atom.
  mlp()            -- the per-element network alone (Sec. 3.1, "~30 x 2").
  md()             -- velocity-Verlet NVE (energy conservation, Sec. 4.2).
  param_grad()     -- force-matching parameter gradient (energy term plus the
                      reverse-over-forward double backward of the force term).

Parity status: every function above is pinned by the CPU tests in
``tests/test_oracle_pins.py`` (closed forms, lattice sums, invariances, finite
differences, a library network, brute-force neighbours, energy drift).  The
full descriptor set has no printed worked example in the paper; beyond those
pins its numerical values are not fixed by the paper itself.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nnp_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

MAXE = 8
MAXL = 8
SF_TYPE_CODE = {"radial": 2, "narrow": 3, "wide": 4}


def build(force: bool = False) -> str:
    """Compile nnp_oracle.c into liboracle.so (gcc, -O2, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp.%d" % os.getpid()
        cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c99", "-D_GNU_SOURCE",
               "-o", tmp, _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


class _Model(ctypes.Structure):
    _fields_ = [
        ("n_elem", ctypes.c_int),
        ("rc", ctypes.c_double),
        ("n_sf", ctypes.c_int * MAXE),
        ("sf_off", ctypes.c_int * MAXE),
        ("sf_type", ctypes.POINTER(ctypes.c_int)),
        ("sf_e1", ctypes.POINTER(ctypes.c_int)),
        ("sf_e2", ctypes.POINTER(ctypes.c_int)),
        ("sf_eta", ctypes.POINTER(ctypes.c_double)),
        ("sf_rs", ctypes.POINTER(ctypes.c_double)),
        ("sf_zeta", ctypes.POINTER(ctypes.c_double)),
        ("sf_lambda", ctypes.POINTER(ctypes.c_double)),
        ("sf_mu", ctypes.POINTER(ctypes.c_double)),
        ("sf_s", ctypes.POINTER(ctypes.c_double)),
        ("n_layers", ctypes.c_int),
        ("width", ctypes.c_int * (MAXL + 1)),
        ("w_off", ctypes.c_int * MAXE),
        ("w", ctypes.POINTER(ctypes.c_double)),
    ]


class _System(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int),
        ("pos", ctypes.POINTER(ctypes.c_double)),
        ("type", ctypes.POINTER(ctypes.c_int)),
        ("box", ctypes.c_double * 3),
    ]


class _Out(ctypes.Structure):
    _fields_ = [
        ("G", ctypes.POINTER(ctypes.c_double)),
        ("dEdG", ctypes.POINTER(ctypes.c_double)),
        ("Ei", ctypes.POINTER(ctypes.c_double)),
        ("F", ctypes.POINTER(ctypes.c_double)),
        ("virial", ctypes.POINTER(ctypes.c_double)),
        ("energy", ctypes.POINTER(ctypes.c_double)),
        ("ldg", ctypes.c_int),
    ]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.POINTER
            lib.or_neighbors.argtypes = [P(_System), ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                         P(ctypes.c_int), P(ctypes.c_int), P(ctypes.c_double)]
            lib.or_neighbors.restype = ctypes.c_int
            lib.or_mlp.argtypes = [P(_Model), ctypes.c_int, P(ctypes.c_double), P(ctypes.c_double)]
            lib.or_mlp.restype = ctypes.c_double
            lib.or_compute.argtypes = [P(_Model), P(_System), ctypes.c_int, P(_Out)]
            lib.or_compute.restype = ctypes.c_int
            lib.or_compute_owned.argtypes = [P(_Model), P(_System), ctypes.c_int, ctypes.c_int, P(_Out)]
            lib.or_compute_owned.restype = ctypes.c_int
            lib.or_compute_subset.argtypes = [P(_Model), P(_System), ctypes.c_int, P(ctypes.c_ubyte), P(_Out)]
            lib.or_compute_subset.restype = ctypes.c_int
            lib.or_md.argtypes = [P(_Model), P(_System), P(ctypes.c_double), P(ctypes.c_double),
                                  P(ctypes.c_double), ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                  P(ctypes.c_double)]
            lib.or_md.restype = ctypes.c_int
            lib.or_param_grad.argtypes = [P(_Model), P(_System), ctypes.c_int, ctypes.c_double,
                                          P(ctypes.c_double), P(ctypes.c_double)]
            lib.or_param_grad.restype = ctypes.c_int
            lib.or_n_params_elem.argtypes = [P(_Model)]
            lib.or_n_params_elem.restype = ctypes.c_int
            lib.or_set_threads.argtypes = [ctypes.c_int]
            lib.or_set_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def set_threads(n: int = 0) -> int:
    """Set the OpenMP thread count (n <= 0 keeps it); returns the count in use."""
    return _load().or_set_threads(int(n))


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _iptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


class Model:
    """Marshals a model description (see ``workloads``) into the oracle's struct."""

    def __init__(self, model: dict):
        sf = model["sf"]
        ne = len(sf)
        if ne > MAXE:
            raise ValueError("too many elements")
        widths = list(model["widths"])
        if len(widths) - 1 > MAXL:
            raise ValueError("too many layers")
        rows = [d for e in range(ne) for d in sf[e]]
        self._type = np.array([SF_TYPE_CODE[d["type"]] for d in rows], dtype=np.int32)
        self._e1 = np.array([d.get("e1", -1) for d in rows], dtype=np.int32)
        self._e2 = np.array([d.get("e2", -1) for d in rows], dtype=np.int32)
        self._eta = np.array([d["eta"] for d in rows], dtype=np.float64)
        self._rs = np.array([d.get("rs", 0.0) for d in rows], dtype=np.float64)
        self._zeta = np.array([d.get("zeta", 1.0) for d in rows], dtype=np.float64)
        self._lam = np.array([d.get("lambda", 1.0) for d in rows], dtype=np.float64)
        self._mu = np.ascontiguousarray(np.concatenate([np.asarray(m, np.float64) for m in model["sf_mu"]]))
        self._s = np.ascontiguousarray(np.concatenate([np.asarray(m, np.float64) for m in model["sf_s"]]))
        self._w = np.ascontiguousarray(np.concatenate([np.asarray(w, np.float64) for w in model["weights"]]))
        st = _Model()
        st.n_elem = ne
        st.rc = float(model["cutoff"])
        off = 0
        for e in range(ne):
            st.n_sf[e] = len(sf[e])
            st.sf_off[e] = off
            off += len(sf[e])
        st.sf_type = _iptr(self._type)
        st.sf_e1 = _iptr(self._e1)
        st.sf_e2 = _iptr(self._e2)
        st.sf_eta = _dptr(self._eta)
        st.sf_rs = _dptr(self._rs)
        st.sf_zeta = _dptr(self._zeta)
        st.sf_lambda = _dptr(self._lam)
        st.sf_mu = _dptr(self._mu)
        st.sf_s = _dptr(self._s)
        st.n_layers = len(widths) - 1
        for l, w in enumerate(widths):
            st.width[l] = int(w)
        self.n_params_elem = 0
        st.w = _dptr(self._w)
        self.st = st
        self.n_params_elem = _load().or_n_params_elem(ctypes.byref(st))
        for e in range(ne):
            st.w_off[e] = e * self.n_params_elem
        if self._w.size != ne * self.n_params_elem:
            raise ValueError("weights size %d != %d" % (self._w.size, ne * self.n_params_elem))
        self.n_elem = ne
        self.n_sf = [len(x) for x in sf]
        self.masses = np.asarray(model["masses"], np.float64)
        self.cutoff = float(model["cutoff"])


class _Sys:
    def __init__(self, pos, types, box):
        self.pos = np.ascontiguousarray(np.asarray(pos, np.float64).reshape(-1, 3))
        self.types = np.ascontiguousarray(np.asarray(types, np.int32).reshape(-1))
        if self.types.size != self.pos.shape[0]:
            raise ValueError("pos/types size mismatch")
        st = _System()
        st.n = self.pos.shape[0]
        st.pos = _dptr(self.pos)
        st.type = _iptr(self.types)
        for a in range(3):
            st.box[a] = float(box[a])
        self.st = st


def _as_model(model):
    return model if isinstance(model, Model) else Model(model)


NB_BRUTE, NB_CELL, NB_AUTO = 0, 1, 2


def neighbors(pos, box, rc, mode=NB_BRUTE, cap=512):
    """Neighbour entries of every atom: list of (j array, d array [M,3])."""
    s = _Sys(pos, np.zeros(len(pos), np.int32), box)
    n = s.st.n
    counts = np.zeros(n, np.int32)
    js = np.zeros((n, cap), np.int32)
    d = np.zeros((n, cap, 3), np.float64)
    mx = _load().or_neighbors(ctypes.byref(s.st), float(rc), int(mode), int(cap), _iptr(counts), _iptr(js), _dptr(d))
    if mx < 0:
        raise RuntimeError("oracle neighbour build failed")
    if mx > cap:
        return neighbors(pos, box, rc, mode, cap=mx)
    return [(js[i, :counts[i]].copy(), d[i, :counts[i]].copy()) for i in range(n)]


def mlp(model, elem, x):
    """(E, dE/dx) of element 'elem''s network at scaled input x (fp64)."""
    m = _as_model(model)
    x = np.ascontiguousarray(np.asarray(x, np.float64))
    dx = np.zeros_like(x)
    E = _load().or_mlp(ctypes.byref(m.st), int(elem), _dptr(x), _dptr(dx))
    return E, dx


def compute(model, pos, types, box, nbmode=NB_AUTO):
    """Energy, per-atom energies, forces, virial, descriptors and dE/dG (fp64).

    Returns a dict with keys energy, Ei [N], F [N,3], virial [3,3] (W_ab = -sum d^a g^b),
    G [N, n_G], dEdG [N, n_G].
    """
    m = _as_model(model)
    s = _Sys(pos, types, box)
    n = s.st.n
    ldg = max(m.n_sf)
    G = np.zeros((n, ldg))
    dEdG = np.zeros((n, ldg))
    Ei = np.zeros(n)
    F = np.zeros((n, 3))
    vir = np.zeros(9)
    E = np.zeros(1)
    o = _Out(_dptr(G), _dptr(dEdG), _dptr(Ei), _dptr(F), _dptr(vir), _dptr(E), ldg)
    if _load().or_compute(ctypes.byref(m.st), ctypes.byref(s.st), int(nbmode), ctypes.byref(o)):
        raise RuntimeError("oracle compute failed")
    return {"energy": float(E[0]), "Ei": Ei, "F": F, "virial": vir.reshape(3, 3), "G": G, "dEdG": dEdG}


def compute_owned(model, pos, types, box, n_own, nbmode=NB_AUTO):
    """compute() with the energy and the virial summed over the energies of the
    first n_own atoms only (a domain's owned atoms, its halo copies after them);
    Ei and F for every atom."""
    m = _as_model(model)
    s = _Sys(pos, types, box)
    n = s.st.n
    ldg = max(m.n_sf)
    null = ctypes.POINTER(ctypes.c_double)()
    Ei = np.zeros(n)
    F = np.zeros((n, 3))
    vir = np.zeros(9)
    E = np.zeros(1)
    o = _Out(null, null, _dptr(Ei), _dptr(F), _dptr(vir), _dptr(E), ldg)
    if _load().or_compute_owned(ctypes.byref(m.st), ctypes.byref(s.st), int(nbmode), int(n_own), ctypes.byref(o)):
        raise RuntimeError("oracle compute_owned failed")
    return {"energy": float(E[0]), "Ei": Ei, "F": F, "virial": vir.reshape(3, 3)}


def compute_subset(model, pos, types, box, idx, nbmode=NB_AUTO):
    """Ei, F, G and dEdG for the atoms idx only (rows in the order of idx)."""
    m = _as_model(model)
    s = _Sys(pos, types, box)
    n = s.st.n
    idx = np.asarray(idx, np.int64)
    tgt = np.zeros(n, np.uint8)
    tgt[idx] = 1
    ldg = max(m.n_sf)
    G = np.zeros((n, ldg))
    dEdG = np.zeros((n, ldg))
    Ei = np.zeros(n)
    F = np.zeros((n, 3))
    null = ctypes.POINTER(ctypes.c_double)()
    o = _Out(_dptr(G), _dptr(dEdG), _dptr(Ei), _dptr(F), null, null, ldg)
    if _load().or_compute_subset(ctypes.byref(m.st), ctypes.byref(s.st), int(nbmode),
                                 tgt.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte)), ctypes.byref(o)):
        raise RuntimeError("oracle compute_subset failed")
    return {"Ei": Ei[idx], "F": F[idx], "G": G[idx], "dEdG": dEdG[idx]}


def md(model, pos, vel, types, box, dt, nsteps, nbmode=NB_AUTO):
    """Velocity-Verlet NVE; returns (pos, vel, log[nsteps+1, 2] of (PE, KE))."""
    m = _as_model(model)
    s = _Sys(pos, types, box)
    p = s.pos.copy()
    v = np.ascontiguousarray(np.asarray(vel, np.float64).reshape(-1, 3)).copy()
    log = np.zeros((nsteps + 1, 2))
    masses = np.ascontiguousarray(m.masses)
    if _load().or_md(ctypes.byref(m.st), ctypes.byref(s.st), _dptr(p), _dptr(v), _dptr(masses),
                     float(dt), int(nsteps), int(nbmode), _dptr(log)):
        raise RuntimeError("oracle md failed")
    return p, v, log


def param_grad(model, pos, types, box, dLdE, u=None, nbmode=NB_AUTO):
    """dLdE * dE/dtheta + sum_m u_m . dF_m/dtheta for one system (packed layout)."""
    m = _as_model(model)
    s = _Sys(pos, types, box)
    g = np.zeros(m.n_elem * m.n_params_elem)
    uu = None
    if u is not None:
        uu = np.ascontiguousarray(np.asarray(u, np.float64).reshape(-1, 3))
    up = _dptr(uu) if uu is not None else ctypes.POINTER(ctypes.c_double)()
    if _load().or_param_grad(ctypes.byref(m.st), ctypes.byref(s.st), int(nbmode), float(dLdE), up, _dptr(g)):
        raise RuntimeError("oracle param_grad failed")
    return g
