"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the benchmark.

This module holds no arithmetic of the method: it only draws positions, types,
velocities, weights and lists descriptor parameter sets.  The descriptor scaling
constants (mu, s) are stored data written by ``oracle/calibrate_scaling.py``.

The paper's trained n2p2 models and QM data (water, Ni, Cu, Si, Ge, Li, Mo;
Sec. 3.3) are not available, so random-weight models with the same structure
stand in for them: a two-element water-like model (cutoff 6.0 A) and a
single-element FCC-metal-like model (cutoff 5.5 A).
"""
from __future__ import annotations

import json
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
KB_EV = 8.617333262e-5           # Boltzmann constant, eV/K
ACC = 9.64853321233100e-3         # 1 eV/(A amu) in A/fs^2
WATER_DENSITY_ATOMS = 3 * 0.0334277  # atoms per A^3 at 1.0 g/cm^3 (0.03343 molecules/A^3)
WATER_CELL = 12.42                # A, 64 molecules at liquid density
MASS = {"O": 15.999, "H": 1.008, "M": 58.6934}

# Seeds of every preset (fixed).
SEED_WATER_MODEL = 1001
SEED_TEACHER_MODEL = 2002
SEED_FCC_MODEL = 3003
SEED_WATER_TINY = 11
SEED_WATER_LATTICE = 12
SEED_FCC = 13
SEED_TRAIN = 14
SEED_VEL = 15


# ----------------------------------------------------------------- descriptors
def radial_etas(n, lo=0.001, hi=0.5):
    """eta_m = lo * (hi/lo)^(m/(n-1)), m = 0..n-1 (log-spaced)."""
    return [lo * (hi / lo) ** (m / (n - 1)) for m in range(n)]


def water_sf_set(resolved=False):
    """Per element (O=0, H=1): 8 radial G2 per neighbour element + 14 narrow angular.

    Angular: for eta in {0.001, 0.01}: lambda=+1 with zeta in {1,2,4,16} and
    lambda=-1 with zeta in {1,2,4}; not resolved by neighbour element: n_G = 30.
    resolved=True: the same 14 for each neighbour-element pair (O,O), (O,H),
    (H,H): n_G = 16 + 42 = 58.
    """
    pairs = ((0, 0), (0, 1), (1, 1)) if resolved else ((-1, -1),)
    per = []
    for _centre in range(2):
        rows = []
        for nb in range(2):
            for eta in radial_etas(8):
                rows.append({"type": "radial", "e1": nb, "e2": -1, "eta": eta, "rs": 0.0})
        for e1, e2 in pairs:
            for eta in (0.001, 0.01):
                for lam, zetas in ((1.0, (1, 2, 4, 16)), (-1.0, (1, 2, 4))):
                    for z in zetas:
                        rows.append({"type": "narrow", "e1": e1, "e2": e2, "eta": eta, "zeta": float(z),
                                     "lambda": lam})
        per.append(rows)
    return per


def fcc_sf_set():
    """One element: 16 radial G2 (eta log-spaced 0.001-0.5) + 24 wide angular.

    Wide angular: zeta in {1,2,4,16} x lambda in {+1,-1} x eta in {0.001, 0.01, 0.05}.  n_G = 40.
    """
    rows = []
    for eta in radial_etas(16):
        rows.append({"type": "radial", "e1": -1, "e2": -1, "eta": eta, "rs": 0.0})
    for eta in (0.001, 0.01, 0.05):
        for lam in (1.0, -1.0):
            for z in (1, 2, 4, 16):
                rows.append({"type": "wide", "e1": -1, "e2": -1, "eta": eta, "zeta": float(z), "lambda": lam})
    return [rows]


def random_weights(widths, n_elem, seed):
    """Packed per-element parameters, W ~ N(0, 1/fan_in) and b ~ N(0, 1/fan_in).

    Layout per element: for each layer l, W_l [out][in] row-major, then b_l [out].
    """
    rng = np.random.default_rng(seed)
    out = []
    for _e in range(n_elem):
        parts = []
        for l in range(len(widths) - 1):
            fin, fout = widths[l], widths[l + 1]
            parts.append(rng.normal(0.0, 1.0 / np.sqrt(fin), size=fout * fin))
            parts.append(rng.normal(0.0, 1.0 / np.sqrt(fin), size=fout))
        out.append(np.concatenate(parts))
    return out


def _scaling(name, sf):
    path = os.path.join(_HERE, "data", "sf_scaling_%s.json" % name)
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return [np.asarray(x, np.float64) for x in d["mu"]], [np.asarray(x, np.float64) for x in d["s"]]
    # identity scaling until calibrated (only the calibration script uses this)
    return [np.zeros(len(r)) for r in sf], [np.ones(len(r)) for r in sf]


def water_model(seed=SEED_WATER_MODEL, hidden=(25, 25), resolved=False):
    """Water-like model; resolved=True takes the element-pair-resolved angular set (n_G = 58)."""
    sf = water_sf_set(resolved)
    name = "water_resolved" if resolved else "water"
    mu, s = _scaling(name, sf)
    widths = [len(sf[0]), *hidden, 1]
    return {"name": name, "elements": ["O", "H"], "masses": [MASS["O"], MASS["H"]], "cutoff": 6.0,
            "sf": sf, "sf_mu": mu, "sf_s": s, "widths": widths, "weights": random_weights(widths, 2, seed)}


def fcc_model(seed=SEED_FCC_MODEL, hidden=(30, 30)):
    sf = fcc_sf_set()
    mu, s = _scaling("fcc", sf)
    widths = [40, *hidden, 1]
    return {"name": "fcc", "elements": ["M"], "masses": [MASS["M"]], "cutoff": 5.5,
            "sf": sf, "sf_mu": mu, "sf_s": s, "widths": widths, "weights": random_weights(widths, 1, seed)}


# ------------------------------------------------------------------ structures
def _min_image_d2(p, q, box):
    d = q - p
    d -= box * np.round(d / box)
    return np.einsum("...k,...k->...", d, d)


def water_random(n_mol=64, box=WATER_CELL, min_sep=0.9, seed=SEED_WATER_TINY):
    """Random sequential placement of 3*n_mol atoms (1/3 O, 2/3 H) in a cubic box.

    A candidate is rejected when any minimum-image distance to the atoms placed so
    far is below min_sep.  Types are assigned in a seeded random order.
    """
    rng = np.random.default_rng(seed)
    n = 3 * n_mol
    L = np.array([box, box, box], np.float64)
    pos = np.zeros((n, 3))
    k = 0
    tries = 0
    while k < n:
        c = rng.uniform(0.0, 1.0, 3) * L
        tries += 1
        if tries > 200000 * n:
            raise RuntimeError("placement failed")
        if k and np.min(_min_image_d2(pos[:k], c, L)) < min_sep * min_sep:
            continue
        pos[k] = c
        k += 1
    types = np.array([0] * n_mol + [1] * (2 * n_mol), np.int32)
    rng.shuffle(types)
    return pos, types, L


def _water_base_cell(rng, box=WATER_CELL):
    """64 molecules: O on a 4x4x4 grid, two H at 0.9572 A with HOH 104.52 deg, random orientation."""
    sp = box / 4.0
    r_oh = 0.9572
    half = np.deg2rad(104.52) / 2.0
    pos, types = [], []
    for ix in range(4):
        for iy in range(4):
            for iz in range(4):
                o = (np.array([ix, iy, iz]) + 0.5) * sp
                q = rng.normal(size=4)
                q /= np.linalg.norm(q)
                a, b, c, d = q
                R = np.array([[a * a + b * b - c * c - d * d, 2 * (b * c - a * d), 2 * (b * d + a * c)],
                              [2 * (b * c + a * d), a * a - b * b + c * c - d * d, 2 * (c * d - a * b)],
                              [2 * (b * d - a * c), 2 * (c * d + a * b), a * a - b * b - c * c + d * d]])
                h1 = R @ np.array([r_oh * np.sin(half), 0.0, r_oh * np.cos(half)])
                h2 = R @ np.array([-r_oh * np.sin(half), 0.0, r_oh * np.cos(half)])
                pos += [o, o + h1, o + h2]
                types += [0, 1, 1]
    return np.array(pos), np.array(types, np.int32)


def water_lattice(reps=(8, 8, 9), sigma=0.1, seed=SEED_WATER_LATTICE):
    """The 192-atom molecular cell replicated reps times, then N(0, sigma) noise on every coordinate.

    110,592 atoms = reps (8,8,9); 2,064,384 = (16,24,28); 1,048,320 = (13,20,21).
    Atom order: replica-major (x fastest), molecule order inside a replica.
    """
    rng = np.random.default_rng(seed)
    base, bt = _water_base_cell(rng)
    nx, ny, nz = reps
    ix, iy, iz = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    shifts = np.stack([ix.ravel(order="F"), iy.ravel(order="F"), iz.ravel(order="F")], 1) * WATER_CELL
    pos = (shifts[:, None, :] + base[None, :, :]).reshape(-1, 3)
    pos += rng.normal(0.0, sigma, size=pos.shape)
    types = np.tile(bt, nx * ny * nz)
    box = np.array([nx, ny, nz], np.float64) * WATER_CELL
    pos -= box * np.floor(pos / box)
    return pos, types, box


def fcc(ncell=(10, 10, 10), a=3.52, sigma=0.05, seed=SEED_FCC, perfect=False):
    """FCC crystal with lattice constant a, ncell unit cells per side, Gaussian displacements."""
    nx, ny, nz = ncell
    basis = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]])
    ix, iy, iz = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    cells = np.stack([ix.ravel(order="F"), iy.ravel(order="F"), iz.ravel(order="F")], 1)
    pos = ((cells[:, None, :] + basis[None, :, :]) * a).reshape(-1, 3)
    if not perfect:
        rng = np.random.default_rng(seed)
        pos = pos + rng.normal(0.0, sigma, size=pos.shape)
    box = np.array([nx, ny, nz], np.float64) * a
    pos -= box * np.floor(pos / box)
    return pos, np.zeros(len(pos), np.int32), box


def train_batch(n_configs=256, mol_range=(22, 170), min_sep=0.9, seed=SEED_TRAIN):
    """Ragged batch of random water-like configurations at liquid density.

    Each configuration has n_mol ~ U{mol_range} molecules (66-510 atoms), a cubic
    box of edge (3 n_mol / rho)^(1/3), and random placement as in water_random.
    """
    rng = np.random.default_rng(seed)
    out = []
    for _b in range(n_configs):
        nm = int(rng.integers(mol_range[0], mol_range[1] + 1))
        L = (3 * nm / WATER_DENSITY_ATOMS) ** (1.0 / 3.0)
        p, t, box = water_random(nm, L, min_sep, seed=int(rng.integers(1 << 30)))
        out.append((p, t, box))
    return out


def maxwell_boltzmann(types, masses, T=300.0, seed=SEED_VEL):
    """Velocities (A/fs) at temperature T with zero total momentum."""
    rng = np.random.default_rng(seed)
    m = np.asarray(masses, np.float64)[np.asarray(types)]
    sd = np.sqrt(KB_EV * T * ACC / m)
    v = rng.normal(size=(len(m), 3)) * sd[:, None]
    p = (m[:, None] * v).sum(0) / m.sum()
    return v - p[None, :]


# Named presets of the benchmark workloads.
PRESETS = {
    "water_tiny": dict(kind="water_random", n_atoms=192),
    "water_110k": dict(kind="water_lattice", reps=(8, 8, 9), n_atoms=110592),
    "water_2m": dict(kind="water_lattice", reps=(16, 24, 28), n_atoms=2064384),
    "water_1m": dict(kind="water_lattice", reps=(13, 20, 21), n_atoms=1048320),
    "fcc_1m": dict(kind="fcc", ncell=(64, 64, 64), n_atoms=1048576),
    "fcc_4k": dict(kind="fcc", ncell=(10, 10, 10), n_atoms=4000),
}


def make(name):
    p = PRESETS[name]
    if p["kind"] == "water_random":
        return water_random()
    if p["kind"] == "water_lattice":
        return water_lattice(p["reps"])
    if p["kind"] == "fcc":
        return fcc(p["ncell"])
    raise KeyError(name)
