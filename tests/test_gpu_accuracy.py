"""Descriptor accuracy at the level of a few float32 ulp, on configurations
whose descriptors have closed forms (Fig. 1b step 1; the standard radial and
wide angular forms): a dimer gives G2 = exp(-eta r^2) f_c(r) for every radial
descriptor, and an isolated trimer gives each wide angular descriptor of the
centre atom as one term 2^(1-zeta) (1 + lambda cos)^zeta exp(-eta (r_ij^2 +
r_ik^2)) f_c(r_ij) f_c(r_ik).  The scaled descriptors G~ = (G - mu)/s carry
|mu/s| up to ~18 in the FCC model, so a descriptor must be accurate to about
an ulp for the per-atom energy to meet 1e-5; these cases test exactly that,
including the near-collinear triplets where (1 + lambda cos)^16 amplifies an
error of cos sixteen-fold."""
import numpy as np
import pytest
import torch

import workloads
from tests.gpuhelp import to_dev

pytestmark = pytest.mark.gpu

U = 2.0 ** -24
BOX = np.array([40.0, 40.0, 40.0])


def _fc(r, rc):
    return np.where(r < rc, 0.5 * (np.cos(np.pi * r / rc) + 1.0), 0.0)


@pytest.fixture(scope="module")
def fcc():
    from paper_2002_00054_b300 import NNP
    m = workloads.fcc_model()
    return m, NNP(m)


def _f32(x):
    return np.asarray(x, np.float32).astype(np.float64)


def test_dimer_radial_to_an_ulp(fcc):
    m, nnp = fcc
    rc = m["cutoff"]
    rng = np.random.default_rng(3)
    errs = []
    for r in np.linspace(0.8, rc - 0.05, 40):
        u = rng.normal(size=3)
        u /= np.linalg.norm(u)
        pos = _f32([[12.0, 13.0, 14.0], [12.0 + r * u[0], 13.0 + r * u[1], 14.0 + r * u[2]]])
        d = pos[1] - pos[0]   # exact: both coordinates are floats within a factor 2
        rr = np.sqrt(d @ d)
        G, _ = nnp.descriptors(*to_dev(pos, np.zeros(2, np.int32)), BOX)
        G = G.double().cpu().numpy()[0]
        # f_c = cos^2 is formed from cos(pi r / (2 rc)) to ~2^-28 absolute: relative to
        # f_c that is 2 x 0.07 ulp / cos, which grows as r -> rc where f_c -> 0
        cth = np.cos(np.pi * rr / (2 * rc))
        for s, sd in enumerate(m["sf"][0]):
            if sd["type"] != "radial":
                continue
            want = np.exp(-sd["eta"] * (rr - sd.get("rs", 0.0)) ** 2) * _fc(rr, rc)
            errs.append((abs(G[s] - want) / want / U, 2.5 + 0.15 / cth))
    e = np.array(errs)
    # one float rounding of the output plus about an ulp of arithmetic
    assert np.all(e[:, 0] <= e[:, 1]), e[np.argmax(e[:, 0] - e[:, 1])]
    assert e[:, 0].mean() <= 0.8, e[:, 0].mean()


@pytest.mark.parametrize("theta_deg", [60.0, 90.0, 120.0, 150.0, 175.0, 179.5, 180.0])
def test_trimer_wide_angular_to_a_few_ulp(fcc, theta_deg):
    m, nnp = fcc
    rc = m["cutoff"]
    rng = np.random.default_rng(int(theta_deg * 10))
    errs = []
    for _ in range(6):
        ra, rb = rng.uniform(2.2, 5.0, 2)
        # a random orientation of the plane of the triplet
        q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
        th = np.radians(theta_deg)
        a = q @ np.array([ra, 0.0, 0.0])
        b = q @ np.array([rb * np.cos(th), rb * np.sin(th), 0.0])
        c0 = np.array([15.0, 16.0, 17.0])
        pos = _f32([c0, c0 + a, c0 + b])
        if np.linalg.norm(pos[1] - pos[2]) < 1.0:
            continue
        da, db = pos[1] - pos[0], pos[2] - pos[0]
        r1, r2 = np.sqrt(da @ da), np.sqrt(db @ db)
        cos = (da @ db) / (r1 * r2)
        G, _ = nnp.descriptors(*to_dev(pos, np.zeros(3, np.int32)), BOX)
        G = G.double().cpu().numpy()[0]
        for s, sd in enumerate(m["sf"][0]):
            if sd["type"] != "wide":
                continue
            z, lam, eta = sd["zeta"], sd["lambda"], sd["eta"]
            want = 2.0 ** (1 - z) * (1 + lam * cos) ** z * np.exp(-eta * (r1 * r1 + r2 * r2)) \
                * _fc(r1, rc) * _fc(r2, rc)
            if want < 1e-30:
                continue
            b = 1 + lam * cos
            # Error model of a term, in ulp: b = 2 - s with s = 1 -/+ cos formed as
            # |u_j -/+ u_k|^2 / 2 to ~2.5 ulp of its own size, so b's absolute error is
            # ~2.5 ulp x (2 - b), which vanishes for (anti)collinear triplets, the ones
            # that dominate zeta = 16, plus the unit vectors' direction rounding for
            # small b (~0.5 ulp absolute).  The power multiplies b's relative error by
            # zeta, its chain of squarings adds up to (zeta - 1)/2 ulp, and the other
            # factors and the output ~3 ulp.
            tol = 3.0 + 0.5 * z + z * 2.5 * (2.0 - b) / b + (z * 0.5 / b if b < 1.0 else 0.0)
            errs.append((abs(G[s] - want) / want / U, tol))
    assert len(errs) > 0
    e = np.array(errs)
    assert np.all(e[:, 0] <= e[:, 1]), e[np.argmax(e[:, 0] - e[:, 1])]
