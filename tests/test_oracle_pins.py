"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

Each test names what fixes the expected value: exact special values of the
cutoff, lattice coordination shells, right-angle / equilateral trimers built
from their angle, algebraic identities, symmetry (translation, rotation,
permutation; Sec. 2 of the paper), finite differences of the energy, a library
network (torch.nn.Sequential in float64), brute-force neighbours, perfect-FCC
symmetry and energy conservation (Sec. 4.2).
"""
import itertools
import math

import numpy as np
import pytest

import oracle
import workloads
from tests.modelkit import angular, model_from_rows, radial

BIG = np.array([40.0, 40.0, 40.0])


def _g(model, pos, types=None, box=BIG):
    pos = np.asarray(pos, float)
    if types is None:
        types = np.zeros(len(pos), np.int32)
    return oracle.compute(model, pos + 10.0, types, box)


# --------------------------------------------------------------- radial / cutoff
def test_dimer_special_values():
    """f_c(rc/2) = 1/2 and f_c(rc/3) = 3/4 exactly (cos(pi/2) = 0, cos(pi/3) = 1/2);
    with eta = ln 2 / r^2 the Gaussian is exactly 1/2."""
    rc = 6.0
    for r, eta, expect in [(3.0, 0.0, 0.5), (2.0, 0.0, 0.75), (3.0, math.log(2) / 9.0, 0.25),
                           (5.999999, 0.0, 0.0), (6.5, 0.0, 0.0)]:
        m = model_from_rows([[radial(eta)]], rc)
        res = _g(m, [[0, 0, 0], [r, 0, 0]])
        assert res["G"][0, 0] == pytest.approx(expect, abs=1e-11)
        assert res["G"][1, 0] == pytest.approx(expect, abs=1e-11)


def test_radial_shift_and_element_filter():
    """rs shifts the Gaussian centre: eta*(r-rs)^2 = 0 at r = rs; the element filter
    keeps only neighbours of the named element."""
    rc = 6.0
    rows = [radial(5.0, rs=3.0, e1=1), radial(0.0, e1=0)]
    m = model_from_rows([rows, rows], rc)
    res = _g(m, [[0, 0, 0], [3.0, 0, 0], [0, 3.0, 0]], types=np.array([0, 1, 0], np.int32))
    # atom 0 sees one element-1 neighbour at exactly rs (Gaussian = 1, fc = 1/2)
    assert res["G"][0, 0] == pytest.approx(0.5, abs=1e-12)
    # and one element-0 neighbour at 3 (fc = 1/2)
    assert res["G"][0, 1] == pytest.approx(0.5, abs=1e-12)


def test_simple_cubic_lattice_shells():
    """eta = 0, simple cubic spacing a: G2 = sum over coordination shells
    6, 12, 8, 6, 24 at a, a*sqrt2, a*sqrt3, 2a, a*sqrt5 (rc between sqrt5 a and sqrt6 a)."""
    a, rc = 2.0, 4.6
    n = 6
    g = np.array(list(itertools.product(range(n), repeat=3)), float) * a
    m = model_from_rows([[radial(0.0)]], rc)
    res = oracle.compute(m, g, np.zeros(len(g), np.int32), np.array([n * a] * 3))
    fc = lambda r: 0.5 * (math.cos(math.pi * r / rc) + 1.0)
    shells = [(6, a), (12, a * math.sqrt(2)), (8, a * math.sqrt(3)), (6, 2 * a), (24, a * math.sqrt(5))]
    expect = sum(k * fc(r) for k, r in shells)
    np.testing.assert_allclose(res["G"][:, 0], expect, rtol=1e-12)


# ------------------------------------------------------------------- angular
@pytest.mark.parametrize("theta_deg", [90.0, 60.0, 120.0, 180.0])
@pytest.mark.parametrize("kind", ["narrow", "wide"])
def test_trimer_from_angle(theta_deg, kind):
    """Isoceles trimer with legs a = rc/2 (f_c = 1/2 exactly) at angle theta:
    the centre's only pair has cos t = cos(theta), r_jk = 2 a sin(theta/2)."""
    rc, a = 6.0, 3.0
    th = math.radians(theta_deg)
    pos = [[0, 0, 0], [a, 0, 0], [a * math.cos(th), a * math.sin(th), 0]]
    eta = 0.02
    terms = [(z, l) for z in (1, 2, 4, 16) for l in (1.0, -1.0)]
    m = model_from_rows([[angular(kind, eta, z, l) for z, l in terms]], rc)
    res = _g(m, pos)
    rjk = 2 * a * math.sin(th / 2)
    ct = math.cos(th)
    for s, (z, l) in enumerate(terms):
        ang = 2.0 ** (1 - z) * (1 + l * ct) ** z
        if kind == "narrow":
            fjk = 0.5 * (math.cos(math.pi * rjk / rc) + 1.0) if rjk < rc else 0.0
            expect = ang * math.exp(-eta * (2 * a * a + rjk * rjk)) * 0.25 * fjk
        else:
            expect = ang * math.exp(-eta * 2 * a * a) * 0.25
        assert res["G"][0, s] == pytest.approx(expect, rel=1e-12, abs=1e-15)


def test_angular_lambda_identity():
    """(1 + c) + (1 - c) = 2 and (1 + c) - (1 - c) = 2c: zeta = 1 pairs of lambda = +-1
    sum to 2 * sum_{j<k} X f f f and differ by 2 * sum_{j<k} cos * X f f f, where the
    pair sums are taken here over brute-force neighbour vectors."""
    rc, eta = 6.0, 0.01
    pos, types, box = workloads.water_random()
    rows = [angular("narrow", eta, 1, 1.0), angular("narrow", eta, 1, -1.0)]
    m = model_from_rows([rows, rows], rc)
    res = oracle.compute(m, pos, types, box)
    nbs = oracle.neighbors(pos, box, rc, mode=oracle.NB_BRUTE)
    fc = lambda r: np.where(r < rc, 0.5 * (np.cos(np.pi * r / rc) + 1.0), 0.0)
    for i in (0, 7, 100):
        d = nbs[i][1]
        r = np.linalg.norm(d, axis=1)
        ja, kb = np.triu_indices(len(r), 1)
        rd = np.linalg.norm(d[kb] - d[ja], axis=1)
        c = np.einsum("ij,ij->i", d[ja], d[kb]) / (r[ja] * r[kb])
        xf = np.exp(-eta * (r[ja] ** 2 + r[kb] ** 2 + rd ** 2)) * fc(r[ja]) * fc(r[kb]) * fc(rd)
        assert res["G"][i, 0] + res["G"][i, 1] == pytest.approx(2 * xf.sum(), rel=1e-11)
        assert res["G"][i, 0] - res["G"][i, 1] == pytest.approx(2 * (c * xf).sum(), rel=1e-9, abs=1e-12)


def test_element_resolved_angular_classes():
    """Angular descriptors resolved by neighbour-element pair: on a trimer whose
    centre sees two neighbours of element 1, the (1, 1) class holds the whole
    unresolved value and the (0, 0) and (0, 1) classes are zero; on the water box
    the three classes of a two-element system partition the pair sum, so they add
    up to the unresolved descriptor (for every eta, lambda, zeta, and both kinds)."""
    rc, a = 6.0, 2.5
    th = math.radians(100.0)
    pos = np.array([[0, 0, 0], [a, 0, 0], [a * math.cos(th), a * math.sin(th), 0]], float)
    terms = [(eta, z, l) for eta in (0.001, 0.02) for z in (1, 2, 4, 16) for l in (1.0, -1.0)]
    for kind in ("narrow", "wide"):
        rows = [angular(kind, e, z, l) for e, z, l in terms]
        for e1, e2 in ((0, 0), (0, 1), (1, 1)):
            rows += [angular(kind, e, z, l, e1=e1, e2=e2) for e, z, l in terms]
        m = model_from_rows([rows, rows], rc)
        res = oracle.compute(m, pos, np.array([0, 1, 1], np.int32), np.array([50.0, 50.0, 50.0]))
        nt = len(terms)
        g = res["G"][0]
        assert np.all(np.abs(g[:nt]) > 0)
        np.testing.assert_array_equal(g[nt:2 * nt], 0.0)        # (0, 0)
        np.testing.assert_array_equal(g[2 * nt:3 * nt], 0.0)    # (0, 1)
        np.testing.assert_allclose(g[3 * nt:], g[:nt], rtol=1e-14)   # (1, 1)
        wpos, wtypes, wbox = workloads.water_random()
        res = oracle.compute(m, wpos, wtypes, wbox)
        G = res["G"]
        parts = G[:, nt:2 * nt] + G[:, 2 * nt:3 * nt] + G[:, 3 * nt:]
        np.testing.assert_allclose(parts, G[:, :nt], rtol=1e-12, atol=1e-300)
        # both classes with one O neighbour are populated in the water box
        assert np.all(np.abs(G[:, 2 * nt:3 * nt]).max(0) > 0)


# ---------------------------------------------------------------- neighbours
def test_neighbors_cell_equals_brute():
    pos, _t, box = workloads.fcc((4, 4, 4))
    rc = 5.5
    a = oracle.neighbors(pos, box, rc, mode=oracle.NB_BRUTE)
    b = oracle.neighbors(pos, box, rc, mode=oracle.NB_CELL)
    for (ja, da), (jb, db) in zip(a, b):
        ka = sorted((int(j), tuple(np.round(d, 9))) for j, d in zip(ja, da))
        kb = sorted((int(j), tuple(np.round(d, 9))) for j, d in zip(jb, db))
        assert ka == kb


@pytest.mark.parametrize("L,rc", [(3.0, 6.0), (4.0, 7.0), (9.0, 6.0)])
def test_neighbors_self_images(L, rc):
    """One atom in a cubic box of edge L: its neighbours are its own images n*L,
    n in Z^3 \\ {0}, |n| L < rc (lattice points counted here by integer loops)."""
    nb = oracle.neighbors(np.array([[0.3, 0.2, 0.1]]), np.array([L, L, L]), rc)
    k = int(math.ceil(rc / L))
    count = sum(1 for n in itertools.product(range(-k, k + 1), repeat=3)
                if n != (0, 0, 0) and (n[0] ** 2 + n[1] ** 2 + n[2] ** 2) * L * L < rc * rc)
    assert len(nb[0][0]) == count


def test_neighbors_symmetric():
    pos, _t, box = workloads.water_random()
    nb = oracle.neighbors(pos, box, 6.0)
    pairs = {(i, int(j), tuple(np.round(d, 8))) for i, (js, ds) in enumerate(nb) for j, d in zip(js, ds)}
    for (i, j, d) in pairs:
        assert (j, i, tuple(-np.array(d) + 0.0)) in pairs or (j, i, tuple(np.round(-np.array(d), 8))) in pairs


# --------------------------------------------------------------- invariances
@pytest.fixture(scope="module")
def water():
    m = workloads.water_model()
    pos, types, box = workloads.water_random()
    return m, pos, types, box, oracle.compute(m, pos, types, box)


def test_translation_invariance(water):
    m, pos, types, box, ref = water
    res = oracle.compute(m, pos + np.array([1.7, -23.1, 5.3]), types, box)
    np.testing.assert_allclose(res["Ei"], ref["Ei"], atol=1e-11)
    np.testing.assert_allclose(res["F"], ref["F"], atol=1e-10)


def test_permutation_invariance(water):
    m, pos, types, box, ref = water
    p = np.random.default_rng(3).permutation(len(pos))
    res = oracle.compute(m, pos[p], types[p], box)
    np.testing.assert_allclose(res["Ei"], ref["Ei"][p], atol=1e-11)
    np.testing.assert_allclose(res["F"], ref["F"][p], atol=1e-10)
    assert res["energy"] == pytest.approx(ref["energy"], abs=1e-10)


def test_cubic_rotation_of_periodic_box(water):
    """(x, y, z) -> (y, -x, z) maps the periodic cubic box onto itself."""
    m, pos, types, box, ref = water
    R = np.array([[0, 1, 0], [-1, 0, 0], [0, 0, 1]], float)
    res = oracle.compute(m, pos @ R.T, types, box)
    np.testing.assert_allclose(res["Ei"], ref["Ei"], atol=1e-11)
    np.testing.assert_allclose(res["F"], ref["F"] @ R.T, atol=1e-10)


def test_random_rotation_of_cluster():
    m = workloads.water_model()
    pos, types, _box = workloads.water_random(12, 7.0, seed=5)
    pos = pos - pos.mean(0)
    q, _ = np.linalg.qr(np.random.default_rng(9).normal(size=(3, 3)))
    big = np.array([60.0, 60.0, 60.0])
    a = oracle.compute(m, pos + 30.0, types, big)
    b = oracle.compute(m, pos @ q.T + 30.0, types, big)
    np.testing.assert_allclose(b["Ei"], a["Ei"], atol=1e-11)
    np.testing.assert_allclose(b["F"], a["F"] @ q.T, atol=1e-10)


def test_perfect_fcc_symmetry():
    m = workloads.fcc_model()
    pos, types, box = workloads.fcc((4, 4, 4), perfect=True)
    res = oracle.compute(m, pos, types, box)
    np.testing.assert_allclose(res["Ei"], res["Ei"][0], rtol=1e-12, atol=1e-12)
    assert np.abs(res["F"]).max() < 1e-9


# ----------------------------------------------------------- finite differences
def _fd_forces(m, pos, types, box, atoms, h=1e-5):
    out = []
    for i in atoms:
        row = []
        for c in range(3):
            p = pos.copy(); p[i, c] += h
            ep = oracle.compute(m, p, types, box)["energy"]
            p[i, c] -= 2 * h
            em = oracle.compute(m, p, types, box)["energy"]
            row.append(-(ep - em) / (2 * h))
        out.append(row)
    return np.array(out)


def test_forces_match_energy_fd_water(water):
    m, pos, types, box, ref = water
    atoms = [0, 5, 191]
    fd = _fd_forces(m, pos, types, box, atoms)
    np.testing.assert_allclose(ref["F"][atoms], fd, atol=1e-7 * max(1.0, np.abs(fd).max()))


def test_forces_match_energy_fd_fcc_multi_image():
    """Box edge 7.04 A < 2 rc: several images of the same atom are neighbours."""
    m = workloads.fcc_model()
    pos, types, box = workloads.fcc((2, 2, 2), sigma=0.1, seed=4)
    ref = oracle.compute(m, pos, types, box)
    atoms = [0, 17]
    fd = _fd_forces(m, pos, types, box, atoms)
    np.testing.assert_allclose(ref["F"][atoms], fd, atol=1e-7 * max(1.0, np.abs(fd).max()))
    np.testing.assert_allclose(ref["F"].sum(0), 0.0, atol=1e-9)


def test_virial_matches_strain_fd():
    """W_ba = -dE/d eps_ab for d -> (I + eps) d: diagonal strain of the periodic box,
    off-diagonal strain of an isolated cluster."""
    m = workloads.water_model()
    pos, types, box = workloads.water_random()
    ref = oracle.compute(m, pos, types, box)
    h = 1e-6
    for a in range(3):
        s = np.ones(3); s[a] += h
        ep = oracle.compute(m, pos * s, types, box * s)["energy"]
        s[a] -= 2 * h
        em = oracle.compute(m, pos * s, types, box * s)["energy"]
        assert ref["virial"][a, a] == pytest.approx(-(ep - em) / (2 * h), rel=1e-6, abs=1e-6)
    cl, ct, _ = workloads.water_random(10, 7.0, seed=8)
    cl = cl - cl.mean(0)
    big = np.array([60.0] * 3)
    r0 = oracle.compute(m, cl + 30, ct, big)
    np.testing.assert_allclose(r0["virial"], r0["virial"].T, atol=1e-9)
    for a, b in [(0, 1), (1, 2), (2, 0)]:
        eps = np.zeros((3, 3)); eps[a, b] = h
        ep = oracle.compute(m, cl @ (np.eye(3) + eps).T + 30, ct, big)["energy"]
        em = oracle.compute(m, cl @ (np.eye(3) - eps).T + 30, ct, big)["energy"]
        assert r0["virial"][b, a] == pytest.approx(-(ep - em) / (2 * h), rel=1e-6, abs=1e-7)


def test_owned_virial_is_the_strain_derivative_of_the_owned_energy():
    """compute_owned: W_A = -dE_A/d eps for E_A = sum of the first n_own atoms'
    energies (finite differences of those energies under strain), and the parts
    for A and its complement add up to the whole system's virial."""
    m = workloads.water_model()
    pos, types, box = workloads.water_random()
    n_own = 100
    r = oracle.compute_owned(m, pos, types, box, n_own)
    assert r["energy"] == pytest.approx(r["Ei"][:n_own].sum(), rel=1e-14)
    h = 1e-6
    for a in range(3):
        s = np.ones(3); s[a] += h
        ep = oracle.compute(m, pos * s, types, box * s)["Ei"][:n_own].sum()
        s[a] -= 2 * h
        em = oracle.compute(m, pos * s, types, box * s)["Ei"][:n_own].sum()
        assert r["virial"][a, a] == pytest.approx(-(ep - em) / (2 * h), rel=1e-6, abs=1e-6)
    # the complement: atoms n_own.. moved to the front
    order = np.r_[np.arange(n_own, len(pos)), np.arange(n_own)]
    rb = oracle.compute_owned(m, pos[order], types[order], box, len(pos) - n_own)
    full = oracle.compute(m, pos, types, box)
    np.testing.assert_allclose(r["virial"] + rb["virial"], full["virial"], rtol=0, atol=1e-10)
    np.testing.assert_allclose(r["F"], full["F"], rtol=0, atol=1e-12)


# ------------------------------------------------------------------- network
def test_mlp_matches_torch_sequential():
    torch = pytest.importorskip("torch")
    m = workloads.water_model()
    widths = m["widths"]
    for e in range(2):
        P = m["weights"][e]
        layers, off = [], 0
        for l in range(len(widths) - 1):
            lin = torch.nn.Linear(widths[l], widths[l + 1]).double()
            n_w = widths[l] * widths[l + 1]
            lin.weight.data = torch.tensor(P[off:off + n_w].reshape(widths[l + 1], widths[l]))
            off += n_w
            lin.bias.data = torch.tensor(P[off:off + widths[l + 1]])
            off += widths[l + 1]
            layers.append(lin)
            if l < len(widths) - 2:
                layers.append(torch.nn.Tanh())
        net = torch.nn.Sequential(*layers)
        x = np.random.default_rng(e).normal(size=widths[0])
        xt = torch.tensor(x, requires_grad=True)
        E_t = net(xt)[0]
        E_t.backward()
        E, dx = oracle.mlp(m, e, x)
        assert E == pytest.approx(E_t.item(), abs=1e-13)
        np.testing.assert_allclose(dx, xt.grad.numpy(), atol=1e-13)


def test_energy_is_sum_of_network_outputs(water):
    m, pos, types, box, ref = water
    assert ref["energy"] == pytest.approx(ref["Ei"].sum(), abs=1e-11)
    for i in (0, 3):
        e = types[i]
        x = (ref["G"][i, :30] - m["sf_mu"][e]) / m["sf_s"][e]
        E, dx = oracle.mlp(m, e, x)
        assert ref["Ei"][i] == pytest.approx(E, abs=1e-12)
        np.testing.assert_allclose(ref["dEdG"][i, :30], dx / m["sf_s"][e], atol=1e-12)


def test_subset_matches_full(water):
    m, pos, types, box, ref = water
    idx = [3, 50, 190]
    sub = oracle.compute_subset(m, pos, types, box, idx)
    np.testing.assert_allclose(sub["Ei"], ref["Ei"][idx], atol=1e-12)
    np.testing.assert_allclose(sub["F"], ref["F"][idx], atol=1e-11)
    np.testing.assert_allclose(sub["G"], ref["G"][idx], atol=1e-12)


# ------------------------------------------------------------------------ NVE
def test_nve_energy_conservation_second_order():
    """Velocity Verlet is second order: the energy error over a fixed time shrinks ~4x
    when dt halves, and stays small."""
    m = workloads.water_model()
    pos, types, box = workloads.water_random()
    vel = workloads.maxwell_boltzmann(types, m["masses"])
    _, _, la = oracle.md(m, pos, vel, types, box, 0.5, 10)
    _, _, lb = oracle.md(m, pos, vel, types, box, 0.25, 20)
    ea = la.sum(1)
    eb = lb.sum(1)
    err_a = abs(ea[-1] - ea[0])
    err_b = abs(eb[-1] - eb[0])
    assert err_a / len(pos) < 5e-4
    assert 2.5 < err_a / err_b < 6.0


# ------------------------------------------------------------ training gradient
def _loss(model, batch, refs, wF):
    B = len(batch)
    n_tot = sum(len(p) for p, _, _ in batch)
    L = 0.0
    for (p, t, box), (Er, Fr) in zip(batch, refs):
        r = oracle.compute(model, p, t, box)
        L += ((r["energy"] - Er) / len(p)) ** 2 / B
        L += wF * ((r["F"] - Fr) ** 2).sum() / (3 * n_tot)
    return L


def _grad(model, batch, refs, wF):
    B = len(batch)
    n_tot = sum(len(p) for p, _, _ in batch)
    g = 0.0
    for (p, t, box), (Er, Fr) in zip(batch, refs):
        r = oracle.compute(model, p, t, box)
        dLdE = 2.0 * (r["energy"] - Er) / len(p) ** 2 / B
        u = 2.0 * wF * (r["F"] - Fr) / (3 * n_tot)
        g = g + oracle.param_grad(model, p, t, box, dLdE, u)
    return g


@pytest.mark.parametrize("wF", [0.0, 10.0])
def test_param_grad_matches_loss_fd(wF):
    m = workloads.water_model(hidden=(8, 6))
    m["sf_mu"] = workloads.water_model()["sf_mu"]
    m["sf_s"] = workloads.water_model()["sf_s"]
    teacher = workloads.water_model(seed=77, hidden=(8, 6))
    teacher["sf_mu"], teacher["sf_s"] = m["sf_mu"], m["sf_s"]
    rng = np.random.default_rng(1)
    batch = [workloads.water_random(nm, (3 * nm / workloads.WATER_DENSITY_ATOMS) ** (1 / 3), seed=20 + nm)
             for nm in (8, 11)]
    refs = []
    for p, t, box in batch:
        r = oracle.compute(teacher, p, t, box)
        refs.append((r["energy"], r["F"] + rng.normal(0, 0.01, r["F"].shape)))
    g = _grad(m, batch, refs, wF)
    w0 = [w.copy() for w in m["weights"]]
    npe = len(w0[0])
    h = 1e-6
    dirs = [rng.normal(size=2 * npe) for _ in range(2)]
    for k in (0, 5, npe - 1, npe + 3):   # single parameters: first layer, output bias ...
        v = np.zeros(2 * npe); v[k] = 1.0
        dirs.append(v)
    for v in dirs:
        def at(sgn):
            m["weights"] = [w0[0] + sgn * h * v[:npe], w0[1] + sgn * h * v[npe:]]
            return _loss(m, batch, refs, wF)
        fd = (at(1) - at(-1)) / (2 * h)
        m["weights"] = w0
        assert g @ v == pytest.approx(fd, rel=2e-6, abs=1e-9)
