"""CUDA path (FP32) against the FP64 oracle on the same seeded inputs: descriptors,
network input gradient, per-atom energies, forces, virial and energy, over the
brute-force (small box, several images) and cell-list neighbour paths, the
narrow (water) and wide (FCC) angular kinds, ragged sizes and edge cases."""
import numpy as np
import pytest
import torch

import oracle
import workloads
from tests.gpuhelp import E_REL, F_ABS, check, energy_err, f32, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def water_nnp():
    from paper_2002_00054_b300 import NNP
    return NNP(workloads.water_model())


@pytest.fixture(scope="module")
def fcc_nnp():
    from paper_2002_00054_b300 import NNP
    return NNP(workloads.fcc_model())


def _case(nnp, model, pos, types, box):
    pos, box = f32(pos), f32(box)
    ref = oracle.compute(model, pos, types, box)
    p, t = to_dev(pos, types)
    out = nnp.compute(p, t, box)
    return ref, out, p, t, box


def _close_by_column(x, ref, rtol, col_floor):
    """|x - ref| <= rtol |ref| + col_floor max|ref column|, element by element."""
    tol = rtol * np.abs(ref) + col_floor * np.abs(ref).max(0)[None, :]
    bad = np.abs(x - ref) > tol
    assert not bad.any(), "%d elements off; worst at %s: %r vs %r" % (
        bad.sum(), np.unravel_index(np.argmax(np.abs(x - ref) / tol), x.shape),
        x.flat[np.argmax(np.abs(x - ref) / tol)], ref.flat[np.argmax(np.abs(x - ref) / tol)])


def test_water_tiny_descriptors(water_nnp):
    m = workloads.water_model()
    pos, types, box = workloads.water_random()
    pos, box = f32(pos), f32(box)
    ref = oracle.compute(m, pos, types, box)
    p, t = to_dev(pos, types)
    G, dEdG = water_nnp.descriptors(p, t, box)
    G = G.double().cpu().numpy()
    gref = ref["G"][:, :30]
    # element by element, relative to each value (float32 output of FP64 sums; the
    # narrow kind's per-triplet factors carry up to ~13 ulp)
    np.testing.assert_allclose(G, gref, rtol=2e-6, atol=0)
    dE = dEdG.double().cpu().numpy()
    dref = ref["dEdG"][:, :30]
    # element by element; the floor (1e-5 of the column's largest value) only guards
    # values that cancel to ~0 in the backprop
    _close_by_column(dE, dref, rtol=1e-4, col_floor=1e-5)


def test_fcc_descriptors_elementwise(fcc_nnp):
    """Wide-kind descriptors and dE/dG of the 4,000-atom FCC box, element by element."""
    m = workloads.fcc_model()
    pos, types, box = workloads.fcc((10, 10, 10))
    pos, box = f32(pos), f32(box)
    ref = oracle.compute(m, pos, types, box)
    p, t = to_dev(pos, types)
    G, dEdG = fcc_nnp.descriptors(p, t, box)
    np.testing.assert_allclose(G.double().cpu().numpy(), ref["G"][:, :40], rtol=1e-6, atol=0)
    dref = ref["dEdG"][:, :40]
    _close_by_column(dEdG.double().cpu().numpy(), dref, rtol=1e-4, col_floor=1e-5)


def test_water_tiny_energy_forces(water_nnp):
    m = workloads.water_model()
    ref, out, *_ = _case(water_nnp, m, *workloads.water_random())
    check(out, ref, what="water 192")


def test_water_lattice_cell_path(water_nnp):
    m = workloads.water_model()
    ref, out, *_ = _case(water_nnp, m, *workloads.water_lattice((2, 2, 2), seed=5))
    assert water_nnp.stats()["n_atoms"] == 1536
    check(out, ref, what="water 1536")


@pytest.mark.parametrize("n_mol", [21, 22, 37])
def test_water_ragged_small_boxes(water_nnp, n_mol):
    """63-111 atoms at liquid density: box < 2 (rc + skin), several images per atom."""
    m = workloads.water_model()
    L = (3 * n_mol / workloads.WATER_DENSITY_ATOMS) ** (1 / 3)
    ref, out, *_ = _case(water_nnp, m, *workloads.water_random(n_mol, L, seed=100 + n_mol))
    check(out, ref, what="water %d" % (3 * n_mol))


def test_dense_water_over_256_neighbours():
    """Water compressed to 0.62 of its edge (~4.2x the density): ~360 neighbours
    inside the cutoff, so the shared-memory capacity exceeds 256 staged neighbours
    and the descriptor pass runs its one-block-pair-at-a-time form (staged indices
    no longer fit 8 bits, no stored pair queues); the force pass rebuilds the
    queues."""
    from paper_2002_00054_b300 import NNP
    m = workloads.water_model()
    pos, types, box = workloads.water_random()
    pos, box = pos * 0.62, box * 0.62
    nnp = NNP(m, max_neighbors=1024)
    ref, out, p, t, fb = _case(nnp, m, pos, types, box)
    assert nnp.stats()["max_cutoff_row"] > 256, nnp.stats()
    check(out, ref, what="dense water")
    out2 = nnp.compute(p, t, fb)   # capacity retuned above 256 for the main pass
    assert nnp.stats()["rc_capacity"] > 256, nnp.stats()
    check(out2, ref, what="dense water, second call")


def test_fcc_4000_cell_path(fcc_nnp):
    m = workloads.fcc_model()
    ref, out, *_ = _case(fcc_nnp, m, *workloads.fcc((10, 10, 10)))
    check(out, ref, what="fcc 4000")


def test_fcc_small_box_images(fcc_nnp):
    m = workloads.fcc_model()
    ref, out, *_ = _case(fcc_nnp, m, *workloads.fcc((2, 2, 2), sigma=0.1, seed=4))
    check(out, ref, what="fcc 32")


def test_cell_path_mixed_row_builders():
    """A 30 A box (4 cells of 7.5 A per side) whose x in [0, 20) is squeezed into
    [0, 10) (twice the density there, half beyond): half the cells have more than
    1,280 atoms in their 27-cell stencil and keep the warp-per-atom row builder,
    the others take the block-per-cell builder that stages the stencil in shared
    memory.
    One evaluation with both builders matches the oracle, and so do the steps
    after (rebuilds with both)."""
    from paper_2002_00054_b300 import NNP
    m = workloads.water_model()
    pos, types, box = workloads.water_random(900, 30.0, seed=31)
    x = np.mod(pos[:, 0], 30.0)
    pos = pos.copy()
    pos[:, 0] = np.where(x < 20.0, x * 0.5, 10.0 + (x - 20.0) * 2.0)
    nnp = NNP(m, max_neighbors=320)
    ref, out, p, t, fb = _case(nnp, m, pos, types, box)
    check(out, ref, what="mixed stencils")
    v = torch.zeros_like(p)
    nnp.step(p, v, t, fb, 0.5, 3)
    check(nnp.compute(p, t, fb), oracle.compute(m, p.double().cpu().numpy(), types, fb), what="mixed stencils, steps")


def test_single_atom_sees_only_itself(fcc_nnp):
    m = workloads.fcc_model()
    ref, out, *_ = _case(fcc_nnp, m, np.array([[0.4, 1.1, 2.0]]), np.array([0], np.int32), np.array([4.0, 4.0, 4.0]))
    check(out, ref, what="one atom")
    assert np.abs(out["F"].cpu().numpy()).max() < 1e-5


def test_empty_system(water_nnp):
    p = torch.zeros((0, 3), dtype=torch.float32, device="cuda")
    t = torch.zeros((0,), dtype=torch.int32, device="cuda")
    out = water_nnp.compute(p, t, [20.0, 20.0, 20.0])
    assert out["energy"].item() == 0.0
    assert out["F"].shape == (0, 3)


def test_bitwise_repeatable(water_nnp):
    pos, types, box = workloads.water_lattice((2, 2, 2), seed=6)
    p, t = to_dev(f32(pos), types)
    a = water_nnp.compute(p, t, f32(box))
    water_nnp.compute(p + 0.3, t, f32(box))   # forces a rebuild in between
    b = water_nnp.compute(p, t, f32(box))
    assert torch.equal(a["F"], b["F"]) and torch.equal(a["Ei"], b["Ei"])
    assert a["energy"].item() == b["energy"].item()


def test_list_reuse_within_skin(water_nnp):
    m = workloads.water_model()
    pos, types, box = workloads.water_lattice((2, 2, 2), seed=7)
    pos, box = f32(pos), f32(box)
    p, t = to_dev(pos, types)
    water_nnp.compute(p, t, box)
    r0 = water_nnp.stats()["rebuilds"]
    rng = np.random.default_rng(0)
    moved = f32(pos + rng.uniform(-0.2, 0.2, pos.shape))   # |d| < 0.35 < skin / 2
    pm, _ = to_dev(moved, types)
    out = water_nnp.compute(pm, t, box)
    assert water_nnp.stats()["rebuilds"] == r0
    check(out, oracle.compute(m, moved, types, box), what="reused list")
    far = f32(pos + rng.uniform(-0.8, 0.8, pos.shape))
    pf, _ = to_dev(far, types)
    out = water_nnp.compute(pf, t, box)
    assert water_nnp.stats()["rebuilds"] == r0 + 1
    check(out, oracle.compute(m, far, types, box), what="rebuilt list")


def test_positions_outside_box(water_nnp):
    """Unwrapped coordinates (atoms shifted by whole boxes) give the same result."""
    m = workloads.water_model()
    pos, types, box = workloads.water_random()
    pos, box = f32(pos), f32(box)
    shift = np.zeros_like(pos)
    shift[::3, 0] = box[0]
    shift[1::5, 2] = -box[2]
    pos2 = f32(pos + shift)
    ref = oracle.compute(m, pos, types, box)
    p, t = to_dev(pos2, types)
    out = water_nnp.compute(p, t, box)
    check(out, ref, e_rel=E_REL, f_abs=F_ABS, what="unwrapped")


def test_stats_counts(water_nnp):
    pos, types, box = workloads.water_random()
    p, t = to_dev(f32(pos), types)
    water_nnp.compute(p, t, f32(box))
    s = water_nnp.stats()
    nb = oracle.neighbors(f32(pos), f32(box), 6.0)
    assert s["cutoff_entries"] == sum(len(x[0]) for x in nb)
    assert s["pairs"] == sum(len(x[0]) * (len(x[0]) - 1) // 2 for x in nb)
    assert 0 < s["triplets"] < s["pairs"]
    # closest pair inside the cutoff (float distance of the same displacement)
    r_min = min(np.sqrt((x[1] ** 2).sum(1)).min() for x in nb if len(x[0]))
    assert abs(s["min_distance"] - r_min) <= 1e-6 * r_min
    # a moved pair is seen by the next call
    q = p.clone()
    q[1] = q[0] + torch.tensor([0.31, 0.0, 0.0], device="cuda")
    water_nnp.compute(q, t, f32(box))
    assert abs(water_nnp.stats()["min_distance"] - 0.31) <= 1e-6


# ------------------------------------------------------------- errors
def test_overflow_is_reported():
    from paper_2002_00054_b300 import NNP, NNPError
    nnp = NNP(workloads.water_model(), max_neighbors=32)
    pos, types, box = workloads.water_random()
    p, t = to_dev(f32(pos), types)
    with pytest.raises(NNPError) as e:
        nnp.compute(p, t, f32(box))
    assert e.value.status == 3
    nnp.close()


def test_nonfinite_and_bad_type_are_reported(water_nnp):
    from paper_2002_00054_b300 import NNPError
    pos, types, box = workloads.water_random()
    p, t = to_dev(f32(pos), types)
    q = p.clone(); q[5, 1] = float("nan")
    with pytest.raises(NNPError) as e:
        water_nnp.compute(q, t, f32(box))
    assert e.value.status == 4
    t2 = t.clone(); t2[3] = 7
    with pytest.raises(NNPError) as e:
        water_nnp.compute(p, t2, f32(box))
    assert e.value.status == 4
    out = water_nnp.compute(p, t, f32(box))   # handle still usable
    assert np.isfinite(out["energy"].item())


def test_box_too_small(water_nnp):
    from paper_2002_00054_b300 import NNPError
    p, t = to_dev(np.zeros((1, 3)), np.zeros(1, np.int32))
    with pytest.raises(NNPError) as e:
        water_nnp.compute(p, t, [3.0, 3.0, 3.0])
    assert e.value.status == 5


@pytest.mark.parametrize("name", ["water", "fcc"])
@pytest.mark.parametrize("form", ["gather", "float"])
def test_force_assembly_forms_agree(name, form, monkeypatch):
    """The default force assembly adds -g_ij into F_j as 64-bit fixed-point
    integers (exact, order-independent sums, one rounding per component);
    NNP_FORCE_GATHER=1 writes g per list slot and gathers through the reverse
    index, NNP_FORCE_SCATTER=1 adds floats with global atomics (the paper's
    scatter form).  Same energies, forces equal up to float summation order,
    the same parity with the oracle, and MD steps (neighbour rebuilds with or
    without a reverse index) keep it."""
    from paper_2002_00054_b300 import NNP
    if name == "water":
        m, (pos, types, box) = workloads.water_model(), workloads.water_lattice((2, 2, 2), seed=5)
    else:
        m, (pos, types, box) = workloads.fcc_model(), workloads.fcc((6, 6, 6), sigma=0.1, seed=6)
    pos, box = f32(pos), f32(box)
    p, t = to_dev(pos, types)
    fixed_h = NNP(m)
    fx = fixed_h.compute(p, t, box)
    fx2 = fixed_h.compute(p, t, box)
    assert torch.equal(fx["F"], fx2["F"])          # reproducible bit for bit
    monkeypatch.setenv("NNP_FORCE_GATHER" if form == "gather" else "NNP_FORCE_SCATTER", "1")
    o_h = NNP(m)
    monkeypatch.delenv("NNP_FORCE_GATHER" if form == "gather" else "NNP_FORCE_SCATTER")
    ot = o_h.compute(p, t, box)
    assert torch.equal(fx["Ei"], ot["Ei"])
    assert (fx["F"] - ot["F"]).abs().max().item() <= 2e-6
    ref = oracle.compute(m, pos, types, box)
    check(fx, ref, what="%s fixed-point scatter" % name)
    check(ot, ref, what="%s %s" % (name, form))
    # continued MD steps with both forms from the same start
    for h in (fixed_h, o_h):
        v = torch.zeros_like(p)
        x = p.clone()
        h.step(x, v, t, box, 0.5, 5)
        check(h.compute(x, t, box), oracle.compute(m, x.double().cpu().numpy(), types, box),
              what="%s after steps" % name)


@pytest.mark.parametrize("name", ["water", "fcc"])
def test_thread_per_atom_descriptors(name):
    """The other mappings of the parallelism ablation (Fig. 6): one thread per
    atom, one thread per (atom, neighbour) with atomic updates of G_i, and one
    CTA per cell with the stencil staged in shared memory, give the raw G of the
    oracle (and of the warp-per-atom kernel) to FP32 summation order (plain
    float sums over ~2000 triplets per atom)."""
    from paper_2002_00054_b300 import NNP
    if name == "water":
        m, (pos, types, box) = workloads.water_model(), workloads.water_lattice((2, 2, 2), seed=7)
    else:
        m, (pos, types, box) = workloads.fcc_model(), workloads.fcc((6, 6, 6), sigma=0.1, seed=8)
    pos, box = f32(pos), f32(box)
    p, t = to_dev(pos, types)
    nnp = NNP(m)
    Gf = nnp.descriptors_flat(p, t, box).double().cpu().numpy()
    Gp = nnp.descriptors_pair(p, t, box).double().cpu().numpy()
    Gc = nnp.descriptors_cell(p, t, box).double().cpu().numpy()
    Gw, _ = nnp.descriptors(p, t, box, dEdG=False)
    Gw = Gw.double().cpu().numpy()
    ng = Gw.shape[1]
    gref = oracle.compute(m, pos, types, box)["G"][:, :ng]
    # plain float sums in both ablation kernels: element by element to ~1e-5
    np.testing.assert_allclose(Gf, gref, rtol=1e-5, atol=0)
    np.testing.assert_allclose(Gp, gref, rtol=1e-5, atol=0)
    np.testing.assert_allclose(Gc, gref, rtol=1e-5, atol=0)
    np.testing.assert_allclose(Gw, gref, rtol=2e-6, atol=0)


def test_cell_order_visiting_is_bitwise(monkeypatch):
    """The main passes visit atoms in cell order (default) or in atom order
    (NNP_CELL_ORDER=0): every atom's arithmetic is its own and the force sums are
    integers, so energies and forces are bit for bit the same, on a box whose
    atoms are stored in a random order."""
    from paper_2002_00054_b300 import NNP
    m = workloads.water_model()
    pos, types, box = workloads.water_lattice((2, 3, 2), seed=9)
    o = np.random.default_rng(3).permutation(len(pos))
    p, t = to_dev(f32(pos[o]), types[o])
    a = NNP(m).compute(p, t, f32(box))
    monkeypatch.setenv("NNP_CELL_ORDER", "0")
    b = NNP(m).compute(p, t, f32(box))
    assert torch.equal(a["F"], b["F"]) and torch.equal(a["Ei"], b["Ei"])
    assert a["energy"].item() == b["energy"].item()
    np.testing.assert_allclose(a["virial"].cpu().numpy(), b["virial"].cpu().numpy(), rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("spill", [False, True])
def test_staged_reuse_is_bitwise(spill, monkeypatch):
    """The force pass reads the neighbours the descriptor pass staged (same
    arithmetic, integer force sums): bitwise the forces of staging them again
    (NNP_STAGE_REUSE=0).  With `spill` both handles first evaluate a system at
    0.75 of liquid density, which lowers the shared-memory capacity below the
    counts of some atoms of liquid water: those take the wide-capacity pass."""
    from paper_2002_00054_b300 import NNP
    m = workloads.water_model()
    pos, types, box = workloads.water_random(seed=78)
    pos, box = f32(pos), f32(box)
    p, t = to_dev(pos, types)
    a = NNP(m)
    monkeypatch.setenv("NNP_STAGE_REUSE", "0")
    b = NNP(m)
    monkeypatch.delenv("NNP_STAGE_REUSE")
    if spill:
        lp, lt, lb = workloads.water_random(box=workloads.WATER_CELL / 0.75 ** (1 / 3), seed=77)
        lp, lt = to_dev(f32(lp), lt)
        for h in (a, b):
            h.compute(lp, lt, f32(lb))
    oa, ob = a.compute(p, t, box), b.compute(p, t, box)
    assert (a.stats()["spilled_atoms"] > 0) == spill
    assert b.stats()["spilled_atoms"] == a.stats()["spilled_atoms"]
    assert torch.equal(oa["F"], ob["F"]) and torch.equal(oa["Ei"], ob["Ei"])
    assert torch.equal(oa["virial"], ob["virial"])
    check(oa, oracle.compute(m, pos, types, box), what="water, staged reuse")

