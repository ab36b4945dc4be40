"""Pins of the oracle's layered soils (Section 4.1's composite column and
Section 4.2's two-layer field): each cell follows the law and parameters of
its own material, and the hierarchy assigns every coarse cell one material.

Readings pinned here:
  * a fine cell's theta, theta' and K are its material's Table 1 law with
    that material's Ks, theta_s, theta_r and shape parameters;
  * a coarse cell takes the material with the largest total restriction
    weight among the fine cells it restricts from (ties: the lower index);
  * conductivities stay cell-centred and faces take the arithmetic mean, so a
    saturated layered column carries the series flux of those face values.
"""
import numpy as np
import pytest

from oracle.dense import dense_newton
from oracle.oracle import ORC_OK, Oracle
from paper_2606_04292_gb300 import workloads as W

MODELS = [W.HAVERKAMP, W.GARDNER, W.VANGENUCHTEN]


def _as_material(soil):
    return W.material(soil["model"], soil["Ks"], soil["theta_s"], soil["theta_r"],
                      soil["p1"], soil["p2"], soil["p3"], soil["p4"])


def _probe(mat):
    """A two-cell column carrying one plain soil: the single-law oracle."""
    p = W.random_problem(1, 2, W.GARDNER, 0)
    p["soil"] = W._soil(mat["model"], mat["Ks"], mat["theta_s"], mat["theta_r"],
                        mat["p1"], mat["p2"], mat["p3"], mat["p4"])
    return Oracle(p)


def _run(prob, nsteps):
    o = Oracle(prob)
    for _ in range(nsteps):
        st, info = o.step()
        assert st == ORC_OK, info
    return o.state()


@pytest.mark.parametrize("model", MODELS)
@pytest.mark.parametrize("dim,n", [(1, (17,)), (2, (9, 11)), (3, (5, 6, 7))])
def test_one_material_reproduces_the_single_law(dim, n, model):
    """One material equal to the soil, or three identical copies of it spread
    at random: the fine operator and right side are bit for bit the
    single-law ones.  The coarse levels differ in the last bits only (a
    single soil restricts its parameters, whose weights sum to one up to
    rounding; a material keeps them exactly), so the converged steps agree
    to far inside the tolerance."""
    p = W.random_problem(dim, n, model, 80 + dim, sink=True)
    N = W.ncells(p)
    m = _as_material(p["soil"])
    idx = np.random.default_rng(3).integers(0, 3, N)
    variants = [W.with_materials(p, [m], np.zeros(N, np.uint8)),
                W.with_materials(p, [m, dict(m), dict(m)], idx)]
    o_ref = Oracle(p)
    o_ref.prepare(p["dt"], 1)
    psi = p["psi0"] + np.random.default_rng(4).uniform(-0.1, 0.1, N)
    r_ref, _ = o_ref.residual(psi)
    for q in variants:
        o = Oracle(q)
        o.prepare(q["dt"], 1)
        assert np.array_equal(o.g(), o_ref.g()) and np.array_equal(o.Kc(), o_ref.Kc())
        assert np.array_equal(o.residual(psi)[0], r_ref)
    ref = _run(p, 3)
    for q in variants:
        assert np.max(np.abs(_run(q, 3) - ref)) <= 1e-10


@pytest.mark.parametrize("dim,n", [(1, (23,)), (2, (13, 10)), (3, (7, 6, 9))])
def test_cell_laws_follow_the_material_index(dim, n):
    """On every level, theta, theta' (and K on the fine level) of a cell equal
    the single-law oracle of the material the cell carries."""
    p = W.random_problem(dim, n, W.VANGENUCHTEN, 90 + dim)
    mats = W.test_materials()
    idx = W.material_pattern(p, "random", 3, 4)
    o = Oracle(W.with_materials(p, mats, idx))
    probes = [_probe(m) for m in mats]
    rng = np.random.default_rng(6)
    assert o.nlevels >= 2
    for lev in range(o.nlevels):
        mm = o.material_map(lev)
        if lev == 0:
            assert np.array_equal(mm, idx)
        for cell in range(o.ncell(lev)):
            psi = -float(np.exp(rng.uniform(np.log(1e-3), np.log(20.0))))
            th, dth, K = o.soil(cell, psi, lev)
            pth, pdth, pK = probes[mm[cell]].soil(0, psi)
            assert th == pth and dth == pdth
            if lev == 0:
                assert K == pK
    # the map is not trivial: all three materials are present on level 1
    assert len(set(o.material_map(1).tolist())) == 3


@pytest.mark.parametrize("kind", ["random", "layers"])
@pytest.mark.parametrize("dim,n", [(1, (40,)), (2, (19, 14)), (3, (9, 7, 8))])
def test_coarse_material_is_the_weighted_majority(dim, n, kind):
    """Coarse material = argmax over materials of the restriction of the
    fine indicator fields, the first index on ties."""
    p = W.random_problem(dim, n, W.GARDNER, 100 + dim)
    o = Oracle(W.with_materials(p, W.test_materials(), W.material_pattern(p, kind, 3, 7)))
    for lev in range(o.nlevels - 1):
        fine = o.material_map(lev)
        weights = np.stack([o.restrict((fine == m).astype(np.float64), lev) for m in range(3)])
        assert np.array_equal(o.material_map(lev + 1), np.argmax(weights, axis=0).astype(np.uint8))


def test_aligned_layers_survive_and_thin_layers_vanish():
    """1D full weighting (1, 3, 3, 1)/8: a band that covers whole coarse cells
    keeps its cells on the coarse level; a single fine cell (weight at most
    3/8 of any coarse cell) does not."""
    p = W.random_problem(1, (32,), W.GARDNER, 5)
    idx = np.zeros(32, np.uint8)
    idx[8:20] = 1          # coarse cells 4..9 of level 1, 2..4 (12 fine cells -> 6 -> 3) of level 2
    idx[27] = 2            # one fine cell
    o = Oracle(W.with_materials(p, W.test_materials(), idx))
    m1 = o.material_map(1)
    want1 = np.zeros(16, np.uint8)
    want1[4:10] = 1
    assert np.array_equal(m1, want1)
    m2 = o.material_map(2)
    assert np.array_equal(np.nonzero(m2 == 1)[0], np.array([2, 3, 4]))
    assert not np.any(m2 == 2)


def _series_profile(Ks, h, P0, P1):
    """Saturated steady column between Dirichlet heads P0 (z = 0) and P1
    (z = Lz): one flux q through every face, face conductances the mean of
    the two cell values (Ks_i at a Dirichlet face, distance h/2), total head
    H = psi + z.  Returns the cell heads psi and q."""
    n = len(Ks)
    Lz = n * h
    Kf = np.concatenate([[Ks[0]], 0.5 * (Ks[:-1] + Ks[1:]), [Ks[-1]]])
    d = np.concatenate([[0.5 * h], np.full(n - 1, h), [0.5 * h]])
    Hb, Ht = P0, P1 + Lz
    q = -(Ht - Hb) / np.sum(d / Kf)            # q = -K dH/dz, positive upward
    H = Hb - np.cumsum(q * d[:-1] / Kf[:-1])
    z = (np.arange(n) + 0.5) * h
    return H - z, q


@pytest.mark.parametrize("dim", [1, 2])
def test_layered_saturated_column_carries_the_series_flux(dim):
    """Saturated layered flow (K = Ks of each cell's material): the series
    profile of the face-mean conductances is the exact discrete solution,
    and the single-soil linear profile is not."""
    nz = 12
    n = {1: (nz,), 2: (5, nz)}[dim]
    kinds = [W.NOFLUX] * (2 * dim - 2) + [W.DIRICHLET, W.DIRICHLET]
    p = W.random_problem(dim, n, W.VANGENUCHTEN, 14, bc_kinds=kinds)
    mats = W.test_materials()
    bands = np.array([0] * 4 + [1] * 3 + [2] * 5, np.uint8)
    nx = p["n"][0] if dim == 2 else 1
    idx = np.repeat(bands, nx)                      # x fastest, bands along z
    Lz = p["L"][dim - 1]
    h = Lz / nz
    P0, P1 = Lz + 1.0, 0.5                          # H falls upward: psi >= P1 > 0
    Ks = np.array([mats[m]["Ks"] for m in bands])
    psi_z, q = _series_profile(Ks, h, P0, P1)
    assert np.all(psi_z > 0) and q > 0
    psi = np.repeat(psi_z, nx)
    p["bc"]["value"][2 * dim - 2] = P0
    p["bc"]["value"][2 * dim - 1] = P1
    p["psi0"] = psi
    o = Oracle(W.with_materials(p, mats, idx))
    o.prepare(p["dt"], 1)
    _, nrm = o.residual(psi)
    scale = np.max(np.abs(o.g()))
    assert nrm <= 1e-13 * scale
    z = (np.arange(nz) + 0.5) * h
    lin = np.repeat(P0 + ((P1 + Lz) - P0) * z / Lz - z, nx)
    _, nrm_lin = o.residual(lin)
    assert nrm_lin > 1e6 * nrm
    # the steady state is also what a time step returns
    st, info = o.step()
    assert st == ORC_OK and np.max(np.abs(o.state() - psi)) <= 1e-9 * np.max(psi)


@pytest.mark.parametrize("dim,n", [(1, (15,)), (2, (8, 9)), (3, (4, 5, 6))])
def test_layered_hydrostatic_state_is_steady(dim, n):
    """psi = H - z between matching Dirichlet heads carries no flux in any
    layering: zero residual, no cycles, the state unchanged."""
    kinds = [W.NOFLUX] * (2 * dim - 2) + [W.DIRICHLET, W.DIRICHLET]
    p = W.random_problem(dim, n, W.GARDNER, 15, bc_kinds=kinds)
    H, Lz = 0.3, p["L"][dim - 1]
    p["bc"]["value"][2 * dim - 2] = H
    p["bc"]["value"][2 * dim - 1] = H - Lz
    nn = p["n"]
    idx = np.arange(W.ncells(p))
    iz = [idx % nn[0], (idx // nn[0]) % nn[1], idx // (nn[0] * nn[1])][dim - 1]
    psi = H - (iz + 0.5) * (Lz / nn[dim - 1])
    p["psi0"] = psi
    o = Oracle(W.with_materials(p, W.test_materials(), W.material_pattern(p, "random", 3, 8)))
    o.prepare(p["dt"], 1)
    _, nrm = o.residual(psi)
    assert nrm <= 1e-13 * np.max(np.abs(o.g()))
    st, info = o.step()
    assert st == ORC_OK and info["cycles"] == 0
    assert np.max(np.abs(o.state() - psi)) <= 1e-12


@pytest.mark.parametrize("scheme", [1, 2])
@pytest.mark.parametrize("dim,n", [(1, (13,)), (2, (7, 6)), (3, (4, 5, 3))])
def test_layered_mass_balance_identity(dim, n, scheme):
    """Conservation with theta taken, per cell, from the single-law oracle of
    that cell's material: sum V (a theta - hist) = boundary inflow - uptake
    - V sum r, to round-off, for any state."""
    kinds = {1: [W.FREE_DRAINAGE, W.DIRICHLET], 2: [W.DIRICHLET, W.FLUX, W.FREE_DRAINAGE, W.DIRICHLET],
             3: [W.NOFLUX, W.DIRICHLET, W.FLUX, W.NOFLUX, W.FREE_DRAINAGE, W.DIRICHLET]}[dim]
    p = W.random_problem(dim, n, W.HAVERKAMP, 30 + dim, bc_kinds=kinds, sink=True, scheme=scheme)
    if scheme == 2:
        p["psi_prev"] = p["psi0"] + np.random.default_rng(2).uniform(-0.05, 0.05, W.ncells(p))
    mats = W.test_materials()
    idx = W.material_pattern(p, "layers", 3, 9)
    o = Oracle(W.with_materials(p, mats, idx))
    assert o.prepare(p["dt"], scheme) == scheme
    psi = o.vcycle(p["psi0"])
    probes = [_probe(m) for m in mats]
    th = np.array([probes[idx[i]].soil(0, x)[0] for i, x in enumerate(psi)])
    S = np.array([o.sink(i, x)[0] for i, x in enumerate(psi)])
    r, _ = o.residual(psi)
    V, a = o.cell_volume(), o.a
    hist = o.array(7)
    lhs = V * np.sum(a * th - hist)
    Q = o.boundary_inflow(psi)
    rhs = Q - V * np.sum(S) - V * np.sum(r)
    scale = V * (np.sum(np.abs(a * th)) + np.sum(np.abs(hist))) + abs(Q)
    assert abs(lhs - rhs) <= 1e-13 * scale, (lhs, rhs)


@pytest.mark.parametrize("dim,n", [(1, (11,)), (2, (6, 7)), (3, (4, 3, 5))])
def test_layered_fas_solution_equals_dense_newton(dim, n):
    """Whatever the coarse levels carry, the FAS answer is the root of the
    fine equations with the per-cell laws."""
    p = W.random_problem(dim, n, W.VANGENUCHTEN, 40 + dim, sink=True, tol=1e-13, coarsest_max_n=2)
    p = W.with_materials(p, W.test_materials(), W.material_pattern(p, "layers", 3, 10))
    o = Oracle(p)
    o.prepare(p["dt"], 1)
    psi_fas, st, info = o.solve_current(p["psi0"])
    assert st == ORC_OK
    psi_dn, res = dense_newton(o, p["psi0"])
    assert res <= 1e-13
    assert np.max(np.abs(psi_fas - psi_dn)) <= 1e-10 * max(1.0, np.max(np.abs(psi_dn)))


def test_material_input_is_validated():
    p = W.random_problem(2, (6, 5), W.GARDNER, 1)
    mats = W.test_materials()
    with pytest.raises(ValueError):
        Oracle(W.with_materials(p, mats, np.full(30, 3, np.uint8)))      # index >= nmat
    with pytest.raises(ValueError):
        Oracle(W.with_materials(p, mats * 3, np.zeros(30, np.uint8)))   # 9 > 8 materials


def test_composite_and_two_layer_workloads_step():
    """Section 4.1's composite column and Section 4.2's two-layer field run
    through the oracle; the composite column's layers are where the paper
    puts them, and the two-layer interface follows zeta(x)."""
    c = W.celia_composite_1d(n=40, nsteps=3)
    idx = c["soil"]["material_index"]
    z = (np.arange(40) + 0.5)
    assert np.all(idx[z < 20] == 0) and np.all(idx[(z >= 20) & (z < 30)] == 1) and np.all(idx[z >= 30] == 2)
    assert [m["model"] for m in c["soil"]["materials"]] == [W.VANGENUCHTEN, W.HAVERKAMP, W.GARDNER]
    _run(c, 3)
    t = W.two_layer_2d(n=16, nsteps=2)
    idx = t["soil"]["material_index"].reshape(16, 16)
    # column x = 50: zeta = 100 (0.1 + 0.45) = 55, cells below z = 55 are the lower soil
    zc = (np.arange(16) + 0.5) * 100.0 / 16
    xc = (np.arange(16) + 0.5) * 100.0 / 16
    zeta = 100.0 * (0.1 * (1.0 - np.cos(np.pi * xc / 100.0)) + 0.45)
    assert np.array_equal(idx, (zc[:, None] < zeta[None, :]).astype(np.uint8))
    assert idx[0, 0] == 1 and idx[-1, 0] == 0
    _run(t, 2)
