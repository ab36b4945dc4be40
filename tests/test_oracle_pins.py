"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: values the
paper prints, closed-form discrete steady states, the structural results of
Section 3 (Prop. 3.1, Lemma 3.1, Theorem 3.1), exact conservation, a
brute-force Newton solve of the whole system, and convergence orders.
"""
import math
import os

import numpy as np
import pytest
from scipy.optimize import brentq

from oracle.dense import dense_newton
from oracle.oracle import ORC_OK, Oracle
from paper_2606_04292_gb300 import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))

CELIA = dict(Ks=0.00944, theta_s=0.287, theta_r=0.075, alpha=1.611e6, beta=3.96,
             A=1.175e6, gamma=4.74)


def load_golden(name):
    vals = {}
    with open(os.path.join(HERE, "golden", name)) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if not line:
                continue
            k, v, dec = line.split()
            vals[k] = (float(v), int(dec))
    return vals


def soil_probe(model, Ks, theta_s, theta_r, p1=0.0, p2=0.0, p3=0.0, p4=0.0):
    """A two-cell column carrying one soil; used to evaluate the laws."""
    p = W.random_problem(1, 2, W.GARDNER, 0)
    p["soil"] = W._soil(model, Ks, theta_s, theta_r, p1, p2, p3, p4)
    return Oracle(p)


def haverkamp_probe():
    c = CELIA
    return soil_probe(W.HAVERKAMP, c["Ks"], c["theta_s"], c["theta_r"], c["alpha"], c["beta"],
                      c["A"], c["gamma"])


# ---------------------------------------------------------------------------
# Constitutive laws (Table 1) pinned by the paper's printed calibration.
# ---------------------------------------------------------------------------
def test_haverkamp_half_suction_points():
    g = load_golden("calibration.txt")
    c = CELIA
    o = haverkamp_probe()
    h_th = c["alpha"] ** (1.0 / c["beta"])
    h_K = c["A"] ** (1.0 / c["gamma"])
    assert round(h_th, g["h_theta_half"][1]) == g["h_theta_half"][0]
    assert round(h_K, g["h_K_half"][1]) == g["h_K_half"][0]
    th, _, _ = o.soil(0, -h_th)
    _, _, K = o.soil(0, -h_K)
    assert abs(th - 0.5 * (c["theta_s"] + c["theta_r"])) <= 1e-15
    assert abs(K - 0.5 * c["Ks"]) <= 1e-17


def test_gardner_calibration():
    g = load_golden("calibration.txt")
    c = CELIA
    h_th = c["alpha"] ** (1.0 / c["beta"])
    aG = math.log(2.0) / h_th
    assert round(aG, g["alpha_G"][1]) == g["alpha_G"][0]
    o = soil_probe(W.GARDNER, c["Ks"], c["theta_s"], c["theta_r"], p1=aG)
    th, _, K = o.soil(0, -h_th)
    assert abs(th - 0.5 * (c["theta_s"] + c["theta_r"])) <= 1e-15
    assert abs(K - 0.5 * c["Ks"]) <= 1e-17


def test_van_genuchten_calibration():
    """The root n* of K_VG(h^K_1/2) = Ks/2 with alpha_VG(n) fixing the WRC
    half point reproduces the printed n*, alpha_VG and m (pins the VG WRC and
    the Mualem HCF with l = 0.5)."""
    g = load_golden("calibration.txt")
    c = CELIA
    h_th = c["alpha"] ** (1.0 / c["beta"])
    h_K = c["A"] ** (1.0 / c["gamma"])

    def alpha_of(n):
        m = 1.0 - 1.0 / n
        return (2.0 ** (1.0 / m) - 1.0) ** (1.0 / n) / h_th

    def f(n):
        o = soil_probe(W.VANGENUCHTEN, c["Ks"], c["theta_s"], c["theta_r"],
                       p1=alpha_of(n), p2=n, p3=g["l_VG"][0])
        th, _, _ = o.soil(0, -h_th)
        assert abs(th - 0.5 * (c["theta_s"] + c["theta_r"])) <= 1e-14
        _, _, K = o.soil(0, -h_K)
        return K / c["Ks"] - 0.5

    n_star = brentq(f, 1.2, 10.0, xtol=1e-14)
    assert round(n_star, g["n_star"][1]) == g["n_star"][0]
    assert round(alpha_of(n_star), g["alpha_VG"][1]) == g["alpha_VG"][0]
    assert round(1.0 - 1.0 / n_star, g["m_VG"][1]) == g["m_VG"][0]


@pytest.mark.parametrize("model", [W.HAVERKAMP, W.GARDNER, W.VANGENUCHTEN])
def test_theta_derivative_matches_central_difference(model):
    p = W.random_problem(1, 4, model, 3)
    o = Oracle(p)
    for psi in [-5.0, -1.3, -0.37, -0.05, -0.004]:
        h = 1e-4 * abs(psi)
        tp, _, _ = o.soil(0, psi + h)
        tm, _, _ = o.soil(0, psi - h)
        th, d, _ = o.soil(0, psi)
        fd = (tp - tm) / (2 * h)
        # truncation O(h^2) plus the round-off of differencing theta ~ theta_s
        tol = 1e-6 * abs(d) + 8 * np.finfo(float).eps * th / h
        assert abs(d - fd) <= tol, (psi, d, fd)
        assert d > 0.0
    # saturated branch: theta_s, Ks, zero capacity (reading for psi >= 0)
    th, d, K = o.soil(0, 0.3)
    assert th == p["soil"]["theta_s"] and d == 0.0 and K == p["soil"]["Ks"]


@pytest.mark.parametrize("model", [W.HAVERKAMP, W.GARDNER, W.VANGENUCHTEN])
def test_theta_monotone_and_bounded(model):
    """Assumption (A1) on psi < 0: theta increasing, theta_r < theta < theta_s."""
    o = Oracle(W.random_problem(1, 4, model, 4))
    s = o.prob["soil"]
    psis = -np.logspace(-4, 2, 200)[::-1]
    ths = [o.soil(0, x)[0] for x in psis]
    assert all(s["theta_r"] <= t < s["theta_s"] for t in ths[:-1])
    assert all(np.diff(ths) >= 0)


def test_sink_reading_shape():
    """Feddes reading of S: zero when over-wet or too dry, increasing on the
    rising branch [h4, h3] (assumption A2), right derivatives at kinks."""
    p = W.random_problem(1, 8, W.VANGENUCHTEN, 5, sink=True)
    o = Oracle(p)
    k = p["sink"]
    cell = p["n"][0] - 1        # top cell, inside the root zone
    S_mid, _ = o.sink(cell, -1.0)
    assert S_mid > 0
    for psi, expect in [(k["h1"], 0.0), (0.5 * (k["h1"] + k["h2"]), 0.5 * S_mid),
                        (k["h2"], S_mid), (k["h3"], S_mid),
                        (0.5 * (k["h3"] + k["h4"]), 0.5 * S_mid), (k["h4"], 0.0), (-100.0, 0.0)]:
        S, _ = o.sink(cell, psi)
        assert abs(S - expect) <= 1e-15 * S_mid + 1e-30, (psi, S, expect)
    for psi in [-40.0, -3.0, -0.2]:
        h = 1e-7
        Sp, _ = o.sink(cell, psi + h)
        S0, dS = o.sink(cell, psi)
        assert abs((Sp - S0) / h - dS) <= 1e-6 * S_mid
    _, dS = o.sink(cell, -40.0)
    assert dS > 0          # rising branch (A2)


@pytest.mark.parametrize("dim", [1, 3])
def test_sink_total_uptake_is_midpoint_rule_of_tp(dim):
    """On the Feddes plateau the whole column takes up Tp per unit area: the
    cells sample beta(d) = exp(-d/lambda)/Z, normalised on [0, D], at their
    centres, so the total is the midpoint rule of an integral equal to one.
    With D on a face, Euler-Maclaurin gives the relative error
    -h^2 (f'(D) - f'(0)) / 24 = -h^2 / (24 lambda^2) + O(h^4) (f = beta); a
    wrong normaliser, depth measured from the wrong end or off the cell
    centre breaks the constant or the order."""
    k = W.feddes_sink()
    lam, D = k["root_decay"], k["root_depth"]
    for n in (40, 80, 160, 320):
        h = 1.0 / n
        assert abs(D / h - round(D / h)) < 1e-9          # root zone ends on a face
        shape = (n,) if dim == 1 else (3, 2, n)
        p = W.random_problem(dim, shape, W.GARDNER, 1, sink=True, L=1.0)
        o = Oracle(p)
        Tp = p["sink"]["Tp"]
        ncol = int(np.prod(shape[:-1]))
        total = sum(o.sink(i, -1.0)[0] for i in range(ncol * n)) * o.cell_volume()
        rel = total / (Tp * 1.0 ** (dim - 1)) - 1.0
        lead = -h * h / (24.0 * lam * lam)
        assert abs(rel - lead) <= 7.0 * h ** 4 / (5760.0 * lam ** 4) * 1.2, (n, rel, lead)


# ---------------------------------------------------------------------------
# Operator assembly: Prop. 3.1 and closed-form discrete steady states.
# ---------------------------------------------------------------------------
BC_SETS = {
    1: [[W.DIRICHLET, W.DIRICHLET], [W.FREE_DRAINAGE, W.FLUX], [W.FREE_DRAINAGE, W.DIRICHLET]],
    2: [[W.NOFLUX, W.NOFLUX, W.DIRICHLET, W.DIRICHLET],
        [W.DIRICHLET, W.NOFLUX, W.FREE_DRAINAGE, W.FLUX]],
    3: [[W.NOFLUX] * 4 + [W.FREE_DRAINAGE, W.DIRICHLET],
        [W.DIRICHLET] * 6],
}
SIZES = {1: (7,), 2: (5, 6), 3: (3, 4, 5)}


@pytest.mark.parametrize("dim", [1, 2, 3])
@pytest.mark.parametrize("bci", [0, 1])
def test_prop31_matrix_structure(dim, bci):
    """Prop. 3.1: m_ii > 0, m_ij >= 0 (M has -m_ij off the diagonal) and the
    off-diagonal row sum equals m_ii on rows without a Dirichlet face; M is
    symmetric.  Checked on every level of the hierarchy."""
    kinds = BC_SETS[dim][bci % len(BC_SETS[dim])]
    p = W.random_problem(dim, SIZES[dim], W.VANGENUCHTEN, 7 + bci, bc_kinds=kinds, hetero=True)
    o = Oracle(p)
    o.prepare(p["dt"], 1)
    for lev in range(o.nlevels):
        M = o.dense_M(lev)
        n = M.shape[0]
        assert np.all(np.diag(M) > 0)
        off = M - np.diag(np.diag(M))
        assert np.all(off <= 0)
        assert np.allclose(M, M.T, rtol=1e-14, atol=0)
        excess = M.sum(axis=1)       # m_ii - sum_{j != i} m_ij >= 0
        assert np.all(excess >= -1e-15 * np.abs(np.diag(M)))
        # interior rows (all faces interior) have zero excess
        nn = o.level_n(lev)
        for i in range(n):
            ii = (i % nn[0], (i // nn[0]) % nn[1], i // (nn[0] * nn[1]))
            interior = all(0 < ii[a] < nn[a] - 1 for a in range(dim))
            if interior:
                assert abs(excess[i]) <= 1e-14 * M[i, i]


@pytest.mark.parametrize("dim,model", [(1, W.HAVERKAMP), (2, W.VANGENUCHTEN), (3, W.GARDNER)])
def test_hydrostatic_state_is_exact_steady_state(dim, model):
    """psi = H - z with matching Dirichlet heads top and bottom and no-flux
    sides has zero flux everywhere: the residual vanishes and a time step
    leaves it unchanged (pins the gravity sign and the elevations)."""
    n = {1: (9,), 2: (6, 7), 3: (3, 4, 5)}[dim]
    kinds = [W.NOFLUX] * (2 * dim - 2) + [W.DIRICHLET, W.DIRICHLET]
    p = W.random_problem(dim, n, model, 11, bc_kinds=kinds, hetero=True)
    H, Lz = 0.3, p["L"][dim - 1]
    p["bc"]["value"][2 * dim - 2] = H - 0.0
    p["bc"]["value"][2 * dim - 1] = H - Lz
    nn = p["n"]
    hz = Lz / nn[dim - 1]
    idx = np.arange(nn[0] * nn[1] * nn[2])
    iz = [idx % nn[0], (idx // nn[0]) % nn[1], idx // (nn[0] * nn[1])][dim - 1]
    psi = H - (iz + 0.5) * hz
    p["psi0"] = psi
    o = Oracle(p)
    o.prepare(p["dt"], 1)
    r, nrm = o.residual(psi)
    scale = np.max(np.abs(o.g()))
    assert nrm <= 1e-13 * scale
    st, info = o.step()
    assert st == ORC_OK and info["cycles"] == 0
    assert np.max(np.abs(o.state() - psi)) <= 1e-12


@pytest.mark.parametrize("dim", [2, 3])
def test_hydrostatic_state_with_face_fields_and_masks(dim):
    """The hydrostatic state psi = H - z stays exact when the bottom head is
    given per face cell (value_field) and the top is Dirichlet only where a
    mask is set (no-flux elsewhere): pins the face indexing of value_field and
    mask_field (lexicographic over the other axes, first fastest)."""
    n = {2: (6, 7), 3: (4, 5, 6)}[dim]
    kinds = [W.NOFLUX] * (2 * dim - 2) + [W.DIRICHLET, W.DIRICHLET]
    p = W.random_problem(dim, n, W.VANGENUCHTEN, 14, bc_kinds=kinds, hetero=True)
    H, Lz = 0.3, p["L"][dim - 1]
    nface = int(np.prod(n[:-1]))
    rng = np.random.default_rng(3)
    p["bc"]["value_field"][2 * dim - 2] = np.full(nface, H)            # bottom: z = 0
    p["bc"]["value"][2 * dim - 1] = H - Lz
    mask = (rng.uniform(size=nface) < 0.5).astype(np.uint8)
    mask[0] = 1
    p["bc"]["mask_field"][2 * dim - 1] = mask
    nn = p["n"]
    hz = Lz / nn[dim - 1]
    idx = np.arange(nn[0] * nn[1] * nn[2])
    iz = [idx % nn[0], (idx // nn[0]) % nn[1], idx // (nn[0] * nn[1])][dim - 1]
    psi = H - (iz + 0.5) * hz
    p["psi0"] = psi
    o = Oracle(p)
    o.prepare(p["dt"], 1)
    _, nrm = o.residual(psi)
    assert nrm <= 1e-13 * np.max(np.abs(o.g()))
    # a bottom head off by 0.1 m in one face cell leaves a defect in exactly the cell above it
    vf = np.full(nface, H)
    k = nface // 2 + 1
    vf[k] = H + 0.1
    p["bc"]["value_field"][2 * dim - 2] = vf
    o2 = Oracle(p)
    o2.prepare(p["dt"], 1)
    r, nrm2 = o2.residual(psi)
    big = np.flatnonzero(np.abs(r) > 1e-9 * np.max(np.abs(o2.g())))
    assert big.tolist() == [k]                     # face cell k lies under fine cell k of the bottom layer
    # a top head off by 0.1 m leaves defects in exactly the top cells whose mask is set
    p["bc"]["value_field"][2 * dim - 2] = np.full(nface, H)
    p["bc"]["value"][2 * dim - 1] = H - Lz + 0.1
    o3 = Oracle(p)
    o3.prepare(p["dt"], 1)
    r, _ = o3.residual(psi)
    big = np.flatnonzero(np.abs(r) > 1e-9 * np.max(np.abs(o3.g())))
    top0 = len(psi) - nface
    assert big.tolist() == (top0 + np.flatnonzero(mask)).tolist()


@pytest.mark.parametrize("face", [0, 3, 4])
def test_face_conductances_restrict_as_the_cell_restriction(face):
    """A coarse boundary conductance is the full-weighting restriction of the
    fine face array over the face's two in-plane axes (R5): the numbers that
    the cell transfer (R6) gives for a 3-d field repeating the fine face
    array along the face normal (whose restriction rows sum to one).  On a
    non-square face with a varying boundary head, a transposed in-plane index
    or a wrong axis breaks it."""
    n = (9, 7, 6)
    kinds = [W.NOFLUX] * 6
    kinds[face] = W.DIRICHLET
    p = W.random_problem(3, n, W.VANGENUCHTEN, 21, bc_kinds=kinds, hetero=True)
    ax = face // 2
    ia, ib = [a for a in range(3) if a != ax]
    p["bc"]["value_field"][face] = np.random.default_rng(5).uniform(-2.0, -0.05, n[ia] * n[ib])
    o = Oracle(p)
    o.prepare(p["dt"], 1)
    kb0, kb1 = o.array(10 + face, 0), o.array(10 + face, 1)
    assert np.ptp(kb0) > 0
    idx = np.indices((n[2], n[1], n[0]))[::-1]          # idx[a] = cell index along axis a (x fastest)
    f3 = kb0[idx[ia] + n[ia] * idx[ib]]
    c3 = o.restrict(f3.ravel(), 0)
    nc = o.level_n(1)
    cidx = np.indices((nc[2], nc[1], nc[0]))[::-1]
    on_plane = (cidx[ax] == 0).ravel()
    ref = np.empty(nc[ia] * nc[ib])
    ref[(cidx[ia] + nc[ia] * cidx[ib]).ravel()[on_plane]] = c3[on_plane]
    assert np.max(np.abs(kb1 - ref)) <= 1e-14 * np.max(np.abs(ref))


@pytest.mark.parametrize("dim", [1, 2])
def test_saturated_linear_head_is_exact(dim):
    """Saturated (psi >= 0, K = Ks) flow between two Dirichlet heads: the
    linear total head is the exact discrete solution.  This pins the
    half-cell distance of the Dirichlet faces."""
    n = {1: (10,), 2: (4, 9)}[dim]
    kinds = [W.NOFLUX] * (2 * dim - 2) + [W.DIRICHLET, W.DIRICHLET]
    p = W.random_problem(dim, n, W.VANGENUCHTEN, 12, bc_kinds=kinds)
    Lz = p["L"][dim - 1]
    P0, P1 = 1.0, 0.5
    p["bc"]["value"][2 * dim - 2] = P0
    p["bc"]["value"][2 * dim - 1] = P1
    nn = p["n"]
    hz = Lz / nn[dim - 1]
    idx = np.arange(nn[0] * nn[1] * nn[2])
    iz = [idx % nn[0], (idx // nn[0]) % nn[1], idx // (nn[0] * nn[1])][dim - 1]
    z = (iz + 0.5) * hz
    Hz = P0 + ((P1 + Lz) - P0) * z / Lz
    psi = Hz - z
    assert np.all(psi >= 0)
    p["psi0"] = psi
    o = Oracle(p)
    o.prepare(p["dt"], 1)
    _, nrm = o.residual(psi)
    assert nrm <= 1e-13 * np.max(np.abs(o.g()))
    # a wrong boundary distance would leave a residual of order Ks*(P1+Lz-P0)/(Lz*hz)
    assert p["soil"]["Ks"] * ((P1 + Lz - P0) / Lz) / hz > 1e6 * nrm


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_constant_flux_column_is_exact(dim):
    """Uniform psi0 < 0 with inflow K(psi0) on top and free drainage at the
    bottom is a steady unit-gradient flow: zero residual (pins the gravity
    term, the prescribed-flux and the free-drainage boundaries)."""
    n = {1: (8,), 2: (5, 6), 3: (3, 4, 5)}[dim]
    kinds = [W.NOFLUX] * (2 * dim - 2) + [W.FREE_DRAINAGE, W.FLUX]
    p = W.random_problem(dim, n, W.HAVERKAMP, 13, bc_kinds=kinds)
    psi0 = -0.4
    o0 = Oracle(p)
    _, _, K0 = o0.soil(0, psi0)
    p["bc"]["value"][2 * dim - 1] = K0
    p["psi0"] = np.full(len(p["psi0"]), psi0)
    o = Oracle(p)
    o.prepare(p["dt"], 1)
    _, nrm = o.residual(p["psi0"])
    assert nrm <= 1e-13 * np.max(np.abs(o.g()))
    # flipping the flux direction must leave a residual
    p["bc"]["value"][2 * dim - 1] = -K0
    o2 = Oracle(p)
    o2.prepare(p["dt"], 1)
    _, nrm2 = o2.residual(p["psi0"])
    assert nrm2 > 1e6 * nrm


@pytest.mark.parametrize("dim", [2, 3])
def test_flux_face_field_column_is_exact(dim):
    """The unit-gradient column with its inflow K(psi0) given per top face
    cell (value_field of a FLUX face) has zero defect; raising one face
    cell's inflow by q leaves the defect g - N = q/h (the inflow enters g) in
    exactly the top cell under it."""
    n = {2: (5, 6), 3: (3, 4, 5)}[dim]
    kinds = [W.NOFLUX] * (2 * dim - 2) + [W.FREE_DRAINAGE, W.FLUX]
    p = W.random_problem(dim, n, W.HAVERKAMP, 15, bc_kinds=kinds)
    psi0 = -0.4
    _, _, K0 = Oracle(p).soil(0, psi0)
    nface = int(np.prod(n[:-1]))
    p["bc"]["value_field"][2 * dim - 1] = np.full(nface, K0)
    p["psi0"] = np.full(len(p["psi0"]), psi0)
    o = Oracle(p)
    o.prepare(p["dt"], 1)
    _, nrm = o.residual(p["psi0"])
    assert nrm <= 1e-13 * np.max(np.abs(o.g()))
    k, q = nface - 2, 3.0 * K0
    vf = np.full(nface, K0)
    vf[k] += q
    p["bc"]["value_field"][2 * dim - 1] = vf
    o2 = Oracle(p)
    o2.prepare(p["dt"], 1)
    r, _ = o2.residual(p["psi0"])
    hz = p["L"][dim - 1] / n[-1]
    cell = len(r) - nface + k
    assert abs(r[cell] - q / hz) <= 1e-12 * q / hz
    r[cell] = 0.0
    assert np.max(np.abs(r)) <= 1e-13 * np.max(np.abs(o2.g()))


@pytest.mark.parametrize("model", [W.HAVERKAMP, W.GARDNER, W.VANGENUCHTEN])
def test_steady_flux_column_converges_to_the_ode_solution(model):
    """A column with a Dirichlet head h_b at the bottom and a prescribed inflow
    q at the top settles to the steady profile of K(h) (dh/dz + 1) = q, the
    ODE dh/dz = q / K(h) - 1 from h(0) = h_b (integrated here by scipy's
    DOP853 to 1e-13, with the law K(h) pinned by the paper's calibration).
    Time steps of 1e5 s reach the discrete steady state; it converges to the
    ODE's values at the cell centres at second order (error ratio -> 4 under
    halving of the cells)."""
    solve_ivp = pytest.importorskip("scipy.integrate").solve_ivp
    dt, hb = 1e5, -1.0
    errs = []
    for n in (32, 64, 128, 256):
        p = W.random_problem(1, (n,), model, 16, bc_kinds=[W.DIRICHLET, W.FLUX], dt=dt,
                             tol=1e-14 * dt, max_cycles=400)
        q = 3.0 * Oracle(p).soil(0, hb)[2]
        p["bc"]["value"] = [hb, q] + [0.0] * 4
        p["psi0"] = np.full(n, hb)
        o = Oracle(p)
        zc = (np.arange(n) + 0.5) / n * p["L"][0]
        ode = solve_ivp(lambda z, h: [q / o.soil(0, h[0])[2] - 1.0], (0.0, zc[-1]), [hb], t_eval=zc,
                        rtol=1e-13, atol=1e-15, method="DOP853")
        last = o.state()
        for _ in range(200):
            assert o.step()[0] == ORC_OK
            cur = o.state()
            moved = np.max(np.abs(cur - last))
            last = cur
            if moved < 1e-12:
                break
        assert moved < 1e-12
        errs.append(np.max(np.abs(cur - ode.y[0])))
    ratios = [errs[k] / errs[k + 1] for k in range(3)]
    assert errs[0] < 2e-4 and all(r > 3.0 for r in ratios[1:]) and ratios[-1] > 3.6, (errs, ratios)


def test_gardner_2d_steady_state_converges_to_the_kirchhoff_solution():
    """Section 4.2's 2D Gardner problem has a closed-form steady state.  With
    K = Ks e^{alpha h} and u = e^{alpha h}, steady flow div(K grad(h + z)) = 0
    (z up) becomes the linear equation lap u + alpha du/dz = 0.  With
    u = e^{-10 alpha} =: u_r on the sides and the bottom and
    u = u_r + (1 - u_r) sin(pi x / L) on the top (the paper's top head),
    separation of variables gives
        u = u_r + (1 - u_r) sin(pi x / L) e^{alpha (L - z) / 2} sinh(beta z) / sinh(beta L),
        beta = sqrt(alpha^2 / 4 + pi^2 / L^2).
    Long implicit steps with the lagged conductivity are a Picard iteration
    whose fixed point is the discrete steady state; it approaches h = ln(u) /
    alpha at second order in the cell size (a wrong gravity sign, Dirichlet
    distance or face average stalls the error at O(1) or O(h))."""
    alpha, L = 0.164, 10.0
    ur = math.exp(-10.0 * alpha)
    beta = math.sqrt(alpha ** 2 / 4.0 + (math.pi / L) ** 2)
    dt = 1e9
    errs = []
    for n in (8, 16, 32):
        p = W.gardner_2d(n=n, dt=dt, nsteps=1, tol=1e-14 * dt, max_cycles=400)
        assert p["soil"]["p1"] == alpha and p["L"][:2] == (L, L)
        c = (np.arange(n) + 0.5) * (L / n)
        X, Z = np.meshgrid(c, c)                      # [z, x]: x fastest when flattened
        u = ur + (1.0 - ur) * np.sin(np.pi * X / L) * np.exp(alpha * (L - Z) / 2.0) * np.sinh(beta * Z) \
            / math.sinh(beta * L)
        exact = (np.log(u) / alpha).reshape(-1)
        o = Oracle(p)
        last = o.state()
        for _ in range(80):
            assert o.step()[0] == ORC_OK
            cur = o.state()
            moved = np.max(np.abs(cur - last))
            last = cur
            if moved < 1e-11:
                break
        assert moved < 1e-11
        errs.append(np.max(np.abs(cur - exact)))
    assert errs[0] < 0.1
    assert errs[0] / errs[1] > 3.3 and errs[1] / errs[2] > 3.3, errs


def test_gardner_3d_steady_state_converges_to_the_kirchhoff_solution():
    """The same closed form in three dimensions: top head
    ln(u_r + (1 - u_r) sin(pi x / L) sin(pi y / L)) / alpha per face cell,
    -10 m on the other faces, beta = sqrt(alpha^2 / 4 + 2 pi^2 / L^2); the
    discrete steady state approaches it at second order (pins the second
    horizontal axis and the face-cell order of a 3-d value field)."""
    alpha, L, dt = 0.164, 10.0, 1e9
    ur = math.exp(-10.0 * alpha)
    beta = math.sqrt(alpha ** 2 / 4.0 + 2.0 * (math.pi / L) ** 2)
    errs = []
    for n in (8, 16):
        p = W.random_problem(3, (n, n, n), W.GARDNER, 0, bc_kinds=[W.DIRICHLET] * 6, L=L, dt=dt,
                             tol=1e-14 * dt, max_cycles=400)
        p["soil"] = W._soil(W.GARDNER, 0.1, 0.45, 0.15, p1=alpha)
        c = (np.arange(n) + 0.5) * (L / n)
        Y, X = np.meshgrid(c, c, indexing="ij")              # top face cells [y, x], x fastest
        p["bc"]["value"] = [-10.0] * 6
        p["bc"]["value_field"][5] = (np.log(ur + (1.0 - ur) * np.sin(np.pi * X / L) * np.sin(np.pi * Y / L))
                                     / alpha).reshape(-1)
        p["psi0"] = np.full(n ** 3, -10.0)
        Z3, Y3, X3 = np.meshgrid(c, c, c, indexing="ij")
        u = ur + (1.0 - ur) * np.sin(np.pi * X3 / L) * np.sin(np.pi * Y3 / L) * np.exp(alpha * (L - Z3) / 2.0) \
            * np.sinh(beta * Z3) / math.sinh(beta * L)
        exact = (np.log(u) / alpha).reshape(-1)
        o = Oracle(p)
        last = o.state()
        for _ in range(80):
            assert o.step()[0] == ORC_OK
            cur = o.state()
            moved = np.max(np.abs(cur - last))
            last = cur
            if moved < 1e-11:
                break
        assert moved < 1e-11
        errs.append(np.max(np.abs(cur - exact)))
    assert errs[0] < 0.2 and errs[0] / errs[1] > 3.2, errs


@pytest.mark.parametrize("scheme", [1, 2])
@pytest.mark.parametrize("dim", [1, 2, 3])
def test_discrete_mass_balance_identity(scheme, dim):
    """Conservation: sum_i V (a theta(psi_i) - hist_i) equals the boundary
    inflow minus uptake minus the xi term plus the volume-weighted residual,
    to round-off, for any psi (interior fluxes telescope)."""
    kinds = {1: [W.FREE_DRAINAGE, W.DIRICHLET], 2: [W.DIRICHLET, W.FLUX, W.FREE_DRAINAGE, W.DIRICHLET],
             3: [W.NOFLUX, W.DIRICHLET, W.FLUX, W.NOFLUX, W.FREE_DRAINAGE, W.DIRICHLET]}[dim]
    n = {1: (11,), 2: (6, 7), 3: (4, 3, 5)}[dim]
    p = W.random_problem(dim, n, W.VANGENUCHTEN, 21 + dim, bc_kinds=kinds, hetero=True,
                         sink=True, xi=3e-4, scheme=scheme)
    rng = np.random.default_rng(5)
    if scheme == 2:
        p["psi_prev"] = p["psi0"] + rng.uniform(-0.05, 0.05, len(p["psi0"]))
    o = Oracle(p)
    assert o.prepare(p["dt"], scheme) == scheme
    psi = o.vcycle(p["psi0"])               # any state: the identity is exact
    V = o.cell_volume()
    a = o.a
    hist = o.array(7)
    pstar = o.array(6)
    th = np.array([o.soil(i, x)[0] for i, x in enumerate(psi)])
    S = np.array([o.sink(i, x)[0] for i, x in enumerate(psi)])
    r, _ = o.residual(psi)
    lhs = V * np.sum(a * th - hist)
    Q = o.boundary_inflow(psi)
    xi = p["opts"]["xi"]
    rhs = Q - V * np.sum(S) - xi * V * np.sum(psi - pstar) - V * np.sum(r)
    scale = V * (np.sum(np.abs(a * th)) + np.sum(np.abs(hist))) + abs(Q)
    assert abs(lhs - rhs) <= 1e-13 * scale, (lhs, rhs)


# ---------------------------------------------------------------------------
# Section 3: Lemma 3.1, Theorem 3.1 and the scalar point update.
# ---------------------------------------------------------------------------
def _splitting(M):
    Lo = np.tril(M, -1)
    D = np.diag(np.diag(M))
    U = np.triu(M, 1)
    return Lo, D, U


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_lemma31_bounds(seed):
    p = W.random_problem(2, (4, 5), W.VANGENUCHTEN, 30 + seed, hetero=True,
                         bc_kinds=[W.DIRICHLET, W.NOFLUX, W.FREE_DRAINAGE, W.DIRICHLET])
    o = Oracle(p)
    o.prepare(p["dt"], 1)
    M = o.dense_M()
    Lo, D, U = _splitting(M)
    rng = np.random.default_rng(seed)
    n = M.shape[0]
    scale = np.mean(np.diag(M))
    kap = rng.uniform(0.01, 1.0, n) * scale
    mu = rng.uniform(0.01, 1.0, n) * scale
    al, be = rng.uniform(0.1, 2.0, 2)
    Uk = U - np.diag(kap)
    rows = np.abs(Uk).sum(axis=1)
    lam_bar, lam_low = rows.max(), rows.min()
    # first bullet: ||alpha I - beta U_kappa||_inf = alpha + beta lam_bar(U_kappa)
    assert abs(np.abs(al * np.eye(n) - be * Uk).sum(axis=1).max() - (al + be * lam_bar)) \
        <= 1e-12 * (al + be * lam_bar)
    # second bullet
    Aop = al * np.diag(mu) + be * (Lo + D + np.diag(kap))
    inv_norm = np.abs(np.linalg.inv(Aop)).sum(axis=1).max()
    assert inv_norm <= 1.0 / (al * mu.min() + be * lam_low) * (1 + 1e-12)


def _changed_after_one_sweep(n, ordering, cell, dim):
    kinds = [W.NOFLUX] * (2 * dim - 2) + [W.FREE_DRAINAGE, W.DIRICHLET]
    # a long step, so that the coupling dominates the storage term and a
    # perturbation decays slowly from cell to cell
    p = W.random_problem(dim, n, W.VANGENUCHTEN, 41, hetero=True, ordering=ordering, newton_iters=0, dt=1e4,
                         tol=1e-16, max_cycles=300, coarsest_max_n=2, bc_kinds=kinds)
    o = Oracle(p)
    o.prepare(p["dt"], 1)
    star, st, info = o.solve_current(p["psi0"])
    floor = np.max(np.abs(o.sweep(star) - star))        # what a sweep moves the converged state
    assert floor <= 1e-12
    psi = star.copy()
    psi[cell] += 0.05
    new = o.sweep(psi)
    return set(np.flatnonzero(np.abs(new - psi) > 1e-10).tolist())


def _expected_changes(n, order, cell):
    """Cells that a Gauss-Seidel sweep in the given order changes when only
    `cell` is off the solution: a visited cell lands off the solution iff a
    neighbour is off it at that moment (else its point solve returns the
    solution), and it changes iff it was off before or lands off now."""
    dim = len(n)
    off = np.zeros(int(np.prod(n)), dtype=bool)
    off[cell] = True
    changed = set()
    for c in order:
        ii = np.unravel_index(c, n[::-1])[::-1]          # x fastest
        nb = []
        for a in range(dim):
            for s in (-1, 1):
                jj = list(ii)
                jj[a] += s
                if 0 <= jj[a] < n[a]:
                    nb.append(int(np.ravel_multi_index(tuple(jj[::-1]), n[::-1])))
        now = any(off[j] for j in nb)
        if off[c] or now:
            changed.add(int(c))
        off[c] = now
    return changed


SWEEP_CASES = [((9,), [4, 5, 8]), ((5, 4), [7, 12, 19]), ((3, 4, 3), [17, 22, 35])]


@pytest.mark.parametrize("n,cells", SWEEP_CASES)
def test_sweep_orders_by_where_a_perturbation_travels(n, cells):
    """Which cells one sweep changes, starting from the solution with one
    cell perturbed, fixes the order of the sweep: lexicographic, ascending
    (Section 3.1), and red-black with the colour of cell 0 first.  A reversed
    or recoloured order moves the perturbation elsewhere."""
    N = int(np.prod(n))
    lex = list(range(N))
    idx = np.arange(N)
    coords = np.stack(np.unravel_index(idx, n[::-1])[::-1])
    colour = coords.sum(axis=0) % 2
    rb = list(idx[colour == 0]) + list(idx[colour == 1])
    for cell in cells:
        assert _changed_after_one_sweep(n, 0, cell, len(n)) == _expected_changes(n, lex, cell), ("lex", cell)
        assert _changed_after_one_sweep(n, 1, cell, len(n)) == _expected_changes(n, rb, cell), ("rb", cell)
    # the rule tells these orders apart on these cells (it cannot tell which
    # axis runs fastest: monotone paths reach the same cells either way)
    assert any(_expected_changes(n, lex[::-1], c) != _expected_changes(n, lex, c) for c in cells)
    assert all(_expected_changes(n, rb, c) != _expected_changes(n, lex, c) for c in cells)


@pytest.mark.parametrize("n", [(9,), (5, 4), (3, 4, 3)])
def test_half_sweeps_are_the_two_colours_of_a_red_black_sweep(n):
    """Half-sweep colour c updates exactly the cells with (i0 + i1 + i2) mod 2
    = c, and colour 0 then colour 1 is one red-black sweep, bit for bit (the
    half-sweeps the GPU stages are compared with)."""
    p = W.random_problem(len(n), n, W.VANGENUCHTEN, 60, sink=True, newton_iters=0)
    o = Oracle(p)
    o.prepare(p["dt"], 1)
    psi = np.array(p["psi0"], dtype=np.float64) + np.random.default_rng(1).uniform(-0.2, 0.2, W.ncells(p))
    coords = np.stack(np.unravel_index(np.arange(psi.size), n[::-1])[::-1])
    colour = coords.sum(axis=0) % 2
    red = o.sweep(psi, color=0)
    assert np.array_equal(red[colour == 1], psi[colour == 1]) and np.all(red[colour == 0] != psi[colour == 0])
    both = o.sweep(red, color=1)
    assert np.array_equal(both[colour == 0], red[colour == 0]) and np.all(both[colour == 1] != red[colour == 1])
    assert np.array_equal(both, o.sweep(psi, ordering=1))


@pytest.mark.parametrize("ordering", [0, 1])
@pytest.mark.parametrize("model", [W.HAVERKAMP, W.VANGENUCHTEN])
def test_theorem31_contraction_per_sweep(ordering, model):
    """With Remark 3.1's shift (equal row sums of U_kappa) the NGS sweep
    contracts the max-norm error by at most
    lam(U_kappa) / (min lambda_i + xi + lam(U_kappa)) each sweep, for the
    lexicographic order and for red-black (both are triangular splittings)."""
    p = W.random_problem(2, (6, 5), model, 40, hetero=True, kappa_mode=1, xi=0.0,
                         ordering=ordering, newton_iters=0, tol=1e-15, max_levels=1,
                         coarse_max_sweeps=5000, coarse_rtol=1e-16,
                         bc_kinds=[W.NOFLUX, W.NOFLUX, W.FREE_DRAINAGE, W.DIRICHLET])
    o = Oracle(p)
    o.prepare(p["dt"], 1)
    star, st, info = o.solve_current(p["psi0"])
    assert info["resid"] <= 1e-13
    M = o.dense_M()
    _, _, U = _splitting(M) if ordering == 0 else (None, None, None)
    kap = o.array(5)
    if ordering == 0:
        u = -U.sum(axis=1)
    else:
        nn = o.level_n(0)
        idx = np.arange(M.shape[0])
        color = (idx % nn[0] + (idx // nn[0]) % nn[1]) % 2
        u = np.where(color == 0, -(M - np.diag(np.diag(M))).sum(axis=1), 0.0)
    rows = kap + u
    assert np.allclose(rows, rows.max(), rtol=1e-12)
    lam = rows.max()
    a = o.a
    rng = np.random.default_rng(1)
    psi = star + rng.uniform(-0.3, 0.3, len(star))
    for s in range(6):
        new = o.sweep(psi)
        e0 = np.max(np.abs(psi - star))
        e1 = np.max(np.abs(new - star))
        lo = np.minimum(new, star)
        hi = np.maximum(new, star)
        dmin = np.array([min(o.soil(i, lo[i])[1], o.soil(i, hi[i])[1]) for i in range(len(star))])
        rho = lam / (a * dmin.min() + 0.0 + lam)
        assert e1 <= rho * e0 * (1 + 1e-9) + 1e-14, (s, e1, e0, rho)
        psi = new


@pytest.mark.parametrize("model", [W.HAVERKAMP, W.GARDNER, W.VANGENUCHTEN])
def test_point_solve_matches_bracketing_root(model):
    p = W.random_problem(1, 6, model, 50, sink=True)
    o = Oracle(p)
    o.prepare(p["dt"], 1)
    a = o.a
    rng = np.random.default_rng(2)
    cell = p["n"][0] - 1
    for _ in range(25):
        cc = 10 ** rng.uniform(-4, 1)
        target = rng.uniform(-3.0, 0.2)
        th, _, _ = o.soil(cell, target)
        S, _ = o.sink(cell, target)
        f = a * th + S + cc * target

        def F(x):
            return a * o.soil(cell, x)[0] + o.sink(cell, x)[0] + cc * x - f

        lo, hi = target - 10.0, target + 10.0
        root = brentq(F, lo, hi, xtol=1e-15, rtol=4 * np.finfo(float).eps)
        x, it = o.point_solve(cell, cc, f, x0=rng.uniform(-3, 0), newton_iters=0)
        assert abs(x - root) <= 1e-12 * max(1.0, abs(root)), (x, root, it)
        x60, _ = o.point_solve(cell, cc, f, x0=root, newton_iters=3)
        assert abs(x60 - root) <= 1e-12 * max(1.0, abs(root))


@pytest.mark.parametrize("model", [W.HAVERKAMP, W.GARDNER, W.VANGENUCHTEN])
def test_fixed_count_point_solve_takes_plain_newton_steps(model):
    """With a fixed count k the point solve takes k textbook Newton steps
    x <- x - F(x)/F'(x), F'(x) = a theta'(x) + S'(x) + c, as long as each
    lands strictly inside the running bracket (eq. point-update, Section
    3.1's Newton steps); a damped or a bisected step breaks it."""
    p = W.random_problem(1, 6, model, 51, sink=True)
    o = Oracle(p)
    o.prepare(p["dt"], 1)
    a = o.a
    rng = np.random.default_rng(7)
    cell = p["n"][0] - 1
    soil = p["soil"]
    smax = o.array(4, 0)[cell]
    used = 0
    for _ in range(40):
        cc = 10 ** rng.uniform(-3, 1)
        target = rng.uniform(-3.0, -0.05)
        f = a * o.soil(cell, target)[0] + o.sink(cell, target)[0] + cc * target
        x0 = target + rng.uniform(-0.05, 0.05) * max(1.0, abs(target))
        lo = (f - a * soil["theta_s"] - smax) / cc
        hi = (f - a * soil["theta_r"]) / cc
        xs, x, ok = [], min(max(x0, lo), hi), True
        for _k in range(2):
            th, dth, _ = o.soil(cell, x)
            S, dS = o.sink(cell, x)
            F = a * th + S + cc * x - f
            if F > 0:
                hi = x
            else:
                lo = x
            xn = x - F / (a * dth + dS + cc)
            if not (lo < xn < hi):
                ok = False
                break
            x = xn
            xs.append(x)
        if not ok:
            continue
        used += 1
        for k in (1, 2):
            got, it = o.point_solve(cell, cc, f, x0=x0, newton_iters=k)
            assert it == k and abs(got - xs[k - 1]) <= 4e-15 * max(1.0, abs(got)), (k, got, xs[k - 1])
    assert used >= 20


# ---------------------------------------------------------------------------
# Coarse operators (Section 3.2, "complete analogy").
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("n,cmax", [((8,), 4), ((9,), 4), ((129,), 4), ((7, 10), 4), ((33, 17), 8),
                                    ((6, 4, 8), 4), ((5, 6, 7), 2), ((256,), 8)])
def test_hierarchy_halves_every_axis_up_to_the_coarsest_size(n, cmax):
    """Levels (R6, R7): every axis with more than one cell goes from N to
    ceil(N/2) until the largest axis has at most coarsest_max_n cells; the
    spacing of each level is L/N."""
    dim = len(n)
    p = W.random_problem(dim, n, W.GARDNER, 3, coarsest_max_n=cmax)
    o = Oracle(p)
    want = [list(n) + [1] * (3 - dim)]
    while max(want[-1]) > cmax:
        want.append([(x + 1) // 2 if x > 1 else 1 for x in want[-1]])
    assert o.nlevels == len(want)
    for lev, w in enumerate(want):
        assert list(o.level_n(lev)) == w, (lev, o.level_n(lev), w)
        assert o.cell_volume(lev) == pytest.approx(np.prod([p["L"][a] / w[a] for a in range(dim)]), rel=1e-15)


COARSE_CASES = [(1, (8,)), (1, (9,)), (2, (8, 6)), (2, (7, 10)), (3, (6, 4, 8)), (3, (5, 6, 7))]


@pytest.mark.parametrize("dim,n", COARSE_CASES)
@pytest.mark.parametrize("model", [W.HAVERKAMP, W.GARDNER, W.VANGENUCHTEN])
def test_coarse_operator_is_rediscretisation_for_constant_coefficients(dim, n, model):
    """Where "complete analogy" has one meaning: a homogeneous soil at a
    uniform state psi0 (so every lagged conductivity, Dirichlet face value and
    soil parameter is one constant).  The level-1 operator N_H must then be
    the same discretisation on the grid of ceil(n/2) cells: equal to the
    fine operator of that coarser problem applied to any vector, Dirichlet
    faces included.  A wrong coarse spacing, a restriction that does not
    preserve constants, or a face conductivity summed instead of averaged
    breaks it."""
    kinds = {1: [W.DIRICHLET, W.DIRICHLET],
             2: [W.DIRICHLET, W.NOFLUX, W.FREE_DRAINAGE, W.DIRICHLET],
             3: [W.NOFLUX, W.DIRICHLET, W.DIRICHLET, W.NOFLUX, W.FREE_DRAINAGE, W.DIRICHLET]}[dim]
    nc = tuple((k + 1) // 2 for k in n)
    psi0, dt = -0.3, 120.0

    def build(shape):
        p = W.random_problem(dim, shape, model, 21, bc_kinds=kinds, coarsest_max_n=2)
        p["bc"]["value"] = [psi0 if k == W.DIRICHLET else 0.0 for k in p["bc"]["kind"]]
        p["psi0"] = np.full(len(p["psi0"]), psi0)
        o = Oracle(p)
        o.prepare(dt, 1)
        return o

    fine, coarse = build(n), build(nc)
    assert fine.nlevels >= 2 and fine.level_n(1)[:dim] == nc
    assert np.max(np.abs(fine.Kc(1) - coarse.Kc(0))) <= 1e-15 * np.max(coarse.Kc(0))
    M_H, M_c = fine.dense_M(1), coarse.dense_M(0)
    assert np.max(np.abs(M_H - M_c)) <= 1e-13 * np.max(np.abs(M_c))
    rng = np.random.default_rng(5)
    x = psi0 + 0.2 * rng.standard_normal(coarse.ncell())
    got, want = fine.apply_N(x, lev=1), coarse.apply_N(x)
    assert np.max(np.abs(got - want)) <= 1e-12 * np.max(np.abs(want))


# ---------------------------------------------------------------------------
# The implicit step: FAS-NGS reaches the plain solution of N_h(psi) = g_h.
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("dim,n", [(1, (9,)), (2, (5, 7)), (3, (4, 3, 5))])
@pytest.mark.parametrize("model", [W.HAVERKAMP, W.GARDNER, W.VANGENUCHTEN])
def test_fas_solution_equals_dense_newton(dim, n, model):
    kinds = [W.NOFLUX] * (2 * dim - 2) + [W.FREE_DRAINAGE, W.DIRICHLET]
    p = W.random_problem(dim, n, model, 60 + dim, bc_kinds=kinds, hetero=True, sink=True,
                         tol=1e-13, coarsest_max_n=2)
    o = Oracle(p)
    o.prepare(p["dt"], 1)
    psi_fas, st, info = o.solve_current(p["psi0"])
    assert st == ORC_OK
    psi_dn, res = dense_newton(o, p["psi0"])
    assert res <= 1e-13
    assert np.max(np.abs(psi_fas - psi_dn)) <= 1e-10 * max(1.0, np.max(np.abs(psi_dn)))


@pytest.mark.parametrize("dim,n", [(1, (9,)), (2, (5, 7)), (3, (4, 3, 5))])
@pytest.mark.parametrize("model", [W.HAVERKAMP, W.GARDNER, W.VANGENUCHTEN])
def test_error_bound_of_the_defect(dim, n, model):
    """The step's error bound (reading R14).  N(psi) - N(psi*) = D (psi - psi*)
    + M (psi - psi*) exactly, D_i the secant slope of a theta + S + xi psi
    between psi_i and psi*_i; M has non-positive off-diagonals and
    non-negative row sums (Prop. 3.1), so at the cell i of the largest error
    |r_i| >= D_i |e_i|.  That inequality holds for every iterate of the cycle;
    the reported bound ||r|| / min_i (a theta'(psi_i) + S'(psi_i) + xi), its
    point-slope form, holds on these iterates too.  psi* is the dense Newton
    solution; iterates within 1e-8 of it are not compared (its own accuracy)."""
    kinds = [W.NOFLUX] * (2 * dim - 2) + [W.FREE_DRAINAGE, W.DIRICHLET]
    compared = 0
    for seed in (70, 71):
        p = W.random_problem(dim, n, model, seed, bc_kinds=kinds, hetero=True, sink=True, tol=1e-13,
                             coarsest_max_n=2)
        o = Oracle(p)
        o.prepare(p["dt"], 1)
        a, xi = o.a, p["opts"]["xi"]
        ex, res = dense_newton(o, p["psi0"])
        assert res <= 1e-13
        psi = np.array(p["psi0"], dtype=np.float64)
        for _ in range(6):
            e = psi - ex
            if np.max(np.abs(e)) < 1e-8:
                break
            r, _ = o.residual(psi)
            i = int(np.argmax(np.abs(e)))
            th_i, S_i = o.soil(i, psi[i])[0], o.sink(i, psi[i])[0]
            th_x, S_x = o.soil(i, ex[i])[0], o.sink(i, ex[i])[0]
            D_sec = (a * (th_i - th_x) + (S_i - S_x)) / (psi[i] - ex[i]) + xi
            assert abs(e[i]) * D_sec <= abs(r[i]) * (1 + 1e-6), (abs(e[i]) * D_sec, abs(r[i]))
            D_pt = np.array([a * o.soil(j, x)[1] + o.sink(j, x)[1] + xi for j, x in enumerate(psi)])
            if D_pt.min() > 0:
                assert np.max(np.abs(e)) <= np.max(np.abs(r)) / D_pt.min()
            compared += 1
            psi = o.vcycle(psi)
    assert compared >= 2


def test_fas_fixed_point_independent_of_hierarchy():
    """The converged FAS answer does not depend on restriction, prolongation
    or coarse operators: V-cycles, plain NGS and both orderings agree."""
    base = W.random_problem(2, (13, 11), W.VANGENUCHTEN, 70, hetero=True, tol=1e-13,
                            bc_kinds=[W.NOFLUX, W.NOFLUX, W.DIRICHLET, W.DIRICHLET])
    sols = []
    for kw in [dict(), dict(ordering=0), dict(max_levels=1, coarse_max_sweeps=100000,
                                              coarse_rtol=1e-15, max_cycles=2)]:
        p = W.with_opts(base, **kw)
        o = Oracle(p)
        o.prepare(p["dt"], 1)
        psi, st, info = o.solve_current(p["psi0"])
        assert st == ORC_OK, (kw, info)
        sols.append(psi)
    for s in sols[1:]:
        assert np.max(np.abs(s - sols[0])) <= 1e-9


def _median_factor(o, psi, cycle, ncyc):
    res = [o.residual(psi)[1]]
    for _ in range(ncyc):
        psi = cycle(psi)
        res.append(o.residual(psi)[1])
        if res[-1] / o.a < 1e-12:
            break
    return float(np.median([res[i + 1] / res[i] for i in range(1, len(res) - 1)]))


def test_multigrid_factor_bounded_under_refinement():
    """Multigrid (Section 3.2): the V(2,2) contraction factor per cycle stays
    well below 1 as the Celia column is refined (N = 128 -> 2048), while a
    plain NGS sweep's factor tends to 1 (why Table 3's GS(100) is slow)."""
    for n in (128, 512, 2048):
        p = W.celia_1d(n=n, nsteps=3)
        o = Oracle(p)
        for _ in range(2):
            o.prepare(p["dt"], 1)
            f = _median_factor(o, o.state(), o.vcycle, 10)
            assert f <= 0.3, (n, f)
            st, _ = o.step()
            assert st == ORC_OK
    p = W.celia_1d(n=2048, nsteps=3)
    o = Oracle(p)
    o.step()
    o.prepare(p["dt"], 1)
    assert _median_factor(o, o.state(), o.sweep, 40) >= 0.9


def _time_error(scheme, nsteps_list, T=1800.0):
    base = W.random_problem(1, 32, W.GARDNER, 80, bc_kinds=[W.DIRICHLET, W.DIRICHLET],
                            tol=1e-14, newton_iters=0)
    base["soil"]["p1"] = 1.0
    base["bc"]["value"][0] = -1.0
    base["bc"]["value"][1] = -0.3
    z = (np.arange(32) + 0.5) / 32
    base["psi0"] = -1.0 + 0.7 * z
    out = {}
    for ns in nsteps_list:
        o = Oracle(base)
        for _ in range(ns):
            st, _ = o.step(T / ns, scheme)
            assert st == ORC_OK
        out[ns] = o.state()
    return out


@pytest.mark.parametrize("scheme,order", [(1, 1.0), (2, 2.0)])
def test_temporal_convergence_order(scheme, order):
    """First-order BDF1 as in the paper's temporal study (Section 4.1); the
    BDF2 reading must show second order (self-convergence against a fine-step
    run on the same grid)."""
    sols = _time_error(scheme, [8, 16, 32, 1024])
    ref = sols[1024]
    errs = [np.max(np.abs(sols[k] - ref)) for k in (8, 16, 32)]
    slopes = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(abs(s - order) <= 0.35 for s in slopes), (errs, slopes)


# ---------------------------------------------------------------------------
# Full multigrid (Section 3.2): coarsest first, the solution interpolated to
# successively finer grids with cycles on each.
# ---------------------------------------------------------------------------
FMG_PROBLEMS = [
    ("2d_vg_fields_dt3600", lambda: W.random_problem(2, (33, 33), W.VANGENUCHTEN, 3, hetero=True, dt=3600.0,
                                                     newton_iters=0)),
    ("3d_drainage_16", lambda: W.with_opts(W.drainage_3d(n=16, precision=0), newton_iters=0)),
]


@pytest.mark.parametrize("mk", [p[1] for p in FMG_PROBLEMS], ids=[p[0] for p in FMG_PROBLEMS])
def test_fmg_pass_beats_one_cycle(mk):
    """Nested iteration with one cycle per level reaches a smaller defect than
    one cycle from the same start (a wrong sign in the interpolated
    correction, or coarse right sides left unrestricted, make it worse)."""
    p = mk()
    o = Oracle(W.with_opts(p, fmg_cycles=1))
    o.prepare(p["dt"], 1)
    psi0 = np.array(p["psi0"], dtype=np.float64)
    _, r_start = o.residual(psi0)
    _, r_v = o.residual(o.vcycle(psi0))
    # the pass on a fresh context: a cycle leaves FAS right sides on the
    # coarse levels, which would stand in for unrestricted ones
    f = Oracle(W.with_opts(p, fmg_cycles=1))
    f.prepare(p["dt"], 1)
    _, r_fmg = f.residual(f.fmg(psi0))
    assert r_fmg < 0.8 * r_v < r_start, (r_start, r_v, r_fmg)


@pytest.mark.parametrize("cycles", [1, 2])
@pytest.mark.parametrize("mk", [p[1] for p in FMG_PROBLEMS], ids=[p[0] for p in FMG_PROBLEMS])
def test_fmg_pass_is_nested_iteration(mk, cycles):
    """The pass written out from the oracle's single stages (Section 3.2's
    nested iteration, R17): right sides g_{l+1} = R g_l and starting iterates
    psi_{l+1} = R psi_l on the way down; on the way up each level first
    takes the interpolated change of the coarser one, psi_l += P(psi_{l+1} -
    R psi_l), then `cycles` cycles on its own right side.  Bit for bit."""
    p = W.with_opts(mk(), fmg_cycles=cycles)
    o = Oracle(p)
    o.prepare(p["dt"], 1)
    nl = o.nlevels
    psi = [np.array(p["psi0"], dtype=np.float64)]
    g = [o.g(0)]
    for l in range(nl - 1):
        psi.append(o.restrict(psi[l], l))
        g.append(o.restrict(g[l], l))
    start = [x.copy() for x in psi]
    for _ in range(cycles):
        psi[nl - 1] = o.vcycle(psi[nl - 1], g[nl - 1], nl - 1)
    for l in range(nl - 2, -1, -1):
        psi[l] = o.prolong_add(psi[l + 1] - start[l + 1], psi[l], l)
        for _ in range(cycles):
            psi[l] = o.vcycle(psi[l], g[l], l)
    fresh = Oracle(p)
    fresh.prepare(p["dt"], 1)
    assert np.array_equal(fresh.fmg(p["psi0"]), psi[0])


def test_fmg_step_reaches_the_cycle_solution():
    """The FMG start changes the iterates, not the solution of the step."""
    p = W.with_opts(FMG_PROBLEMS[1][1](), tol=1e-12, max_cycles=200)
    a, b = Oracle(p), Oracle(W.with_opts(p, fmg_cycles=1))
    sa, ia = a.step()
    sb, ib = b.step()
    assert sa == sb == ORC_OK
    assert ib["resid"] <= 1e-12 and ib["resid0"] == pytest.approx(ia["resid0"])
    assert np.max(np.abs(a.state() - b.state())) <= 1e-9 * np.max(np.abs(a.state()))


# ---------------------------------------------------------------------------
# The cycle's structure (Section 3.2): steps 1-7 of the two-grid FAS step with
# the coarse solve replaced by gamma recursive cycles (gamma = 2 on the
# gamma_levels finest levels when gamma_levels > 0, V below), and the
# coarsest level swept until its defect is coarse_rtol times the initial one
# or coarse_max_sweeps sweeps have run (R7).  Written here from the oracle's
# single stages; the recursion must give the oracle's cycle bit for bit.
# ---------------------------------------------------------------------------
def _fas_cycle(o, opts, psi, g, lev):
    nl = o.nlevels
    if lev == nl - 1:
        _, d0 = o.residual(psi, g, lev)
        for _ in range(opts["coarse_max_sweeps"]):
            psi = o.sweep(psi, g, lev)
            _, d = o.residual(psi, g, lev)
            if not d > opts["coarse_rtol"] * d0:
                break
        return psi
    for _ in range(opts["nu1"]):                                   # 1 pre-smoothing
        psi = o.sweep(psi, g, lev)
    d, _ = o.residual(psi, g, lev)                                 # 2 defect
    psibar = o.restrict(psi, lev)                                  # 3 restriction
    dH = o.restrict(d, lev)
    gH = o.apply_N(psibar, lev + 1) + dH                           # 4 coarse right side
    gam = max(opts["cycle_gamma"], 1)
    if opts["gamma_levels"] > 0 and lev >= opts["gamma_levels"]:
        gam = 1
    psiH = psibar.copy()
    for _ in range(gam):                                           # 5 coarse solve
        psiH = _fas_cycle(o, opts, psiH, gH, lev + 1)
    psi = o.prolong_add(psiH - psibar, psi, lev)                   # 6 correction
    for _ in range(opts["nu2"]):                                   # 7 post-smoothing
        psi = o.sweep(psi, g, lev)
    return psi


@pytest.mark.parametrize("gamma,glev,nu1,nu2", [(1, 0, 2, 2), (2, 0, 1, 1), (2, 1, 0, 2), (2, 2, 2, 1), (3, 1, 1, 0)])
@pytest.mark.parametrize("dim", [2, 3])
def test_cycle_is_fas_steps_1_to_7_recursively(dim, gamma, glev, nu1, nu2):
    shape = (21, 17) if dim == 2 else (13, 10, 9)
    p = W.random_problem(dim, shape, W.VANGENUCHTEN, 40 + dim, hetero=True, sink=True, newton_iters=0,
                         cycle_gamma=gamma, gamma_levels=glev, nu1=nu1, nu2=nu2, coarse_max_sweeps=7)
    o = Oracle(p)
    assert o.nlevels >= 3
    o.prepare(p["dt"], 1)
    psi = np.array(p["psi0"], dtype=np.float64)
    g = o.g()
    for _ in range(2):
        ref = o.vcycle(psi)
        mine = _fas_cycle(o, p["opts"], psi, g, 0)
        assert np.array_equal(mine, ref)
        psi = ref
