"""CUDA path vs the CPU oracle, stage by stage and step by step (needs a GPU).

Tolerances (FP64 mode): the two sides evaluate the same formulas with
different libm routines, summation order and fused multiply-adds, so single
stages agree to ~1e-13 relative; iterated results (V-cycles, steps) to the
1e-10 norm-wise relative bound ||dpsi||_inf <= 1e-10 ||psi_ref||_inf.
Mixed mode is checked against the a-posteriori bound
||psi_mixed - psi_ref||_inf <= (||r_mixed|| + ||r_ref||) / min_i(a theta'_i + xi)
(the diagonal-dominance argument of Lemma 3.1 applied to the whole Jacobian).
Mixed mode evaluates K(psi*), theta and the defect in float-float arithmetic
(laws within DD_EPS = 6e-12 relative, the bound of the soil-law tests), so its
discrete system differs from the oracle's by at most DD_EPS times the size of
each term; the oracle's residual of a mixed result may exceed the GPU's own by
that much (_law_allowance), on top of the stop tolerance.
"""
import numpy as np
import pytest

from law_allowance import law_allowance
from oracle.oracle import ORC_OK, Oracle
from paper_2606_04292_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2606_04292_gb300 import richards as R  # noqa: E402

STAGE_RTOL = 1e-12
STEP_RTOL = 1e-10
DD_EPS = 6e-12


def _law_allowance(orc, prob, psi):
    return law_allowance(orc, prob, psi, DD_EPS)


# FP64-outer mixed mode (precision 2): the system and the deciding defect are
# FP64, so the oracle's residual of its result exceeds the GPU's own only by
# the rounding of the two FP64 evaluations (different libm routines, FMA
# contraction, summation order): a few tens of ulps of each term's magnitude.
FP64_ROUNDING_EPS = 32 * np.finfo(float).eps


def _fp64_rounding(orc, prob, psi):
    return law_allowance(orc, prob, psi, FP64_ROUNDING_EPS)


def rel(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


def sweep_agrees(orc, prob, lev, got, ref, old, g):
    """A half-sweep result against the oracle's: within STAGE_RTOL norm-wise,
    or, per cell, within the round-off sensitivity of its point equation
    a theta(x) + S(x) + (xi + kappa + m_ii) x = g + sum_j m_ij x_j + kappa x_old:
    16 eps (sum of the magnitudes of its terms) / (its derivative).  A cell
    whose coupling and capacity are both tiny (e.g. a coarse cell of a dry
    column in cm, m_ii ~ 1e-7, a theta' ~ 1e-8 near saturation) has a root
    that rounding alone moves by far more than 1e-12 relative."""
    if rel(got, ref) <= STAGE_RTOL:
        return True
    M = orc.dense_M(lev)
    o = prob["opts"]
    kappa = o["kappa"] if o["kappa_mode"] == 0 else 0.0
    a, xi = orc.a, o["xi"]
    laws = np.array([orc.soil(i, x, lev)[:2] for i, x in enumerate(ref)])
    sinks = np.array([orc.sink(i, x, lev) for i, x in enumerate(ref)])
    offd = np.abs(M - np.diag(np.diag(M))) @ np.abs(ref)
    scale = (a * np.abs(laws[:, 0]) + np.abs(sinks[:, 0]) + np.abs(g) + offd + np.diag(M) * np.abs(ref)
             + kappa * (np.abs(old) + np.abs(ref)) + xi * np.abs(ref))
    deriv = a * laws[:, 1] + sinks[:, 1] + xi + kappa + np.diag(M)
    tol = STAGE_RTOL * np.max(np.abs(ref)) + 16 * np.finfo(float).eps * scale / deriv
    return bool(np.all(np.abs(got - ref) <= tol))


def pair(prob, **opts):
    p = W.with_opts(prob, **opts) if opts else prob
    return R.Solver(p), Oracle(p), p


def layered(dim, n, model, seed, kind, **kw):
    """A random problem whose soil is three materials (one per law) in a
    random or wavy-banded index map."""
    p = W.random_problem(dim, n, model, seed, **kw)
    return W.with_materials(p, W.test_materials(), W.material_pattern(p, kind, 3, seed))


PROBLEMS = [
    ("1d_haverkamp_dir", lambda: W.random_problem(1, 37, W.HAVERKAMP, 1,
                                                   bc_kinds=[W.DIRICHLET, W.DIRICHLET], psi_range=(-1.5, -0.1))),
    ("1d_vg_sink_flux", lambda: W.random_problem(1, 64, W.VANGENUCHTEN, 2, bc_kinds=[W.FREE_DRAINAGE, W.FLUX],
                                                 hetero=True, sink=True)),
    ("2d_vg_strip", lambda: W.strip_2d(n=33, dt=60.0)),
    ("2d_gardner_mixed_bc", lambda: W.random_problem(2, (23, 18), W.GARDNER, 3,
                                                     bc_kinds=[W.DIRICHLET, W.NOFLUX, W.FREE_DRAINAGE, W.FLUX],
                                                     hetero=True)),
    ("3d_vg_hetero_sink", lambda: W.random_problem(3, (17, 12, 9), W.VANGENUCHTEN, 4, hetero=True, sink=True)),
    ("3d_haverkamp_dir", lambda: W.random_problem(3, (10, 11, 13), W.HAVERKAMP, 5,
                                                   bc_kinds=[W.DIRICHLET] * 6)),
    # (W(2,2) down to 4^3: with one fixed Newton step and the adaptive coarse
    # stop, the slower-converging W(0,2) default can part from the oracle by a
    # few cycles on one-ulp differences; W(0,2) has its own test with Newton to
    # round-off below.  An 8^3 coarsest level with one sweep, right for
    # 256^3, leaves 16^3 two levels, too few for the tight-tolerance oracle
    # runs.)
    ("3d_drainage_16", lambda: W.drainage_3d(n=16, precision=0, nu1=2, coarsest_max_n=4, coarse_max_sweeps=2,
                                             inner_rtol=1e-4)),
    ("2d_gardner_paper_32", lambda: W.gardner_2d(n=32)),
    ("1d_celia_composite_40", lambda: W.celia_composite_1d(n=40)),
    ("2d_layers_3mat", lambda: layered(2, (23, 19), W.VANGENUCHTEN, 6, "layers",
                                       bc_kinds=[W.NOFLUX, W.DIRICHLET, W.FREE_DRAINAGE, W.DIRICHLET])),
    ("3d_random_3mat_sink", lambda: layered(3, (11, 9, 13), W.HAVERKAMP, 7, "random", sink=True)),
    ("2d_two_layer_paper_32", lambda: W.two_layer_2d(n=32)),
]
IDS = [p[0] for p in PROBLEMS]


@pytest.mark.parametrize("mk", [p[1] for p in PROBLEMS], ids=IDS)
@pytest.mark.parametrize("scheme", [1, 2])
def test_prepare_matches_oracle(mk, scheme):
    prob = mk()
    if scheme == 2:
        rng = np.random.default_rng(9)
        prob["psi_prev"] = prob["psi0"] + rng.uniform(-0.02, 0.02, len(prob["psi0"]))
    gs, orc, p = pair(prob)
    assert gs.prepare(p["dt"], scheme) == scheme
    assert orc.prepare(p["dt"], scheme) == scheme
    assert gs.nlevels == orc.nlevels
    for lev in range(orc.nlevels):
        assert gs.level_n(lev) == orc.level_n(lev)
        assert rel(gs.get_level(lev, 2), orc.Kc(lev)) <= STAGE_RTOL, lev
        for f in range(2 * p["dim"]):
            kg, ko = gs.get_level(lev, 10 + f), orc.array(10 + f, lev)
            assert np.max(np.abs(kg - ko)) <= STAGE_RTOL * max(np.max(np.abs(ko)), 1e-300), (lev, f)
    assert rel(gs.get_level(0, 1), orc.g(0)) <= STAGE_RTOL


@pytest.mark.parametrize("mk", [p[1] for p in PROBLEMS], ids=IDS)
@pytest.mark.parametrize("scheme", [1, 2])
def test_mixed_prepare_matches_oracle_within_float_float_bound(mk, scheme):
    """Mixed mode takes K(psi*), theta(psi^n), theta(psi^{n-1}) and g in
    float-float: the finest level's Kc and g agree with the oracle to DD_EPS."""
    prob = W.with_opts(mk(), precision=1)
    if scheme == 2:
        rng = np.random.default_rng(9)
        prob["psi_prev"] = prob["psi0"] + rng.uniform(-0.02, 0.02, len(prob["psi0"]))
    gs, orc, p = pair(prob)
    assert gs.prepare(p["dt"], scheme) == scheme
    assert orc.prepare(p["dt"], scheme) == scheme
    assert rel(gs.get_level(0, 2), orc.Kc(0)) <= DD_EPS
    for f in range(2 * p["dim"]):
        kg, ko = gs.get_level(0, 10 + f), orc.array(10 + f, 0)
        assert np.max(np.abs(kg - ko)) <= DD_EPS * max(np.max(np.abs(ko)), 1e-300), f
    assert rel(gs.get_level(0, 1), orc.g(0)) <= DD_EPS


@pytest.mark.parametrize("mk", [p[1] for p in PROBLEMS], ids=IDS)
@pytest.mark.parametrize("newton", [0, 2])
def test_halfsweeps_match_oracle_on_every_level(mk, newton):
    """Red then black half-sweep on every level.  With Newton run to round-off
    the states are random; with the fixed two-step Newton of the solver they
    are near the root, as inside a solve (far from it, two unconverged steps
    can take different bracketing branches on a one-ulp difference)."""
    prob = mk()
    gs, orc, p = pair(prob, newton_iters=newton)
    gs.prepare(p["dt"], 1)
    orc.prepare(p["dt"], 1)
    rng = np.random.default_rng(3)
    for lev in range(orc.nlevels):
        n = orc.ncell(lev)
        if newton == 0:
            psi = rng.uniform(-1.5, -0.05, n)
            g = orc.apply_N(rng.uniform(-1.5, -0.05, n), lev)
        else:
            psi = rng.uniform(-1.5, -0.05, n)
            g = orc.apply_N(psi + rng.uniform(-1e-3, 1e-3, n), lev)
        gs.set_level(lev, 0, psi)
        gs.set_level(lev, 1, g)
        ref = psi
        for color in (0, 1):
            old = ref
            ref = orc.sweep(ref, g, lev, color)
            gs.sweep(lev, color)
            got = gs.get_level(lev, 0)
            assert sweep_agrees(orc, p, lev, got, ref, old, g), (lev, color, rel(got, ref))


# big nested 3-d levels take the shared-memory tiled transfers (FP64 here,
# the same template as the FP32 inner cycles), boundary tiles included
TRANSFER_PROBLEMS = PROBLEMS + [
    ("3d_vg_tiled_64x32x16", lambda: W.random_problem(3, (64, 32, 16), W.VANGENUCHTEN, 17, hetero=True,
                                                      bc_kinds=[W.DIRICHLET, W.NOFLUX, W.NOFLUX, W.DIRICHLET,
                                                                W.FREE_DRAINAGE, W.DIRICHLET])),
    ("3d_vg_tiled_96x40x24", lambda: W.random_problem(3, (96, 40, 24), W.VANGENUCHTEN, 18, sink=True)),
]


@pytest.mark.parametrize("mk", [p[1] for p in TRANSFER_PROBLEMS], ids=[p[0] for p in TRANSFER_PROBLEMS])
def test_residual_restrict_tau_prolong_match_oracle(mk):
    prob = mk()
    gs, orc, p = pair(prob)
    gs.prepare(p["dt"], 1)
    orc.prepare(p["dt"], 1)
    rng = np.random.default_rng(4)
    psi = p["psi0"] + rng.uniform(-0.05, 0.05, len(p["psi0"]))
    gs.set_level(0, 0, psi)
    nrm = gs.residual(0)
    r, nrm_ref = orc.residual(psi)
    d = gs.get_level(0, 7)
    scale = np.max(np.abs(orc.g()))
    assert np.max(np.abs(d - r)) <= 1e-12 * scale
    assert abs(nrm - nrm_ref) <= 1e-12 * scale
    if orc.nlevels < 2:
        return
    gs.restrict_tau(0)
    pbar = orc.restrict(psi)
    dH = orc.restrict(r)
    gH = orc.apply_N(pbar, 1) + dH
    assert rel(gs.get_level(1, 6), pbar) <= STAGE_RTOL
    assert np.max(np.abs(gs.get_level(1, 7) - dH)) <= 1e-12 * scale
    assert np.max(np.abs(gs.get_level(1, 1) - gH)) <= 1e-12 * np.max(np.abs(gH))
    uH = pbar + rng.uniform(-0.01, 0.01, len(pbar))
    gs.set_level(1, 0, uH)
    gs.prolong(0)
    ref = orc.prolong_add(uH - pbar, psi)
    assert rel(gs.get_level(0, 0), ref) <= STAGE_RTOL


@pytest.mark.parametrize("mk", [p[1] for p in PROBLEMS], ids=IDS)
@pytest.mark.parametrize("gamma,glev", [(1, 0), (2, 0), (2, 1)])
def test_vcycle_matches_oracle(mk, gamma, glev):
    """Iterate-for-iterate V-cycles.  Point solves run to round-off and the
    coarsest level does a fixed number of sweeps: with a fixed two-step Newton
    the cycle map is discontinuous (whether a step bisects can flip on one
    ulp; the oracle alone moves by ~1e-3 under a 1e-15 input perturbation on
    the drainage case), and the coarse stop rule is a threshold decision."""
    prob = mk()
    gs, orc, p = pair(prob, coarse_rtol=0.0, coarse_max_sweeps=12, newton_iters=0, cycle_gamma=gamma,
                       gamma_levels=glev)
    gs.prepare(p["dt"], 1)
    orc.prepare(p["dt"], 1)
    ref = p["psi0"]
    for _ in range(2):
        gs.vcycle()
        ref = orc.vcycle(ref)
        assert rel(gs.get_level(0, 0), ref) <= STEP_RTOL


FMG_IDS = ["1d_haverkamp_dir", "2d_gardner_mixed_bc", "3d_vg_hetero_sink", "3d_drainage_16", "2d_layers_3mat"]
FMG_PROBLEMS = [p for p in PROBLEMS if p[0] in FMG_IDS]


@pytest.mark.parametrize("mk", [p[1] for p in FMG_PROBLEMS], ids=[p[0] for p in FMG_PROBLEMS])
@pytest.mark.parametrize("fmg", [1, 2])
def test_fmg_pass_matches_oracle(mk, fmg):
    """The full multigrid pass alone (max_cycles = 0), iterate for iterate."""
    prob = mk()
    gs, orc, p = pair(prob, coarse_rtol=0.0, coarse_max_sweeps=12, newton_iters=0, fmg_cycles=fmg, max_cycles=0)
    gs.step(p["dt"], 1, check=False)
    orc.prepare(p["dt"], 1)
    ref = orc.fmg(p["psi0"])
    assert rel(gs.state(), ref) <= STEP_RTOL


@pytest.mark.parametrize("mk", [p[1] for p in FMG_PROBLEMS], ids=[p[0] for p in FMG_PROBLEMS])
def test_fmg_steps_match_oracle(mk):
    """Whole FMG-started steps (Newton to round-off and a fixed coarsest sweep
    count, as in the cycle tests: with the sink the system need not be
    monotone, and iterates that part on one ulp may reach another root)."""
    prob = mk()
    gs, orc, p = pair(prob, tol=1e-11, max_cycles=200, fmg_cycles=1, newton_iters=0, coarse_rtol=0.0,
                      coarse_max_sweeps=12)
    for k in range(2):
        st, info = gs.step(p["dt"], p["scheme"], check=False)
        sto, info_o = orc.step(p["dt"], p["scheme"])
        assert st == sto, (k, info, info_o)
        assert abs(info["cycles"] - info_o["cycles"]) <= 1, (k, info, info_o)
        assert rel(gs.state(), orc.state()) <= STEP_RTOL, k


@pytest.mark.parametrize("mk", [p[1] for p in FMG_PROBLEMS], ids=[p[0] for p in FMG_PROBLEMS])
def test_mixed_fmg_within_stated_bound(mk):
    """Mixed mode with a full multigrid start of every inner solve."""
    prob = W.with_opts(mk(), precision=1, fmg_cycles=1)
    gs = R.Solver(prob)
    orc = Oracle(W.with_opts(prob, tol=1e-13, newton_iters=0, fmg_cycles=0))
    cur, prev = np.array(prob["psi0"], dtype=np.float64), None
    for k in range(2):
        st, info = gs.step(prob["dt"], prob["scheme"], check=False)
        assert st == R.RICH_OK, info
        psi_m = gs.state()
        orc.set_state(cur, prev)
        assert orc.step(prob["dt"], prob["scheme"])[0] == ORC_OK
        psi_r = orc.state()
        orc.set_state(cur, prev)
        orc.prepare(prob["dt"], info["scheme_used"])
        bound = _mixed_bound(orc, psi_m, psi_r)
        assert np.max(np.abs(psi_m - psi_r)) <= bound * (1 + 1e-6) + 1e-15, k
        prev, cur = cur, psi_m


@pytest.mark.parametrize("mk", [p[1] for p in PROBLEMS], ids=IDS)
def test_fp64_steps_match_oracle(mk):
    """Whole steps, both sides cycling to a tight tolerance (1e-11) so that the
    comparison is between two converged solutions of the same system."""
    prob = mk()
    gs, orc, p = pair(prob, tol=1e-11, max_cycles=200)
    for k in range(3):
        st, info = gs.step(p["dt"], p["scheme"], check=False)
        sto, info_o = orc.step(p["dt"], p["scheme"])
        assert st == sto, (k, info, info_o)
        assert abs(info["cycles"] - info_o["cycles"]) <= 1, (k, info, info_o)
        assert rel(gs.state(), orc.state()) <= STEP_RTOL, k


def test_celia_column_full_run():
    """The paper's 1-d column (config: N=128, dt = 10 s, 36 BDF1 steps)."""
    prob = W.celia_1d()
    gs, orc, p = pair(prob)
    for k in range(p["nsteps"]):
        st, info = gs.step()
        sto, info_o = orc.step()
        assert st == R.RICH_OK and sto == ORC_OK
        assert info["cycles"] == info_o["cycles"]
    assert rel(gs.state(), orc.state()) <= STEP_RTOL


def test_strip_2d_bdf2_steps():
    prob = W.strip_2d(n=65, nsteps=6, tol=1e-11, max_cycles=200)
    gs, orc, p = pair(prob)
    for k in range(p["nsteps"]):
        st, info = gs.step()
        sto, info_o = orc.step()
        assert st == sto
        assert rel(gs.state(), orc.state()) <= STEP_RTOL, k


def test_strip_2d_513_bdf2_steps():
    """The 2-d infiltration workload at its full size (513^2, the hierarchy odd
    on every level: 513, 257, ..., 5), FP64, BDF2: three steps, both sides
    cycling to 1e-11, agree to the 1e-10 norm-wise bound."""
    prob = W.strip_2d(n=513, nsteps=3, tol=1e-11, max_cycles=200)
    gs, orc, p = pair(prob)
    for k in range(p["nsteps"]):
        st, info = gs.step()
        sto, info_o = orc.step()
        assert st == sto == R.RICH_OK, (k, info, info_o)
        assert rel(gs.state(), orc.state()) <= STEP_RTOL, k


def _mixed_bound(orc, psi_m, psi_r):
    """(||r_m|| + ||r_r||) / min_i a theta'(zeta_i), zeta_i on [psi_m, psi_r]."""
    a = orc.a
    xi = orc.prob["opts"]["xi"]
    _, rm = orc.residual(psi_m)
    _, rr = orc.residual(psi_r)
    lo, hi = np.minimum(psi_m, psi_r), np.maximum(psi_m, psi_r)
    dmin = np.inf
    for i in range(len(psi_m)):
        d = min(orc.soil(i, lo[i])[1], orc.soil(i, hi[i])[1])
        dmin = min(dmin, a * d + xi)
    if dmin <= 0:
        return np.inf
    return (rm + rr) / dmin


@pytest.mark.parametrize("mk", [p[1] for p in PROBLEMS if "sink" not in p[0]],
                         ids=[p[0] for p in PROBLEMS if "sink" not in p[0]])
@pytest.mark.parametrize("predictor", [0, 1])
def test_mixed_precision_within_stated_bound(mk, predictor):
    prob = mk()
    prob = W.with_opts(prob, precision=1, predictor=predictor)
    gs = R.Solver(prob)
    orc = Oracle(W.with_opts(prob, tol=1e-13, newton_iters=0))
    cur, prev = np.array(prob["psi0"], dtype=np.float64), None
    for k in range(3):
        st, info = gs.step(prob["dt"], prob["scheme"], check=False)
        assert st == R.RICH_OK, info
        assert info["resid"] <= prob["opts"]["tol"]
        orc.set_state(cur, prev)           # same history as the GPU step
        assert orc.step(prob["dt"], prob["scheme"])[0] == ORC_OK
        psi_m, psi_r = gs.state(), orc.state()
        orc.set_state(cur, prev)
        orc.prepare(prob["dt"], info["scheme_used"])
        _, rm = orc.residual(psi_m)        # the oracle re-derives the FP64 residual
        assert rm / orc.a <= prob["opts"]["tol"] * (1 + 1e-6) + _law_allowance(orc, prob, psi_m)
        bound = _mixed_bound(orc, psi_m, psi_r)
        err = np.max(np.abs(psi_m - psi_r))
        assert err <= bound * (1 + 1e-6), (k, err, bound)
        prev, cur = cur, psi_m


@pytest.mark.parametrize("mk", [p[1] for p in PROBLEMS], ids=IDS)
@pytest.mark.parametrize("scheme", [1, 2])
def test_fp64_outer_prepare_matches_oracle(mk, scheme):
    """The FP64-outer mixed mode assembles the FP64 system: the finest level's
    Kc, boundary conductances and g agree with the oracle to STAGE_RTOL."""
    prob = W.with_opts(mk(), precision=2)
    if scheme == 2:
        rng = np.random.default_rng(9)
        prob["psi_prev"] = prob["psi0"] + rng.uniform(-0.02, 0.02, len(prob["psi0"]))
    gs, orc, p = pair(prob)
    assert gs.prepare(p["dt"], scheme) == scheme
    assert orc.prepare(p["dt"], scheme) == scheme
    assert rel(gs.get_level(0, 2), orc.Kc(0)) <= STAGE_RTOL
    for f in range(2 * p["dim"]):
        kg, ko = gs.get_level(0, 10 + f), orc.array(10 + f, 0)
        assert np.max(np.abs(kg - ko)) <= STAGE_RTOL * max(np.max(np.abs(ko)), 1e-300), f
    assert rel(gs.get_level(0, 1), orc.g(0)) <= STAGE_RTOL


LAG_PROBLEMS = [p for p in PROBLEMS if p[0] in ("3d_vg_hetero_sink", "2d_layers_3mat", "1d_celia_composite_40")]


@pytest.mark.parametrize("mk", [p[1] for p in LAG_PROBLEMS], ids=[p[0] for p in LAG_PROBLEMS])
@pytest.mark.parametrize("precision", [0, 1, 2])
def test_bdf2_lag_at_psi_n_matches_oracle(mk, precision):
    """bdf2_lag = 1 (K and the xi term lagged at psi^n in a BDF2 step): the
    finest level's Kc and g agree with the oracle's (to STAGE_RTOL in FP64 and
    with the FP64 outer layer, to DD_EPS in float-float), and three FP64 steps
    agree to STEP_RTOL."""
    prob = W.with_opts(mk(), precision=precision, bdf2_lag=1, xi=1e-3)
    rng = np.random.default_rng(9)
    prob["psi_prev"] = prob["psi0"] + rng.uniform(-0.05, 0.05, len(prob["psi0"]))
    gs, orc, p = pair(prob)
    assert gs.prepare(p["dt"], 2) == 2
    assert orc.prepare(p["dt"], 2) == 2
    tol = DD_EPS if precision == 1 else STAGE_RTOL
    assert rel(gs.get_level(0, 2), orc.Kc(0)) <= tol
    assert rel(gs.get_level(0, 1), orc.g(0)) <= tol
    if precision == 0:
        gs, orc, p = pair(prob)
        for k in range(3):
            st, info = gs.step(p["dt"], 2)
            sto, info_o = orc.step(p["dt"], 2)
            assert st == sto == R.RICH_OK, (k, info, info_o)
            assert rel(gs.state(), orc.state()) <= STEP_RTOL, k


@pytest.mark.parametrize("mk", [p[1] for p in PROBLEMS if "sink" not in p[0]],
                         ids=[p[0] for p in PROBLEMS if "sink" not in p[0]])
@pytest.mark.parametrize("predictor", [0, 1])
def test_fp64_outer_passes_the_oracle_stop_test(mk, predictor):
    """precision 2: every step's result satisfies the oracle's own FP64 stop
    test, up to FP64 rounding only (no float-float law allowance), and lies
    within the stated bound of the oracle's tight solution."""
    prob = W.with_opts(mk(), precision=2, predictor=predictor)
    gs = R.Solver(prob)
    orc = Oracle(W.with_opts(prob, tol=1e-13, newton_iters=0))
    cur, prev = np.array(prob["psi0"], dtype=np.float64), None
    for k in range(3):
        st, info = gs.step(prob["dt"], prob["scheme"], check=False)
        assert st == R.RICH_OK, info
        assert info["resid"] <= prob["opts"]["tol"]
        orc.set_state(cur, prev)
        assert orc.step(prob["dt"], prob["scheme"])[0] == ORC_OK
        psi_m, psi_r = gs.state(), orc.state()
        orc.set_state(cur, prev)
        orc.prepare(prob["dt"], info["scheme_used"])
        _, rm = orc.residual(psi_m)
        assert rm / orc.a <= prob["opts"]["tol"] * (1 + 1e-6) + _fp64_rounding(orc, prob, psi_m), (k, rm / orc.a)
        # the GPU's deciding defect is the oracle's to FP64 rounding
        assert abs(info["resid"] - rm / orc.a) <= 1e-9 * prob["opts"]["tol"] + _fp64_rounding(orc, prob, psi_m), k
        bound = _mixed_bound(orc, psi_m, psi_r)
        err = np.max(np.abs(psi_m - psi_r))
        assert err <= bound * (1 + 1e-6), (k, err, bound)
        prev, cur = cur, psi_m


def test_fp64_outer_with_unrounded_fields_and_sink():
    """General float64 per-cell fields (no value exact in FP32), a sink, BDF2,
    every law: the FP64-outer result passes the oracle's FP64 stop test and
    the float-float result passes it within the law allowance."""
    for model, seed in ((W.VANGENUCHTEN, 41), (W.HAVERKAMP, 42), (W.GARDNER, 43)):
        base = W.random_problem(3, (14, 13, 12), model, seed, hetero=True, sink=True, scheme=2)
        f = base["soil"]["p1_field"]
        assert np.any(f.astype(np.float32).astype(np.float64) != f)
        for precision in (1, 2):
            prob = W.with_opts(base, precision=precision)
            gs = R.Solver(prob)
            orc = Oracle(prob)
            cur, prev = np.array(prob["psi0"], dtype=np.float64), None
            for k in range(3):
                st, info = gs.step(prob["dt"], prob["scheme"], check=False)
                assert st == R.RICH_OK, (model, precision, info)
                psi = gs.state()
                orc.set_state(cur, prev)
                orc.prepare(prob["dt"], info["scheme_used"])
                _, rm = orc.residual(psi)
                allow = _fp64_rounding(orc, prob, psi) if precision == 2 else _law_allowance(orc, prob, psi)
                assert rm / orc.a <= prob["opts"]["tol"] * (1 + 1e-6) + allow, (model, precision, k)
                prev, cur = cur, psi


def _face_field_problem():
    """3-d problem whose boundary data are per face cell: inflow value_field on
    the top (FLUX), a Dirichlet side with a mask and a head per face cell, free
    drainage at the bottom, a sink."""
    p = W.random_problem(3, (12, 10, 14), W.VANGENUCHTEN, 8, hetero=True, sink=True,
                         bc_kinds=[W.DIRICHLET, W.NOFLUX, W.NOFLUX, W.NOFLUX, W.FREE_DRAINAGE, W.FLUX])
    rng = np.random.default_rng(9)
    n0, n1, n2 = p["n"]
    p["bc"]["value_field"][5] = rng.uniform(0.0, 2e-6, n0 * n1)          # top: z-face cells over (x, y)
    p["bc"]["value_field"][0] = rng.uniform(-1.5, -0.2, n1 * n2)         # x-low: face cells over (y, z)
    p["bc"]["mask_field"][0] = (rng.uniform(size=n1 * n2) < 0.6).astype(np.uint8)
    return p


WATER_PROBLEMS = [
    ("1d_vg_sink_flux_xi", lambda: W.with_opts(W.random_problem(1, 64, W.VANGENUCHTEN, 2, bc_kinds=[W.FREE_DRAINAGE,
                                                                                                  W.FLUX],
                                                              hetero=True, sink=True, scheme=2), xi=3e-4)),
    ("2d_gardner_mixed_bc", lambda: W.random_problem(2, (23, 18), W.GARDNER, 3,
                                                     bc_kinds=[W.DIRICHLET, W.NOFLUX, W.FREE_DRAINAGE, W.FLUX],
                                                     hetero=True, scheme=2)),
    ("3d_vg_hetero_sink", lambda: W.random_problem(3, (17, 12, 9), W.VANGENUCHTEN, 4, hetero=True, sink=True)),
    ("3d_layers_3mat_sink", lambda: layered(3, (12, 10, 11), W.GARDNER, 8, "layers", sink=True, scheme=2,
                                            bc_kinds=[W.NOFLUX, W.FLUX, W.DIRICHLET, W.NOFLUX, W.FREE_DRAINAGE,
                                                      W.DIRICHLET])),
    ("3d_face_fields_sink", _face_field_problem),
]


@pytest.mark.parametrize("mk", [p[1] for p in WATER_PROBLEMS], ids=[p[0] for p in WATER_PROBLEMS])
@pytest.mark.parametrize("precision", [0, 1, 2])
def test_water_balance_and_error_bound_of_each_step(mk, precision):
    """info.mass_defect equals the oracle's water balance of the GPU state
    (sum V (a theta - hist + S + xi (psi - psi*)) - boundary inflow, over a);
    info.err_bound bounds the distance to the oracle's tight solution."""
    prob = W.with_opts(mk(), precision=precision)
    gs = R.Solver(prob)
    orc = Oracle(W.with_opts(prob, tol=1e-13, newton_iters=0))
    xi = prob["opts"]["xi"]
    cur, prev = np.array(prob["psi0"], dtype=np.float64), None
    for k in range(3):
        st, info = gs.step(prob["dt"], prob["scheme"], check=False)
        assert st == R.RICH_OK, info
        psi = gs.state()
        orc.set_state(cur, prev)
        orc.prepare(prob["dt"], info["scheme_used"])
        V, a = orc.cell_volume(), orc.a
        hist, pstar = orc.array(7), orc.array(6)
        th = np.array([orc.soil(i, x)[0] for i, x in enumerate(psi)])
        S = np.array([orc.sink(i, x)[0] for i, x in enumerate(psi)])
        Q = orc.boundary_inflow(psi)
        want = (V * np.sum(a * th - hist) + V * np.sum(S) + xi * V * np.sum(psi - pstar) - Q) / a
        scale = (V * (np.sum(np.abs(a * th)) + np.sum(np.abs(hist))) + abs(Q)) / a
        assert abs(info["mass_defect"] - want) <= 1e-11 * scale, (k, info["mass_defect"], want, scale)
        orc.set_state(cur, prev)
        assert orc.step(prob["dt"], info["scheme_used"])[0] == ORC_OK
        err = np.max(np.abs(psi - orc.state()))
        if np.isfinite(info["err_bound"]):
            assert err <= info["err_bound"] * (1 + 1e-6) + 1e-15, (k, err, info["err_bound"])
        prev, cur = cur, psi


def test_mixed_precision_reaches_fp64_solution_at_tight_tolerance():
    """The FP64 outer correction is not limited by FP32: at tol 1e-13 the
    mixed result equals the FP64 solution to 1e-9."""
    prob = W.with_opts(W.random_problem(3, (15, 14, 13), W.VANGENUCHTEN, 6, hetero=True),
                       precision=1, tol=1e-13, max_outer=40)
    gs = R.Solver(prob)
    orc = Oracle(W.with_opts(prob, tol=1e-14, newton_iters=0))
    st, info = gs.step()
    assert st == R.RICH_OK, info
    assert orc.step()[0] == ORC_OK
    assert rel(gs.state(), orc.state()) <= 1e-9


@pytest.mark.parametrize("n", [1, 2, 3])
def test_tiny_and_degenerate_grids(n):
    for dim in (1, 2, 3):
        prob = W.random_problem(dim, (n,) * dim, W.VANGENUCHTEN, 7,
                                bc_kinds=[W.DIRICHLET] * (2 * dim), kappa=0.01)
        gs, orc, p = pair(prob)
        st, info = gs.step()
        sto, _ = orc.step()
        assert st == sto
        assert rel(gs.state(), orc.state()) <= STEP_RTOL


def test_hydrostatic_state_unchanged_on_gpu():
    prob = W.random_problem(3, (9, 8, 7), W.VANGENUCHTEN, 8, hetero=True,
                            bc_kinds=[W.NOFLUX] * 4 + [W.DIRICHLET, W.DIRICHLET])
    H = 0.2
    prob["bc"]["value"][4], prob["bc"]["value"][5] = H, H - 1.0
    idx = np.arange(9 * 8 * 7)
    z = (idx // 72 + 0.5) / 7
    prob["psi0"] = H - z
    gs = R.Solver(prob)
    st, info = gs.step()
    assert st == R.RICH_OK and info["cycles"] == 0
    assert np.max(np.abs(gs.state() - prob["psi0"])) <= 1e-13


def test_error_statuses():
    prob = W.random_problem(2, (8, 8), W.VANGENUCHTEN, 9)
    gs = R.Solver(prob)
    bad = dict(prob["soil"], Ks=-1.0)
    with pytest.raises(R.RichardsError) as e:
        gs.set_soil(bad)
    assert e.value.status == R.RICH_EINVAL
    bad_bc = dict(prob["bc"], kind=[W.FREE_DRAINAGE] + list(prob["bc"]["kind"][1:]))
    with pytest.raises(R.RichardsError):
        gs.set_bc(bad_bc)
    with pytest.raises(R.RichardsError):
        gs.set_state(np.full(64, np.nan))
    gs.set_state(prob["psi0"])
    st, info = R.Solver(W.with_opts(prob, max_cycles=1, tol=1e-30)).step(check=False)
    assert st == R.RICH_ENOCONV


@pytest.mark.slow
@pytest.mark.parametrize("precision", [1, 2])
def test_full_size_drainage_step_solves_the_oracle_system(precision):
    """At the benchmark's size (256^3, BDF2 workload with unrounded float64
    fields, first step) the GPU result satisfies the oracle's own FP64 stop
    test: exactly up to FP64 rounding with the FP64 outer layer, within the
    float-float law allowance with the float-float one."""
    prob = W.drainage_3d(n=256, precision=precision)
    gs = R.Solver(prob)
    st, info = gs.step()
    assert st == R.RICH_OK, info
    psi = gs.state()
    del gs
    orc = Oracle(prob)
    orc.prepare(prob["dt"], info["scheme_used"])
    _, nrm = orc.residual(psi)
    allow = _fp64_rounding(orc, prob, psi) if precision == 2 else _law_allowance(orc, prob, psi)
    assert nrm / orc.a <= prob["opts"]["tol"] * (1 + 1e-6) + allow, (nrm / orc.a, allow, info)


def test_graph_replay_matches_direct_launches():
    """The captured FP32 inner solve (cycle graphs inside a conditional while
    node that takes the inner stop test on the device) makes exactly the
    launches and decisions of the host-driven loop it replaced."""
    prob = W.with_opts(W.random_problem(3, (40, 36, 33), W.VANGENUCHTEN, 12, hetero=True, sink=True, scheme=2),
                       precision=1)
    stream = torch.cuda.Stream()
    a = R.Solver(prob, stream=stream.cuda_stream, opts=dict(graphs=1))
    b = R.Solver(prob, stream=stream.cuda_stream, opts=dict(graphs=0))
    for _ in range(3):
        sa, ia = a.step()
        sb, ib = b.step()
        assert sa == sb == R.RICH_OK
        assert ia["cycles"] == ib["cycles"] and ia["cell_updates"] == ib["cell_updates"]
    assert np.array_equal(a.state(), b.state())
    assert a.graph_status() == ""                  # both graphs were built and used
    a.profile(True)
    a.step()
    prof = a.profile_read()
    assert any(r["name"] == "sweep32" and r["launches"] > 0 for r in prof)


@pytest.mark.parametrize("fmg", [0, 1])
@pytest.mark.parametrize("graphs", [0, 1])
def test_mixed_without_presmoothing_reuses_the_stop_test_defect(fmg, graphs):
    """W(0,2) inner cycles start from the inner stop test's finest-level
    defect (and from g before the first cycle) instead of recomputing it: the
    steps meet the stop test on the oracle's own FP64 residual, stay within
    the error bound, converge in as many cycles as a W(1,2) run needs at most
    1.6 times over, and graph replay equals direct launches."""
    prob = W.with_opts(W.drainage_3d(n=32, coarsest_max_n=4), nu1=0, nu2=2, fmg_cycles=fmg)
    gs = R.Solver(prob, opts=dict(graphs=graphs))
    ref = R.Solver(W.with_opts(prob, nu1=1))
    orc = Oracle(W.with_opts(prob, tol=1e-13, newton_iters=0, fmg_cycles=0))
    cur, prev = np.array(prob["psi0"], dtype=np.float64), None
    for k in range(3):
        st, info = gs.step(prob["dt"], prob["scheme"], check=False)
        st1, info1 = ref.step(prob["dt"], prob["scheme"], check=False)
        assert st == st1 == R.RICH_OK, (info, info1)
        assert info["cycles"] <= 1.6 * info1["cycles"] + 1, (info, info1)
        psi_m = gs.state()
        orc.set_state(cur, prev)
        assert orc.step(prob["dt"], prob["scheme"])[0] == ORC_OK
        psi_r = orc.state()
        orc.set_state(cur, prev)
        orc.prepare(prob["dt"], info["scheme_used"])
        _, rm = orc.residual(psi_m)
        assert rm / orc.a <= prob["opts"]["tol"] * (1 + 1e-6) + _law_allowance(orc, prob, psi_m)
        assert np.max(np.abs(psi_m - psi_r)) <= _mixed_bound(orc, psi_m, psi_r) * (1 + 1e-6), k
        prev, cur = cur, psi_m
    if graphs:
        other = R.Solver(prob, opts=dict(graphs=0))
        for _ in range(3):
            other.step(prob["dt"], prob["scheme"])
        assert np.array_equal(other.state(), gs.state())


@pytest.mark.parametrize("mk", [p[1] for p in FMG_PROBLEMS], ids=[p[0] for p in FMG_PROBLEMS])
def test_fp64_steps_without_presmoothing_match_oracle(mk):
    """FP64 W(0,2) steps: each cycle reuses the finest defect of the stop test
    before it (the oracle recomputes it); iterates as the oracle's."""
    prob = mk()
    gs, orc, p = pair(prob, nu1=0, nu2=2, tol=1e-11, max_cycles=300, newton_iters=0, coarse_rtol=0.0,
                      coarse_max_sweeps=12)
    for k in range(2):
        st, info = gs.step(p["dt"], p["scheme"], check=False)
        sto, info_o = orc.step(p["dt"], p["scheme"])
        assert st == sto, (k, info, info_o)
        assert abs(info["cycles"] - info_o["cycles"]) <= 1, (k, info, info_o)
        assert rel(gs.state(), orc.state()) <= STEP_RTOL, k


def test_rejected_state_leaves_the_context_unchanged():
    """A state with a NaN or an infinity (in psi or psi_prev) is rejected
    with EINVAL after the device check, and the previous state stays."""
    prob = W.random_problem(3, (9, 8, 7), W.GARDNER, 16, scheme=2)
    gs = R.Solver(prob)
    gs.step()
    before = gs.state()
    for bad, prev in [(np.nan, None), (np.inf, None), (0.0, -np.inf)]:
        psi = before.copy()
        psi[17] = bad if bad != 0.0 else psi[17]
        pp = None if prev is None else np.full_like(before, prev)
        with pytest.raises(R.RichardsError) as e:
            gs.set_state(psi, pp)
        assert e.value.status == R.RICH_EINVAL
        assert np.array_equal(gs.state(), before)
    st, info = gs.step()
    assert st == R.RICH_OK


@pytest.mark.parametrize("precision", [1, 2])
@pytest.mark.parametrize("model", [W.VANGENUCHTEN, W.HAVERKAMP, W.GARDNER])
def test_state_handed_back_steps_like_the_resident_one(precision, model):
    """A caller that reads every step's result back and hands it in again
    (psi^n the result, psi^{n-1} the state it stepped from) advances bit for
    bit like a context that keeps its state on the device: a state equal to
    the context's own keeps that state's cached theta, which is what the
    resident context steps with."""
    prob = W.random_problem(3, (19, 14, 11), model, 31, hetero=True, sink=True, scheme=2, precision=precision)
    a, b = R.Solver(prob), R.Solver(prob)
    psi, prev = b.state(), None
    for k in range(4):
        sa, ia = a.step(check=False)
        if k:
            b.set_state(psi, prev)
        sb, ib = b.step(check=False)
        assert sa == sb == R.RICH_OK, (k, ia, ib)
        assert (ia["cycles"], ia["outer_iters"]) == (ib["cycles"], ib["outer_iters"]), k
        prev, psi = psi, b.state()
        assert np.array_equal(a.state(), psi), k
    a.close()
    b.close()


@pytest.mark.parametrize("which", ["psi", "prev"])
def test_changed_state_does_not_reuse_the_theta_cache(which):
    """A state that differs from the context's own in one cell of psi^n (or
    of psi^{n-1}) takes theta afresh there: the BDF2 step equals that of a
    new context given the same state.  (A stale cache would move the
    history term of that cell by theta' x 0.05 m, ~1e-3, far above the
    1e-12 allowed.)"""
    prob = W.random_problem(3, (19, 14, 11), W.VANGENUCHTEN, 32, hetero=True, scheme=2, precision=2)
    b = R.Solver(prob)
    psi0 = b.state()
    st, info = b.step()                      # b: psi^n = X, psi^{n-1} = psi0, both cached
    X, Y = b.state(), psi0.copy()
    k = X.size // 2 + 7
    if which == "psi":
        X[k] -= 0.05
    else:
        Y[k] -= 0.05
    b.set_state(X, Y)
    c = R.Solver(prob)
    c.set_state(X, Y)
    sb, ib = b.step(check=False)
    sc, ic = c.step(check=False)
    assert sb == sc == R.RICH_OK
    assert rel(b.state(), c.state()) <= 1e-12
    b.close()
    c.close()


def test_pipelined_half_sweeps_equal_one_cell_per_thread():
    """Levels of >= 2^20 cells take the pipelined half-sweep (sweep_planes
    cells along z per thread, blocks away from the y/z boundaries without
    those tests); the same point updates in the same order per cell, so the
    mixed steps are bit for bit those of one cell per thread.  Odd sizes
    leave a partial row pair and a partial plane chunk."""
    prob = W.drainage_3d(n=103)
    states = []
    for planes in (1, 2, 4, 8):
        gs = R.Solver(prob, opts=dict(sweep_planes=planes))
        for _ in range(2):
            st, info = gs.step(check=False)
            assert st == R.RICH_OK, (planes, info)
        states.append(gs.state())
        gs.close()
    for st in states[1:]:
        assert np.array_equal(st, states[0])


# ---------------------------------------------------------------------------
# The paper's lexicographic ordering on the GPU (ordering 0: hyperplanes
# i0 + i1 + i2 = const in turn), iterate for iterate against the oracle's
# sequential sweep.
# ---------------------------------------------------------------------------
LEX_IDS = ["1d_haverkamp_dir", "2d_gardner_mixed_bc", "3d_vg_hetero_sink", "3d_haverkamp_dir",
           "1d_celia_composite_40", "2d_layers_3mat"]
LEX_PROBLEMS = [p for p in PROBLEMS if p[0] in LEX_IDS]


@pytest.mark.parametrize("mk", [p[1] for p in LEX_PROBLEMS], ids=[p[0] for p in LEX_PROBLEMS])
@pytest.mark.parametrize("newton", [0, 2])
def test_lexicographic_sweeps_match_oracle_on_every_level(mk, newton):
    """One lexicographic sweep on every level (Newton to round-off on random
    states; the fixed two-step Newton near the root)."""
    prob = W.with_opts(mk(), ordering=0)
    gs, orc, p = pair(prob, newton_iters=newton)
    gs.prepare(p["dt"], 1)
    orc.prepare(p["dt"], 1)
    rng = np.random.default_rng(13)
    for lev in range(orc.nlevels):
        n = orc.ncell(lev)
        psi = rng.uniform(-1.5, -0.05, n)
        g = orc.apply_N(rng.uniform(-1.5, -0.05, n) if newton == 0 else psi + rng.uniform(-1e-3, 1e-3, n), lev)
        gs.set_level(lev, 0, psi)
        gs.set_level(lev, 1, g)
        ref = orc.sweep(psi, g, lev, -1, ordering=0)
        gs.sweep(lev, -1)
        got = gs.get_level(lev, 0)
        assert sweep_agrees(orc, p, lev, got, ref, psi, g), (lev, rel(got, ref))
    with pytest.raises(R.RichardsError):
        gs.sweep(0, 0)                    # half-sweeps belong to the red-black ordering


def test_lexicographic_differs_from_red_black():
    """The two orderings are different smoothers (same fixed point): one
    sweep from the same state gives different iterates."""
    prob = W.random_problem(2, (12, 10), W.VANGENUCHTEN, 21)
    lex, rb = R.Solver(W.with_opts(prob, ordering=0)), R.Solver(prob)
    for gs in (lex, rb):
        gs.prepare(prob["dt"], 1)
        gs.sweep(0, -1)
    assert rel(lex.get_level(0, 0), rb.get_level(0, 0)) > 1e-6


@pytest.mark.parametrize("mk", [p[1] for p in LEX_PROBLEMS], ids=[p[0] for p in LEX_PROBLEMS])
@pytest.mark.parametrize("gamma", [1, 2])
def test_lexicographic_cycles_match_oracle(mk, gamma):
    prob = W.with_opts(mk(), ordering=0)
    gs, orc, p = pair(prob, coarse_rtol=0.0, coarse_max_sweeps=12, newton_iters=0, cycle_gamma=gamma,
                      gamma_levels=0)
    gs.prepare(p["dt"], 1)
    orc.prepare(p["dt"], 1)
    ref = p["psi0"]
    for _ in range(2):
        gs.vcycle()
        ref = orc.vcycle(ref)
        assert rel(gs.get_level(0, 0), ref) <= STEP_RTOL


@pytest.mark.parametrize("mk", [p[1] for p in LEX_PROBLEMS], ids=[p[0] for p in LEX_PROBLEMS])
def test_lexicographic_fp64_steps_match_oracle(mk):
    prob = W.with_opts(mk(), ordering=0)
    gs, orc, p = pair(prob, tol=1e-11, max_cycles=200)
    for k in range(3):
        st, info = gs.step(p["dt"], p["scheme"], check=False)
        sto, info_o = orc.step(p["dt"], p["scheme"])
        assert st == sto, (k, info, info_o)
        assert abs(info["cycles"] - info_o["cycles"]) <= 1, (k, info, info_o)
        assert rel(gs.state(), orc.state()) <= STEP_RTOL, k


@pytest.mark.parametrize("mk", [p[1] for p in LEX_PROBLEMS if "sink" not in p[0]],
                         ids=[p[0] for p in LEX_PROBLEMS if "sink" not in p[0]])
def test_lexicographic_mixed_within_stated_bound(mk):
    """Mixed mode with the lexicographic FP32 inner smoother."""
    prob = W.with_opts(mk(), precision=1, ordering=0)
    gs = R.Solver(prob)
    orc = Oracle(W.with_opts(prob, tol=1e-13, newton_iters=0))
    cur, prev = np.array(prob["psi0"], dtype=np.float64), None
    for k in range(2):
        st, info = gs.step(prob["dt"], prob["scheme"], check=False)
        assert st == R.RICH_OK, info
        psi_m = gs.state()
        orc.set_state(cur, prev)
        assert orc.step(prob["dt"], prob["scheme"])[0] == ORC_OK
        psi_r = orc.state()
        orc.set_state(cur, prev)
        orc.prepare(prob["dt"], info["scheme_used"])
        _, rm = orc.residual(psi_m)
        assert rm / orc.a <= prob["opts"]["tol"] * (1 + 1e-6) + _law_allowance(orc, prob, psi_m)
        assert np.max(np.abs(psi_m - psi_r)) <= _mixed_bound(orc, psi_m, psi_r) * (1 + 1e-6), k
        prev, cur = cur, psi_m


def test_celia_column_lexicographic_full_run():
    """Section 4.1's column with the paper's own sweep order: cycle counts
    and the final state as the oracle's lexicographic run."""
    prob = W.with_opts(W.celia_1d(), ordering=0)
    gs, orc, p = pair(prob)
    for k in range(p["nsteps"]):
        st, info = gs.step()
        sto, info_o = orc.step()
        assert st == R.RICH_OK and sto == ORC_OK
        assert info["cycles"] == info_o["cycles"], k
    assert rel(gs.state(), orc.state()) <= STEP_RTOL


def test_face_fields_fp64_steps_match_oracle():
    prob = _face_field_problem()
    gs, orc, p = pair(prob, tol=1e-11, max_cycles=200)
    for k in range(3):
        st, info = gs.step(p["dt"], p["scheme"], check=False)
        sto, info_o = orc.step(p["dt"], p["scheme"])
        assert st == sto == R.RICH_OK, (k, info, info_o)
        assert rel(gs.state(), orc.state()) <= STEP_RTOL, k
        assert abs(info["mass_defect"]) <= 1e-9


def test_launch_shapes_give_the_same_bits():
    """The launch shapes the autotuner chooses among (cells per thread along
    z, block sizes of the half-sweeps and of the defect kernel) never change
    what is computed: steps with hand-set shapes on every grid level, and with
    the autotuned ones, equal the default launches bit for bit."""
    prob = W.with_opts(W.drainage_3d(n=64, nsteps=4), precision=2, tail_cells=64)
    ref = R.Solver(prob)
    odd = R.Solver(prob)
    shapes = [(2, 64, 32), (4, 32, 256), (1, 256, 64), (8, 128, 128)]
    for lev in range(min(odd.nlevels - 1, len(shapes))):
        pl, bx, rb = shapes[lev]
        n2 = odd.level_n(lev)[2]
        odd.set_launch(lev, pl if n2 >= 2 * pl or pl == 1 else 1, bx if pl == 1 or bx <= 128 else 128, rb)
    tuned = R.Solver(prob)
    for k in range(3):
        sa, ia = ref.step()
        sb, ib = odd.step()
        sc, ic = tuned.step()
        assert sa == sb == sc == R.RICH_OK
        assert ia["cycles"] == ib["cycles"] == ic["cycles"], (k, ia, ib, ic)
        assert np.array_equal(ref.state(), odd.state()), k
        assert np.array_equal(ref.state(), tuned.state()), k
        if k == 0:
            tuned.prepare(prob["dt"], prob["scheme"])
            choice = tuned.autotune(reps=2)
            assert len(choice) == tuned.nlevels
            assert all(pl in (1, 2, 4, 8) and bx in (0, 32, 64, 128, 256) for pl, bx, _ in choice)
    with pytest.raises(R.RichardsError):
        odd.set_launch(0, 3, 64, 64)
    with pytest.raises(R.RichardsError):
        odd.set_launch(1, 2, 256, 64)


@pytest.mark.parametrize("precision,extra", [(2, {}), (1, {}), (2, {"fmg_cycles": 1})])
def test_colour_split_layout_gives_the_same_bits(precision, extra):
    """The colour-split layout of the finest FP32 level's per-cell parameters
    (a 128^3 grid: even n0, over 2^20 cells) changes only where the values
    sit: steps with it equal steps with the natural layout bit for bit, with
    per-cell soil fields, a sink and (one case) an FMG start of each inner
    solve."""
    base = W.drainage_3d(n=128, precision=precision, **extra)
    base = dict(base, sink=W.feddes_sink(Tp=W.TP_5MM_PER_DAY * 50))
    split = R.Solver(W.with_opts(base, layout=0))
    natural = R.Solver(W.with_opts(base, layout=1))
    for k in range(3):
        sa, ia = split.step()
        sb, ib = natural.step()
        assert sa == sb == R.RICH_OK
        assert ia["cycles"] == ib["cycles"] and ia["outer_iters"] == ib["outer_iters"], (k, ia, ib)
        assert np.array_equal(split.state(), natural.state()), k


@pytest.mark.parametrize("n,gamma", [(64, 2), (96, 1), (50, 2)])
def test_cooperative_coarse_cycle_gives_the_same_bits(n, gamma):
    """The coarse levels of the FP32 inner cycles as one cooperative launch
    per visit (grid barriers between stages) compute what the stage launches
    compute: steps with it equal steps without it bit for bit, nested (64, 96)
    and odd (50: 25, 13, 7 cells per axis) hierarchies, V- and W-cycles, with
    the inner cycle captured into a CUDA graph and launched directly."""
    prob = W.drainage_3d(n=n, nsteps=3, precision=2, cycle_gamma=gamma, gamma_levels=0, tail_cells=64,
                         coarsest_max_n=4)
    stream = torch.cuda.Stream()
    coop = R.Solver(prob, stream=stream.cuda_stream)
    coop.set_coop(1 << 18)
    plain = R.Solver(prob, stream=stream.cuda_stream)
    direct = R.Solver(W.with_opts(prob, graphs=0), stream=stream.cuda_stream)
    direct.set_coop(1 << 18)
    for k in range(3):
        sa, ia = coop.step()
        sb, ib = plain.step()
        sc, ic = direct.step()
        assert sa == sb == sc == R.RICH_OK
        assert ia["cycles"] == ib["cycles"] == ic["cycles"], (k, ia, ib, ic)
        assert ia["cell_updates"] == ib["cell_updates"] == ic["cell_updates"], (k, ia, ib, ic)
        assert np.array_equal(coop.state(), plain.state()), k
        assert np.array_equal(coop.state(), direct.state()), k
    direct.profile(True)
    direct.step()
    names = {r["name"] for r in direct.profile_read()}
    assert "coop32" in names, names
