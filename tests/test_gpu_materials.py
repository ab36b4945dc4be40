"""Layered soils on the GPU (richards_set_materials) against the oracle.

The stage, cycle, step, FMG, mixed-precision and water-balance parity tests
of test_gpu_parity.py run on layered problems too (Section 4.1's composite
column, Section 4.2's two-layer field, three-law random and banded maps).
This file checks what is particular to materials: the material of every
cell on every level and its parameters (integer and copied values: bit for
bit), the per-cell laws of richards_soil_eval, the paper's two layered
workloads over whole runs, input validation, and switching back to a
single soil.  Tolerances as in test_gpu_parity.py and test_gpu_soil.py.
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
DD_RTOL = 6e-12


def rel(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


def layered(dim, n, model, seed, kind, **kw):
    p = W.random_problem(dim, n, model, seed, **kw)
    return W.with_materials(p, W.test_materials(), W.material_pattern(p, kind, 3, seed))


MAPS = [("1d_41_layers", 1, (41,), "layers"), ("1d_64_random", 1, (64,), "random"),
        ("2d_27x14_random", 2, (27, 14), "random"), ("2d_32x32_layers", 2, (32, 32), "layers"),
        ("3d_13x9x10_random", 3, (13, 9, 10), "random"), ("3d_16x8x12_layers", 3, (16, 8, 12), "layers")]


@pytest.mark.parametrize("dim,n,kind", [m[1:] for m in MAPS], ids=[m[0] for m in MAPS])
def test_material_maps_and_parameters_match_oracle(dim, n, kind):
    """Material index and p1, p2 of every cell on every level, bit for bit
    (the coarse majority is taken on the host with the oracle's weights and
    order of summation)."""
    prob = layered(dim, n, W.VANGENUCHTEN, 11 + dim, kind)
    gs, orc = R.Solver(prob), Oracle(prob)
    assert gs.nlevels == orc.nlevels >= 2
    for lev in range(orc.nlevels):
        mm = orc.material_map(lev)
        assert np.array_equal(gs.get_level(lev, 8), mm.astype(np.float64)), lev
        assert np.array_equal(gs.get_level(lev, 3), orc.array(2, lev)), lev
        assert np.array_equal(gs.get_level(lev, 4), orc.array(3, lev)), lev
    assert len(set(orc.material_map(1).tolist())) >= 2


def test_layered_soil_eval_matches_oracle():
    """richards_soil_eval with each cell's law: FP64 within 1e-12, float-float
    within 6e-12 of the oracle (van Genuchten-Mualem K where the oracle's plain
    form is accurate, t = (alpha h)^n in [1e-3, 99]; elsewhere against FP64)."""
    prob = layered(3, (12, 11, 10), W.GARDNER, 21, "random")
    gs, orc = R.Solver(prob), Oracle(prob)
    rng = np.random.default_rng(5)
    psi = -np.exp(rng.uniform(np.log(1e-4), np.log(60.0), gs.N))
    psi[::13] = rng.uniform(0.0, 1.0, psi[::13].size)
    ref = np.array([orc.soil(i, x) for i, x in enumerate(psi)])
    th_o, K_o = ref[:, 0], ref[:, 2]
    mats = prob["soil"]["materials"]
    idx = prob["soil"]["material_index"]
    ok = np.ones(gs.N, bool)
    for i in range(gs.N):
        m = mats[idx[i]]
        if m["model"] == W.VANGENUCHTEN and psi[i] < 0:
            t = (m["p1"] * -psi[i]) ** m["p2"]
            ok[i] = 1e-3 <= t <= 99.0
    assert 0.5 < ok.mean() < 1.0
    th64, K64 = gs.soil_eval(psi, arith=0)
    thdd, Kdd = gs.soil_eval(psi, arith=1)
    floor = 1e-20 * np.max(K_o)
    assert rel(th64, th_o) <= STAGE_RTOL
    assert np.max(np.abs(K64 - K_o)[ok] / np.maximum(K_o[ok], floor)) <= STAGE_RTOL
    assert rel(thdd, th_o) <= DD_RTOL
    assert np.max(np.abs(Kdd - K64) / np.maximum(K64, floor)) <= DD_RTOL
    sat = psi >= 0
    ts = np.array([mats[m]["theta_s"] for m in idx])
    Ks = np.array([mats[m]["Ks"] for m in idx])
    assert np.array_equal(th64[sat], ts[sat]) and np.array_equal(K64[sat], Ks[sat])


def test_composite_column_full_run():
    """Section 4.1's composite column (N = 128, dt = 10 s, 36 BDF1 steps):
    cycle counts equal, final state within the step bound."""
    prob = W.celia_composite_1d()
    gs, orc = R.Solver(prob), Oracle(prob)
    for k in range(prob["nsteps"]):
        st, info = gs.step()
        sto, info_o = orc.step()
        assert st == R.RICH_OK and sto == ORC_OK, k
        assert info["cycles"] == info_o["cycles"], (k, info, info_o)
    assert rel(gs.state(), orc.state()) <= STEP_RTOL


@pytest.mark.parametrize("precision", [0, 1])
def test_two_layer_field_steps(precision):
    """Section 4.2's two-layer field on 64^2 (FMG start, 10 + 10 sweeps,
    kappa = 0.1).  FP64: steps within the step bound of the oracle's.  Mixed:
    from the same history, the oracle's own FP64 residual of each GPU step
    meets the stop test (plus the float-float law allowance), and the state
    lies within the reported error bound of the oracle's tight solution."""
    prob = W.with_opts(W.two_layer_2d(n=64), precision=precision)
    if precision == 0:
        prob = W.with_opts(prob, tol=1e-11)
    gs = R.Solver(prob)
    orc = Oracle(W.with_opts(prob, tol=1e-11 if precision == 0 else 1e-13))
    cur, prev = np.array(prob["psi0"], dtype=np.float64), None
    for k in range(4):
        st, info = gs.step(check=False)
        assert st == R.RICH_OK, (k, info)
        psi = gs.state()
        if precision == 0:
            assert orc.step()[0] == ORC_OK
            assert rel(psi, orc.state()) <= STEP_RTOL, k
            continue
        orc.set_state(cur, prev)
        orc.prepare(prob["dt"], info["scheme_used"])
        _, rm = orc.residual(psi)
        assert rm / orc.a <= prob["opts"]["tol"] * (1 + 1e-6) + law_allowance(orc, prob, psi, DD_RTOL), k
        orc.set_state(cur, prev)
        assert orc.step(prob["dt"], info["scheme_used"])[0] == ORC_OK
        if np.isfinite(info["err_bound"]):
            assert np.max(np.abs(psi - orc.state())) <= info["err_bound"] * (1 + 1e-6) + 1e-15, k
        prev, cur = cur, psi


def test_set_materials_rejects_bad_input():
    prob = layered(2, (9, 8), W.VANGENUCHTEN, 3, "random")
    gs = R.Solver(prob)
    mats = W.test_materials()
    idx = prob["soil"]["material_index"]
    for bad_mats, bad_idx in [([], idx), (mats * 3, idx), (mats[:2], np.full(72, 2, np.uint8)),
                              ([dict(mats[0], Ks=-1.0)] + mats[1:], idx),
                              ([dict(mats[0], p2=0.9)] + mats[1:], idx),
                              ([dict(mats[1], theta_r=0.5)] + mats[1:], idx)]:
        with pytest.raises(R.RichardsError) as e:
            gs.set_materials(bad_mats, bad_idx)
        assert e.value.status == R.RICH_EINVAL
    with pytest.raises(R.RichardsError):
        gs.set_materials(mats, idx[:10])


@pytest.mark.parametrize("precision", [0, 1])
def test_switching_between_layered_and_single_soils(precision):
    """A single soil set after materials gives bit for bit the steps of a
    fresh single-soil context; one material covering every cell gives the
    single-law fine operator exactly and its steps within the step bound
    (its coarse parameters are exact, the single soil's restricted)."""
    base = W.with_opts(W.random_problem(2, (21, 17), W.HAVERKAMP, 30, sink=True), precision=precision)
    ref = R.Solver(base)
    ref.step()
    ref.step()
    gs = R.Solver(layered(2, (21, 17), W.HAVERKAMP, 30, "layers", sink=True, precision=precision))
    gs.step()
    gs.set_soil(base["soil"])
    gs.set_state(base["psi0"])
    gs.step()
    gs.step()
    assert np.array_equal(gs.state(), ref.state())
    s = base["soil"]
    tight = W.with_opts(base, tol=1e-11, max_cycles=200, max_outer=40)
    one = W.with_materials(tight, [W.material(s["model"], s["Ks"], s["theta_s"], s["theta_r"], s["p1"], s["p2"],
                                              s["p3"], s["p4"])], np.zeros(21 * 17, np.uint8))
    g1 = R.Solver(one)
    r1 = R.Solver(tight)
    g1.prepare(base["dt"], 1)
    r1.prepare(base["dt"], 1)
    for which in (1, 2, 12, 13):
        a, b = g1.get_level(0, which), r1.get_level(0, which)
        if precision == 0:
            assert np.array_equal(a, b), which
        else:      # float-float pairs split from a field or from a scalar may differ in their last bits
            assert np.max(np.abs(a - b)) <= DD_RTOL * max(np.max(np.abs(b)), 1e-300), which
    g1.set_state(base["psi0"])
    r1.set_state(base["psi0"])
    for k in range(2):
        st1, i1 = g1.step(check=False)
        st2, i2 = r1.step(check=False)
        assert st1 == st2 == R.RICH_OK, (k, i1, i2)
        if precision == 0:
            assert rel(g1.state(), r1.state()) <= STEP_RTOL, k
        elif k == 0:     # same history: both within their error bounds of one exact step
            assert np.max(np.abs(g1.state() - r1.state())) <= (i1["err_bound"] + i2["err_bound"]) * (1 + 1e-6)
