"""Soil laws on the GPU (Table 1) against the oracle, FP64 and float-float.

richards_soil_eval evaluates theta(psi) and K(psi) per cell with the cell's
own parameters.  FP64 must agree with the oracle to the 1e-12 stage bound of
the other parity tests (different libm routines, each within a few ulp, and
exp arguments up to ~60 in magnitude).

The oracle's van Genuchten-Mualem K is the plain definition
Se^l (1 - (1 - Se^{1/m})^m)^2 with Se^{1/m} = 1/(1 + t), t = (alpha h)^n.  It
cancels at both ends: 1 - Se^{1/m} loses ~1e-16/t relative near saturation,
and 1 - (1 - Se^{1/m})^m ~1e-16 (1 + t)/m as t grows; against 40-digit values
its error stays below 1e-13 for t in [1e-3, 99].  The GPU takes a
cancellation-free form.  So K is compared with the oracle for t in that band,
and over the whole range float-float is compared with the GPU's FP64.

Float-float keeps 48-bit significands, so an exp argument x of magnitude up
to 60 carries an absolute error ~60 * 2^-48 ~ 2e-13, i.e. a relative error
2e-13 in exp(x).  theta chains two such exponentials after a log (~1e-12 at
most), the van Genuchten-Mualem K three plus the squared expm1 term (~3e-12);
the bounds below add a factor ~2 on those.
"""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2606_04292_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2606_04292_gb300 import richards as R  # noqa: E402

FP64_RTOL = 1e-12
DD_RTOL = {"theta": 2e-12, "K": 6e-12}

MODELS = [("vangenuchten", W.VANGENUCHTEN), ("haverkamp", W.HAVERKAMP), ("gardner", W.GARDNER)]


def _heads(N, seed):
    """Pressure heads over the whole range the laws see: |psi| from 1e-9 to
    1e5 log-uniform (negative), plus saturated values and exact zeros."""
    rng = np.random.Generator(np.random.PCG64(seed))
    psi = -np.exp(rng.uniform(np.log(1e-9), np.log(1e5), N))
    psi[::17] = rng.uniform(0.0, 2.0, psi[::17].size)
    psi[5::41] = 0.0
    return psi


def _oracle_laws(orc, psi):
    th = np.empty(psi.size)
    K = np.empty(psi.size)
    for i, x in enumerate(psi):
        t, _, k = orc.soil(i, x)
        th[i], K[i] = t, k
    return th, K


def _relerr(got, want):
    # relative per element; values below 1e-20 of the largest (the far tails,
    # which float-float keeps to float precision only below ~1e-31) count absolutely
    floor = 1e-20 * max(np.max(np.abs(want)), 1e-300)
    return np.max(np.abs(got - want) / np.maximum(np.abs(want), floor))


@pytest.mark.parametrize("name,model", MODELS, ids=[m[0] for m in MODELS])
@pytest.mark.parametrize("hetero", [False, True], ids=["uniform", "fields"])
def test_soil_eval_matches_oracle(name, model, hetero):
    prob = W.random_problem(3, (16, 16, 12), model, 40 + model, hetero=hetero)
    gs = R.Solver(prob)
    orc = Oracle(prob)
    psi = _heads(gs.N, 7 + model)
    th_o, K_o = _oracle_laws(orc, psi)
    ok = np.ones(psi.size, bool)
    if model == W.VANGENUCHTEN:
        soil = prob["soil"]
        n = np.asarray(soil["p2_field"]) if soil.get("p2_field") is not None else np.full(psi.size, soil["p2"])
        Se = (th_o - soil["theta_r"]) / (soil["theta_s"] - soil["theta_r"])
        with np.errstate(divide="ignore"):
            t = Se ** (-n / (n - 1.0)) - 1.0
        ok = (t >= 1e-3) & (t <= 99.0)
        assert 0.1 < ok.mean() < 0.9           # both ranges are exercised
    th64, K64 = gs.soil_eval(psi, arith=0)
    assert _relerr(th64, th_o) <= FP64_RTOL
    assert _relerr(K64[ok], K_o[ok]) <= FP64_RTOL
    thdd, Kdd = gs.soil_eval(psi, arith=1)
    assert _relerr(thdd, th_o) <= DD_RTOL["theta"], _relerr(thdd, th_o)
    assert _relerr(Kdd[ok], K_o[ok]) <= DD_RTOL["K"], _relerr(Kdd[ok], K_o[ok])
    assert _relerr(Kdd, K64) <= DD_RTOL["K"], _relerr(Kdd, K64)
    sat = psi >= 0
    ts = prob["soil"]["theta_s"]
    assert np.all(th64[sat] == ts)
    assert np.all(np.abs(thdd[sat] - ts) <= 2.0 ** -46 * ts)     # theta_s as a float pair


def test_soil_eval_rejects_bad_arith():
    prob = W.random_problem(2, (8, 8), W.VANGENUCHTEN, 3)
    gs = R.Solver(prob)
    with pytest.raises(R.RichardsError) as e:
        gs.soil_eval(np.zeros(gs.N), arith=2)
    assert e.value.status == R.RICH_EINVAL
