"""The FP64 elementary functions of the soil laws against CUDA's (needs a GPU).

The FP64 laws (Table 1) take their powers and exponentials through the
library's table-driven exp, expm1, log and log1p.  Each must stay within a few
ulps of CUDA's own function (itself within ~1 ulp of the correctly rounded
value) over the ranges the laws reach and across the edges of its reduction
(the table steps, the series thresholds at 1/128, 1 for log, ln2/512 for exp),
and hand the rest to CUDA's function unchanged.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2606_04292_gb300 import richards as R  # noqa: E402

ULPS = 4


def _eval(fn, x):
    L = R.lib()
    xd = torch.tensor(np.asarray(x, dtype=np.float64), device="cuda")
    yd = torch.empty_like(xd)
    dp = lambda t: C.cast(C.c_void_p(t.data_ptr()), C.POINTER(C.c_double))
    assert L.richards_math_eval(fn, dp(xd), dp(yd), len(x), None) == R.RICH_OK
    return yd.cpu().numpy()


def _ulp_err(got, want):
    scale = np.spacing(np.abs(want))
    return np.abs(got - want) / np.where(scale > 0, scale, np.finfo(float).tiny)


def _inputs(rng, fn):
    u = lambda a, b, n=20000: rng.uniform(a, b, n)
    if fn in (0, 1):                                   # exp, expm1
        edges = np.concatenate([k * np.log(2) / 256 + np.array([-1e-15, 0.0, 1e-15]) for k in range(-1200, 1200)])
        xs = [u(-700, 700), u(-30, 30), u(-1, 1), u(-0.01, 0.01), u(-1e-4, 1e-4),
              np.log(2) / 512 * np.array([-1.0001, -0.9999, 0.9999, 1.0001]), 0.0078125 * np.array([-1.001, -0.999,
                                                                                                    0.999, 1.001]),
              edges, -np.logspace(-300, 2.8, 2000), np.logspace(-300, 2.8, 2000)]
    elif fn == 2:                                      # log
        xs = [np.exp(u(-700, 700)), u(0.9, 1.1), u(0.99, 1.01), u(1e-3, 1e4), 2.0 ** np.arange(-1000, 1000),
              1 + np.array([-0.0078125, -0.0078124, 0.0078124, 0.0078125, 0.0078126]),
              1 + np.arange(512) / 256.0, (1 + np.arange(512) / 256.0) * 0.5,
              np.nextafter(1 + np.arange(1, 512) / 256.0, 0.0)]
    else:                                              # log1p
        xs = [u(0, 1), u(0, 1e-2), u(0, 1e-6), np.exp(u(-700, 40)), np.logspace(-300, 300, 4000),
              np.array([0.0078124, 0.0078125, 0.0078126]), np.arange(512) / 256.0, u(-0.0078, 0.0078), u(1, 1000)]
    return np.concatenate(xs)


@pytest.mark.parametrize("fn,name", [(0, "exp"), (1, "expm1"), (2, "log"), (3, "log1p")])
def test_table_driven_functions_within_a_few_ulps_of_cuda(fn, name):
    rng = np.random.default_rng(7 + fn)
    x = _inputs(rng, fn)
    got, want = _eval(fn, x), _eval(fn + 4, x)
    ok = np.isfinite(want)
    assert np.array_equal(np.isfinite(got), ok), name
    err = _ulp_err(got[ok], want[ok])
    worst = int(np.argmax(err))
    assert err[worst] <= ULPS, (name, x[ok][worst], got[ok][worst], want[ok][worst], err[worst])


def test_outside_the_law_ranges_cuda_decides():
    """Arguments outside the ranges each function serves itself go to CUDA's
    function: |x| > 700 for exp and expm1; x <= 0, subnormal, infinite or NaN
    for log; s < -1/128, infinite or NaN for log1p."""
    outside = {0: [-800.0, 710.0, np.inf, -np.inf, np.nan],
               1: [-800.0, 710.0, np.inf, -np.inf, np.nan],
               2: [1e-310, 0.0, -1.0, np.inf, np.nan],
               3: [-800.0, -1.0, -0.5, -0.0079, np.inf, np.nan]}
    for fn, xs in outside.items():
        x = np.array(xs)
        got, want = _eval(fn, x), _eval(fn + 4, x)
        assert np.array_equal(got, want, equal_nan=True), (fn, got, want)
