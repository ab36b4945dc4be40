"""The C-ABI library builds, loads and exports every declared entry point;
argument validation that needs no device returns EINVAL (no GPU needed)."""
import ctypes as C
import os
import re

from paper_2606_04292_gb300 import richards as R
from paper_2606_04292_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "richards.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(richards_[a-z_0-9]+)\s*\(", src)
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    L = R.lib()
    decl = declared_functions()
    assert len(decl) >= 20
    for name in decl:
        assert hasattr(L, name), name
    assert set(decl) == set(R.exported_symbols())


def test_create_rejects_invalid_arguments_without_a_device():
    L = R.lib()
    o = R.make_opts(W.default_opts())
    h = C.c_void_p()
    inf = float("inf")
    bad_grids = [R.richards_grid(0, (C.c_int * 3)(4, 1, 1), (C.c_double * 3)(1, 1, 1)),
                 R.richards_grid(4, (C.c_int * 3)(4, 4, 4), (C.c_double * 3)(1, 1, 1)),
                 R.richards_grid(1, (C.c_int * 3)(4, 2, 1), (C.c_double * 3)(1, 1, 1)),
                 R.richards_grid(2, (C.c_int * 3)(4, 0, 1), (C.c_double * 3)(1, 1, 1)),
                 R.richards_grid(2, (C.c_int * 3)(4, 4, 1), (C.c_double * 3)(1, -1, 1)),
                 R.richards_grid(2, (C.c_int * 3)(4, 4, 1), (C.c_double * 3)(inf, 1, 1)),
                 R.richards_grid(2, (C.c_int * 3)(4, 65536, 1), (C.c_double * 3)(1, 1, 1)),
                 R.richards_grid(3, (C.c_int * 3)(4, 4, 65536), (C.c_double * 3)(1, 1, 1)),
                 R.richards_grid(3, (C.c_int * 3)(2048, 1024, 1024), (C.c_double * 3)(1, 1, 1))]
    for g in bad_grids:
        assert L.richards_create(C.byref(g), C.byref(o), None, C.byref(h)) == R.RICH_EINVAL
    g = R.richards_grid(2, (C.c_int * 3)(4, 4, 1), (C.c_double * 3)(1, 1, 1))
    for key, val in [("ordering", 2), ("ordering", -1), ("kappa_mode", 1), ("precision", 3), ("tol", 0.0), ("nu1", -1),
                     ("newton_iters", -2), ("xi", -1.0), ("sweep_planes", 3), ("sweep_planes", 0), ("predictor", 2), ("fmg_cycles", -1),
                     ("nu2", -1), ("coarse_max_sweeps", 0), ("max_cycles", -1), ("coarsest_max_n", 0), ("tol", float("nan")),
                     ("newton_iters", 201), ("precision", -1), ("kappa", -1.0), ("inner_cycles", 0), ("max_outer", -1),
                     ("tail_cells", -1), ("cycle_gamma", 0), ("cycle_gamma", 4), ("gamma_levels", -1), ("graphs", 2),
                     ("fmg_cycles", 17), ("layout", 2), ("bdf2_lag", 2), ("bdf2_lag", -1)]:
        oo = R.make_opts(W.default_opts(**{key: val}))
        assert L.richards_create(C.byref(g), C.byref(oo), None, C.byref(h)) == R.RICH_EINVAL, key
    assert L.richards_create(None, C.byref(o), None, C.byref(h)) == R.RICH_EINVAL


def test_null_context_calls_are_rejected():
    L = R.lib()
    assert L.richards_step(None, 1.0, 1, None) == R.RICH_EINVAL
    assert L.richards_set_soil(None, None) == R.RICH_EINVAL
    assert L.richards_get_state(None, None, 0) == R.RICH_EINVAL
    assert L.richards_nlevels(None) == 0
    L.richards_destroy(None)


def test_device_bytes_estimate_is_host_only_and_monotone():
    from paper_2606_04292_gb300 import serve
    a = serve.request_bytes(W.drainage_3d(n=32, precision=0))
    b = serve.request_bytes(W.drainage_3d(n=32))            # mixed keeps FP32 copies too
    c = serve.request_bytes(W.drainage_3d(n=64))
    assert 0 < a < b < c
    assert c > 7 * b                                        # ~8x the cells
    L = R.lib()
    g = R.richards_grid(0, (C.c_int * 3)(4, 1, 1), (C.c_double * 3)(1, 1, 1))
    assert L.richards_device_bytes(C.byref(g), C.byref(R.make_opts(W.default_opts())), 0, 0) == -1
