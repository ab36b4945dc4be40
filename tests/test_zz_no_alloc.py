"""The allocation-free small-grid step against the regular step (needs a GPU).

richards_step_small_noalloc serves callers that may not allocate device
memory while they run (a memory pool that owns the device, a real-time loop
where an allocation may block, a plug-in limited to the memory handed to it).
It must give the same state as richards_step on a context, call after call,
within the step tolerance of the other GPU tests, and reject the inputs the
regular set-up calls reject.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2606_04292_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2606_04292_gb300 import richards as R  # noqa: E402

STEP_RTOL = 1e-10


def _dptr(t):
    return C.cast(C.c_void_p(t.data_ptr()), C.POINTER(C.c_double)) if t is not None else None


def _structs(prob, keep):
    """C structs for the call; per-cell and per-face fields as device arrays."""
    grid = R.richards_grid(prob["dim"], (C.c_int * 3)(*prob["n"]), (C.c_double * 3)(*prob["L"]))
    s = prob["soil"]
    soil = R.richards_soil(s["model"], s["Ks"], s["theta_s"], s["theta_r"], s["p1"], s["p2"], s["p3"], s["p4"])
    for key in ("Ks_field", "p1_field", "p2_field"):
        if s.get(key) is not None:
            t = torch.tensor(np.asarray(s[key], dtype=np.float64), device="cuda")
            keep.append(t)
            setattr(soil, key, _dptr(t))
    b = prob["bc"]
    bc = R.richards_bc()
    for f in range(6):
        bc.kind[f] = int(b["kind"][f])
        bc.value[f] = float(b["value"][f])
        if b["value_field"][f] is not None:
            t = torch.tensor(np.asarray(b["value_field"][f], dtype=np.float64), device="cuda")
            keep.append(t)
            bc.value_field[f] = _dptr(t)
        if b["mask_field"][f] is not None:
            t = torch.tensor(np.asarray(b["mask_field"][f], dtype=np.uint8), device="cuda")
            keep.append(t)
            bc.mask_field[f] = C.cast(C.c_void_p(t.data_ptr()), C.POINTER(C.c_ubyte))
    k = prob["sink"]
    sink = R.richards_sink(int(k["enabled"]), k["Tp"], k["root_depth"], k["root_decay"], k["h1"], k["h2"], k["h3"],
                           k["h4"])
    opts = R.make_opts(prob["opts"])
    return grid, soil, bc, sink, opts


def _noalloc_step(prob, psi_n, psi_prev, keep, out=None):
    L = R.lib()
    grid, soil, bc, sink, opts = _structs(prob, keep)
    out = torch.empty_like(psi_n) if out is None else out
    info = R.richards_step_info()
    st = L.richards_step_small_noalloc(C.byref(grid), C.byref(soil), C.byref(bc), C.byref(sink), C.byref(opts),
                                       float(prob["dt"]), int(prob["scheme"]), _dptr(psi_n), _dptr(psi_prev),
                                       _dptr(out), C.byref(info),
                                       C.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st, info.as_dict(), out


CASES = [
    ("3d_vg_fields_sink_bdf2", lambda: W.random_problem(3, (16, 16, 16), W.VANGENUCHTEN, 31, hetero=True, sink=True,
                                                        scheme=2)),
    ("2d_strip_mask_bdf2", lambda: W.strip_2d(n=63)),
    ("1d_celia_bdf1", lambda: W.celia_1d(n=128)),
    ("3d_vg_wcycle", lambda: W.random_problem(3, (15, 14, 13), W.VANGENUCHTEN, 33, hetero=True, cycle_gamma=2)),
]


@pytest.mark.parametrize("mk", [c[1] for c in CASES], ids=[c[0] for c in CASES])
def test_noalloc_step_matches_regular_step_twice(mk):
    prob = W.with_opts(mk(), precision=0)
    ref = R.Solver(prob)
    keep = []
    psi = torch.tensor(np.asarray(prob["psi0"], dtype=np.float64), device="cuda")
    prev = None
    for call in range(2):
        st_ref, info_ref = ref.step(check=False)
        st, info, out = _noalloc_step(prob, psi, prev, keep)
        assert st == st_ref == R.RICH_OK, (call, st, st_ref)
        assert info["cycles"] == info_ref["cycles"], (call, info, info_ref)
        got, want = out.cpu().numpy(), ref.state()
        err = np.max(np.abs(got - want)) / np.max(np.abs(want))
        assert err <= STEP_RTOL, (call, err)
        prev, psi = psi, out


def test_noalloc_rejects_grid_above_maximum():
    prob = W.random_problem(3, (17, 16, 16), W.VANGENUCHTEN, 32)
    assert 17 * 16 * 16 > 4096
    keep = []
    psi = torch.zeros(17 * 16 * 16, dtype=torch.float64, device="cuda")
    st, _, _ = _noalloc_step(prob, psi, None, keep)
    assert st == R.RICH_EINVAL


@pytest.mark.parametrize("alias", ["psi_n", "psi_prev"])
def test_noalloc_output_may_alias_an_input(alias):
    """BDF2 with rotating buffers: the output written over psi^n or over
    psi^{n-1} gives the regular step's state."""
    prob = W.with_opts(W.random_problem(3, (12, 11, 10), W.VANGENUCHTEN, 34, hetero=True, scheme=2), precision=0)
    ref = R.Solver(prob)
    keep = []
    psi = torch.tensor(np.asarray(prob["psi0"], dtype=np.float64), device="cuda")
    prev = None
    for call in range(3):
        assert ref.step(check=False)[0] == R.RICH_OK
        if prev is None:
            out = torch.empty_like(psi)
        else:
            out = psi if alias == "psi_n" else prev
        keep_prev = psi.clone()
        st, _, out = _noalloc_step(prob, psi, prev, keep, out=out)
        assert st == R.RICH_OK, (call, st)
        got, want = out.cpu().numpy(), ref.state()
        assert np.max(np.abs(got - want)) / np.max(np.abs(want)) <= STEP_RTOL, call
        prev, psi = keep_prev, out


BAD_SOILS = [
    ("haverkamp_alpha", W.HAVERKAMP, dict(p1=0.0)),
    ("haverkamp_beta", W.HAVERKAMP, dict(p2=-1.0)),
    ("haverkamp_A", W.HAVERKAMP, dict(p3=0.0)),
    ("haverkamp_gamma", W.HAVERKAMP, dict(p4=float("nan"))),
    ("gardner_alpha", W.GARDNER, dict(p1=-2.0)),
    ("vg_n", W.VANGENUCHTEN, dict(p2=1.0)),
    ("vg_l", W.VANGENUCHTEN, dict(p3=float("inf"))),
    ("vg_alpha", W.VANGENUCHTEN, dict(p1=0.0)),
]


@pytest.mark.parametrize("model,bad", [(b[1], b[2]) for b in BAD_SOILS], ids=[b[0] for b in BAD_SOILS])
def test_noalloc_rejects_what_set_soil_rejects(model, bad):
    prob = W.random_problem(2, (8, 8), model, 35)
    prob["soil"] = dict(prob["soil"], **bad)
    with pytest.raises(R.RichardsError) as e:
        R.Solver(prob)
    assert e.value.status == R.RICH_EINVAL
    psi = torch.tensor(np.asarray(prob["psi0"], dtype=np.float64), device="cuda")
    st, _, _ = _noalloc_step(prob, psi, None, [])
    assert st == R.RICH_EINVAL


def test_noalloc_rejects_bad_sink_and_boundary_values():
    prob = W.random_problem(2, (8, 8), W.VANGENUCHTEN, 36, sink=True)
    psi = torch.tensor(np.asarray(prob["psi0"], dtype=np.float64), device="cuda")
    for sink in (dict(prob["sink"], Tp=-1.0), dict(prob["sink"], root_decay=float("nan"))):
        st, _, _ = _noalloc_step(dict(prob, sink=sink), psi, None, [])
        assert st == R.RICH_EINVAL
    bc = dict(prob["bc"], value=list(prob["bc"]["value"]))
    bc["value"][3] = float("nan")
    st, _, _ = _noalloc_step(dict(prob, bc=bc), psi, None, [])
    assert st == R.RICH_EINVAL
