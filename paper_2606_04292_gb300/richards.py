"""Thin ctypes binding of the C ABI in ``include/richards.h``.

Argument marshalling only: every stage of the solver runs in the CUDA library
``_lib/librichards_gb300.so``.  Loading fails loudly when the library is
missing; there is no fallback.  Functions keep the C names
(``richards_create``, ``richards_step``, ...); :class:`Solver` wraps them for
a problem ``dict`` as produced by :mod:`paper_2606_04292_gb300.workloads`.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

RICH_OK, RICH_EINVAL, RICH_ENOMEM, RICH_ENOCONV, RICH_ENAN, RICH_ETIMEOUT, RICH_ECUDA, RICH_EBUSY = range(8)
STATUS_NAMES = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ENOCONV", 4: "ENAN", 5: "ETIMEOUT", 6: "ECUDA",
                7: "EBUSY"}


class RichardsError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class richards_grid(C.Structure):
    _fields_ = [("dim", C.c_int), ("n", C.c_int * 3), ("L", C.c_double * 3)]


class richards_soil(C.Structure):
    _fields_ = [("model", C.c_int), ("Ks", C.c_double), ("theta_s", C.c_double), ("theta_r", C.c_double),
                ("p1", C.c_double), ("p2", C.c_double), ("p3", C.c_double), ("p4", C.c_double),
                ("Ks_field", C.POINTER(C.c_double)), ("p1_field", C.POINTER(C.c_double)),
                ("p2_field", C.POINTER(C.c_double))]


class richards_material(C.Structure):
    _fields_ = [("model", C.c_int), ("Ks", C.c_double), ("theta_s", C.c_double), ("theta_r", C.c_double),
                ("p1", C.c_double), ("p2", C.c_double), ("p3", C.c_double), ("p4", C.c_double)]


class richards_bc(C.Structure):
    _fields_ = [("kind", C.c_int * 6), ("value", C.c_double * 6),
                ("value_field", C.POINTER(C.c_double) * 6), ("mask_field", C.POINTER(C.c_ubyte) * 6)]


class richards_sink(C.Structure):
    _fields_ = [("enabled", C.c_int), ("Tp", C.c_double), ("root_depth", C.c_double),
                ("root_decay", C.c_double), ("h1", C.c_double), ("h2", C.c_double), ("h3", C.c_double),
                ("h4", C.c_double)]


class richards_opts(C.Structure):
    _fields_ = [("nu1", C.c_int), ("nu2", C.c_int), ("coarse_max_sweeps", C.c_int), ("coarse_rtol", C.c_double),
                ("coarsest_max_n", C.c_int), ("max_levels", C.c_int), ("kappa_mode", C.c_int),
                ("kappa", C.c_double), ("xi", C.c_double), ("tol", C.c_double), ("max_cycles", C.c_int),
                ("ordering", C.c_int), ("newton_iters", C.c_int), ("precision", C.c_int),
                ("inner_cycles", C.c_int), ("inner_rtol", C.c_double), ("max_outer", C.c_int),
                ("tail_cells", C.c_int), ("cycle_gamma", C.c_int), ("gamma_levels", C.c_int),
                ("graphs", C.c_int), ("sweep_planes", C.c_int), ("predictor", C.c_int),
                ("fmg_cycles", C.c_int), ("layout", C.c_int), ("bdf2_lag", C.c_int)]


class richards_step_info(C.Structure):
    _fields_ = [("cycles", C.c_int), ("outer_iters", C.c_int), ("scheme_used", C.c_int),
                ("resid0", C.c_double), ("resid", C.c_double), ("cell_updates", C.c_longlong),
                ("mass_defect", C.c_double), ("err_bound", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class richards_column(C.Structure):
    _fields_ = [("n", C.c_int), ("L", C.c_double), ("soil", richards_soil), ("bc_kind", C.c_int * 2),
                ("bc_value", C.c_double * 2)]


class richards_kernel_stat(C.Structure):
    _fields_ = [("name", C.c_char * 32), ("level", C.c_int), ("launches", C.c_longlong), ("ms", C.c_double),
                ("cells", C.c_longlong)]


_DP = C.POINTER(C.c_double)
_VP = C.c_void_p
_lib = None

_SIGS = {
    "richards_create": (C.c_int, [C.POINTER(richards_grid), C.POINTER(richards_opts), _VP, C.POINTER(_VP)]),
    "richards_set_soil": (C.c_int, [_VP, C.POINTER(richards_soil)]),
    "richards_set_materials": (C.c_int, [_VP, C.POINTER(richards_material), C.c_int, C.POINTER(C.c_ubyte)]),
    "richards_set_bc": (C.c_int, [_VP, C.POINTER(richards_bc)]),
    "richards_set_sink": (C.c_int, [_VP, C.POINTER(richards_sink)]),
    "richards_set_state": (C.c_int, [_VP, _DP, _DP, C.c_double]),
    "richards_step": (C.c_int, [_VP, C.c_double, C.c_int, C.POINTER(richards_step_info)]),
    "richards_solve": (C.c_int, [_VP, C.c_double, C.c_int, C.c_int, C.POINTER(richards_step_info)]),
    "richards_get_state": (C.c_int, [_VP, _DP, C.c_int]),
    "richards_time": (C.c_double, [_VP]),
    "richards_ncell": (C.c_longlong, [_VP]),
    "richards_last_error": (C.c_char_p, [_VP]),
    "richards_destroy": (None, [_VP]),
    "richards_prepare": (C.c_int, [_VP, C.c_double, C.c_int, C.POINTER(C.c_int)]),
    "richards_nlevels": (C.c_int, [_VP]),
    "richards_level_dims": (C.c_int, [_VP, C.c_int, C.POINTER(C.c_int)]),
    "richards_soil_eval": (C.c_int, [_VP, _DP, _DP, _DP, C.c_int, C.c_int]),
    "richards_get_level": (C.c_int, [_VP, C.c_int, C.c_int, _DP, C.c_longlong]),
    "richards_set_level": (C.c_int, [_VP, C.c_int, C.c_int, _DP, C.c_longlong]),
    "richards_sweep": (C.c_int, [_VP, C.c_int, C.c_int]),
    "richards_residual": (C.c_int, [_VP, C.c_int, _DP]),
    "richards_restrict_tau": (C.c_int, [_VP, C.c_int]),
    "richards_prolong": (C.c_int, [_VP, C.c_int]),
    "richards_vcycle": (C.c_int, [_VP]),
    "richards_profile": (C.c_int, [_VP, C.c_int]),
    "richards_profile_read": (C.c_int, [_VP, C.POINTER(richards_kernel_stat), C.c_int]),
    "richards_batch_submit": (C.c_int, [C.POINTER(_VP), C.c_int, C.c_double, C.c_int, C.c_int]),
    "richards_batch_poll": (C.c_int, [C.POINTER(_VP), C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int),
                                      C.POINTER(richards_step_info)]),
    "richards_device_bytes": (C.c_longlong, [C.POINTER(richards_grid), C.POINTER(richards_opts), C.c_int, C.c_int]),
    "richards_columns_create": (C.c_int, [C.c_int, C.POINTER(richards_column), C.POINTER(richards_sink),
                                          C.POINTER(richards_opts), _VP, C.POINTER(_VP)]),
    "richards_columns_destroy": (None, [_VP]),
    "richards_columns_ncell": (C.c_longlong, [_VP]),
    "richards_columns_set_state": (C.c_int, [_VP, _DP, _DP]),
    "richards_columns_run": (C.c_int, [_VP, C.c_double, C.c_int, C.c_int]),
    "richards_columns_get_state": (C.c_int, [_VP, _DP, C.c_int]),
    "richards_columns_stats": (C.c_int, [_VP, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int), _DP,
                                         C.POINTER(C.c_longlong)]),
    "richards_columns_set_threads": (C.c_int, [_VP, C.c_int]),
    "richards_columns_autotune": (C.c_int, [_VP, C.c_double, C.c_int, C.POINTER(C.c_int)]),
    "richards_math_eval": (C.c_int, [C.c_int, _DP, _DP, C.c_longlong, _VP]),
    "richards_autotune": (C.c_int, [_VP, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "richards_set_launch": (C.c_int, [_VP, C.c_int, C.c_int, C.c_int, C.c_int]),
    "richards_set_coop": (C.c_int, [_VP, C.c_longlong]),
    "richards_graph_status": (C.c_char_p, [_VP]),
    "richards_batcher_create": (C.c_int, [_VP, C.c_int, C.POINTER(_VP)]),
    "richards_batcher_destroy": (None, [_VP]),
    "richards_batcher_last_error": (C.c_char_p, [_VP]),
    "richards_batcher_step": (C.c_int, [_VP, C.POINTER(_VP), C.c_int, _DP, C.POINTER(C.c_int), C.POINTER(C.c_int),
                                        C.POINTER(richards_step_info)]),
    "richards_batcher_advance": (C.c_int, [_VP, C.POINTER(_VP), C.c_int, _DP, C.POINTER(C.c_int),
                                           C.POINTER(C.c_int), C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int),
                                           C.POINTER(richards_step_info)]),
    "richards_step_small_noalloc": (C.c_int, [C.POINTER(richards_grid), C.POINTER(richards_soil),
                                              C.POINTER(richards_bc), C.POINTER(richards_sink),
                                              C.POINTER(richards_opts), C.c_double, C.c_int, _DP, _DP, _DP,
                                              C.POINTER(richards_step_info), _VP]),
}


def library_path():
    return _build.LIB


def lib(build_if_missing=True):
    """Load the CUDA library (building it when stale).  Raises if unavailable."""
    global _lib
    if _lib is None:
        path = _build.build() if build_if_missing else _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library missing: {path}")
        L = C.CDLL(path)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def exported_symbols():
    return list(_SIGS)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _dp(a):
    return a.ctypes.data_as(_DP)


def _check(st, ctx=None):
    if st != RICH_OK:
        msg = lib().richards_last_error(ctx).decode() if ctx else ""
        raise RichardsError(st, msg)


def make_opts(o):
    return richards_opts(o["nu1"], o["nu2"], o["coarse_max_sweeps"], o["coarse_rtol"], o["coarsest_max_n"],
                         o["max_levels"], o["kappa_mode"], o["kappa"], o["xi"], o["tol"], o["max_cycles"],
                         o["ordering"], o["newton_iters"], o["precision"], o["inner_cycles"], o["inner_rtol"],
                         o["max_outer"], o["tail_cells"], o.get("cycle_gamma", 1), o.get("gamma_levels", 0),
                         o.get("graphs", 1), o.get("sweep_planes", 2), o.get("predictor", 0),
                         o.get("fmg_cycles", 0), o.get("layout", 0), o.get("bdf2_lag", 0))


def current_stream():
    """Handle of torch's current CUDA stream (0 when torch is unavailable)."""
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except ImportError:
        pass
    return 0


class Solver:
    """One problem on the GPU through the C ABI."""

    def __init__(self, prob, stream=None, opts=None):
        L = lib()
        self.prob = prob
        self._keep = []
        o = dict(prob["opts"])
        if opts:
            o.update(opts)
        self.opts = o
        grid = richards_grid(prob["dim"], (C.c_int * 3)(*prob["n"]), (C.c_double * 3)(*prob["L"]))
        h = C.c_void_p()
        st = L.richards_create(C.byref(grid), C.byref(make_opts(o)),
                               C.c_void_p(current_stream() if stream is None else stream), C.byref(h))
        if st != RICH_OK:
            raise RichardsError(st, "richards_create failed")
        self.h = h
        self.N = int(L.richards_ncell(self.h))
        self.set_soil(prob["soil"])
        self.set_bc(prob["bc"])
        self.set_sink(prob["sink"])
        self.set_state(prob["psi0"], prob.get("psi_prev"))

    def close(self):
        if getattr(self, "h", None):
            lib().richards_destroy(self.h)
            self.h = None

    __del__ = close

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- set-up ----------------------------------------------------------
    def set_soil(self, s):
        if s.get("materials"):
            self.set_materials(s["materials"], s["material_index"])
            return
        soil = richards_soil(s["model"], s["Ks"], s["theta_s"], s["theta_r"], s["p1"], s["p2"], s["p3"], s["p4"])
        for key in ("Ks_field", "p1_field", "p2_field"):
            if s.get(key) is not None:
                arr = _f64(s[key])
                self._keep.append(arr)
                setattr(soil, key, _dp(arr))
        _check(lib().richards_set_soil(self.h, C.byref(soil)), self.h)

    def set_materials(self, mats, index):
        """Layered soil: a list of per-material law dicts and a uint8 index per cell."""
        arr = (richards_material * len(mats))(*[
            richards_material(m["model"], m["Ks"], m["theta_s"], m["theta_r"], m["p1"], m["p2"], m["p3"], m["p4"])
            for m in mats])
        idx = np.ascontiguousarray(index, dtype=np.uint8)
        if idx.size != self.N:
            raise RichardsError(RICH_EINVAL, "material index size mismatch")
        _check(lib().richards_set_materials(self.h, arr, len(mats), idx.ctypes.data_as(C.POINTER(C.c_ubyte))),
               self.h)

    def set_bc(self, b):
        bc = richards_bc()
        for f in range(6):
            bc.kind[f] = int(b["kind"][f])
            bc.value[f] = float(b["value"][f])
            if b["value_field"][f] is not None:
                arr = _f64(b["value_field"][f])
                self._keep.append(arr)
                bc.value_field[f] = _dp(arr)
            if b["mask_field"][f] is not None:
                arr = np.ascontiguousarray(b["mask_field"][f], dtype=np.uint8)
                self._keep.append(arr)
                bc.mask_field[f] = arr.ctypes.data_as(C.POINTER(C.c_ubyte))
        _check(lib().richards_set_bc(self.h, C.byref(bc)), self.h)

    def set_sink(self, k):
        sink = richards_sink(int(k["enabled"]), k["Tp"], k["root_depth"], k["root_decay"], k["h1"], k["h2"],
                             k["h3"], k["h4"])
        _check(lib().richards_set_sink(self.h, C.byref(sink)), self.h)

    def set_state(self, psi, psi_prev=None, t=0.0):
        psi = _f64(psi)
        pp = None if psi_prev is None else _f64(psi_prev)
        _check(lib().richards_set_state(self.h, _dp(psi), None if pp is None else _dp(pp), float(t)), self.h)

    # -- time stepping ---------------------------------------------------
    def step(self, dt=None, scheme=None, check=True):
        info = richards_step_info()
        st = lib().richards_step(self.h, float(self.prob["dt"] if dt is None else dt),
                                 int(self.prob["scheme"] if scheme is None else scheme), C.byref(info))
        if check and st not in (RICH_OK,):
            _check(st, self.h)
        return st, info.as_dict()

    def graph_status(self):
        """"" when the inner cycles run as CUDA graphs, else why not."""
        return lib().richards_graph_status(self.h).decode()

    def state(self):
        out = np.empty(self.N)
        _check(lib().richards_get_state(self.h, _dp(out), 0), self.h)
        return out

    def state_to_device(self, ptr):
        _check(lib().richards_get_state(self.h, C.cast(C.c_void_p(ptr), _DP), 1), self.h)

    @property
    def time(self):
        return lib().richards_time(self.h)

    # -- inspection ------------------------------------------------------
    def prepare(self, dt=None, scheme=None):
        used = C.c_int()
        _check(lib().richards_prepare(self.h, float(self.prob["dt"] if dt is None else dt),
                                      int(self.prob["scheme"] if scheme is None else scheme), C.byref(used)),
               self.h)
        return used.value

    @property
    def nlevels(self):
        return lib().richards_nlevels(self.h)

    def level_n(self, lev):
        n = (C.c_int * 3)()
        _check(lib().richards_level_dims(self.h, lev, n), self.h)
        return tuple(n)

    def level_ncell(self, lev):
        n = self.level_n(lev)
        return n[0] * n[1] * n[2]

    def soil_eval(self, psi, arith=0):
        """(theta, K) at the heads psi, one per fine cell; arith 1: float-float."""
        psi = _f64(psi)
        th, K = np.empty(self.N), np.empty(self.N)
        _check(lib().richards_soil_eval(self.h, _dp(psi), _dp(th), _dp(K), int(arith), 0), self.h)
        return th, K

    def get_level(self, lev, which):
        n = self.level_n(lev)
        if which >= 10:
            ax = (which - 10) // 2
            cnt = n[0] * n[1] * n[2] // n[ax]
        else:
            cnt = n[0] * n[1] * n[2]
        out = np.empty(cnt)
        _check(lib().richards_get_level(self.h, lev, which, _dp(out), cnt), self.h)
        return out

    def set_level(self, lev, which, arr):
        arr = _f64(arr)
        _check(lib().richards_set_level(self.h, lev, which, _dp(arr), arr.size), self.h)

    def sweep(self, lev=0, color=-1):
        _check(lib().richards_sweep(self.h, lev, color), self.h)

    def residual(self, lev=0):
        nrm = C.c_double()
        _check(lib().richards_residual(self.h, lev, C.byref(nrm)), self.h)
        return nrm.value

    def restrict_tau(self, lev=0):
        _check(lib().richards_restrict_tau(self.h, lev), self.h)

    def prolong(self, lev=0):
        _check(lib().richards_prolong(self.h, lev), self.h)

    def vcycle(self):
        _check(lib().richards_vcycle(self.h), self.h)

    # -- launch shapes ---------------------------------------------------
    def autotune(self, reps=5):
        """Time the candidate launch shapes of every big grid level on the
        current prepared state and keep the fastest; returns per level
        (planes, block_x, resid_block_x), 0 = default."""
        n = self.nlevels
        pl, bx, rb = (C.c_int * n)(), (C.c_int * n)(), (C.c_int * n)()
        _check(lib().richards_autotune(self.h, int(reps), pl, bx, rb), self.h)
        return [(pl[k], bx[k], rb[k]) for k in range(n)]

    def set_coop(self, max_cells):
        _check(lib().richards_set_coop(self.h, int(max_cells)), self.h)

    def set_launch(self, level, planes=0, block_x=0, resid_block_x=0):
        _check(lib().richards_set_launch(self.h, int(level), int(planes), int(block_x), int(resid_block_x)), self.h)

    # -- kernel timing ---------------------------------------------------
    def profile(self, enable=True, mode=1):
        """mode 1: time every launch; 2: time the finest level, count the rest;
        3: count only."""
        _check(lib().richards_profile(self.h, int(mode) if enable else 0), self.h)

    def profile_read(self):
        buf = (richards_kernel_stat * 256)()
        n = lib().richards_profile_read(self.h, buf, 256)
        if n < 0:
            raise RichardsError(RICH_EINVAL, "profile_read failed")
        return [dict(name=buf[i].name.decode(), level=buf[i].level, launches=buf[i].launches, ms=buf[i].ms,
                     cells=buf[i].cells) for i in range(n)]


class Columns:
    """A batch of independent 1D columns (``richards_columns_*``).

    ``probs``: list of 1D problem dicts (``workloads.columns()`` or
    ``random_problem(1, ...)``); soil fields are not used (scalar soil per
    column); the sink and the options of the first problem apply to all.
    """

    def __init__(self, probs, stream=None, opts=None):
        L = lib()
        self.probs = probs
        o = dict(probs[0]["opts"])
        if opts:
            o.update(opts)
        self.opts = o
        arr = (richards_column * len(probs))()
        for k, p in enumerate(probs):
            s = p["soil"]
            arr[k].n = int(p["n"][0])
            arr[k].L = float(p["L"][0])
            arr[k].soil = richards_soil(s["model"], s["Ks"], s["theta_s"], s["theta_r"], s["p1"], s["p2"],
                                        s["p3"], s["p4"])
            for f in range(2):
                arr[k].bc_kind[f] = int(p["bc"]["kind"][f])
                arr[k].bc_value[f] = float(p["bc"]["value"][f])
        k0 = probs[0]["sink"]
        sink = richards_sink(int(k0["enabled"]), k0["Tp"], k0["root_depth"], k0["root_decay"], k0["h1"],
                             k0["h2"], k0["h3"], k0["h4"])
        h = C.c_void_p()
        st = L.richards_columns_create(len(probs), arr, C.byref(sink), C.byref(make_opts(o)),
                                       C.c_void_p(current_stream() if stream is None else stream), C.byref(h))
        if st != RICH_OK:
            raise RichardsError(st, "richards_columns_create failed")
        self.h = h
        self.ncol = len(probs)
        self.N = int(L.richards_columns_ncell(h))
        self.offsets = np.cumsum([0] + [int(p["n"][0]) for p in probs])
        psi = np.concatenate([np.asarray(p["psi0"], dtype=np.float64) for p in probs])
        self.set_state(psi)

    def close(self):
        if getattr(self, "h", None):
            lib().richards_columns_destroy(self.h)
            self.h = None

    __del__ = close

    def set_state(self, psi, psi_prev=None):
        psi = _f64(psi)
        pp = None if psi_prev is None else _f64(psi_prev)
        st = lib().richards_columns_set_state(self.h, _dp(psi), None if pp is None else _dp(pp))
        if st != RICH_OK:
            raise RichardsError(st, "richards_columns_set_state failed")

    def run(self, dt, nsteps, scheme=1):
        return lib().richards_columns_run(self.h, float(dt), int(nsteps), int(scheme))

    def state(self):
        out = np.empty(self.N)
        st = lib().richards_columns_get_state(self.h, _dp(out), 0)
        if st != RICH_OK:
            raise RichardsError(st, "richards_columns_get_state failed")
        return out

    def column(self, psi, k):
        return psi[self.offsets[k]:self.offsets[k + 1]]

    def stats(self):
        n = self.ncol
        status = (C.c_int * n)()
        cycles = (C.c_int * n)()
        outer = (C.c_int * n)()
        resid = np.empty(n)
        upd = (C.c_longlong * n)()
        st = lib().richards_columns_stats(self.h, status, cycles, outer, _dp(resid), upd)
        if st != RICH_OK:
            raise RichardsError(st, "richards_columns_stats failed")
        return dict(status=np.array(status[:]), cycles=np.array(cycles[:]), outer=np.array(outer[:]),
                    resid=resid, updates=np.array(upd[:], dtype=np.int64))

    def set_threads(self, t):
        return lib().richards_columns_set_threads(self.h, int(t))

    def autotune(self, dt, scheme=1):
        t = C.c_int()
        st = lib().richards_columns_autotune(self.h, float(dt), int(scheme), C.byref(t))
        if st != RICH_OK:
            raise RichardsError(st, "richards_columns_autotune failed")
        return t.value


class Batcher:
    """Batched steps of many resident solvers (``richards_batcher_*``): step()
    advances every listed Solver by one step, advance() each by its own
    number of steps on its own schedule (continuous batching); the FP32 inner
    cycles of all solvers in an inner solve share launches."""

    def __init__(self, max_contexts=64, stream=None):
        h = C.c_void_p()
        st = lib().richards_batcher_create(C.c_void_p(current_stream() if stream is None else stream),
                                           int(max_contexts), C.byref(h))
        if st != RICH_OK:
            raise RichardsError(st, "richards_batcher_create failed")
        self.h = h
        self.cap = int(max_contexts)

    def close(self):
        if getattr(self, "h", None):
            lib().richards_batcher_destroy(self.h)
            self.h = None

    __del__ = close

    def step(self, solvers, dts, schemes):
        """One step of each solver; returns (status list, info dict list)."""
        n = len(solvers)
        hs = (C.c_void_p * n)(*[s.h.value for s in solvers])
        dt = _f64(dts)
        sc = (C.c_int * n)(*[int(x) for x in schemes])
        status = (C.c_int * n)()
        info = (richards_step_info * n)()
        st = lib().richards_batcher_step(self.h, hs, n, _dp(dt), sc, status, info)
        if st != RICH_OK:
            raise RichardsError(st, lib().richards_batcher_last_error(self.h).decode())
        return [int(x) for x in status], [info[k].as_dict() for k in range(n)]

    def advance(self, solvers, dts, schemes, steps_left, max_ticks=0):
        """Continuous batching (``richards_batcher_advance``): each solver
        takes up to steps_left[k] more steps on its own schedule; returns
        when one of them has done all its steps (or after max_ticks ticks).
        Returns (steps_left, steps_done, status, info) lists; info[k] sums
        cycles, outer iterations and updates over the steps done."""
        n = len(solvers)
        hs = (C.c_void_p * n)(*[s.h.value for s in solvers])
        dt = _f64(dts)
        sc = (C.c_int * n)(*[int(x) for x in schemes])
        left = (C.c_int * n)(*[int(x) for x in steps_left])
        done = (C.c_int * n)()
        status = (C.c_int * n)()
        info = (richards_step_info * n)()
        st = lib().richards_batcher_advance(self.h, hs, n, _dp(dt), sc, left, int(max_ticks), done, status, info)
        if st != RICH_OK:
            raise RichardsError(st, lib().richards_batcher_last_error(self.h).decode())
        return ([int(x) for x in left], [int(x) for x in done], [int(x) for x in status],
                [info[k].as_dict() for k in range(n)])
