"""ctypes wrapper of the CPU FP64 oracle -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this module.  It loads ``oracle/liborc.so`` (built from
``richards_oracle.c`` by :func:`build`) and exposes a small class ``Oracle``
that takes the same problem ``dict`` as the CUDA binding (see
``paper_2606_04292_gb300.workloads``).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "richards_oracle.c")
LIB = os.path.join(HERE, "liborc.so")

ORC_OK, ORC_EINVAL, ORC_ENOCONV, ORC_ENAN = 0, 1, 3, 4


def build(force=False):
    """Compile the oracle with gcc: -O2, no fast-math, no FP contraction."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= max(
            os.path.getmtime(SRC), os.path.getmtime(os.path.join(HERE, "richards_oracle.h"))):
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    base = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-o", tmp, SRC]
    # OpenMP only shares the cells of one red-black colour among threads
    # (orc_sweep_rb_threads); without it that sweep runs on one thread
    if subprocess.run(base + ["-fopenmp", "-lm"], capture_output=True).returncode != 0:
        subprocess.check_call(base + ["-lm"])
    os.replace(tmp, LIB)
    return LIB


class _Grid(C.Structure):
    _fields_ = [("dim", C.c_int), ("n", C.c_int * 3), ("L", C.c_double * 3)]


class _Soil(C.Structure):
    _fields_ = [("model", C.c_int), ("Ks", C.c_double), ("theta_s", C.c_double),
                ("theta_r", C.c_double), ("p1", C.c_double), ("p2", C.c_double),
                ("p3", C.c_double), ("p4", C.c_double),
                ("Ks_field", C.POINTER(C.c_double)), ("p1_field", C.POINTER(C.c_double)),
                ("p2_field", C.POINTER(C.c_double))]


class _Material(C.Structure):
    _fields_ = [("model", C.c_int), ("Ks", C.c_double), ("theta_s", C.c_double),
                ("theta_r", C.c_double), ("p1", C.c_double), ("p2", C.c_double),
                ("p3", C.c_double), ("p4", C.c_double)]


class _BC(C.Structure):
    _fields_ = [("kind", C.c_int * 6), ("value", C.c_double * 6),
                ("value_field", C.POINTER(C.c_double) * 6),
                ("mask_field", C.POINTER(C.c_ubyte) * 6)]


class _Sink(C.Structure):
    _fields_ = [("enabled", C.c_int), ("Tp", C.c_double), ("root_depth", C.c_double),
                ("root_decay", C.c_double), ("h1", C.c_double), ("h2", C.c_double),
                ("h3", C.c_double), ("h4", C.c_double)]


class _Opts(C.Structure):
    _fields_ = [("nu1", C.c_int), ("nu2", C.c_int), ("coarse_max_sweeps", C.c_int),
                ("coarse_rtol", C.c_double), ("coarsest_max_n", C.c_int),
                ("max_levels", C.c_int), ("kappa_mode", C.c_int), ("kappa", C.c_double),
                ("xi", C.c_double), ("tol", C.c_double), ("max_cycles", C.c_int),
                ("ordering", C.c_int), ("newton_iters", C.c_int), ("cycle_gamma", C.c_int),
                ("gamma_levels", C.c_int), ("fmg_cycles", C.c_int), ("bdf2_lag", C.c_int)]


class _Info(C.Structure):
    _fields_ = [("cycles", C.c_int), ("resid", C.c_double), ("resid0", C.c_double)]


_lib = None
_DP = C.POINTER(C.c_double)


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(LIB)
        L.orc_create.restype = C.c_void_p
        L.orc_create.argtypes = [C.POINTER(_Grid), C.POINTER(_Soil), C.POINTER(_BC),
                                 C.POINTER(_Sink), C.POINTER(_Opts)]
        L.orc_destroy.argtypes = [C.c_void_p]
        L.orc_nlevels.argtypes = [C.c_void_p]
        L.orc_level_n.argtypes = [C.c_void_p, C.c_int, C.POINTER(C.c_int)]
        L.orc_level_ncell.restype = C.c_long
        L.orc_level_ncell.argtypes = [C.c_void_p, C.c_int]
        L.orc_face_ncell.restype = C.c_long
        L.orc_face_ncell.argtypes = [C.c_void_p, C.c_int, C.c_int]
        L.orc_set_state.argtypes = [C.c_void_p, _DP, _DP]
        L.orc_get_state.argtypes = [C.c_void_p, _DP]
        L.orc_prepare.argtypes = [C.c_void_p, C.c_double, C.c_int]
        L.orc_a.restype = C.c_double
        L.orc_a.argtypes = [C.c_void_p]
        L.orc_apply_N.argtypes = [C.c_void_p, C.c_int, _DP, _DP]
        L.orc_residual.restype = C.c_double
        L.orc_residual.argtypes = [C.c_void_p, C.c_int, _DP, _DP, _DP]
        L.orc_sweep.argtypes = [C.c_void_p, C.c_int, _DP, _DP, C.c_int]
        L.orc_sweep_ordering.argtypes = [C.c_void_p, C.c_int, _DP, _DP, C.c_int]
        L.orc_sweep_rb_threads.argtypes = [C.c_void_p, C.c_int, _DP, _DP, C.c_int]
        L.orc_sweep_rb_threads.restype = C.c_int
        L.orc_restrict.argtypes = [C.c_void_p, C.c_int, _DP, _DP]
        L.orc_prolong_add.argtypes = [C.c_void_p, C.c_int, _DP, _DP]
        L.orc_vcycle.argtypes = [C.c_void_p, C.c_int, _DP, _DP]
        L.orc_step.argtypes = [C.c_void_p, C.c_double, C.c_int, C.POINTER(_Info)]
        L.orc_solve_current.argtypes = [C.c_void_p, _DP, C.POINTER(_Info)]
        L.orc_fmg.argtypes = [C.c_void_p, _DP]
        L.orc_set_materials.restype = C.c_int
        L.orc_set_materials.argtypes = [C.c_void_p, C.POINTER(_Material), C.c_int, C.POINTER(C.c_ubyte)]
        L.orc_level_material.restype = None
        L.orc_level_material.argtypes = [C.c_void_p, C.c_int, C.POINTER(C.c_ubyte)]
        L.orc_get_array.argtypes = [C.c_void_p, C.c_int, C.c_int, _DP]
        L.orc_set_g.argtypes = [C.c_void_p, _DP]
        L.orc_soil_eval.argtypes = [C.c_void_p, C.c_int, C.c_long, C.c_double, _DP, _DP, _DP]
        L.orc_sink_eval.argtypes = [C.c_void_p, C.c_int, C.c_long, C.c_double, _DP, _DP]
        L.orc_point_solve.restype = C.c_double
        L.orc_point_solve.argtypes = [C.c_void_p, C.c_int, C.c_long, C.c_double, C.c_double,
                                      C.c_double, C.c_int, C.POINTER(C.c_int)]
        L.orc_dense_M.argtypes = [C.c_void_p, C.c_int, _DP]
        L.orc_boundary_inflow.restype = C.c_double
        L.orc_boundary_inflow.argtypes = [C.c_void_p, _DP]
        L.orc_cell_volume.restype = C.c_double
        L.orc_cell_volume.argtypes = [C.c_void_p, C.c_int]
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(_DP)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class Oracle:
    """One problem on the CPU.  Holds references to every array handed over."""

    def __init__(self, prob):
        L = lib()
        self.prob = prob
        self._keep = []
        g = _Grid(prob["dim"], (C.c_int * 3)(*prob["n"]), (C.c_double * 3)(*prob["L"]))
        s = prob["soil"]
        soil = _Soil(s["model"], s["Ks"], s["theta_s"], s["theta_r"], s["p1"], s["p2"],
                     s["p3"], s["p4"])
        for key in ("Ks_field", "p1_field", "p2_field"):
            if s.get(key) is not None:
                arr = _f64(s[key])
                self._keep.append(arr)
                setattr(soil, key, _dp(arr))
        b = prob["bc"]
        bc = _BC()
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
        k = prob["sink"]
        sink = _Sink(int(k["enabled"]), k["Tp"], k["root_depth"], k["root_decay"],
                     k["h1"], k["h2"], k["h3"], k["h4"])
        o = prob["opts"]
        opts = _Opts(o["nu1"], o["nu2"], o["coarse_max_sweeps"], o["coarse_rtol"],
                     o["coarsest_max_n"], o["max_levels"], o["kappa_mode"], o["kappa"],
                     o["xi"], o["tol"], o["max_cycles"], o["ordering"], o["newton_iters"],
                     o.get("cycle_gamma", 1), o.get("gamma_levels", 0), o.get("fmg_cycles", 0),
                     o.get("bdf2_lag", 0))
        self.h = L.orc_create(C.byref(g), C.byref(soil), C.byref(bc), C.byref(sink),
                              C.byref(opts))
        if not self.h:
            raise ValueError("oracle rejected the problem")
        if s.get("materials"):
            mats = (_Material * len(s["materials"]))(*[
                _Material(m["model"], m["Ks"], m["theta_s"], m["theta_r"], m["p1"], m["p2"], m["p3"], m["p4"])
                for m in s["materials"]])
            idx = np.ascontiguousarray(s["material_index"], dtype=np.uint8)
            if L.orc_set_materials(self.h, mats, len(s["materials"]),
                                   idx.ctypes.data_as(C.POINTER(C.c_ubyte))) != ORC_OK:
                raise ValueError("oracle rejected the materials")
        self.N = int(L.orc_level_ncell(self.h, 0))
        self.set_state(prob["psi0"], prob.get("psi_prev"))

    def __del__(self):
        if getattr(self, "h", None):
            lib().orc_destroy(self.h)
            self.h = None

    # -- hierarchy -------------------------------------------------------
    @property
    def nlevels(self):
        return lib().orc_nlevels(self.h)

    def level_n(self, lev):
        n = (C.c_int * 3)()
        lib().orc_level_n(self.h, lev, n)
        return tuple(n)

    def ncell(self, lev=0):
        return int(lib().orc_level_ncell(self.h, lev))

    def nface(self, lev, face):
        return int(lib().orc_face_ncell(self.h, lev, face))

    # -- state -----------------------------------------------------------
    def set_state(self, psi, psi_prev=None):
        psi = _f64(psi)
        if psi_prev is None:
            lib().orc_set_state(self.h, _dp(psi), None)
        else:
            pp = _f64(psi_prev)
            lib().orc_set_state(self.h, _dp(psi), _dp(pp))

    def state(self):
        out = np.empty(self.N)
        lib().orc_get_state(self.h, _dp(out))
        return out

    def prepare(self, dt, scheme):
        return lib().orc_prepare(self.h, float(dt), int(scheme))

    @property
    def a(self):
        return lib().orc_a(self.h)

    def array(self, which, lev=0):
        if which >= 10:
            n = self.nface(lev, which - 10)
        elif which in (6, 7):
            n = self.N
        else:
            n = self.ncell(lev)
        out = np.empty(n)
        lib().orc_get_array(self.h, lev, which, _dp(out))
        return out

    def Kc(self, lev=0):
        return self.array(0, lev)

    def g(self, lev=0):
        return self.array(1, lev)

    def set_g(self, g):
        g = _f64(g)
        lib().orc_set_g(self.h, _dp(g))

    # -- operators -------------------------------------------------------
    def apply_N(self, psi, lev=0):
        psi = _f64(psi)
        out = np.empty_like(psi)
        lib().orc_apply_N(self.h, lev, _dp(psi), _dp(out))
        return out

    def residual(self, psi, g=None, lev=0):
        psi = _f64(psi)
        g = self.g(lev) if g is None else _f64(g)
        r = np.empty_like(psi)
        nrm = lib().orc_residual(self.h, lev, _dp(psi), _dp(g), _dp(r))
        return r, nrm

    def sweep(self, psi, g=None, lev=0, color=-1, ordering=None):
        psi = _f64(psi).copy()
        g = self.g(lev) if g is None else _f64(g)
        if ordering is None:
            lib().orc_sweep(self.h, lev, _dp(psi), _dp(g), int(color))
        else:
            lib().orc_sweep_ordering(self.h, lev, _dp(psi), _dp(g), int(ordering))
        return psi

    def sweep_threads(self, psi, nthreads=0, g=None, lev=0):
        """One red-black sweep on nthreads OpenMP threads (0: all); the same
        result as sweep(psi, ordering=1).  Returns (psi, threads used)."""
        psi = _f64(psi).copy()
        g = self.g(lev) if g is None else _f64(g)
        used = lib().orc_sweep_rb_threads(self.h, lev, _dp(psi), _dp(g), int(nthreads))
        return psi, int(used)

    def restrict(self, fine, lev=0):
        fine = _f64(fine)
        out = np.empty(self.ncell(lev + 1))
        lib().orc_restrict(self.h, lev, _dp(fine), _dp(out))
        return out

    def prolong_add(self, coarse, fine, lev=0):
        coarse = _f64(coarse)
        fine = _f64(fine).copy()
        lib().orc_prolong_add(self.h, lev, _dp(coarse), _dp(fine))
        return fine

    def vcycle(self, psi, g=None, lev=0):
        psi = _f64(psi).copy()
        g = self.g(lev) if g is None else _f64(g)
        lib().orc_vcycle(self.h, lev, _dp(psi), _dp(g))
        return psi

    def step(self, dt=None, scheme=None):
        info = _Info()
        st = lib().orc_step(self.h, float(dt if dt is not None else self.prob["dt"]),
                            int(scheme if scheme is not None else self.prob["scheme"]),
                            C.byref(info))
        return st, dict(cycles=info.cycles, resid=info.resid, resid0=info.resid0)

    def fmg(self, psi):
        """Full multigrid pass (fmg_cycles per level) from psi on the prepared step."""
        psi = _f64(psi).copy()
        lib().orc_fmg(self.h, _dp(psi))
        return psi

    def solve_current(self, psi):
        psi = _f64(psi).copy()
        info = _Info()
        st = lib().orc_solve_current(self.h, _dp(psi), C.byref(info))
        return psi, st, dict(cycles=info.cycles, resid=info.resid, resid0=info.resid0)

    # -- pointwise -------------------------------------------------------
    def soil(self, cell, psi, lev=0):
        th, dth, K = C.c_double(), C.c_double(), C.c_double()
        lib().orc_soil_eval(self.h, lev, int(cell), float(psi), C.byref(th), C.byref(dth),
                            C.byref(K))
        return th.value, dth.value, K.value

    def sink(self, cell, psi, lev=0):
        S, dS = C.c_double(), C.c_double()
        lib().orc_sink_eval(self.h, lev, int(cell), float(psi), C.byref(S), C.byref(dS))
        return S.value, dS.value

    def point_solve(self, cell, cc, f, x0, newton_iters=0, lev=0):
        it = C.c_int()
        x = lib().orc_point_solve(self.h, lev, int(cell), float(cc), float(f), float(x0),
                                  int(newton_iters), C.byref(it))
        return x, it.value

    def dense_M(self, lev=0):
        n = self.ncell(lev)
        M = np.empty((n, n))
        lib().orc_dense_M(self.h, lev, _dp(M))
        return M

    def boundary_inflow(self, psi):
        psi = _f64(psi)
        return lib().orc_boundary_inflow(self.h, _dp(psi))

    def material_map(self, lev=0):
        out = np.zeros(self.ncell(lev), dtype=np.uint8)
        lib().orc_level_material(self.h, lev, out.ctypes.data_as(C.POINTER(C.c_ubyte)))
        return out

    def cell_volume(self, lev=0):
        return lib().orc_cell_volume(self.h, lev)
