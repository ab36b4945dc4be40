"""Seeded synthetic inputs for the Richards solver.

This module only *describes* problems: grid sizes, soil parameters, boundary
descriptors, sink parameters, initial states and time-step settings.  It holds
none of the method's arithmetic (no constitutive law that a result is
computed with, no operator, no solver), so that both the CUDA path and the
CPU oracle can consume the same inputs without sharing any code that
computes a result.  The one law-shaped helper, ``head_at_saturation``,
inverts Table 1's theta only to choose starting heads for the serving trace:
any head is a valid input, and no result is checked against it.

Problem layout (a plain ``dict``):

* ``dim``: 1, 2 or 3.  The last active axis (``dim-1``) is the vertical axis,
  with elevation ``z`` increasing upward (the bottom face is ``z = 0``).
* ``n``: cells per axis, a 3-tuple; axes ``>= dim`` have ``n = 1``.
* ``L``: domain length per axis (the units of the problem; cm for the
  Celia column, m elsewhere).
* ``soil``: ``model`` (``HAVERKAMP``/``GARDNER``/``VANGENUCHTEN``), scalars
  ``Ks, theta_s, theta_r, p1..p4`` and optional per-cell fields
  ``Ks_field, p1_field, p2_field`` (x-fastest, float64).
  Parameter meaning per model (Table 1 of the paper):
  Haverkamp p1=alpha, p2=beta, p3=A, p4=gamma; Gardner p1=alpha;
  van Genuchten p1=alpha, p2=n, p3=l (pore-connectivity, 0.5).
* ``bc``: per face ``2*axis+side`` (side 0 = low end, 1 = high end):
  ``kind`` (``DIRICHLET``/``NOFLUX``/``FLUX``/``FREE_DRAINAGE``), ``value``
  (head for Dirichlet, inflow rate for flux), optional ``value_field`` and
  ``mask_field`` over the face cells (lexicographic over the other axes).
* ``sink``: Feddes-type root-water-uptake parameters (``enabled``, ``Tp``,
  ``root_depth``, ``root_decay``, ``h1..h4``).
* ``psi0`` (and optionally ``psi_prev``): initial state, float64, x-fastest.
* ``dt``, ``nsteps``, ``scheme`` (1 = BDF1, 2 = BDF2).
* ``opts``: solver options (sweeps, kappa mode, xi, tolerance, ...).

Every parameter and per-cell field is a plain float64 draw: the library makes
whatever lower-precision copies it needs on the device itself.
"""
from __future__ import annotations

import copy
import math

import numpy as np

HAVERKAMP, GARDNER, VANGENUCHTEN = 0, 1, 2
DIRICHLET, NOFLUX, FLUX, FREE_DRAINAGE = 0, 1, 2, 3

MODEL_NAMES = {HAVERKAMP: "haverkamp", GARDNER: "gardner", VANGENUCHTEN: "vangenuchten"}

# 5 mm/day of potential transpiration, in m/s.
TP_5MM_PER_DAY = 5.0e-3 / 86400.0


def default_opts(**kw):
    o = dict(nu1=2, nu2=2, coarse_max_sweeps=50, coarse_rtol=0.1,
             coarsest_max_n=4, max_levels=0,
             kappa_mode=0, kappa=0.0, xi=0.0,
             tol=1e-8, max_cycles=60,
             ordering=1,          # 0 = lexicographic, 1 = red-black
             newton_iters=2,      # 0 = to tolerance; k > 0 = exactly k steps
             precision=0,         # 0 = FP64 plain, 1 = FP32 inner / float-float outer, 2 = FP64 outer
             inner_cycles=8, inner_rtol=1e-3, max_outer=20,
             tail_cells=4096, cycle_gamma=1, gamma_levels=0, graphs=1, sweep_planes=2, predictor=0,
             fmg_cycles=0,
             layout=0,
             bdf2_lag=0)          # BDF2 lag of K and the xi term: 0 = 2 psi^n - psi^(n-1), 1 = psi^n
    o.update(kw)
    return o


def no_sink():
    return dict(enabled=0, Tp=0.0, root_depth=0.3, root_decay=0.1,
                h1=-0.10, h2=-0.25, h3=-5.0, h4=-80.0)


def feddes_sink(Tp=TP_5MM_PER_DAY):
    return dict(enabled=1, Tp=Tp, root_depth=0.3, root_decay=0.1,
                h1=-0.10, h2=-0.25, h3=-5.0, h4=-80.0)


def _bc(kinds, values=None):
    kinds = list(kinds) + [NOFLUX] * (6 - len(kinds))
    values = list(values or []) + [0.0] * (6 - len(values or []))
    return dict(kind=kinds, value=values, value_field=[None] * 6, mask_field=[None] * 6)


def _soil(model, Ks, theta_s, theta_r, p1=0.0, p2=0.0, p3=0.0, p4=0.0,
          Ks_field=None, p1_field=None, p2_field=None):
    return dict(model=model, Ks=float(Ks), theta_s=float(theta_s), theta_r=float(theta_r),
                p1=float(p1), p2=float(p2), p3=float(p3), p4=float(p4),
                Ks_field=Ks_field, p1_field=p1_field, p2_field=p2_field)


def ncells(prob):
    n = prob["n"]
    return int(n[0] * n[1] * n[2])


# ---------------------------------------------------------------------------
# The paper's 1D Celia/Haverkamp column (Section 4.1, Table 2), in cm and s.
# ---------------------------------------------------------------------------
def celia_1d(n=128, dt=10.0, nsteps=36, **optkw):
    soil = _soil(HAVERKAMP, Ks=0.00944, theta_s=0.287, theta_r=0.075,
                 p1=1.611e6, p2=3.96, p3=1.175e6, p4=4.74)
    bc = _bc([DIRICHLET, DIRICHLET], [-61.5, -20.7])   # bottom, top (cm)
    # The paper's shift kappa = 0.1 goes with its tau = 0.1 s; at dt = 10 s it
    # under-relaxes the dry cells so strongly that the cycles stall, so the
    # 10 s workload uses kappa = 0 (pass kappa=0.1, dt=0.1 for the paper's run).
    opts = default_opts(kappa_mode=0, kappa=0.0, xi=0.0)
    opts.update(optkw)
    return dict(name=f"celia1d_n{n}", dim=1, n=(n, 1, 1), L=(40.0, 1.0, 1.0),
                soil=soil, bc=bc, sink=no_sink(),
                psi0=np.full(n, -61.5), psi_prev=None,
                dt=dt, nsteps=nsteps, scheme=1, opts=opts)


# ---------------------------------------------------------------------------
# 2D strip infiltration (513^2 over 1 m^2, van Genuchten), in m and s.
# ---------------------------------------------------------------------------
def strip_2d(n=513, dt=60.0, nsteps=100, **optkw):
    soil = _soil(VANGENUCHTEN, Ks=1e-5, theta_s=0.368, theta_r=0.102,
                 p1=3.35, p2=2.0, p3=0.5)
    # axis 0 = x, axis 1 = z (vertical).  Faces: 0 x-low, 1 x-high, 2 bottom, 3 top.
    bc = _bc([NOFLUX, NOFLUX, DIRICHLET, DIRICHLET], [0.0, 0.0, -10.0, -0.1])
    h = 1.0 / n
    xc = (np.arange(n) + 0.5) * h
    bc["mask_field"][3] = (np.abs(xc - 0.5) <= 0.1).astype(np.uint8)
    # BDF2 with K lagged at psi^n: the wetting front into soil at -10 m is one
    # cell wide, and the extrapolated lag 2 psi^n - psi^(n-1) there jumps from
    # dry to saturated conductivity between steps; from about step 20 the
    # V-cycles then alternate between two states instead of converging (the
    # oracle shows the same).  bdf2_lag=0 selects the extrapolated lag.
    opts = default_opts(kappa_mode=0, kappa=0.0, xi=0.0, bdf2_lag=1)
    opts.update(optkw)
    return dict(name=f"strip2d_n{n}", dim=2, n=(n, n, 1), L=(1.0, 1.0, 1.0),
                soil=soil, bc=bc, sink=no_sink(),
                psi0=np.full(n * n, -10.0), psi_prev=None,
                dt=dt, nsteps=nsteps, scheme=2, opts=opts)


# ---------------------------------------------------------------------------
# The paper's 2D infiltration test (Section 4.2): Gardner soil on (0, 10)^2 m,
# time in days, h = -10 m initially and on every boundary but the top, where
# eq. top-bc prescribes h(x) = ln(e^{-10 alpha} + (1 - e^{-10 alpha})
# sin(pi x / 10)) / alpha (0 at x = 5, -10 at the corners); 3 days at
# tau = 0.1 day on 128^2 cells.
# ---------------------------------------------------------------------------
def gardner_2d(n=128, dt=0.1, nsteps=30, **optkw):
    alpha = 0.164
    soil = _soil(GARDNER, Ks=0.1, theta_s=0.45, theta_r=0.15, p1=alpha)
    # faces: 0 x-low, 1 x-high, 2 bottom, 3 top (axis 1 vertical)
    bc = _bc([DIRICHLET, DIRICHLET, DIRICHLET, DIRICHLET], [-10.0, -10.0, -10.0, 0.0])
    xc = (np.arange(n) + 0.5) * (10.0 / n)
    e = math.exp(-10.0 * alpha)
    bc["value_field"][3] = np.log(e + (1.0 - e) * np.sin(np.pi * xc / 10.0)) / alpha
    opts = default_opts(kappa_mode=0, kappa=0.0, xi=0.0)
    opts.update(optkw)
    return dict(name=f"gardner2d_n{n}", dim=2, n=(n, n, 1), L=(10.0, 10.0, 1.0),
                soil=soil, bc=bc, sink=no_sink(),
                psi0=np.full(n * n, -10.0), psi_prev=None,
                dt=dt, nsteps=nsteps, scheme=1, opts=opts)


# ---------------------------------------------------------------------------
# Layered soils (spatially varying laws).  A soil dict may carry
# "materials" (list of per-material laws and parameters) and
# "material_index" (uint8 per cell); each cell then uses its material.
# ---------------------------------------------------------------------------
def material(model, Ks, theta_s, theta_r, p1=0.0, p2=0.0, p3=0.0, p4=0.0):
    return dict(model=int(model), Ks=float(Ks), theta_s=float(theta_s), theta_r=float(theta_r),
                p1=float(p1), p2=float(p2), p3=float(p3), p4=float(p4))


def celia_composite_1d(n=128, dt=10.0, nsteps=36, **optkw):
    """Section 4.1's composite column (cm, s): Gardner for 30 <= z < 40,
    Haverkamp for 20 <= z < 30, van Genuchten-Mualem elsewhere, with the
    shared Ks, theta_s, theta_r of Table 2 and the parameters of Table 4."""
    prob = celia_1d(n=n, dt=dt, nsteps=nsteps, **optkw)
    Ks, ts, tr = 0.00944, 0.287, 0.075
    mats = [material(VANGENUCHTEN, Ks, ts, tr, p1=0.03165, p2=3.349, p3=0.5),
            material(HAVERKAMP, Ks, ts, tr, p1=1.611e6, p2=3.96, p3=1.175e6, p4=4.74),
            material(GARDNER, Ks, ts, tr, p1=0.01877)]
    z = (np.arange(n) + 0.5) * (40.0 / n)
    idx = np.zeros(n, dtype=np.uint8)
    idx[(z >= 20.0) & (z < 30.0)] = 1
    idx[(z >= 30.0) & (z < 40.0)] = 2
    prob["soil"] = dict(prob["soil"], materials=mats, material_index=idx)
    prob["name"] = f"celia_composite1d_n{n}"
    return prob


def two_layer_2d(n=256, dt=0.01, nsteps=100, **optkw):
    """Section 4.2's two-layer van Genuchten-Mualem field (cm, hours) on
    (0, 100)^2: the interface zeta(x) = 100 (0.1 (1 - cos(pi x / 100)) + 0.45),
    psi = -z initially, psi = 0 on the top and bottom, no flux on the sides;
    FMG with 10 pre- and 10 post-smoothing sweeps, kappa = 0.1, xi = 0."""
    upper = material(VANGENUCHTEN, 0.25, 0.50, 0.120, p1=0.025, p2=3.00, p3=0.5)
    lower = material(VANGENUCHTEN, 2.00, 0.46, 0.034, p1=0.016, p2=1.37, p3=0.5)
    h = 100.0 / n
    xc = (np.arange(n) + 0.5) * h
    zc = (np.arange(n) + 0.5) * h
    zeta = 100.0 * (0.1 * (1.0 - np.cos(np.pi * xc / 100.0)) + 0.45)
    idx = (zc[:, None] < zeta[None, :]).astype(np.uint8).reshape(-1)     # [z, x], x fastest
    soil = _soil(VANGENUCHTEN, Ks=upper["Ks"], theta_s=upper["theta_s"], theta_r=upper["theta_r"],
                 p1=upper["p1"], p2=upper["p2"], p3=0.5)
    soil.update(materials=[upper, lower], material_index=idx)
    bc = _bc([NOFLUX, NOFLUX, DIRICHLET, DIRICHLET], [0.0, 0.0, 0.0, 0.0])
    opts = default_opts(kappa_mode=0, kappa=0.1, xi=0.0, nu1=10, nu2=10, fmg_cycles=1)
    opts.update(optkw)
    psi0 = -np.repeat(zc, n)
    return dict(name=f"two_layer2d_n{n}", dim=2, n=(n, n, 1), L=(100.0, 100.0, 1.0),
                soil=soil, bc=bc, sink=no_sink(), psi0=psi0, psi_prev=None,
                dt=dt, nsteps=nsteps, scheme=1, opts=opts)


def test_materials():
    """Three materials in m and s, one per law, with distinct Ks, theta_s and
    theta_r."""
    return [material(VANGENUCHTEN, 1e-5, 0.368, 0.102, p1=3.35, p2=2.0, p3=0.5),
            material(HAVERKAMP, 2.5e-5, 0.287, 0.075, p1=1.611e6 * 100.0 ** -3.96,
                     p2=3.96, p3=1.175e6 * 100.0 ** -4.74, p4=4.74),
            material(GARDNER, 4e-6, 0.45, 0.15, p1=2.0)]


def with_materials(prob, mats, index):
    """A copy of prob whose soil carries the given materials and per-cell index."""
    p = copy.copy(prob)
    p["soil"] = dict(prob["soil"], materials=list(mats),
                     material_index=np.ascontiguousarray(index, dtype=np.uint8))
    return p


def material_pattern(prob, kind, nmat, seed):
    """A material index for prob's grid: "random" (independent per cell) or
    "layers" (bands in the vertical axis bounded by wavy interfaces)."""
    nn = prob["n"]
    N = nn[0] * nn[1] * nn[2]
    rng = np.random.Generator(np.random.PCG64(seed))
    if kind == "random":
        return rng.integers(0, nmat, N).astype(np.uint8)
    dim = prob["dim"]
    idx = np.arange(N)
    pos = [idx % nn[0], (idx // nn[0]) % nn[1], idx // (nn[0] * nn[1])]
    z = (pos[dim - 1] + 0.5) / nn[dim - 1]
    x = (pos[0] + 0.5) / nn[0] if dim > 1 else np.zeros(N)
    cuts = np.sort(rng.uniform(0.15, 0.85, nmat - 1))
    amp = rng.uniform(0.0, 0.1, nmat - 1)
    out = np.zeros(N, dtype=np.uint8)
    for k in range(nmat - 1):
        out += (z >= cuts[k] + amp[k] * np.sin(2.0 * np.pi * x)).astype(np.uint8)
    return out


def gaussian_log_field(shape, corr_cells, seed):
    """Standardised Gaussian random field with covariance ~ exp(-r^2/corr^2).

    White noise (seeded PCG64) convolved, with periodic wrap via FFT, with a
    Gaussian kernel of standard deviation corr/sqrt(2) cells; then shifted and
    scaled to sample mean 0 and standard deviation 1.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    w = rng.standard_normal(shape)
    s = corr_cells / math.sqrt(2.0)
    F = np.fft.rfftn(w)
    freqs = [np.fft.fftfreq(m) for m in shape[:-1]] + [np.fft.rfftfreq(shape[-1])]
    grids = np.meshgrid(*freqs, indexing="ij")
    k2 = sum(g * g for g in grids)
    F *= np.exp(-2.0 * (math.pi ** 2) * (s ** 2) * k2)
    G = np.fft.irfftn(F, s=shape, axes=list(range(len(shape))))
    G = (G - G.mean()) / G.std()
    return G


# ---------------------------------------------------------------------------
# 3D drainage (256^3 over 1 m^3, heterogeneous van Genuchten), m and s.
# ---------------------------------------------------------------------------
def drainage_3d(n=256, dt=300.0, nsteps=50, seed_ks=3, seed_vg=4, **optkw):
    shape_zyx = (n, n, n)
    G = gaussian_log_field(shape_zyx, 8.0, seed_ks)          # indexed [z, y, x]
    Ks = np.exp(math.log(1e-5) + 1.0 * G).reshape(-1)   # x fastest
    rng = np.random.Generator(np.random.PCG64(seed_vg))
    alpha = rng.uniform(2.0, 5.0, n ** 3)
    nvg = rng.uniform(1.5, 2.5, n ** 3)
    soil = _soil(VANGENUCHTEN, Ks=1e-5, theta_s=0.368, theta_r=0.102,
                 p1=3.5, p2=2.0, p3=0.5, Ks_field=Ks, p1_field=alpha, p2_field=nvg)
    # faces: x-low, x-high, y-low, y-high, bottom (free drainage), top (no flux)
    bc = _bc([NOFLUX, NOFLUX, NOFLUX, NOFLUX, FREE_DRAINAGE, NOFLUX])
    # W-cycles on the two finest levels (V below): on this heterogeneous,
    # partly saturated field they need ~2.4x fewer cycles than V-cycles, as
    # many as full W-cycles.  Two post- and no pre-smoothing sweeps, W(0,2):
    # 13.9 cycles per step against 10.6 for W(2,2), but each cycle reuses the
    # inner stop test's finest-level defect, so a step costs 13% less (28.9
    # against 33.3 ms at 256^3, when it was measured).  Each FP32 inner solve
    # reduces its defect 5e3-fold (two or three outer corrections reach tol
    # 1e-8), and levels of up to 512 cells run in the single-block tail.  One safeguarded Newton step per point update
    # gives the same cycles per step here as two in 8% less time.  Coarsening
    # stops at 8^3: as many cycles as with a 4^3 level below it, 6% less
    # time; one sweep there and an inner target of 2e-4 save another 2%.
    opts = default_opts(kappa_mode=0, kappa=0.0, xi=0.0, precision=1, cycle_gamma=2, gamma_levels=2,
                        nu1=0, nu2=2, coarse_max_sweeps=1, coarsest_max_n=8, inner_rtol=2e-4, tail_cells=512,
                        newton_iters=1)
    opts.update(optkw)
    return dict(name=f"drainage3d_n{n}", dim=3, n=(n, n, n), L=(1.0, 1.0, 1.0),
                soil=soil, bc=bc, sink=no_sink(),
                psi0=np.zeros(n ** 3), psi_prev=None,
                dt=dt, nsteps=nsteps, scheme=2, opts=opts)


# ---------------------------------------------------------------------------
# Batched root-uptake columns (lengths U{64..1024} over 1 m), m and s.
# ---------------------------------------------------------------------------
def columns(ncol=4096, seed=5, dt=600.0, nsteps=144, nmin=64, nmax=1024, **optkw):
    rng = np.random.Generator(np.random.PCG64(seed))
    lengths = rng.integers(nmin, nmax + 1, ncol)
    alpha = rng.uniform(0.5, 5.0, ncol)
    nvg = rng.uniform(1.2, 3.0, ncol)
    Ks = np.exp(rng.uniform(math.log(1e-7), math.log(1e-4), ncol))
    out = []
    for c in range(ncol):
        m = int(lengths[c])
        soil = _soil(VANGENUCHTEN, Ks=Ks[c], theta_s=0.368, theta_r=0.102,
                     p1=alpha[c], p2=nvg[c], p3=0.5)
        bc = _bc([FREE_DRAINAGE, FLUX], [0.0, 0.0])
        # two safeguarded Newton steps per point update (the default): one
        # step is 6% faster on this workload, but columns with a top inflow
        # and a varying initial head then stall in the FP32 inner solve and
        # end non-finite (the step is rejected with psi^n kept)
        opts = default_opts(kappa_mode=0, kappa=0.0, xi=0.0, precision=1)
        opts.update(optkw)
        out.append(dict(name=f"column{c}_n{m}", dim=1, n=(m, 1, 1), L=(1.0, 1.0, 1.0),
                        soil=soil, bc=bc, sink=feddes_sink(),
                        psi0=np.full(m, -1.0), psi_prev=None,
                        dt=dt, nsteps=nsteps, scheme=1, opts=opts))
    return out


# ---------------------------------------------------------------------------
# Serving trace: Poisson arrivals of mixed 2D/3D solves.
# ---------------------------------------------------------------------------
def head_at_saturation(soil, Se):
    """Pressure head (m, < 0) at effective saturation Se of a uniform soil
    (the inverse of theta(psi) of Table 1)."""
    a = soil["p1"]
    if soil["model"] == HAVERKAMP:           # Se = alpha / (alpha + h^beta)
        return -float((a * (1.0 / Se - 1.0)) ** (1.0 / soil["p2"]))
    if soil["model"] == GARDNER:             # Se = exp(alpha psi)
        return float(math.log(Se) / a)
    n = soil["p2"]
    m = 1.0 - 1.0 / n                        # Se = (1 + (alpha h)^n)^-m
    return -float((Se ** (-1.0 / m) - 1.0) ** (1.0 / n) / a)


def serving_trace(rate=200.0, seconds=60.0, seed=6, sizes2d=(129, 257, 513, 1025),
                  sizes3d=(65, 129, 257), max_requests=None):
    rng = np.random.Generator(np.random.PCG64(seed))
    t = 0.0
    reqs = []
    while True:
        t += rng.exponential(1.0 / rate)
        if t > seconds:
            break
        if max_requests is not None and len(reqs) >= max_requests:
            break
        is3d = rng.random() < 0.5
        n = int(rng.choice(sizes3d if is3d else sizes2d))
        model = int(rng.integers(0, 3))
        Ks = float(math.exp(rng.uniform(math.log(1e-7), math.log(1e-4))))
        if model == HAVERKAMP:
            s = rng.uniform(0.8, 1.2)
            # C1 parameters converted from cm to m: A*100^-gamma, alpha*100^-beta
            soil = _soil(HAVERKAMP, Ks, 0.287, 0.075, p1=1.611e6 * 100.0 ** -3.96 * s,
                         p2=3.96, p3=1.175e6 * 100.0 ** -4.74 * s, p4=4.74)
        elif model == GARDNER:
            soil = _soil(GARDNER, Ks, 0.368, 0.102, p1=float(rng.uniform(1.0, 5.0)))
        else:
            soil = _soil(VANGENUCHTEN, Ks, 0.368, 0.102, p1=float(rng.uniform(0.5, 5.0)),
                         p2=float(rng.uniform(1.2, 3.0)), p3=0.5)
        steps = int(rng.integers(20, 201))
        sink = feddes_sink() if rng.random() < 0.5 else no_sink()
        # initial (and lower boundary) head at an effective saturation of
        # 0.1-0.3 of this soil: dry, but not so dry that K(psi*) underflows
        # to 0 where theta' is 0 too (with xi = 0 that system is singular)
        dry = head_at_saturation(soil, float(rng.uniform(0.1, 0.3)))
        wet = head_at_saturation(soil, 0.95)
        if is3d:
            bc = _bc([NOFLUX, NOFLUX, NOFLUX, NOFLUX, FREE_DRAINAGE, DIRICHLET],
                     [0, 0, 0, 0, 0, wet])
            prob = dict(name=f"req{len(reqs)}_3d_n{n}", dim=3, n=(n, n, n), L=(1.0, 1.0, 1.0),
                        psi0=np.full(n ** 3, dry), dt=300.0)
        else:
            bc = _bc([NOFLUX, NOFLUX, DIRICHLET, DIRICHLET], [0, 0, dry, wet])
            h = 1.0 / n
            xc = (np.arange(n) + 0.5) * h
            bc["mask_field"][3] = (np.abs(xc - 0.5) <= 0.1).astype(np.uint8)
            prob = dict(name=f"req{len(reqs)}_2d_n{n}", dim=2, n=(n, n, 1), L=(1.0, 1.0, 1.0),
                        psi0=np.full(n * n, dry), dt=60.0)
        prob.update(soil=soil, bc=bc, sink=sink, psi_prev=None, nsteps=steps, scheme=2,
                    opts=default_opts(precision=1), arrival=t)
        reqs.append(prob)
    return reqs


# ---------------------------------------------------------------------------
# Small random problems for parity tests (odd sizes, every BC kind and model).
# ---------------------------------------------------------------------------
def random_problem(dim, n, model, seed, bc_kinds=None, hetero=False, sink=False,
                   psi_range=(-2.0, -0.05), L=1.0, dt=60.0, scheme=1, **optkw):
    rng = np.random.Generator(np.random.PCG64(seed))
    nn = [1, 1, 1]
    for a in range(dim):
        nn[a] = int(n[a]) if hasattr(n, "__len__") else int(n)
    N = nn[0] * nn[1] * nn[2]
    if model == HAVERKAMP:
        soil = _soil(HAVERKAMP, 1e-5, 0.287, 0.075, p1=1.611e6 * 100.0 ** -3.96,
                     p2=3.96, p3=1.175e6 * 100.0 ** -4.74, p4=4.74)
        if hetero:
            soil["p1_field"] = soil["p1"] * rng.uniform(0.7, 1.3, N)
            soil["p2_field"] = rng.uniform(3.0, 4.5, N)
    elif model == GARDNER:
        soil = _soil(GARDNER, 1e-5, 0.45, 0.15, p1=2.0)
        if hetero:
            soil["p1_field"] = rng.uniform(1.0, 5.0, N)
    else:
        soil = _soil(VANGENUCHTEN, 1e-5, 0.368, 0.102, p1=3.35, p2=2.0, p3=0.5)
        if hetero:
            soil["p1_field"] = rng.uniform(2.0, 5.0, N)
            soil["p2_field"] = rng.uniform(1.5, 2.5, N)
    if hetero:
        soil["Ks_field"] = np.exp(np.log(1e-5) + rng.standard_normal(N))
    if bc_kinds is None:
        bc_kinds = [NOFLUX] * (2 * dim - 2) + [FREE_DRAINAGE, DIRICHLET]
    vals = []
    for k in bc_kinds:
        if k == DIRICHLET:
            vals.append(float(rng.uniform(*psi_range)))
        elif k == FLUX:
            vals.append(float(rng.uniform(0.0, 2e-6)))
        else:
            vals.append(0.0)
    bc = _bc(bc_kinds, vals)
    psi0 = rng.uniform(psi_range[0], psi_range[1], N)
    opts = default_opts(kappa_mode=0, kappa=0.0, xi=0.0)
    opts.update(optkw)
    return dict(name=f"rand{dim}d_m{model}_s{seed}", dim=dim, n=tuple(nn),
                L=(L, L, L), soil=soil, bc=bc,
                sink=feddes_sink(Tp=TP_5MM_PER_DAY * 50) if sink else no_sink(),
                psi0=psi0, psi_prev=None, dt=dt, nsteps=3, scheme=scheme, opts=opts)


def with_opts(prob, **kw):
    p = copy.copy(prob)
    p["opts"] = dict(prob["opts"])
    p["opts"].update(kw)
    return p
