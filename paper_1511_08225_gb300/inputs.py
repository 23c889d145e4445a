"""Seeded synthetic inputs for the speed-limited PIC path.

This module builds problem descriptions and draws initial particle states.
It holds none of the timestep's arithmetic (no push, deposit or field solve),
so both the CUDA library's tests and the FP64 oracle can take their inputs
from it.  Everything is drawn from ``numpy.random.Generator(PCG64(seed))``.

Normalised units throughout: electron plasma frequency, electron Debye length,
electron thermal speed, eps0, e and m_e are all 1, so the reference density
n0 is 1 and an electron with temperature T_e = 1 has thermal speed 1.

Problem dictionaries (the plain description both implementations accept):

    n_cells, dx, dt, periodic, phi_lo, phi_hi, eps0, seed,
    species: [{name, q, m, w, v0, kind, T, capacity}],
    source:  {mode, lo_cells, len_cells, rate, ref_species}

``kind`` is 0 = beta == 1 (plain PIC), 1 = Heaviside, 2 = "relativistic"
(Sec. II of the paper).  ``T`` is the temperature of the physical source
Maxwellian (0 = the species is not injected).  ``w`` is the g-weight of one
macroparticle (real particles per macroparticle per unit area).
"""
from __future__ import annotations

import math

import numpy as np
from scipy import integrate

BETA_ONE, BETA_HEAVISIDE, BETA_RELATIVISTIC = 0, 1, 2
SRC_NONE, SRC_LOSS_MATCHED, SRC_RATE, SRC_WALL = 0, 1, 2, 3

SEED = 20151126


def make_rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


# ------------------------------------------------------------------ g loading
def _g_factor(kind: int, r: np.ndarray, v0: float) -> np.ndarray:
    """Density ratio g0/f0 of a speed-limited load, i.e. how much more often a
    macroparticle of speed r must be drawn than a physical particle (Sec. II:
    f = beta g).  Bounded by 1 + r/v0 for all three kinds."""
    r = np.asarray(r, dtype=np.float64)
    if kind == BETA_ONE:
        return np.ones_like(r)
    if kind == BETA_HEAVISIDE:
        return np.maximum(1.0, r / v0)
    return np.sqrt(r * r + v0 * v0) / v0


def mean_g_factor(kind: int, vth: float, v0: float, vdim: int = 3) -> float:
    """<g0/f0> over a Maxwellian of thermal speed vth (vdim = 1 or 3)."""
    if kind == BETA_ONE:
        return 1.0
    if vdim == 3:
        def dens(r):
            return 4.0 * math.pi * r * r * (2 * math.pi * vth * vth) ** -1.5 * math.exp(
                -r * r / (2 * vth * vth))
    else:
        def dens(r):
            return 2.0 * (2 * math.pi * vth * vth) ** -0.5 * math.exp(-r * r / (2 * vth * vth))
    top = 40.0 * vth
    pts = [v0] if v0 < top else None
    val, _ = integrate.quad(lambda r: dens(r) * float(_g_factor(kind, np.array(r), v0)),
                            0.0, top, points=pts, limit=400, epsabs=0, epsrel=1e-12)
    return val


def _isotropic(rng, n):
    z = rng.uniform(-1.0, 1.0, n)
    ph = rng.uniform(0.0, 2 * math.pi, n)
    s = np.sqrt(1.0 - z * z)
    return np.stack([s * np.cos(ph), s * np.sin(ph), z], axis=1)


def g_velocities(rng, n: int, vth: float, v0: float, kind: int, vdim: int = 3) -> np.ndarray:
    """Draw n velocities from g0 = f0 * (g0/f0), f0 a Maxwellian (vth per
    component), by rejection from the envelope f0 * (1 + r/v0): a mixture of
    the Maxwellian itself (mass 1) and the Maxwellian weighted by r/v0 (speed
    drawn from r^2/(2 vth^2) ~ Gamma(2) in 3V, ~ Exp(1) in 1V).  Returns
    (n, 3) float64; in 1V only the x component is non-zero."""
    out = np.zeros((n, 3))
    if kind == BETA_ONE:
        if vdim == 3:
            out[:] = rng.normal(0.0, vth, (n, 3))
        else:
            out[:, 0] = rng.normal(0.0, vth, n)
        return out
    mean_r = vth * (2.0 * math.sqrt(2.0 / math.pi) if vdim == 3 else math.sqrt(2.0 / math.pi))
    p_weighted = (mean_r / v0) / (1.0 + mean_r / v0)
    filled = 0
    while filled < n:
        m = max(1024, int(1.3 * (n - filled)))
        pick_w = rng.random(m) < p_weighted
        r = np.empty(m)
        if vdim == 3:
            r[~pick_w] = np.sqrt((rng.normal(0.0, vth, (int((~pick_w).sum()), 3)) ** 2).sum(1))
            r[pick_w] = vth * np.sqrt(2.0 * rng.gamma(2.0, 1.0, int(pick_w.sum())))
        else:
            r[~pick_w] = np.abs(rng.normal(0.0, vth, int((~pick_w).sum())))
            r[pick_w] = vth * np.sqrt(2.0 * rng.exponential(1.0, int(pick_w.sum())))
        acc = rng.random(m) * (1.0 + r / v0) <= _g_factor(kind, r, v0)
        r = r[acc][: n - filled]
        k = r.size
        if vdim == 3:
            out[filled:filled + k] = r[:, None] * _isotropic(rng, k)
        else:
            out[filled:filled + k, 0] = r * np.where(rng.random(k) < 0.5, -1.0, 1.0)
        filled += k
    return out


def uniform_cells(rng, n: int, n_cells: int, lo: float = 0.0, hi: float | None = None):
    """Positions uniform in [lo, hi) cells, as (int32 cell, float32 offset in [0,1))."""
    hi = float(n_cells) if hi is None else hi
    xc = rng.uniform(lo, hi, n)
    cell = np.floor(xc).astype(np.int64)
    off = (xc - cell).astype(np.float32)
    # float32 rounding can turn 0.99999997 into 1.0: move such points into the next cell
    bump = off >= np.float32(1.0)
    off[bump] = 0.0
    cell[bump] += 1
    cell = np.minimum(cell, n_cells - 1)
    return cell.astype(np.int32), off


# ------------------------------------------------------------------ problems
def species(name, q, m, T, v0, kind, n0=1.0, ppc=100, dx=0.5, vdim=3, capacity=None,
            n_load=None, inject_T=None):
    vth = math.sqrt(T / m)
    w = n0 * dx * mean_g_factor(kind, vth, v0, vdim) / ppc
    return {"name": name, "q": float(q), "m": float(m), "w": float(w), "v0": float(v0),
            "kind": int(kind), "T": float(T if inject_T is None else inject_T),
            "T_load": float(T), "vth": vth, "ppc": int(ppc), "vdim": int(vdim),
            "capacity": int(capacity) if capacity is not None else None}


def periodic_problem(n_cells=256, dx=0.5, dt=0.2, ppc=100, mass_ratio=100.0, T_e=1.0,
                     T_i=1.0, v0=0.2, kind=BETA_HEAVISIDE, seed=SEED, vdim=3):
    """1D periodic electron-ion plasma (the 256-cell, 51,200-particle case when
    called with defaults).  Velocities Maxwellian (g-loaded), positions uniform."""
    sp = [species("e", -1.0, 1.0, T_e, v0, kind, ppc=ppc, dx=dx, vdim=vdim),
          species("i", 1.0, mass_ratio, T_i, v0, kind, ppc=ppc, dx=dx, vdim=vdim)]
    for s in sp:
        s["T"] = 0.0  # no source on a periodic grid
        s["capacity"] = int(ppc * n_cells * 1.0) + 64
    return {"n_cells": int(n_cells), "dx": float(dx), "dt": float(dt), "periodic": True,
            "phi_lo": 0.0, "phi_hi": 0.0, "eps0": 1.0, "seed": int(seed), "species": sp,
            "source": {"mode": SRC_NONE, "lo_cells": 0.0, "len_cells": 0.0, "rate": 0.0,
                       "ref_species": 1}}


def sheath_problem(n_cells=4096, dx=0.5, v0=0.05, ppc=1000, mass_ratio=73440.0, T_e=1.0,
                   T_i=0.1, kind=BETA_HEAVISIDE, dt=None, seed=SEED, capacity_factor=1.5,
                   source_mode=SRC_LOSS_MATCHED, rate=0.0):
    """1D bounded argon-like sheath: absorbing walls at phi = 0, electrons and
    ions loaded uniformly, a central source band (45%..55% of the domain)
    re-injecting physical Maxwellian pairs.  dt defaults to dx / v0."""
    dt = dx / v0 if dt is None else dt
    sp = [species("e", -1.0, 1.0, T_e, v0, kind, ppc=ppc, dx=dx),
          species("i", 1.0, mass_ratio, T_i, v0, kind, ppc=ppc, dx=dx)]
    for s in sp:
        s["capacity"] = int(capacity_factor * ppc * n_cells) + 1024
    return {"n_cells": int(n_cells), "dx": float(dx), "dt": float(dt), "periodic": False,
            "phi_lo": 0.0, "phi_hi": 0.0, "eps0": 1.0, "seed": int(seed), "species": sp,
            "source": {"mode": int(source_mode), "lo_cells": 0.45 * n_cells,
                       "len_cells": 0.10 * n_cells, "rate": float(rate), "ref_species": 1}}


ARGON_MASS_RATIO = 39.9 * 1836.0


def paper_sheath_problem(kind=BETA_HEAVISIDE, n_cells=100, dx=0.25, v0=0.016, dt=None,
                         delta_phi=12.5 / 2.2, T_i=0.5 / 2.2, ppc=1000, seed=SEED,
                         capacity_factor=3.0):
    """The collisionless argon sheath of Sec. IV in normalised units: T_e = 1 and
    the density of the source plasma is 1, so lengths are in its Debye length
    (0.16 cm in the paper).  100 cells of dx = 0.25 (L = 25, the paper's 4 cm),
    plates at phi(0) = -12.5 V / 2.2 eV and phi(L) = 0, electrons and argon ions
    (m_i/m_e = 39.9 x 1836, T_i = 0.5/2.2) entering through the right plate from a
    stationary plasma (SRC_WALL), from an empty box.  kind BETA_ONE is plain PIC
    with dt = dx / (5 v_te); the speed-limited run uses v0 = 0.016 v_te and
    dt = dx / v0 (312.5 PIC steps).  The weights give ~ppc macroparticles per cell
    at density 1 (w = dx <1/beta> / ppc, as for a load)."""
    if dt is None:
        dt = dx / 5.0 if kind == BETA_ONE else dx / v0
    sp = [species("e", -1.0, 1.0, 1.0, v0, kind, ppc=ppc, dx=dx),
          species("i", 1.0, ARGON_MASS_RATIO, T_i, v0, kind, ppc=ppc, dx=dx)]
    for s in sp:
        s["capacity"] = int(capacity_factor * ppc * n_cells) + 4096
    return {"n_cells": int(n_cells), "dx": float(dx), "dt": float(dt), "periodic": False,
            "phi_lo": -float(delta_phi), "phi_hi": 0.0, "eps0": 1.0, "seed": int(seed),
            "species": sp,
            "source": {"mode": SRC_WALL, "lo_cells": 0.0, "len_cells": 0.0, "rate": 1.0,
                       "ref_species": 1}}


def empty_state(prob: dict):
    """No particles (the sheath fills from its source)."""
    return [(np.zeros(0, np.int32), np.zeros(0, np.float32), np.zeros((0, 3), np.float32))
            for _ in prob["species"]]


def load_state(prob: dict, seed: int | None = None, quiet: bool = False):
    """Initial FP32 particle state for every species: a list of
    (cell int32[n], offset float32[n], v float32[n,3]) with ppc * n_cells
    particles per species, velocities drawn from the speed-limited load g0.

    quiet=False: positions uniform over the grid (independent draws).
    quiet=True: every cell holds the same ppc velocities at offsets (k+1/2)/ppc,
    and each species' weight w is reset so that sum(w beta) over a cell is
    exactly n0 dx: the load is neutral cell by cell, with no noise field."""
    rng = make_rng(prob["seed"] if seed is None else seed)
    if quiet:
        out = []
        N = int(prob["n_cells"])
        for sp in prob["species"]:
            ppc = int(sp["ppc"])
            v = g_velocities(rng, ppc, sp["vth"], sp["v0"], sp["kind"], sp.get("vdim", 3))
            r = np.sqrt((v * v).sum(1))
            sp["w"] = float(prob["dx"] / (1.0 / _g_factor(sp["kind"], r, sp["v0"])).sum())
            cell = np.repeat(np.arange(N, dtype=np.int32), ppc)
            off = np.tile(((np.arange(ppc) + 0.5) / ppc).astype(np.float32), N)
            out.append((cell, off, np.tile(v.astype(np.float32), (N, 1))))
        return out
    out = []
    for sp in prob["species"]:
        n = int(sp["ppc"]) * int(prob["n_cells"])
        cell, off = uniform_cells(rng, n, int(prob["n_cells"]))
        v = g_velocities(rng, n, sp["vth"], sp["v0"], sp["kind"], sp.get("vdim", 3))
        out.append((cell, off, v.astype(np.float32)))
    return out


def quiet_symmetric_state(prob: dict, seed: int | None = None):
    """A quiet start whose velocity set is symmetric: every cell holds the same ppc
    velocities, ppc/2 draws of g0 and their negatives side by side, at offsets
    (k+1/2)/ppc, and each species' weight w is reset so that sum(w beta) over a cell
    is exactly n0 dx.  The load is neutral cell by cell and carries no net flux or
    net d(beta)/dv, so nothing but the walls and the source disturbs it."""
    rng = make_rng(prob["seed"] if seed is None else seed)
    out = []
    N = int(prob["n_cells"])
    for sp in prob["species"]:
        ppc = int(sp["ppc"])
        h = g_velocities(rng, ppc // 2, sp["vth"], sp["v0"], sp["kind"], sp.get("vdim", 3))
        v = np.empty((2 * (ppc // 2), 3), dtype=np.float32)
        v[0::2] = h
        v[1::2] = -v[0::2]
        v64 = v.astype(np.float64)  # the weight is set from the stored FP32 velocities
        r = np.sqrt((v64 * v64).sum(1))
        sp["w"] = float(prob["dx"] / (1.0 / _g_factor(sp["kind"], r, sp["v0"])).sum())
        n = v.shape[0]
        cell = np.repeat(np.arange(N, dtype=np.int32), n)
        off = np.tile(((np.arange(n) + 0.5) / n).astype(np.float32), N)
        out.append((cell, off, np.tile(v, (N, 1))))
    return out


def random_state(rng, n: int, n_cells: int, vscale: float = 1.0):
    """Generic FP32 state for parity cases: uniform cells, Gaussian velocities."""
    cell, off = uniform_cells(rng, n, n_cells)
    v = rng.normal(0.0, vscale, (n, 3)).astype(np.float32)
    return cell, off, v


# ------------------------------------------------------------------ 2D problems
def plasma2d_problem(nx=1024, ny=1024, dx=1.0, v0=0.1, ppc=64, mass_ratio=1836.0, T_e=1.0,
                     T_i=0.1, kind=BETA_HEAVISIDE, dt=None, seed=SEED, capacity_factor=1.25,
                     source_mode=SRC_LOSS_MATCHED, rate=0.0, cg_rtol=1e-8, cg_maxit=20000,
                     solver="cg"):
    """2D3V electron-ion plasma between two absorbing plates at phi = 0 (y = 0 and
    y = ny dx), periodic in x, loaded uniformly (ppc per species per cell), with a
    central source band (45%..55% of y) re-injecting physical Maxwellian pairs.
    dt defaults to dx / v0.  Weights are per unit length in z: w = n0 dx^2 <1/beta> / ppc.
    solver: "cg" (Jacobi-PCG, warm-started) or "fft" (direct, nx a power of two)."""
    dt = dx / v0 if dt is None else dt
    sp = []
    for name, q, m, T in (("e", -1.0, 1.0, T_e), ("i", 1.0, mass_ratio, T_i)):
        s = species(name, q, m, T, v0, kind, ppc=ppc, dx=dx)
        s["w"] *= dx  # area weighting: n0 dx^2 <1/beta> / ppc
        s["capacity"] = int(capacity_factor * ppc * nx * ny) + 4096
        sp.append(s)
    return {"ndim": 2, "nx": int(nx), "ny": int(ny), "dx": float(dx), "dt": float(dt),
            "phi_lo": 0.0, "phi_hi": 0.0, "eps0": 1.0, "seed": int(seed), "species": sp,
            "source": {"mode": int(source_mode), "lo_cells": 0.45 * ny, "len_cells": 0.10 * ny,
                       "rate": float(rate), "ref_species": 1},
            "cg_rtol": float(cg_rtol), "cg_maxit": int(cg_maxit), "solver": solver}


def load_state2d(prob: dict, seed: int | None = None):
    """Initial FP32 2D state per species: (cell int32 = cy*nx + cx, offset float32
    (n, 2), v float32 (n, 3)), ppc * nx * ny particles per species, positions
    uniform over the domain, velocities from the speed-limited load g0."""
    rng = make_rng(prob["seed"] if seed is None else seed)
    nx, ny = int(prob["nx"]), int(prob["ny"])
    out = []
    for sp in prob["species"]:
        n = int(sp["ppc"]) * nx * ny
        cx, ox = uniform_cells(rng, n, nx)
        cy, oy = uniform_cells(rng, n, ny)
        v = g_velocities(rng, n, sp["vth"], sp["v0"], sp["kind"], 3)
        cell = (cy.astype(np.int64) * nx + cx).astype(np.int32)
        out.append((cell, np.stack([ox, oy], axis=1).astype(np.float32), v.astype(np.float32)))
    return out


# ------------------------------------------------------------------ batches
def batch_problems(m=256, seed=SEED, cells=(512, 8192), ppc=(100, 1000),
                   mass_ratios=(1836.0, 73440.0), v0=(0.01, 0.5), dx=0.5, T_e=1.0, T_i=0.1):
    """m independent sheaths of uneven size: cells ~ U{lo..hi}, ppc ~ U{lo..hi},
    m_i/m_e drawn from mass_ratios with equal probability, v0 log-uniform in
    [v0_lo, v0_hi] (in v_te), dt = dx / v0, T_e/T_i = 10 (instance i is seeded
    seed + i)."""
    rng = make_rng(seed)
    out = []
    for i in range(m):
        n = int(rng.integers(cells[0], cells[1] + 1))
        pc = int(rng.integers(ppc[0], ppc[1] + 1))
        mr = float(mass_ratios[int(rng.integers(0, len(mass_ratios)))])
        vv = float(math.exp(rng.uniform(math.log(v0[0]), math.log(v0[1]))))
        out.append(sheath_problem(n_cells=n, dx=dx, v0=vv, ppc=pc, mass_ratio=mr, T_e=T_e,
                                  T_i=T_i, seed=seed + i))
    return out


# ------------------------------------------------------------------ wave-particle test (Sec. V)
def wave_problem(kind=BETA_HEAVISIDE, v0=2.0, n_cells=200, dx=0.5, ppc=1000, dt=None,
                 phi0=0.1, vphi=1.0, ramp_periods=20.0, seed=SEED):
    """Test electrons (1D1V: vy = vz = 0, T_e = 1) in a periodic box of one
    wavelength, L = n_cells dx, driven by the prescribed wave
    phi = phi0(t) sin(k (x - vphi t)), k = 2 pi / L, ramped up over ramp_periods
    wave periods (e phi0 / T_e = 0.1 and vphi = v_te as in Sec. V).  dt = dx / v0
    for the speed-limited runs, dx / 4 for plain PIC (kind BETA_ONE)."""
    if dt is None:
        dt = dx / 4.0 if kind == BETA_ONE else dx / v0
    s = species("e", -1.0, 1.0, 1.0, v0, kind, ppc=ppc, dx=dx, vdim=1)
    s["T"] = 0.0
    s["capacity"] = int(ppc * n_cells) + 64
    L = n_cells * dx
    return {"n_cells": int(n_cells), "dx": float(dx), "dt": float(dt), "periodic": True,
            "phi_lo": 0.0, "phi_hi": 0.0, "eps0": 1.0, "seed": int(seed), "species": [s],
            "source": {"mode": SRC_NONE, "lo_cells": 0.0, "len_cells": 0.0, "rate": 0.0,
                       "ref_species": 0},
            "wave": {"phi0": float(phi0), "k": 2.0 * math.pi / L, "vphi": float(vphi),
                     "ramp": float(ramp_periods) * L / float(vphi)}}
