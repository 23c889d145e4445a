"""FP64 CPU oracle for the speed-limited PIC step (Werner et al., arXiv 1511.08225).

TEST INFRASTRUCTURE.  This module and the C file beside it state, slowly and
plainly, what one SLPIC timestep computes.  Only the test suite, the package
smoke check and the benchmark's CPU-baseline leg may import it; the product
library never does.  It imports nothing from the CUDA package.

The heavy per-particle loops are in ``slpic_oracle.c`` (plain C, FP64); this
file loads it with ctypes and strings the steps together in the order of
Appendix A, Eq. (slpicIntegration):

    solve rho^n -> phi^n -> E^n
    for each particle: gather E^n(x^n), v^{n+1/2} = v^{n-1/2} + (q/m) E tau*,
        x^{n+1} = x^n + beta(|v^{n+1/2}|) v^{n+1/2} dt, walls
    inject source particles (first pushed next step)
    rho^{n+1} = sum_p q w beta(|v^{n+1/2}|) S(x - x^{n+1})

Readings of the paper that this file takes (the paper is silent on them):
the loaded velocity is v^{-1/2}; rho^0 is deposited with beta(|v^{-1/2}|);
injected particles are deposited into rho^{n+1} with beta of their initial
velocity and take their first push in the next step.

A speed limit that varies in space (Sec. II) is given as prob["v0_profile"]:
one factor lam_c > 0 per cell, so that a particle in cell c has the limit
v0_s lam_c.  The push of a step takes the factor of the cell the particle starts
in, the deposit that of the cell it is deposited from, the wall source that of
the last cell (the one the entering particles are placed in).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "slpic_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

BETA_ONE, BETA_HEAVISIDE, BETA_RELATIVISTIC = 0, 1, 2
SRC_NONE, SRC_LOSS_MATCHED, SRC_RATE, SRC_WALL = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile the oracle C file into liboracle.so (gcc, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "slpic_oracle.h"))
    ):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
             "-shared", _SRC, "-o", tmp, "-lm"]
        )
        os.replace(tmp, _LIB)
    return _LIB


_lib = None
_D = ctypes.c_double
_P = ctypes.c_void_p
_L = ctypes.c_long
_I = ctypes.c_int


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        L = _lib
        L.orc_beta.restype = _D
        L.orc_beta.argtypes = [_I, _D, _D]
        for name in ("orc_beta_integral", "orc_beta_integral_closed"):
            f = getattr(L, name)
            f.restype = _D
            f.argtypes = [_I, _P, _P, _D, _D]
        L.orc_beta_integral_mmid.restype = _D
        L.orc_beta_integral_mmid.argtypes = [_I, _P, _P, _D, _D, _D, ctypes.POINTER(_L)]
        L.orc_time_closed.restype = _D
        L.orc_time_closed.argtypes = [_I, _P, _P, _D, _D]
        L.orc_rk4_limited.restype = None
        L.orc_rk4_limited.argtypes = [_I, _P, _P, _D, _D, _L, _P]
        L.orc_poisson1d_dirichlet.restype = None
        L.orc_poisson1d_dirichlet.argtypes = [_I, _D, _D, _P, _D, _D, _P]
        L.orc_poisson1d_periodic.restype = None
        L.orc_poisson1d_periodic.argtypes = [_I, _D, _D, _P, _P]
        L.orc_efield1d.restype = None
        L.orc_efield1d.argtypes = [_I, _I, _D, _P, _P]
        L.orc_deposit1d.restype = None
        L.orc_deposit1d.argtypes = [_I, _I, _D, _L, _P, _P, _P, _I, _D, _P, _D, _P]
        L.orc_beta_f32.restype = ctypes.c_float
        L.orc_beta_f32.argtypes = [_I, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                   ctypes.c_float]
        L.orc_deposit_q40.restype = None
        L.orc_deposit_q40.argtypes = [_I, _I, _L, _P, _P, _P, _I, ctypes.c_float, _P, _P]
        L.orc_push1d.restype = None
        L.orc_push1d.argtypes = [_I, _I, _D, _D, _P, _L, _P, _P, _P, _D, _I, _D, _P, _P]
        L.orc_splitmix64_at.restype = ctypes.c_uint64
        L.orc_splitmix64_at.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
        L.orc_stream_key.restype = ctypes.c_uint64
        L.orc_stream_key.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32]
        L.orc_u24.restype = ctypes.c_float
        L.orc_u24.argtypes = [ctypes.c_uint64]
        L.orc_inject.restype = None
        L.orc_inject.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32, _L,
                                 ctypes.c_float, ctypes.c_float, _D, _D, _P, _P]
        L.orc_poisson2d_direct.restype = None
        L.orc_poisson2d_direct.argtypes = [_I, _I, _D, _D, _P, _D, _D, _P]
        L.orc_poisson2d_cg.restype = _I
        L.orc_poisson2d_cg.argtypes = [_I, _I, _D, _D, _P, _D, _D, _D, _I, _P,
                                       ctypes.POINTER(_D)]
        L.orc_efield2d.restype = None
        L.orc_efield2d.argtypes = [_I, _I, _D, _P, _P, _P]
        L.orc_deposit2d.restype = None
        L.orc_deposit2d.argtypes = [_I, _I, _D, _L, _P, _P, _P, _P, _I, _D, _D, _P]
        L.orc_deposit2d_q40.restype = None
        L.orc_deposit2d_q40.argtypes = [_I, _I, _L, _P, _P, _P, _I, ctypes.c_float, _P]
        L.orc_push2d.restype = None
        L.orc_push2d.argtypes = [_I, _I, _D, _D, _P, _P, _L, _P, _P, _P, _P, _D, _I, _D, _P]
        L.orc_inject_wall.restype = None
        L.orc_inject_wall.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32, _L, _I,
                                      _D, _D, _D, _I, _D, _P, _P]
        L.orc_inject2d.restype = None
        L.orc_inject2d.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32, _L,
                                   ctypes.c_float, ctypes.c_float, _I, _D, _D, _P, _P, _P]
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _vec3(x) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(x, dtype=np.float64).reshape(3))


# ---------------------------------------------------------------- scalar pieces
def beta(kind: int, r: float, v0: float) -> float:
    """Sec. II, Eqs. (relativisticBeta) / (heavisideBeta)."""
    return lib().orc_beta(kind, r, v0)


def beta_integral(kind, u, a, dt, v0) -> float:
    """Appendix A, Eq. (slpicIntegrationV): tau* = int beta(|v(t)|) dt."""
    u, a = _vec3(u), _vec3(a)
    return lib().orc_beta_integral(kind, _ptr(u), _ptr(a), dt, v0)


def beta_integral_mmid(kind, u, a, dt, v0, rel_tol=1e-2):
    """The paper's modified-midpoint evaluation (Appendix A); returns (tau*, substeps)."""
    u, a = _vec3(u), _vec3(a)
    n = ctypes.c_long(0)
    t = lib().orc_beta_integral_mmid(kind, _ptr(u), _ptr(a), dt, v0, rel_tol, ctypes.byref(n))
    return t, n.value


def beta_integral_closed(kind, u, a, dt, v0) -> float:
    u, a = _vec3(u), _vec3(a)
    return lib().orc_beta_integral_closed(kind, _ptr(u), _ptr(a), dt, v0)


def time_closed(kind, u, a, v0, tau) -> float:
    u, a = _vec3(u), _vec3(a)
    return lib().orc_time_closed(kind, _ptr(u), _ptr(a), v0, tau)


def rk4_limited(kind, u, a, dt, v0, n_sub=1_000_000) -> np.ndarray:
    """Brute-force RK4 of Eq. (LimPtclDyn): [v(dt), x(dt)-x(0), int beta dt]."""
    u, a = _vec3(u), _vec3(a)
    out = np.zeros(7)
    lib().orc_rk4_limited(kind, _ptr(u), _ptr(a), dt, v0, n_sub, _ptr(out))
    return out


def push_velocity(kind, u, a, dt, v0) -> np.ndarray:
    """v^{n+1/2} = v^{n-1/2} + a tau* (Appendix A)."""
    u, a = _vec3(u), _vec3(a)
    return u + a * beta_integral(kind, u, a, dt, v0)


# ---------------------------------------------------------------- grid pieces
def poisson1d(rho: np.ndarray, dx: float, periodic: bool, phi_lo=0.0, phi_hi=0.0,
              eps0=1.0) -> np.ndarray:
    """Appendix A, Eq. (LimPtclDynAppendixDotE), 1D nodal 3-point stencil."""
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    if periodic:
        n_cells = rho.size
        phi = np.zeros(n_cells)
        lib().orc_poisson1d_periodic(n_cells, dx, eps0, _ptr(rho), _ptr(phi))
    else:
        n_cells = rho.size - 1
        phi = np.zeros(n_cells + 1)
        lib().orc_poisson1d_dirichlet(n_cells, dx, eps0, _ptr(rho), phi_lo, phi_hi,
                                      _ptr(phi))
    return phi


def efield1d(phi: np.ndarray, dx: float, periodic: bool) -> np.ndarray:
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    n_cells = phi.size if periodic else phi.size - 1
    E = np.zeros_like(phi)
    lib().orc_efield1d(n_cells, int(periodic), dx, _ptr(phi), _ptr(E))
    return E


def deposit_q40(n_cells, periodic, cell, offset, v, kind, v0, lam=None) -> np.ndarray:
    """The quantised int64 deposit rule (bit-exact contract, see the C file);
    lam: per-cell FP32 factors of v0, or None."""
    cell = np.ascontiguousarray(cell, dtype=np.int32)
    offset = np.ascontiguousarray(offset, dtype=np.float32)
    v = np.ascontiguousarray(v, dtype=np.float32).reshape(-1, 3)
    nn = n_cells if periodic else n_cells + 1
    acc = np.zeros(nn, dtype=np.int64)
    lam_p = None
    if lam is not None:
        lam = np.ascontiguousarray(lam, dtype=np.float32)
        assert lam.size == n_cells
        lam_p = _ptr(lam)
    lib().orc_deposit_q40(n_cells, int(periodic), cell.size, _ptr(cell), _ptr(offset),
                          _ptr(v), kind, np.float32(v0), lam_p, _ptr(acc))
    return acc


def beta_f32(kind, vx, vy, vz, v0) -> np.float32:
    return np.float32(lib().orc_beta_f32(kind, vx, vy, vz, v0))


def splitmix64_at(key: int, i: int) -> int:
    return lib().orc_splitmix64_at(key, i)


def stream_key(seed: int, step: int, species: int) -> int:
    return lib().orc_stream_key(seed, step, species)


# ---------------------------------------------------------------- 2D grid pieces
# Node (i, j) of an nx x (ny+1) grid is entry [j, i] (periodic in x, plates at j = 0, ny).
def poisson2d_direct(rho: np.ndarray, dx: float, phi_lo=0.0, phi_hi=0.0, eps0=1.0):
    """5-point Poisson (Appendix A, Eq. LimPtclDynAppendixDotE, in 2D) solved
    directly: DFT in x, Thomas per mode in y.  rho, phi: (ny+1, nx)."""
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    ny, nx = rho.shape[0] - 1, rho.shape[1]
    phi = np.zeros_like(rho)
    lib().orc_poisson2d_direct(nx, ny, dx, eps0, _ptr(rho), phi_lo, phi_hi, _ptr(phi))
    return phi


def poisson2d_cg(rho: np.ndarray, dx: float, phi0=None, phi_lo=0.0, phi_hi=0.0, eps0=1.0,
                 rtol=1e-8, maxit=100000):
    """Jacobi-preconditioned CG on the same system from the guess phi0;
    returns (phi, iterations (-1: not converged), relative residual)."""
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    ny, nx = rho.shape[0] - 1, rho.shape[1]
    phi = np.zeros_like(rho) if phi0 is None else np.array(phi0, dtype=np.float64)
    res = ctypes.c_double(0.0)
    it = lib().orc_poisson2d_cg(nx, ny, dx, eps0, _ptr(rho), phi_lo, phi_hi, rtol, maxit,
                                _ptr(phi), ctypes.byref(res))
    return phi, it, res.value


def efield2d(phi: np.ndarray, dx: float):
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    ny, nx = phi.shape[0] - 1, phi.shape[1]
    Ex, Ey = np.zeros_like(phi), np.zeros_like(phi)
    lib().orc_efield2d(nx, ny, dx, _ptr(phi), _ptr(Ex), _ptr(Ey))
    return Ex, Ey


def deposit2d_q40(nx, ny, cell, offset, v, kind, v0) -> np.ndarray:
    """The quantised 2D deposit rule (bit-exact contract, see the C file);
    offset (n, 2) = (dx_, dy_); returns int64 (ny+1, nx)."""
    cell = np.ascontiguousarray(cell, dtype=np.int32)
    offset = np.ascontiguousarray(offset, dtype=np.float32).reshape(-1, 2)
    v = np.ascontiguousarray(v, dtype=np.float32).reshape(-1, 3)
    acc = np.zeros((ny + 1, nx), dtype=np.int64)
    lib().orc_deposit2d_q40(nx, ny, cell.size, _ptr(cell), _ptr(offset), _ptr(v), kind,
                            np.float32(v0), _ptr(acc))
    return acc


# ---------------------------------------------------------------- the simulation
class OracleSim:
    """Plain FP64 SLPIC in 1D3V on one grid (Appendix A; Sec. IV geometry).

    ``prob`` is the plain problem dictionary also understood by the CUDA
    binding (grid, dt, boundary, species, source, seed).
    """

    def __init__(self, prob: dict):
        self.prob = prob
        self.N = int(prob["n_cells"])
        self.dx = float(prob["dx"])
        self.dt = float(prob["dt"])
        self.periodic = bool(prob["periodic"])
        self.eps0 = float(prob.get("eps0", 1.0))
        self.nn = self.N if self.periodic else self.N + 1
        self.sp = prob["species"]
        ns = len(self.sp)
        self.set_profile(prob.get("v0_profile"))
        self.x = [np.zeros(0) for _ in range(ns)]
        self.v = [np.zeros((0, 3)) for _ in range(ns)]
        self.step_index = 0
        self.frac = [0.0] * ns
        self.flux = np.zeros((ns, 2), dtype=np.int64)  # cumulative absorptions
        self.last_absorbed = np.zeros((ns, 2), dtype=np.int64)
        self.last_injected = np.zeros(ns, dtype=np.int64)
        self.dens = np.zeros((ns, self.nn))
        self.rho = np.zeros(self.nn)
        self.phi = np.zeros(self.nn)
        self.E = np.zeros(self.nn)

    def set_profile(self, lam):
        """Per-cell factors of every species' v0 (FP32 numbers, > 0), or None
        for a uniform limit; takes effect from the next push or deposit."""
        if lam is None:
            self.lam = None
            return
        lam = np.asarray(lam, dtype=np.float32).astype(np.float64)
        assert lam.shape == (self.N,) and (lam > 0).all()
        self.lam = np.ascontiguousarray(lam)

    def _lam_ptr(self):
        return None if self.lam is None else _ptr(self.lam)

    def v0_of_cells(self, s: int, cells) -> np.ndarray:
        """The FP64 limit of species s in the given cells."""
        v0 = float(self.sp[s]["v0"])
        cells = np.asarray(cells, dtype=np.int64)
        if self.lam is None:
            return np.full(cells.shape, v0)
        return v0 * self.lam[cells]

    # --- loading -----------------------------------------------------------
    def load(self, s: int, x: np.ndarray, v: np.ndarray):
        self.x[s] = np.concatenate([self.x[s], np.asarray(x, dtype=np.float64)])
        self.v[s] = np.concatenate([self.v[s], np.asarray(v, dtype=np.float64).reshape(-1, 3)])

    def load_cells(self, s: int, cell, offset, v):
        """Take the FP32 (cell, offset, v) state: x = (cell + offset) dx in FP64."""
        x = (np.asarray(cell, dtype=np.float64) + np.asarray(offset, dtype=np.float32)
             .astype(np.float64)) * self.dx
        self.load(s, x, np.asarray(v, dtype=np.float32).astype(np.float64))

    def start(self):
        """Deposit rho^0 (beta of the loaded v^{-1/2}) and solve for E^0."""
        self.deposit()
        self.solve()

    # --- steps of Appendix A -----------------------------------------------
    def deposit(self):
        L = lib()
        self.dens = np.zeros((len(self.sp), self.nn))
        for s, sp in enumerate(self.sp):
            x = np.ascontiguousarray(self.x[s])
            v = np.ascontiguousarray(self.v[s])
            L.orc_deposit1d(self.N, int(self.periodic), self.dx, x.size, _ptr(x), _ptr(v),
                            None, int(sp["kind"]), float(sp["v0"]), self._lam_ptr(),
                            float(sp["w"]), _ptr(self.dens[s]))
        self.rho = sum(float(sp["q"]) * self.dens[s] for s, sp in enumerate(self.sp))

    def solve(self, t=None):
        """Poisson for E^n (Appendix A); with a prescribed wave (Sec. V test
        particles, prob["wave"] = {phi0, k, vphi, ramp}) the field is instead
        -d/dx of phi0(t) sin(k (x - vphi t)), phi0(t) = phi0 min(1, t/ramp), at the
        nodes and at time t (default: the current level, step_index * dt)."""
        p = self.prob
        w = p.get("wave")
        if w is not None and float(w["k"]) > 0.0:
            t = self.step_index * self.dt if t is None else t
            amp = float(w["phi0"])
            if float(w.get("ramp", 0.0)) > 0.0:
                amp *= min(1.0, t / float(w["ramp"]))
            xj = np.arange(self.nn) * self.dx
            ph = float(w["k"]) * (xj - float(w["vphi"]) * t)
            self.phi = amp * np.sin(ph)
            self.E = -amp * float(w["k"]) * np.cos(ph)
            return
        self.phi = poisson1d(self.rho, self.dx, self.periodic, p.get("phi_lo", 0.0),
                             p.get("phi_hi", 0.0), self.eps0)
        self.E = efield1d(self.phi, self.dx, self.periodic)

    def push(self):
        L = lib()
        E = np.ascontiguousarray(self.E)
        for s, sp in enumerate(self.sp):
            n = self.x[s].size
            x = np.ascontiguousarray(self.x[s])
            v = np.ascontiguousarray(self.v[s])
            alive = np.ones(n, dtype=np.uint8)
            flux = np.zeros(2, dtype=np.int64)
            L.orc_push1d(self.N, int(self.periodic), self.dx, self.dt, _ptr(E), n, _ptr(x),
                         _ptr(v), _ptr(alive), float(sp["q"]) / float(sp["m"]),
                         int(sp["kind"]), float(sp["v0"]), self._lam_ptr(), _ptr(flux))
            keep = alive.astype(bool)
            self.x[s] = x[keep]
            self.v[s] = v[keep]
            self.last_absorbed[s] = flux
            self.flux[s] += flux

    def injection_counts(self) -> list[int]:
        """Macroparticles per species this step (source readings of Sec. IV):
        LOSS_MATCHED re-injects the physical count of reference-species
        particles absorbed this step; RATE injects rate*dt physical pairs.
        A physical count S becomes S / w_s macroparticles (g-source = f-source),
        with the fractional part carried to the next step."""
        src = self.prob.get("source", {"mode": SRC_NONE})
        mode = int(src.get("mode", SRC_NONE))
        if mode == SRC_NONE:
            return [0] * len(self.sp)
        if mode == SRC_LOSS_MATCHED:
            ref = int(src["ref_species"])
            S = float(self.last_absorbed[ref].sum()) * float(self.sp[ref]["w"])
        else:
            S = float(src["rate"]) * self.dt
        out = []
        for s, sp in enumerate(self.sp):
            if float(sp.get("T", 0.0)) <= 0.0:
                out.append(0)
                continue
            if mode == SRC_WALL:
                # one-sided flux of a stationary Maxwellian of density `rate`
                vth = np.sqrt(float(sp["T"]) / float(sp["m"]))
                S = float(src["rate"]) * vth / np.sqrt(2.0 * np.pi) * self.dt
            self.frac[s] += S / float(sp["w"])
            k = int(np.floor(self.frac[s]))
            self.frac[s] -= k
            out.append(k)
        return out

    def inject(self):
        src = self.prob.get("source", {"mode": SRC_NONE})
        counts = self.injection_counts()
        L = lib()
        for s, sp in enumerate(self.sp):
            k = counts[s]
            self.last_injected[s] = k
            if k == 0:
                continue
            x = np.zeros(k)
            v = np.zeros((k, 3))
            vth = np.sqrt(float(sp["T"]) / float(sp["m"]))
            if int(src.get("mode", SRC_NONE)) == SRC_WALL:
                L.orc_inject_wall(int(self.prob["seed"]), self.step_index, s, k, self.N,
                                  self.dx, self.dt, vth, int(sp["kind"]),
                                  float(self.v0_of_cells(s, [self.N - 1])[0]), _ptr(x), _ptr(v))
            else:
                L.orc_inject(int(self.prob["seed"]), self.step_index, s, k,
                             np.float32(src["lo_cells"]), np.float32(src["len_cells"]),
                             self.dx, vth, _ptr(x), _ptr(v))
            self.load(s, x, v)

    def step(self, n: int = 1):
        for _ in range(n):
            self.push()
            self.inject()
            self.deposit()
            self.solve((self.step_index + 1) * self.dt)
            self.step_index += 1

    # --- diagnostics ---------------------------------------------------------
    def diagnostics(self) -> dict:
        """Counts, g-weight, physical count (w beta), physical kinetic energy
        sum(1/2 m w beta |v|^2) (f = beta g, Sec. II) and field energy."""
        out = {"count": [], "sum_w": [], "sum_wbeta": [], "kinetic": []}
        for s, sp in enumerate(self.sp):
            v = self.v[s]
            r = np.sqrt((v * v).sum(axis=1))
            cells = np.minimum(np.floor(self.x[s] / self.dx).astype(np.int64), self.N - 1)
            b = _beta_vec(int(sp["kind"]), r, self.v0_of_cells(s, cells))
            w = float(sp["w"])
            out["count"].append(int(v.shape[0]))
            out["sum_w"].append(w * v.shape[0])
            out["sum_wbeta"].append(float(w * b.sum()))
            out["kinetic"].append(float(0.5 * float(sp["m"]) * w * (b * r * r).sum()))
        wts = np.ones(self.nn)
        if not self.periodic:
            wts[0] = wts[-1] = 0.5
        out["field_energy"] = float(0.5 * self.eps0 * self.dx * (wts * self.E ** 2).sum())
        out["flux"] = self.flux.copy()
        out["step"] = self.step_index
        return out


def _beta_vec(kind, r, v0):
    if kind == BETA_ONE:
        return np.ones_like(r)
    if kind == BETA_HEAVISIDE:
        return np.where(r <= v0, 1.0, v0 / np.maximum(r, 1e-300))
    return v0 / np.sqrt(r * r + v0 * v0)


class OracleSim2D:
    """Plain FP64 SLPIC in 2D3V: periodic in x, absorbing plates in y (the 2D
    form of Appendix A with bilinear weighting).  The field is solved directly
    (DFT x Thomas) unless ``cg=True``, which uses the Jacobi-PCG of the C file
    warm-started from the previous potential.

    ``prob``: nx, ny, dx, dt, phi_lo, phi_hi, eps0, seed, species (as in 1D),
    source {mode, lo_cells, len_cells (in y), rate, ref_species}, cg_rtol.
    """

    def __init__(self, prob: dict, cg: bool = False):
        self.prob = prob
        self.nx, self.ny = int(prob["nx"]), int(prob["ny"])
        self.dx, self.dt = float(prob["dx"]), float(prob["dt"])
        self.eps0 = float(prob.get("eps0", 1.0))
        self.cg = cg
        self.sp = prob["species"]
        ns = len(self.sp)
        self.x = [np.zeros(0) for _ in range(ns)]
        self.y = [np.zeros(0) for _ in range(ns)]
        self.v = [np.zeros((0, 3)) for _ in range(ns)]
        self.step_index = 0
        self.frac = [0.0] * ns
        self.flux = np.zeros((ns, 2), dtype=np.int64)
        self.last_absorbed = np.zeros((ns, 2), dtype=np.int64)
        shape = (self.ny + 1, self.nx)
        self.dens = np.zeros((ns,) + shape)
        self.rho = np.zeros(shape)
        self.phi = np.zeros(shape)
        self.Ex = np.zeros(shape)
        self.Ey = np.zeros(shape)
        self.cg_iters = 0

    def load(self, s, x, y, v):
        self.x[s] = np.concatenate([self.x[s], np.asarray(x, dtype=np.float64)])
        self.y[s] = np.concatenate([self.y[s], np.asarray(y, dtype=np.float64)])
        self.v[s] = np.concatenate([self.v[s], np.asarray(v, dtype=np.float64).reshape(-1, 3)])

    def load_cells(self, s, cell, offset, v):
        """FP32 (cell = cy*nx + cx, offset (dx_, dy_), v) -> FP64 positions."""
        cell = np.asarray(cell, dtype=np.int64)
        off = np.asarray(offset, dtype=np.float32).reshape(-1, 2).astype(np.float64)
        x = ((cell % self.nx) + off[:, 0]) * self.dx
        y = ((cell // self.nx) + off[:, 1]) * self.dx
        self.load(s, x, y, np.asarray(v, dtype=np.float32).astype(np.float64))

    def start(self):
        self.deposit()
        self.solve()

    def deposit(self):
        L = lib()
        self.dens = np.zeros((len(self.sp), self.ny + 1, self.nx))
        for s, sp in enumerate(self.sp):
            x, y = np.ascontiguousarray(self.x[s]), np.ascontiguousarray(self.y[s])
            v = np.ascontiguousarray(self.v[s])
            L.orc_deposit2d(self.nx, self.ny, self.dx, x.size, _ptr(x), _ptr(y), _ptr(v), None,
                            int(sp["kind"]), float(sp["v0"]), float(sp["w"]),
                            _ptr(self.dens[s]))
        self.rho = sum(float(sp["q"]) * self.dens[s] for s, sp in enumerate(self.sp))

    def solve(self):
        p = self.prob
        lo, hi = p.get("phi_lo", 0.0), p.get("phi_hi", 0.0)
        if self.cg:
            self.phi, self.cg_iters, _ = poisson2d_cg(
                self.rho, self.dx, self.phi, lo, hi, self.eps0, p.get("cg_rtol", 1e-8))
        else:
            self.phi = poisson2d_direct(self.rho, self.dx, lo, hi, self.eps0)
        self.Ex, self.Ey = efield2d(self.phi, self.dx)

    def push(self):
        L = lib()
        Ex, Ey = np.ascontiguousarray(self.Ex), np.ascontiguousarray(self.Ey)
        for s, sp in enumerate(self.sp):
            n = self.x[s].size
            x, y = np.ascontiguousarray(self.x[s]), np.ascontiguousarray(self.y[s])
            v = np.ascontiguousarray(self.v[s])
            alive = np.ones(n, dtype=np.uint8)
            flux = np.zeros(2, dtype=np.int64)
            L.orc_push2d(self.nx, self.ny, self.dx, self.dt, _ptr(Ex), _ptr(Ey), n, _ptr(x),
                         _ptr(y), _ptr(v), _ptr(alive), float(sp["q"]) / float(sp["m"]),
                         int(sp["kind"]), float(sp["v0"]), _ptr(flux))
            keep = alive.astype(bool)
            self.x[s], self.y[s], self.v[s] = x[keep], y[keep], v[keep]
            self.last_absorbed[s] = flux
            self.flux[s] += flux

    def inject(self):
        src = self.prob.get("source", {"mode": SRC_NONE})
        mode = int(src.get("mode", SRC_NONE))
        if mode == SRC_NONE:
            return
        if mode == SRC_LOSS_MATCHED:
            ref = int(src["ref_species"])
            S = float(self.last_absorbed[ref].sum()) * float(self.sp[ref]["w"])
        else:
            S = float(src["rate"]) * self.dt
        L = lib()
        for s, sp in enumerate(self.sp):
            if float(sp.get("T", 0.0)) <= 0.0:
                continue
            self.frac[s] += S / float(sp["w"])
            k = int(np.floor(self.frac[s]))
            self.frac[s] -= k
            if k == 0:
                continue
            x, y, v = np.zeros(k), np.zeros(k), np.zeros((k, 3))
            vth = np.sqrt(float(sp["T"]) / float(sp["m"]))
            L.orc_inject2d(int(self.prob["seed"]), self.step_index, s, k,
                           np.float32(src["lo_cells"]), np.float32(src["len_cells"]), self.nx,
                           self.dx, vth, _ptr(x), _ptr(y), _ptr(v))
            self.load(s, x, y, v)

    def step(self, n: int = 1):
        for _ in range(n):
            self.push()
            self.inject()
            self.deposit()
            self.solve()
            self.step_index += 1
