"""Thin ctypes binding of the 2D entry points of libslpic.so (include/slpic2d.h).

Argument marshalling only, as in ``binding``: the library does every step of
the 2D method; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import binding
from .binding import SLPIC_MAX_SPECIES, SLPIC_OK, SlpicError, slpic_species

#: every function declared in include/slpic2d.h
EXPORTS2D = (
    "slpic2d_create", "slpic2d_destroy", "slpic2d_last_error", "slpic2d_set_stream",
    "slpic2d_load_particles", "slpic2d_prepare", "slpic2d_step", "slpic2d_synchronize",
    "slpic2d_fields", "slpic2d_charge_raw", "slpic2d_particle_count", "slpic2d_get_particles",
    "slpic2d_diagnostics", "slpic2d_solve_poisson", "slpic2d_enable_kernel_timing",
    "slpic2d_kernel_times", "slpic2d_set_warm_start",
)

SLPIC2D_WARM_PREV, SLPIC2D_WARM_ZERO, SLPIC2D_WARM_UNET, SLPIC2D_WARM_UNET_DELTA = 0, 1, 2, 3


class slpic2d_config(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("dx", ctypes.c_double),
                ("dt", ctypes.c_double), ("phi_lo", ctypes.c_double),
                ("phi_hi", ctypes.c_double), ("eps0", ctypes.c_double),
                ("max_speed", ctypes.c_double), ("seed", ctypes.c_uint64),
                ("n_species", ctypes.c_int32), ("src_mode", ctypes.c_int32),
                ("src_ref_species", ctypes.c_int32), ("cg_maxit", ctypes.c_int32),
                ("src_lo_cells", ctypes.c_double), ("src_len_cells", ctypes.c_double),
                ("src_rate", ctypes.c_double), ("cg_rtol", ctypes.c_double),
                ("species", slpic_species * SLPIC_MAX_SPECIES),
                ("solver", ctypes.c_int32), ("reserved", ctypes.c_int32)]


SLPIC2D_SOLVER_CG, SLPIC2D_SOLVER_FFT = 0, 1


class slpic2d_diag(ctypes.Structure):
    _fields_ = [("step", ctypes.c_int64), ("time", ctypes.c_double),
                ("count", ctypes.c_int64 * SLPIC_MAX_SPECIES),
                ("absorbed", (ctypes.c_int64 * 2) * SLPIC_MAX_SPECIES),
                ("injected", ctypes.c_int64 * SLPIC_MAX_SPECIES),
                ("cg_iterations", ctypes.c_int32), ("iterative_last", ctypes.c_int32),
                ("cg_iterations_total", ctypes.c_int64), ("cg_rel_residual", ctypes.c_double)]


_ready = False


def load_library() -> ctypes.CDLL:
    global _ready
    L = binding.load_library()
    if _ready:
        return L
    P, I, I32, I64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int32, ctypes.c_int64
    sig = {
        "slpic2d_create": (I, [ctypes.POINTER(slpic2d_config), ctypes.POINTER(P)]),
        "slpic2d_destroy": (I, [P]),
        "slpic2d_last_error": (ctypes.c_char_p, [P]),
        "slpic2d_set_stream": (I, [P, P]),
        "slpic2d_load_particles": (I, [P, I, I64, P, P, P]),
        "slpic2d_prepare": (I, [P]),
        "slpic2d_step": (I, [P, I64]),
        "slpic2d_synchronize": (I, [P]),
        "slpic2d_fields": (I, [P, P, P, P, P]),
        "slpic2d_charge_raw": (I, [P, I, P]),
        "slpic2d_particle_count": (I, [P, I, ctypes.POINTER(I64)]),
        "slpic2d_get_particles": (I, [P, I, P, P, P, ctypes.POINTER(I64)]),
        "slpic2d_diagnostics": (I, [P, ctypes.POINTER(slpic2d_diag)]),
        "slpic2d_solve_poisson": (I, [P, P, P, ctypes.POINTER(I32), ctypes.POINTER(ctypes.c_double)]),
        "slpic2d_enable_kernel_timing": (I, [P, I]),
        "slpic2d_set_warm_start": (I, [P, I32, P]),
        "slpic2d_kernel_times": (I, [P, ctypes.POINTER(ctypes.c_double),
                                     ctypes.POINTER(ctypes.c_double),
                                     ctypes.POINTER(ctypes.c_double), ctypes.POINTER(I64)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _ready = True
    return L


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _check(h, rc: int, where: str):
    if rc != SLPIC_OK:
        L = load_library()
        msg = (L.slpic2d_last_error(h) if h else L.slpic_create_error()) or b""
        raise SlpicError(rc, where, msg.decode())


def config_from_problem(prob: dict) -> slpic2d_config:
    """slpic2d_config from the plain 2D problem dictionary of ``inputs``."""
    c = slpic2d_config()
    c.nx, c.ny = int(prob["nx"]), int(prob["ny"])
    c.dx, c.dt = float(prob["dx"]), float(prob["dt"])
    c.phi_lo, c.phi_hi = float(prob.get("phi_lo", 0.0)), float(prob.get("phi_hi", 0.0))
    c.eps0 = float(prob.get("eps0", 1.0))
    c.max_speed = float(prob.get("max_speed", 0.0))
    c.seed = int(prob["seed"])
    c.n_species = len(prob["species"])
    src = prob.get("source", {"mode": 0})
    c.src_mode = int(src.get("mode", 0))
    c.src_ref_species = int(src.get("ref_species", 0))
    c.src_lo_cells = float(src.get("lo_cells", 0.0))
    c.src_len_cells = float(src.get("len_cells", 0.0))
    c.src_rate = float(src.get("rate", 0.0))
    c.cg_rtol = float(prob.get("cg_rtol", 1e-8))
    c.cg_maxit = int(prob.get("cg_maxit", 20000))
    c.solver = {"cg": SLPIC2D_SOLVER_CG, "fft": SLPIC2D_SOLVER_FFT}[prob.get("solver", "cg")]
    for s, sp in enumerate(prob["species"]):
        d = c.species[s]
        d.q, d.m, d.w, d.v0 = float(sp["q"]), float(sp["m"]), float(sp["w"]), float(sp["v0"])
        d.T_src = float(sp.get("T", 0.0))
        d.capacity = int(sp["capacity"])
        d.beta_kind = int(sp["kind"])
    return c


def slpic2d_create(cfg: slpic2d_config):
    h = ctypes.c_void_p()
    _check(None, load_library().slpic2d_create(ctypes.byref(cfg), ctypes.byref(h)),
           "slpic2d_create")
    return h


def slpic2d_destroy(h):
    load_library().slpic2d_destroy(h)


def slpic2d_set_stream(h, stream: int):
    _check(h, load_library().slpic2d_set_stream(h, ctypes.c_void_p(stream)), "slpic2d_set_stream")


def slpic2d_load_particles(h, s: int, cell, offset, v):
    cell = np.ascontiguousarray(cell, dtype=np.int32)
    offset = np.ascontiguousarray(offset, dtype=np.float32).reshape(-1, 2)
    v = np.ascontiguousarray(v, dtype=np.float32).reshape(-1, 3)
    _check(h, load_library().slpic2d_load_particles(h, s, cell.size, _ptr(cell), _ptr(offset),
                                                    _ptr(v)), "slpic2d_load_particles")


def slpic2d_prepare(h):
    _check(h, load_library().slpic2d_prepare(h), "slpic2d_prepare")


def slpic2d_step(h, n: int):
    _check(h, load_library().slpic2d_step(h, n), "slpic2d_step")


def slpic2d_synchronize(h):
    _check(h, load_library().slpic2d_synchronize(h), "slpic2d_synchronize")


def slpic2d_fields(h, nx: int, ny: int):
    shape = (ny + 1, nx)
    rho, phi = np.zeros(shape), np.zeros(shape)
    Ex, Ey = np.zeros(shape, np.float32), np.zeros(shape, np.float32)
    _check(h, load_library().slpic2d_fields(h, _ptr(rho), _ptr(phi), _ptr(Ex), _ptr(Ey)),
           "slpic2d_fields")
    return rho, phi, Ex, Ey


def slpic2d_charge_raw(h, s: int, nx: int, ny: int) -> np.ndarray:
    acc = np.zeros((ny + 1, nx), dtype=np.int64)
    _check(h, load_library().slpic2d_charge_raw(h, s, _ptr(acc)), "slpic2d_charge_raw")
    return acc


def slpic2d_particle_count(h, s: int) -> int:
    n = ctypes.c_int64(0)
    _check(h, load_library().slpic2d_particle_count(h, s, ctypes.byref(n)),
           "slpic2d_particle_count")
    return n.value


def slpic2d_get_particles(h, s: int):
    n = slpic2d_particle_count(h, s)
    cell = np.zeros(max(n, 1), np.int32)
    off = np.zeros((max(n, 1), 2), np.float32)
    v = np.zeros((max(n, 1), 3), np.float32)
    cap = ctypes.c_int64(max(n, 1))
    _check(h, load_library().slpic2d_get_particles(h, s, _ptr(cell), _ptr(off), _ptr(v),
                                                   ctypes.byref(cap)), "slpic2d_get_particles")
    k = cap.value
    return cell[:k], off[:k], v[:k]


def slpic2d_diagnostics(h) -> dict:
    d = slpic2d_diag()
    _check(h, load_library().slpic2d_diagnostics(h, ctypes.byref(d)), "slpic2d_diagnostics")
    return {"step": d.step, "time": d.time, "count": list(d.count),
            "absorbed": [list(a) for a in d.absorbed], "injected": list(d.injected),
            "cg_iterations": d.cg_iterations, "iterative_last": d.iterative_last,
            "cg_iterations_total": d.cg_iterations_total,
            "cg_rel_residual": d.cg_rel_residual}


def slpic2d_solve_poisson(h, rho: np.ndarray, phi0: np.ndarray | None = None):
    """Standalone CG solve of the configured 2D system; returns (phi, iterations,
    relative residual)."""
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    phi = np.zeros_like(rho) if phi0 is None else np.array(phi0, dtype=np.float64)
    it = ctypes.c_int32(0)
    res = ctypes.c_double(0.0)
    _check(h, load_library().slpic2d_solve_poisson(h, _ptr(rho), _ptr(phi), ctypes.byref(it),
                                                   ctypes.byref(res)), "slpic2d_solve_poisson")
    return phi, it.value, res.value


def slpic2d_set_warm_start(h, mode: int, net=None):
    """net: a binding_unet.UNet (or its raw handle) for SLPIC2D_WARM_UNET."""
    nh = getattr(net, "h", net)
    _check(h, load_library().slpic2d_set_warm_start(h, mode, nh), "slpic2d_set_warm_start")


def slpic2d_enable_kernel_timing(h, on: bool = True):
    _check(h, load_library().slpic2d_enable_kernel_timing(h, int(on)),
           "slpic2d_enable_kernel_timing")


def slpic2d_kernel_times(h):
    """(particle_ms, inject_ms, field_ms, steps): mean per-step kernel times."""
    a, b, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    n = ctypes.c_int64()
    _check(h, load_library().slpic2d_kernel_times(h, ctypes.byref(a), ctypes.byref(b),
                                                  ctypes.byref(c), ctypes.byref(n)),
           "slpic2d_kernel_times")
    return a.value, b.value, c.value, n.value


class Simulation2D:
    """Owning wrapper around one slpic2d handle."""

    def __init__(self, prob: dict):
        self.prob = prob
        self.nx, self.ny = int(prob["nx"]), int(prob["ny"])
        self.cfg = config_from_problem(prob)
        self.h = slpic2d_create(self.cfg)

    def close(self):
        if self.h:
            slpic2d_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def load(self, s, cell, offset, v):
        slpic2d_load_particles(self.h, s, cell, offset, v)

    def load_state(self, state):
        for s, (cell, off, v) in enumerate(state):
            self.load(s, cell, off, v)

    def prepare(self):
        slpic2d_prepare(self.h)

    def step(self, n: int = 1):
        slpic2d_step(self.h, n)

    def synchronize(self):
        slpic2d_synchronize(self.h)

    def set_warm_start(self, mode: int, net=None):
        slpic2d_set_warm_start(self.h, mode, net)

    def fields(self):
        return slpic2d_fields(self.h, self.nx, self.ny)

    def charge_raw(self, s: int):
        return slpic2d_charge_raw(self.h, s, self.nx, self.ny)

    def particles(self, s: int):
        return slpic2d_get_particles(self.h, s)

    def diagnostics(self):
        return slpic2d_diagnostics(self.h)

    def solve_poisson(self, rho, phi0=None):
        return slpic2d_solve_poisson(self.h, rho, phi0)
