"""Thin ctypes binding of libslpic.so (include/slpic.h), same entry-point names.

Argument marshalling only: every step of the simulation runs in the CUDA
library.  Loading fails loudly if the library is missing; there is no CPU
fallback.  Host arrays are numpy arrays; the ``*_dev`` entry points take
torch CUDA tensors (or raw device pointers).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libslpic.so")

SLPIC_OK = 0
SLPIC_ERR_INVALID = -1
SLPIC_ERR_CFL = -2
SLPIC_ERR_OOM = -3
SLPIC_ERR_CAPACITY = -4
SLPIC_ERR_NOCONVERGE = -5
SLPIC_ERR_TIMEOUT = -6
SLPIC_ERR_CUDA = -7
ERR_NAMES = {0: "OK", -1: "INVALID", -2: "CFL", -3: "OOM", -4: "CAPACITY",
             -5: "NOCONVERGE", -6: "TIMEOUT", -7: "CUDA"}

SLPIC_BETA_ONE, SLPIC_BETA_HEAVISIDE, SLPIC_BETA_RELATIVISTIC = 0, 1, 2
SLPIC_BC_DIRICHLET_ABSORB, SLPIC_BC_PERIODIC = 0, 1
SLPIC_SRC_NONE, SLPIC_SRC_LOSS_MATCHED, SLPIC_SRC_RATE, SLPIC_SRC_WALL = 0, 1, 2, 3
SLPIC_MAX_SPECIES = 4

#: every function declared in include/slpic.h
EXPORTS = (
    "slpic_create", "slpic_destroy", "slpic_last_error", "slpic_create_error",
    "slpic_set_stream", "slpic_load_particles", "slpic_load_particles_dev",
    "slpic_load_particles_f64", "slpic_prepare", "slpic_step", "slpic_synchronize",
    "slpic_fields", "slpic_density", "slpic_charge_raw", "slpic_particle_count",
    "slpic_get_particles", "slpic_diagnostics", "slpic_save", "slpic_restore",
    "slpic_enable_kernel_timing", "slpic_kernel_times", "slpic_kernel_spans",
    "slpic_set_wait_limit",
    "slpic_kernels_per_step",
    "slpic_particle_step_noalloc", "slpic_create_batch", "slpic_set_speed_limit",
    "slpic_set_timestep", "slpic_set_wave", "slpic_get_tuning", "slpic_set_tuning",
    "slpic_autotune", "slpic_fields_async", "slpic_set_speed_limit_profile",
)


class slpic_species(ctypes.Structure):
    _fields_ = [("q", ctypes.c_double), ("m", ctypes.c_double), ("w", ctypes.c_double),
                ("v0", ctypes.c_double), ("T_src", ctypes.c_double),
                ("capacity", ctypes.c_int64), ("beta_kind", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class slpic_config(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int32), ("n_cells", ctypes.c_int32),
                ("dx", ctypes.c_double), ("dt", ctypes.c_double),
                ("bc", ctypes.c_int32), ("n_species", ctypes.c_int32),
                ("phi_lo", ctypes.c_double), ("phi_hi", ctypes.c_double),
                ("eps0", ctypes.c_double), ("max_speed", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("src_mode", ctypes.c_int32),
                ("src_ref_species", ctypes.c_int32), ("src_lo_cells", ctypes.c_double),
                ("src_len_cells", ctypes.c_double), ("src_rate", ctypes.c_double),
                ("species", slpic_species * SLPIC_MAX_SPECIES)]


class slpic_diag(ctypes.Structure):
    _fields_ = [("step", ctypes.c_int64), ("time", ctypes.c_double),
                ("count", ctypes.c_int64 * SLPIC_MAX_SPECIES),
                ("sum_w", ctypes.c_double * SLPIC_MAX_SPECIES),
                ("sum_wbeta", ctypes.c_double * SLPIC_MAX_SPECIES),
                ("kinetic", ctypes.c_double * SLPIC_MAX_SPECIES),
                ("field_energy", ctypes.c_double),
                ("absorbed", (ctypes.c_int64 * 2) * SLPIC_MAX_SPECIES),
                ("injected", ctypes.c_int64 * SLPIC_MAX_SPECIES),
                ("iterative", ctypes.c_int64 * SLPIC_MAX_SPECIES)]


class slpic_tuning(ctypes.Structure):
    _fields_ = [("compact_every", ctypes.c_int32), ("particle_kernel", ctypes.c_int32),
                ("batch_waves", ctypes.c_int32), ("batch_min_share", ctypes.c_int32)]


class SlpicError(RuntimeError):
    def __init__(self, code: int, where: str, msg: str):
        super().__init__(f"{where}: SLPIC_ERR_{ERR_NAMES.get(code, code)} ({code}): {msg}")
        self.code = code


_lib = None


def load_library(path: str | None = None) -> ctypes.CDLL:
    """Load libslpic.so (built by ``build()``); raise if it is not there."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(
            f"{path} not found: build the CUDA library first "
            "(python -m paper_1511_08225_gb300.build); there is no CPU fallback")
    L = ctypes.CDLL(path)
    P, I, I64, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
    sig = {
        "slpic_create": (I, [ctypes.POINTER(slpic_config), ctypes.POINTER(P)]),
        "slpic_create_batch": (I, [ctypes.POINTER(slpic_config), I, ctypes.POINTER(P)]),
        "slpic_set_speed_limit": (I, [P, I, I, D]),
        "slpic_set_speed_limit_profile": (I, [P, P, I]),
        "slpic_set_timestep": (I, [P, D]),
        "slpic_set_wave": (I, [P, D, D, D, D]),
        "slpic_get_tuning": (I, [P, ctypes.POINTER(slpic_tuning)]),
        "slpic_set_tuning": (I, [P, ctypes.POINTER(slpic_tuning)]),
        "slpic_autotune": (I, [P, ctypes.c_int32, ctypes.POINTER(slpic_tuning),
                               ctypes.POINTER(D)]),
        "slpic_destroy": (I, [P]),
        "slpic_last_error": (ctypes.c_char_p, [P]),
        "slpic_create_error": (ctypes.c_char_p, []),
        "slpic_set_stream": (I, [P, P]),
        "slpic_load_particles": (I, [P, I, I, I64, P, P, P]),
        "slpic_load_particles_dev": (I, [P, I, I, I64, P, P, P]),
        "slpic_load_particles_f64": (I, [P, I, I, I64, P, P]),
        "slpic_prepare": (I, [P]),
        "slpic_step": (I, [P, I64]),
        "slpic_synchronize": (I, [P]),
        "slpic_fields": (I, [P, I, P, P, P]),
        "slpic_fields_async": (I, [P, I, P, P, P]),
        "slpic_density": (I, [P, I, I, P]),
        "slpic_charge_raw": (I, [P, I, I, P]),
        "slpic_particle_count": (I, [P, I, I, ctypes.POINTER(I64)]),
        "slpic_get_particles": (I, [P, I, I, I64, P, P, P, ctypes.POINTER(I64)]),
        "slpic_diagnostics": (I, [P, I, ctypes.POINTER(slpic_diag)]),
        "slpic_save": (I, [P, P, ctypes.POINTER(ctypes.c_size_t)]),
        "slpic_restore": (I, [P, P, ctypes.c_size_t]),
        "slpic_enable_kernel_timing": (I, [P, I64]),
        "slpic_kernel_times": (I, [P, ctypes.POINTER(D), ctypes.POINTER(D), ctypes.POINTER(D),
                                   ctypes.POINTER(I64)]),
        "slpic_kernel_spans": (I, [P, P, P]),
        "slpic_set_wait_limit": (I, [P, I64]),
        "slpic_kernels_per_step": (I, [P, ctypes.POINTER(I)]),
        "slpic_particle_step_noalloc": (I, [ctypes.POINTER(slpic_config), I, I64, P, P, P, P, P,
                                            P, ctypes.POINTER(I64), P, P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _check(h, rc: int, where: str):
    if rc != SLPIC_OK:
        L = load_library()
        msg = (L.slpic_last_error(h) if h else L.slpic_create_error()) or b""
        raise SlpicError(rc, where, msg.decode())


def config_from_problem(prob: dict) -> slpic_config:
    """Problem dictionary (see inputs.py) -> slpic_config."""
    c = slpic_config()
    c.ndim = 1
    c.n_cells = int(prob["n_cells"])
    c.dx = float(prob["dx"])
    c.dt = float(prob["dt"])
    c.bc = SLPIC_BC_PERIODIC if prob["periodic"] else SLPIC_BC_DIRICHLET_ABSORB
    c.phi_lo = float(prob.get("phi_lo", 0.0))
    c.phi_hi = float(prob.get("phi_hi", 0.0))
    c.eps0 = float(prob.get("eps0", 1.0))
    c.max_speed = float(prob.get("max_speed", 0.0))
    c.seed = int(prob.get("seed", 0))
    src = prob.get("source", {"mode": SLPIC_SRC_NONE})
    c.src_mode = int(src.get("mode", SLPIC_SRC_NONE))
    c.src_ref_species = int(src.get("ref_species", 0))
    c.src_lo_cells = float(src.get("lo_cells", 0.0))
    c.src_len_cells = float(src.get("len_cells", 0.0))
    c.src_rate = float(src.get("rate", 0.0))
    sps = prob["species"]
    c.n_species = len(sps)
    for i, sp in enumerate(sps):
        s = c.species[i]
        s.q, s.m, s.w = float(sp["q"]), float(sp["m"]), float(sp["w"])
        s.v0 = float(sp["v0"])
        s.T_src = float(sp.get("T", 0.0))
        cap = sp.get("capacity")
        s.capacity = int(cap) if cap else 1 << 20
        s.beta_kind = int(sp["kind"])
    return c


# ---------------------------------------------------------------- raw entry points
def slpic_create(cfg: slpic_config) -> ctypes.c_void_p:
    L = load_library()
    h = ctypes.c_void_p()
    rc = L.slpic_create(ctypes.byref(cfg), ctypes.byref(h))
    _check(None, rc, "slpic_create")
    return h


def slpic_destroy(h):
    load_library().slpic_destroy(h)


def slpic_set_stream(h, stream: int):
    _check(h, load_library().slpic_set_stream(h, ctypes.c_void_p(stream)), "slpic_set_stream")


def slpic_load_particles(h, instance, species, cell, offset, v):
    cell = np.ascontiguousarray(cell, dtype=np.int32)
    offset = np.ascontiguousarray(offset, dtype=np.float32)
    v = np.ascontiguousarray(v, dtype=np.float32).reshape(-1, 3)
    n = cell.size
    if offset.size != n or v.shape[0] != n:
        raise ValueError("cell, offset and v must describe the same number of particles")
    _check(h, load_library().slpic_load_particles(h, instance, species, n, _ptr(cell),
                                                  _ptr(offset), _ptr(v)),
           "slpic_load_particles")


def slpic_load_particles_dev(h, instance, species, cell, offset, v):
    """cell/offset/v: torch CUDA tensors (int32 [n], float32 [n], float32 [n,3])."""
    n = int(cell.numel())
    for t in (cell, offset, v):
        if not t.is_cuda or not t.is_contiguous():
            raise ValueError("device loads need contiguous CUDA tensors")
    _check(h, load_library().slpic_load_particles_dev(
        h, instance, species, n, ctypes.c_void_p(cell.data_ptr()),
        ctypes.c_void_p(offset.data_ptr()), ctypes.c_void_p(v.data_ptr())),
        "slpic_load_particles_dev")


def slpic_load_particles_f64(h, instance, species, x, v):
    x = np.ascontiguousarray(x, dtype=np.float64)
    v = np.ascontiguousarray(v, dtype=np.float64).reshape(-1, 3)
    _check(h, load_library().slpic_load_particles_f64(h, instance, species, x.size, _ptr(x),
                                                      _ptr(v)), "slpic_load_particles_f64")


def slpic_prepare(h):
    _check(h, load_library().slpic_prepare(h), "slpic_prepare")


def slpic_step(h, nsteps: int):
    _check(h, load_library().slpic_step(h, int(nsteps)), "slpic_step")


def slpic_synchronize(h):
    _check(h, load_library().slpic_synchronize(h), "slpic_synchronize")


def slpic_fields(h, instance, nn: int):
    rho, phi = np.zeros(nn), np.zeros(nn)
    E = np.zeros(nn, dtype=np.float32)
    _check(h, load_library().slpic_fields(h, instance, _ptr(rho), _ptr(phi), _ptr(E)),
           "slpic_fields")
    return rho, phi, E


def slpic_density(h, instance, species, nn: int):
    n = np.zeros(nn)
    _check(h, load_library().slpic_density(h, instance, species, _ptr(n)), "slpic_density")
    return n


def slpic_charge_raw(h, instance, species, nn: int):
    acc = np.zeros(nn, dtype=np.int64)
    _check(h, load_library().slpic_charge_raw(h, instance, species, _ptr(acc)),
           "slpic_charge_raw")
    return acc


def slpic_particle_count(h, instance, species) -> int:
    n = ctypes.c_int64()
    _check(h, load_library().slpic_particle_count(h, instance, species, ctypes.byref(n)),
           "slpic_particle_count")
    return n.value


def slpic_get_particles(h, instance, species):
    n = slpic_particle_count(h, instance, species)
    cell = np.zeros(n, dtype=np.int32)
    off = np.zeros(n, dtype=np.float32)
    v = np.zeros((n, 3), dtype=np.float32)
    got = ctypes.c_int64()
    _check(h, load_library().slpic_get_particles(h, instance, species, n, _ptr(cell), _ptr(off),
                                                 _ptr(v), ctypes.byref(got)),
           "slpic_get_particles")
    k = got.value
    return cell[:k], off[:k], v[:k]


def slpic_diagnostics(h, instance=0) -> dict:
    d = slpic_diag()
    _check(h, load_library().slpic_diagnostics(h, instance, ctypes.byref(d)),
           "slpic_diagnostics")
    return {"step": d.step, "time": d.time, "count": list(d.count), "sum_w": list(d.sum_w),
            "sum_wbeta": list(d.sum_wbeta), "kinetic": list(d.kinetic),
            "field_energy": d.field_energy,
            "absorbed": [[d.absorbed[s][0], d.absorbed[s][1]] for s in range(SLPIC_MAX_SPECIES)],
            "injected": list(d.injected), "iterative": list(d.iterative)}


def slpic_save(h) -> bytes:
    L = load_library()
    size = ctypes.c_size_t(0)
    _check(h, L.slpic_save(h, None, ctypes.byref(size)), "slpic_save")
    buf = ctypes.create_string_buffer(size.value)
    _check(h, L.slpic_save(h, buf, ctypes.byref(size)), "slpic_save")
    return buf.raw[: size.value]


def slpic_restore(h, blob: bytes):
    buf = ctypes.create_string_buffer(blob, len(blob))
    _check(h, load_library().slpic_restore(h, buf, len(blob)), "slpic_restore")


def slpic_enable_kernel_timing(h, max_steps: int):
    _check(h, load_library().slpic_enable_kernel_timing(h, int(max_steps)),
           "slpic_enable_kernel_timing")


def slpic_kernel_times(h):
    """(particle_ms, hard_ms, field_ms, steps) per step of the last timed replay."""
    a, b, c, n = ctypes.c_double(), ctypes.c_double(), ctypes.c_double(), ctypes.c_int64()
    _check(h, load_library().slpic_kernel_times(h, ctypes.byref(a), ctypes.byref(b),
                                                ctypes.byref(c), ctypes.byref(n)),
           "slpic_kernel_times")
    return a.value, b.value, c.value, n.value


def slpic_kernel_spans(h):
    """(ms[3], launches[3]): summed device time and launch count of the particle
    kernel, the iterative-push kernel and the field kernel since creation."""
    ms = np.zeros(3)
    n = np.zeros(3, dtype=np.int64)
    _check(h, load_library().slpic_kernel_spans(h, _ptr(ms), _ptr(n)), "slpic_kernel_spans")
    return ms, n


def slpic_set_wait_limit(h, cycles: int):
    """Spin limit of the particle kernel's pipeline waits, in SM clock cycles (0 =
    the default, about a second)."""
    _check(h, load_library().slpic_set_wait_limit(h, int(cycles)), "slpic_set_wait_limit")


def slpic_kernels_per_step(h) -> int:
    n = ctypes.c_int()
    _check(h, load_library().slpic_kernels_per_step(h, ctypes.byref(n)), "slpic_kernels_per_step")
    return n.value


def slpic_particle_step_noalloc(cfg: slpic_config, species: int, cell_in, state_in, E,
                                cell_out, state_out, charge_out, stream: int = 0):
    """Allocation-free particle step on torch CUDA tensors (see slpic.h).
    Returns (n_out, [absorbed_lo, absorbed_hi])."""
    n = int(cell_in.numel())
    n_out = ctypes.c_int64()
    absorbed = (ctypes.c_int64 * 2)()
    rc = load_library().slpic_particle_step_noalloc(
        ctypes.byref(cfg), species, n, ctypes.c_void_p(cell_in.data_ptr()),
        ctypes.c_void_p(state_in.data_ptr()), ctypes.c_void_p(E.data_ptr()),
        ctypes.c_void_p(cell_out.data_ptr()), ctypes.c_void_p(state_out.data_ptr()),
        ctypes.c_void_p(charge_out.data_ptr()), ctypes.byref(n_out), absorbed,
        ctypes.c_void_p(stream))
    if rc != SLPIC_OK:
        raise SlpicError(rc, "slpic_particle_step_noalloc", "")
    return n_out.value, [absorbed[0], absorbed[1]]


# ---------------------------------------------------------------- convenience wrapper
class Simulation:
    """One simulation handle built from a problem dictionary (see inputs.py)."""

    def __init__(self, prob: dict):
        self.prob = prob
        self.cfg = config_from_problem(prob)
        self.nn = int(prob["n_cells"]) + (0 if prob["periodic"] else 1)
        self.ns = len(prob["species"])
        self.h = slpic_create(self.cfg)
        if prob.get("v0_profile") is not None:
            try:
                slpic_set_speed_limit_profile(self.h, prob["v0_profile"])
            except SlpicError:
                self.close()
                raise

    def close(self):
        if self.h:
            slpic_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def load(self, species, cell, offset, v):
        slpic_load_particles(self.h, 0, species, cell, offset, v)

    def load_state(self, state):
        for s, (c, o, v) in enumerate(state):
            self.load(s, c, o, v)

    def prepare(self):
        slpic_prepare(self.h)

    def step(self, n=1):
        slpic_step(self.h, n)

    def synchronize(self):
        slpic_synchronize(self.h)

    def fields(self):
        return slpic_fields(self.h, 0, self.nn)

    def charge_raw(self, s):
        return slpic_charge_raw(self.h, 0, s, self.nn)

    def density(self, s):
        return slpic_density(self.h, 0, s, self.nn)

    def count(self, s):
        return slpic_particle_count(self.h, 0, s)

    def particles(self, s):
        return slpic_get_particles(self.h, 0, s)

    def diagnostics(self):
        return slpic_diagnostics(self.h, 0)

    def save(self):
        return slpic_save(self.h)

    def restore(self, blob):
        slpic_restore(self.h, blob)


def slpic_set_speed_limit(h, instance, species, v0):
    _check(h, load_library().slpic_set_speed_limit(h, instance, species, v0),
           "slpic_set_speed_limit")


def slpic_set_speed_limit_profile(h, lam):
    """Per-cell factors of v0 (one per cell), or None for a uniform limit."""
    if lam is None:
        rc = load_library().slpic_set_speed_limit_profile(h, None, 0)
    else:
        lam = np.ascontiguousarray(lam, dtype=np.float64)
        rc = load_library().slpic_set_speed_limit_profile(
            h, lam.ctypes.data_as(ctypes.c_void_p), int(lam.size))
    _check(h, rc, "slpic_set_speed_limit_profile")


def slpic_set_timestep(h, dt):
    _check(h, load_library().slpic_set_timestep(h, dt), "slpic_set_timestep")


def slpic_set_wave(h, phi0, k, vphi, t_ramp=0.0):
    _check(h, load_library().slpic_set_wave(h, phi0, k, vphi, t_ramp), "slpic_set_wave")


def _tuning_dict(t: slpic_tuning) -> dict:
    return {f: getattr(t, f) for f, _ in slpic_tuning._fields_}


def slpic_get_tuning(h) -> dict:
    t = slpic_tuning()
    _check(h, load_library().slpic_get_tuning(h, ctypes.byref(t)), "slpic_get_tuning")
    return _tuning_dict(t)


def slpic_set_tuning(h, **settings):
    """Change some of compact_every, particle_kernel, batch_waves, batch_min_share."""
    t = slpic_tuning(**slpic_get_tuning(h))
    for k, v in settings.items():
        setattr(t, k, int(v))
    _check(h, load_library().slpic_set_tuning(h, ctypes.byref(t)), "slpic_set_tuning")


def slpic_autotune(h, steps_per_trial: int = 64):
    """(chosen settings, ms per step); the simulation advances by the trials."""
    t = slpic_tuning()
    ms = ctypes.c_double()
    _check(h, load_library().slpic_autotune(h, steps_per_trial, ctypes.byref(t), ctypes.byref(ms)),
           "slpic_autotune")
    return _tuning_dict(t), ms.value


def slpic_create_batch(cfgs) -> ctypes.c_void_p:
    arr = (slpic_config * len(cfgs))(*cfgs)
    h = ctypes.c_void_p()
    rc = load_library().slpic_create_batch(arr, len(cfgs), ctypes.byref(h))
    _check(None, rc, "slpic_create_batch")
    return h


class Batch:
    """A batch of independent simulations (slpic_create_batch) stepped together;
    per-instance calls take the instance index."""

    def __init__(self, probs):
        self.probs = list(probs)
        self.h = slpic_create_batch([config_from_problem(p) for p in self.probs])
        self.nn = [int(p["n_cells"]) + (0 if p["periodic"] else 1) for p in self.probs]

    def close(self):
        if self.h:
            slpic_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def load(self, inst, species, cell, offset, v):
        slpic_load_particles(self.h, inst, species, cell, offset, v)

    def load_state(self, inst, state):
        for s, (c, o, v) in enumerate(state):
            self.load(inst, s, c, o, v)

    def prepare(self):
        slpic_prepare(self.h)

    def step(self, n=1):
        slpic_step(self.h, n)

    def synchronize(self):
        slpic_synchronize(self.h)

    def fields(self, inst):
        return slpic_fields(self.h, inst, self.nn[inst])

    def charge_raw(self, inst, s):
        return slpic_charge_raw(self.h, inst, s, self.nn[inst])

    def count(self, inst, s):
        return slpic_particle_count(self.h, inst, s)

    def particles(self, inst, s):
        return slpic_get_particles(self.h, inst, s)

    def diagnostics(self, inst):
        return slpic_diagnostics(self.h, inst)


# ------------------------------------------------------------------ plain FP64 form
#: every function declared in include/slpic_fp64.h
EXPORTS_FP64 = (
    "slpic_fp64_create", "slpic_fp64_destroy", "slpic_fp64_last_error", "slpic_fp64_set_stream",
    "slpic_fp64_load_particles", "slpic_fp64_prepare", "slpic_fp64_step",
    "slpic_fp64_synchronize", "slpic_fp64_fields", "slpic_fp64_particle_count",
    "slpic_fp64_get_particles",
)
_fp64_ready = False


def _fp64_lib():
    global _fp64_ready
    L = load_library()
    if not _fp64_ready:
        P, I, I64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64
        sig = {
            "slpic_fp64_create": (I, [ctypes.POINTER(slpic_config), ctypes.POINTER(P)]),
            "slpic_fp64_destroy": (I, [P]),
            "slpic_fp64_last_error": (ctypes.c_char_p, [P]),
            "slpic_fp64_set_stream": (I, [P, P]),
            "slpic_fp64_load_particles": (I, [P, I, I64, P, P]),
            "slpic_fp64_prepare": (I, [P]),
            "slpic_fp64_step": (I, [P, I64]),
            "slpic_fp64_synchronize": (I, [P]),
            "slpic_fp64_fields": (I, [P, P, P, P]),
            "slpic_fp64_particle_count": (I, [P, I, ctypes.POINTER(I64)]),
            "slpic_fp64_get_particles": (I, [P, I, I64, P, P, ctypes.POINTER(I64)]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _fp64_ready = True
    return L


def _check64(h, rc, where):
    if rc != SLPIC_OK:
        L = _fp64_lib()
        msg = (L.slpic_fp64_last_error(h) if h else L.slpic_create_error()) or b""
        raise SlpicError(rc, where, msg.decode())


class SimulationFP64:
    """The plain FP64 form (include/slpic_fp64.h) of the same problem."""

    def __init__(self, prob: dict):
        self.prob = prob
        self.nn = int(prob["n_cells"]) + (0 if prob["periodic"] else 1)
        self.ns = len(prob["species"])
        cfg = config_from_problem(prob)
        h = ctypes.c_void_p()
        _check64(None, _fp64_lib().slpic_fp64_create(ctypes.byref(cfg), ctypes.byref(h)),
                 "slpic_fp64_create")
        self.h = h

    def close(self):
        if self.h:
            _fp64_lib().slpic_fp64_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream: int):
        _check64(self.h, _fp64_lib().slpic_fp64_set_stream(self.h, ctypes.c_void_p(stream)),
                 "slpic_fp64_set_stream")

    def load(self, s, x, v):
        x = np.ascontiguousarray(x, dtype=np.float64)
        v = np.ascontiguousarray(v, dtype=np.float64).reshape(-1, 3)
        _check64(self.h, _fp64_lib().slpic_fp64_load_particles(self.h, s, x.size, _ptr(x), _ptr(v)),
                 "slpic_fp64_load_particles")

    def load_cells(self, s, cell, offset, v):
        dx = float(self.prob["dx"])
        x = (np.asarray(cell, np.float64) + np.asarray(offset, np.float32).astype(np.float64)) * dx
        self.load(s, x, np.asarray(v, np.float32).astype(np.float64))

    def prepare(self):
        _check64(self.h, _fp64_lib().slpic_fp64_prepare(self.h), "slpic_fp64_prepare")

    def step(self, n=1):
        _check64(self.h, _fp64_lib().slpic_fp64_step(self.h, n), "slpic_fp64_step")

    def synchronize(self):
        _check64(self.h, _fp64_lib().slpic_fp64_synchronize(self.h), "slpic_fp64_synchronize")

    def fields(self):
        rho, phi, E = np.zeros(self.nn), np.zeros(self.nn), np.zeros(self.nn)
        _check64(self.h, _fp64_lib().slpic_fp64_fields(self.h, _ptr(rho), _ptr(phi), _ptr(E)),
                 "slpic_fp64_fields")
        return rho, phi, E

    def count(self, s):
        n = ctypes.c_int64(0)
        _check64(self.h, _fp64_lib().slpic_fp64_particle_count(self.h, s, ctypes.byref(n)),
                 "slpic_fp64_particle_count")
        return n.value

    def particles(self, s):
        n = self.count(s)
        x = np.zeros(max(n, 1))
        v = np.zeros((max(n, 1), 3))
        got = ctypes.c_int64(0)
        _check64(self.h, _fp64_lib().slpic_fp64_get_particles(self.h, s, max(n, 1), _ptr(x), _ptr(v),
                                                              ctypes.byref(got)),
                 "slpic_fp64_get_particles")
        return x[:got.value], v[:got.value]
