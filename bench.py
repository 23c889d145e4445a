"""Benchmark: SLPIC particle-steps/s on the 1D bounded argon-like sheath.

Workload (one GPU, weak-scaled: every rank runs its own independent sheath):
4,096 cells, dx = 0.5 lambda_De, electrons + ions with m_i/m_e = 73,440 and
T_e/T_i = 10, 1,000 macroparticles per cell per species (8.19M at load),
Heaviside beta with v0 = 0.02 v_te and dt = dx/v0, absorbing phi = 0 walls, a
central source band re-injecting the ions' losses (LOSS_MATCHED).  A step is
one full pass of the timestep: gather, push, move, walls, deposit,
compaction, injection, FP64 Poisson solve.  Inputs are synthetic and seeded.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line (rank 0).  Under torchrun every rank simulates its own
instance; the timed region is bracketed by a barrier and device
synchronisation and the slowest rank's time is reported.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "SLPIC particle-steps/s incl. deposit+field solve, 1xGB300"
UNIT = "particle-steps/s"
BYTES_PER_PARTICLE_STEP = 40  # int32 cell + float4 state, read once and written once
FALLBACK_HBM_GBS = 6800.0
V0 = 0.02
PPC = 1000
N_CELLS = 4096


def v0_profile(kind, n_cells):
    """Per-cell factors of v0 for --v0-profile: 'sine' is 1/2 at the walls and 1
    at the centre, lam_c = 1/2 + 1/2 sin(pi x_c / L) at the cell centres."""
    if kind == "none":
        return None
    x = (np.arange(n_cells) + 0.5) / n_cells
    return (0.5 + 0.5 * np.sin(np.pi * x)).astype(np.float32)


def workload_config(n_gpus, profile="none"):
    limit = ("v0=0.02 v_te" if profile == "none" else
             "v0=0.02 v_te x lam(x), lam = 1/2 + 1/2 sin(pi x/L) per cell (speed limit varying "
             "in space)")
    return {
        "workload": "1D bounded argon-like sheath (1D3V): 4096 cells, dx=0.5 lambda_De, "
                    "m_i/m_e=73440, T_e/T_i=10, 1000 ppc/species (8.19M particles at load), "
                    f"Heaviside beta, {limit}, dt=dx/v0, phi=0 absorbing walls, "
                    "central LOSS_MATCHED source",
        "n_cells": N_CELLS, "ppc_per_species": PPC, "v0": V0, "species": 2,
        "precision": "FP32 push, int64 fixed-point deposit, FP64 Poisson",
        "l2": "state larger than L2 (8.19M x 20 B = 164 MB read + 164 MB written per step)",
        "parallelism": f"independent instance per GPU x{n_gpus}",
    }


def make_problem(seed):
    from paper_1511_08225_gb300 import inputs
    return inputs.sheath_problem(n_cells=N_CELLS, ppc=PPC, v0=V0, seed=seed)


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi sampling (200 ms) while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.rows = []
        self.proc = None
        self.t_on = self.t_off = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append((time.time(), line.strip()))

    def mark(self, on):
        if on:
            self.t_on = time.time()
        else:
            self.t_off = time.time()

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = [r for t, r in self.rows if self.t_on and self.t_off and self.t_on <= t <= self.t_off]
        if not rows:
            rows = [r for _, r in self.rows]
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            f = [x.strip() for x in r.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)),
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ roofline inputs
def hbm_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            d = json.load(open(p))
            for k in ("hbm_gbs", "hbm_GBs", "hbm"):
                if k in d and d[k]:
                    return float(d[k]), "measured"
        except (ValueError, OSError):
            pass
    return FALLBACK_HBM_GBS, "fallback"


def kernel_source_hash():
    h = hashlib.sha256()
    for f in ("kernels.cu", "particle_step.cuh", "push_math.cuh", "slpic_internal.cuh"):
        h.update(open(os.path.join(ROOT, "paper_1511_08225_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


PROFILE_SUMMARY = os.path.join(ROOT, "profiles", "k_particles_tma_sheath4096.md")


def profiled_traffic(n_particles):
    """DRAM bytes per launch of the particle kernel from the committed ncu
    summary (its `key: value` lines), scaled to this launch's particle count;
    None if the summary is missing or the kernel source changed since."""
    if not os.path.exists(PROFILE_SUMMARY):
        return None
    kv = {}
    for line in open(PROFILE_SUMMARY):
        line = line.strip().lstrip("-").strip()
        if ":" in line:
            k, v = line.split(":", 1)
            kv[k.strip().strip("`")] = v.strip().strip("`")
    try:
        if kv.get("source_hash") != kernel_source_hash():
            return None
        per_particle = float(kv["dram_bytes_per_launch"]) / float(kv["particles_per_launch"])
    except (KeyError, ValueError):
        return None
    return per_particle * n_particles


# ------------------------------------------------------------------ CPU oracle
def oracle_rate(prob, state, budget_s=None, max_particles=None, rng_seed=0, n_steps=None):
    """Time the FP64 oracle on a random particle subsample of the same workload (its
    own run from that state): exactly n_steps steps, or else steps until budget_s of
    CPU time is spent (at least one).  Returns (particle-steps/s, particle-steps,
    seconds, steps)."""
    from oracle import oracle as orc
    rng = np.random.default_rng(rng_seed)
    o = orc.OracleSim(prob)
    n_total = sum(s[0].size for s in state)
    frac = 1.0 if max_particles is None else min(1.0, max_particles / n_total)
    for s, (c, off, v) in enumerate(state):
        k = max(1, int(round(c.size * frac)))
        idx = rng.choice(c.size, size=k, replace=False) if k < c.size else np.arange(c.size)
        o.load_cells(s, c[idx], off[idx], v[idx])
    o.start()
    done, k, t0 = 0, 0, time.perf_counter()
    while True:
        n = sum(x.size for x in o.x)
        o.step(1)
        done += n
        k += 1
        if n_steps is not None:
            if k >= n_steps:
                break
        elif time.perf_counter() - t0 >= budget_s:
            break
    dt = time.perf_counter() - t0
    return done / dt, done, dt, k


def _oracle_rate_job(job):
    prob, state, n_steps, max_particles, seed = job
    r, done, dt, _ = oracle_rate(prob, state, n_steps=n_steps, max_particles=max_particles,
                                 rng_seed=0 if max_particles else seed)
    return r, done, dt


def oracle_rate_all_cores(prob, state, n_steps, per_worker=40_000, workers=None, timeout=None):
    """The oracle as it stands on every host core at once: independent copies in a
    spawn-started pool, each stepping its own random subsample of per_worker
    particles of the workload for the same n_steps steps (the step range a one-core
    run of the same size covers); copy 0 steps the one-core run's own subsample.  Returns (the sum of their particle-steps/s,
    workers, seconds of the slowest copy).  Raises on any failure, and on a pool that
    does not answer within `timeout` seconds, so the caller never hangs on it."""
    import multiprocessing as mp
    workers = int(workers or os.cpu_count() or 1)
    rng = np.random.default_rng(7)
    n_total = sum(s[0].size for s in state)
    frac = min(1.0, per_worker / max(n_total, 1))
    jobs = [(prob, state, int(n_steps), per_worker, 0)]  # copy 0: the one-core sample
    for w in range(1, workers):
        sub = []
        for c, off, v in state:
            k = max(1, int(round(c.size * frac))) if c.size else 0
            idx = rng.choice(c.size, size=k, replace=False) if k else np.zeros(0, np.int64)
            sub.append((c[idx], off[idx], v[idx]))
        jobs.append((prob, sub, int(n_steps), None, w))
    ctx = mp.get_context("spawn")
    with ctx.Pool(workers) as pool:
        res = pool.map_async(_oracle_rate_job, jobs, chunksize=1).get(timeout=timeout)
    return sum(r for r, _, _ in res), workers, max(dt for _, _, dt in res)


def cpu_baseline(prob, state, budget_s, per_worker=40_000):
    """cpu_baseline of the JSON line: the oracle on one core for about budget_s, then
    the same number of steps on every host core at once (independent copies; the
    first copy steps the same subsample as the one-core run)."""
    r, done, dt, nst = oracle_rate(prob, state, budget_s=budget_s, max_particles=per_worker,
                                   rng_seed=0)
    one = {"value": r, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": f"steps 1..{nst} of the oracle's own run from a random "
                     f"{per_worker:,}-particle subsample of the workload's load (same grid, "
                     f"source), {done} particle-steps in {dt:.1f} s, one thread"}
    try:
        ra, nw, slow = oracle_rate_all_cores(prob, state, nst, per_worker=per_worker,
                                             timeout=4 * dt + 120)
        return {"value": ra, "unit": UNIT, "cores": nw, "kind": "oracle",
                "sample": f"{nw} independent copies of the oracle, one per host core, each "
                          f"running steps 1..{nst} from its own random {per_worker:,}-particle "
                          f"subsample of the workload's load (the one-core run's step range); "
                          f"the sum of their rates; slowest copy {slow:.1f} s",
                "single_core": one, "cores_x_single_core": nw * r}
    except Exception as e:  # keep the one-core figure
        one["all_cores_error"] = repr(e)[:200]
        return one


def run_reference(args):
    """--impl reference: the FP64 CPU oracle as it stands, same metric/config."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from paper_1511_08225_gb300 import inputs
    from oracle import oracle as orc
    orc.build()
    prob = make_problem(inputs.SEED)
    lam = v0_profile(args.v0_profile, prob["n_cells"])
    if lam is not None:
        prob["v0_profile"] = lam
    state = inputs.load_state(prob)
    # calibrate the per-particle cost, then size each step's sample so that
    # warmup + steps end in about two minutes
    rate, _, _, _ = oracle_rate(prob, state, 0.5, max_particles=20_000)
    total_steps = max(1, args.steps + args.warmup)
    # at most 250k particles a step: far above the calibration sample the oracle's cost
    # per particle grows (a whole 8.19M-particle step ran about 7x slower per particle)
    per_step_particles = int(max(200, min(250_000, rate * 120.0 / total_steps)))
    rng = np.random.default_rng(1)
    o = orc.OracleSim(prob)
    n_total = sum(s[0].size for s in state)
    frac = per_step_particles / n_total
    for s, (c, off, v) in enumerate(state):
        k = max(1, int(round(c.size * frac)))
        idx = rng.choice(c.size, size=k, replace=False)
        o.load_cells(s, c[idx], off[idx], v[idx])
    o.start()
    for _ in range(args.warmup):
        o.step(1)
    done = 0
    t0 = time.perf_counter()
    for _ in range(args.steps):
        done += sum(x.size for x in o.x)
        o.step(1)
    dt = time.perf_counter() - t0
    value = done / dt
    sample = (f"each step advances a fixed random subsample of {per_step_particles} "
              f"particles of the 8.19M-particle workload's load (same grid, source), the "
              f"oracle's own run from it; the GPU arm times its state after its settle steps, "
              f"which the oracle could not reach in minutes")
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / max(1, args.steps),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "impl": "reference",
        "config": workload_config(args.gpus, args.v0_profile),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ GPU arm
def aggregate_ranks(ms, particle_steps, dist, device):
    """Whole-job figures over the ranks (weak scaling, one independent instance per
    rank): the slowest rank's time and the particle-steps of all ranks.  Without a
    process group the rank's own figures."""
    if not dist:
        return ms, particle_steps
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    ps = torch.tensor([particle_steps], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(ps, op=dist.ReduceOp.SUM)
    return float(t[0]), float(ps[0])


def smi_once(gpu_index):
    """One nvidia-smi sample of the clocks (the 200 ms sampler may not fire inside a
    short timed region): (sm_mhz, sm_max_mhz, [active throttle reasons]) or None."""
    try:
        out = subprocess.run(
            ["nvidia-smi", f"--id={gpu_index}", f"--query-gpu={ClockSampler.Q}",
             "--format=csv,noheader,nounits"], capture_output=True, text=True, timeout=10)
        f = [x.strip() for x in out.stdout.strip().split(",")]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        return float(f[1]), float(f[2]), [n for n, v in zip(names, f[5:9]) if v.lower() == "active"]
    except (OSError, ValueError, IndexError, subprocess.SubprocessError):
        return None


def run_gpu(args):
    import torch

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_1511_08225_gb300 import binding, inputs
    from paper_1511_08225_gb300 import build as pkg_build
    pkg_build.build()
    binding.load_library()

    seed = inputs.SEED + rank
    prob = make_problem(seed)
    lam = v0_profile(args.v0_profile, prob["n_cells"])
    if lam is not None:
        prob["v0_profile"] = lam
    state = inputs.load_state(prob)
    n_load = sum(s[0].size for s in state)

    stream = torch.cuda.Stream()
    sim = binding.Simulation(prob)
    binding.slpic_set_stream(sim.h, stream.cuda_stream)
    binding.slpic_set_tuning(sim.h, compact_every=args.compact_every)
    sim.load_state(state)
    sim.prepare()

    def barrier():
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    def live():
        return sum(sim.count(s) for s in range(2))

    def phi_range():
        _, phi, _ = sim.fields()
        return float(phi.min()), float(phi.max())

    # settle: the configured sheath has no steady state from any start; within about
    # 100/omega_pe it runs away, and after ~2,000 steps it sits in a stationary
    # saturated state.  The timed steps are taken there, past the transient.
    t_set = time.perf_counter()
    sim.step(args.settle)
    sim.synchronize()
    settle_s = time.perf_counter() - t_set
    clocks = ClockSampler(local)
    clocks.start()
    sim.step(args.warmup)
    tuning = binding.slpic_get_tuning(sim.h)
    if args.autotune:  # outside the timed region; the trials advance the run
        tuning, _ = binding.slpic_autotune(sim.h, steps_per_trial=256)
    sim.synchronize()
    blob = sim.save()  # checkpoint: the timed steps are replayed for the event timing
    n0 = live()
    dg0 = sim.diagnostics()
    ph0 = phi_range()
    sp0, nl0 = binding.slpic_kernel_spans(sim.h)
    smi0 = smi_once(local)
    barrier()
    clocks.mark(True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    sim.step(args.steps)
    ev1.record(stream)
    ev1.synchronize()
    barrier()
    clocks.mark(False)
    smi1 = smi_once(local)
    ms = ev0.elapsed_time(ev1)
    sim.synchronize()
    n1 = live()
    dg1 = sim.diagnostics()
    ph1 = phi_range()
    sp1, nl1 = binding.slpic_kernel_spans(sim.h)
    clocks.stop()
    # device time of each kernel over the timed steps themselves (first CTA start to
    # last CTA end, on the GPU's global timer)
    span_ms = (sp1 - sp0) / args.steps
    # the same steps replayed from the checkpoint with CUDA events bracketing the
    # kernels (event nodes in the graph add a little launch latency per interval)
    sim.restore(blob)
    binding.slpic_enable_kernel_timing(sim.h, args.steps if args.steps <= 4096 else 4096)
    sim.step(args.steps if args.steps <= 4096 else 4096)
    push_ms, hard_ms_ev, field_ms_ev, nrec = binding.slpic_kernel_times(sim.h)
    binding.slpic_enable_kernel_timing(sim.h, 0)
    n_replay = min(args.steps, 4096)
    # the replay ends where the timed steps did (checked when it covers all of them)
    replay_same = None if n_replay < args.steps else sim.diagnostics()["step"] == dg1["step"]
    n_replay_end = live()  # the live count where the replay ends
    iterative_per_step = (sum(dg1["iterative"]) - sum(dg0["iterative"])) / args.steps

    t_max, particle_steps = aggregate_ranks(ms, 0.5 * (n0 + n1) * args.steps, dist, "cuda")
    value = particle_steps / (t_max * 1e-3)

    # roofline of the particle kernel (dominant kernel): algorithmic bytes over its
    # CUDA-event duration on the library's stream, the timed steps replayed; the
    # particles per launch are the mean live count over the replayed steps
    n_mean = 0.5 * (n0 + n1)
    n_launch = 0.5 * (n0 + n_replay_end)
    peak, peak_kind = hbm_peak()
    if push_ms <= 0:
        push_ms = span_ms[0]
        n_launch = n_mean
    achieved = BYTES_PER_PARTICLE_STEP * n_launch / (push_ms * 1e-3) / 1e9
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak,
            "traffic": profiled_traffic(n_launch) if lam is None else None,
            "particles_per_launch": n_launch,
            "kernel": (f"{'k_particles_tma' if tuning['particle_kernel'] == 0 else 'k_particles'}"
                       f"{'' if lam is None else ' (speed-limit profile variant)'} "
                       f"(in-place steps; k_particles_compact every {tuning['compact_every']})"),
            "kernel_ms": push_ms,
            "kernel_ms_timing": "CUDA events on the library's stream bracketing the particle "
                                "kernel, the timed steps replayed from a checkpoint",
            "hard_kernel_ms": float(span_ms[1]), "field_kernel_ms": float(span_ms[2]),
            "split_ms": {"particle": float(span_ms[0]), "hard": float(span_ms[1]),
                         "field": float(span_ms[2]), "sum": float(span_ms.sum()),
                         "step": t_max / args.steps,
                         "launches": [int(x) for x in (nl1 - nl0)],
                         "timing": "device global timer, first CTA start to last CTA end of "
                                   "each launch, over the timed steps themselves"},
            "events_ms": {"particle": push_ms, "hard": hard_ms_ev, "field": field_ms_ev,
                          "steps": int(nrec),
                          "replayed": ("all the timed steps" if n_replay == args.steps else
                                       f"the first {n_replay} of the timed steps"),
                          "replay_reached_the_same_step": replay_same},
            "iterative_pushes_per_step": iterative_per_step,
            "bytes_per_particle_step": BYTES_PER_PARTICLE_STEP,
            "peak_source": f"{peak_kind} HBM copy bandwidth (burst)", "tuning": tuning,
            "autotuned": bool(args.autotune)}

    # the timed state, stated: field energy and potential at both ends of the region
    timed_state = {
        "settle_steps": args.settle, "settle_s": round(settle_s, 2),
        "step_range": [int(dg0["step"]), int(dg1["step"])],
        "field_energy": [dg0["field_energy"], dg1["field_energy"]],
        "e_phi_over_Te_max": [ph0[1], ph1[1]], "e_phi_over_Te_min": [ph0[0], ph1[0]],
        "physical_count_e_i": [dg1["sum_wbeta"][0], dg1["sum_wbeta"][1]],
        "note": "the configured sheath has no steady state under SLPIC (it runs away from "
                "a random, a quiet or an empty start within ~100/omega_pe); the timed steps "
                "are in the stationary saturated state reached after the settle steps",
    }

    # end to end through the C ABI with pinned host buffers: the settled particles
    # loaded from host memory, then the steps with a read-back after every step
    e2e = None
    settled = None
    if rank == 0 or world > 1 or not args.no_fp64:
        settled = [sim.particles(s) for s in range(2)]
    if rank == 0 or world > 1:
        e2e = run_e2e(prob, settled, args, binding, torch, stream)

    # the plain FP64 form of the same step from the same settled particles (the
    # comparison point of the metric)
    fp64 = None
    if rank == 0 and not args.no_fp64 and lam is None:  # the FP64 form has no profile
        fp64 = run_fp64(prob, settled, args, binding, torch, stream, value)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(prob, state, args.cpu_budget)

    clk = clocks.summary()
    clk["one_shot"] = {"before": smi0, "after": smi1}
    if clk["sm_mhz"] is None:
        shots = [x for x in (smi0, smi1) if x]
        if shots:
            clk.update({"sm_mhz": float(np.median([x[0] for x in shots])),
                        "sm_max_mhz": max(x[1] for x in shots),
                        "reasons": sorted({r for x in shots for r in x[2]}),
                        "samples": len(shots)})

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "impl": "gb300",
            "config": workload_config(world, args.v0_profile),
            "particles_at_load": n_load, "particles_timed_mean": n_mean,
            "timed_state": timed_state,
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "fp64_form": fp64,
            "gpu_launches": int((nl1 - nl0).sum()), "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    sim.close()
    if dist:
        dist.destroy_process_group()
    return 0


def run_fp64(prob, settled, args, binding, torch, stream, mixed_value):
    """Particle-steps/s of the plain FP64 form (include/slpic_fp64.h): same
    problem, the same settled particles, the same warm-up, min(steps, 50) timed
    steps."""
    g = binding.SimulationFP64(prob)
    g.set_stream(stream.cuda_stream)
    for s, (c, o, v) in enumerate(settled):
        g.load_cells(s, c, o, v)
    g.prepare()
    g.step(args.warmup)
    g.synchronize()
    n0 = sum(g.count(s) for s in range(len(settled)))
    steps = max(1, min(args.steps, 50))
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    g.step(steps)
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    g.synchronize()
    n1 = sum(g.count(s) for s in range(len(settled)))
    g.close()
    val = 0.5 * (n0 + n1) * steps / (ms * 1e-3)
    return {"value": val, "unit": UNIT, "steps": steps, "warmup": args.warmup,
            "ms_per_step": ms / steps, "speedup_of_mixed": mixed_value / val,
            "state": "the mixed form's settled particles, loaded in FP64",
            "form": "FP64 x + 3 FP64 v (32 B/particle), FP64 push (closed-form time, Newton), "
                    "FP64 atomic CIC deposit, FP64 prefix-sum Poisson, survivors packed "
                    "every step; 3 launches per step"}


def run_e2e(prob, settled, args, binding, torch, stream):
    """Same metric through the public API with pinned host memory: each timed
    run loads the (settled) particles from host, then every step is followed by a
    device-to-host read of rho, phi and E (the step's result)."""
    pinned = []
    for c, o, v in settled:
        tc = torch.from_numpy(np.ascontiguousarray(c)).pin_memory()
        to = torch.from_numpy(np.ascontiguousarray(o)).pin_memory()
        tv = torch.from_numpy(np.ascontiguousarray(v)).pin_memory()
        pinned.append((tc.numpy(), to.numpy(), tv.numpy()))
    nn = prob["n_cells"] + 1
    # a ring of two pinned read-back buffers: the copy of step k's fields overlaps
    # step k+1
    ring = [(torch.empty(nn, dtype=torch.float64).pin_memory().numpy(),
             torch.empty(nn, dtype=torch.float64).pin_memory().numpy(),
             torch.empty(nn, dtype=torch.float32).pin_memory().numpy()) for _ in range(2)]
    L = binding.load_library()
    steps = max(1, min(args.steps, args.e2e_steps))
    sim = binding.Simulation(prob)
    binding.slpic_set_stream(sim.h, stream.cuda_stream)
    binding.slpic_set_tuning(sim.h, compact_every=args.compact_every)
    torch.cuda.synchronize()
    h2d = sum(a.nbytes + b.nbytes + c.nbytes for a, b, c in pinned)
    t0 = time.perf_counter()
    for s, (c, o, v) in enumerate(pinned):
        sim.load(s, c, o, v)
    for k in range(steps):
        sim.step(1)
        rho, phi, E = ring[k & 1]
        rc = L.slpic_fields_async(sim.h, 0, binding._ptr(rho), binding._ptr(phi),
                                  binding._ptr(E))
        if rc:
            raise RuntimeError(f"slpic_fields_async failed: {rc}")
    sim.synchronize()
    t1 = time.perf_counter()
    # the last read-back is the state's fields
    chk = sim.fields()
    if not (np.array_equal(chk[1], ring[(steps - 1) & 1][1]) and
            np.array_equal(chk[2], ring[(steps - 1) & 1][2])):
        raise RuntimeError("asynchronous read-back differs from slpic_fields")
    rho, phi, E = ring[0]
    d = sim.diagnostics()
    n_end = sum(d["count"][:2])
    n_start = sum(c.size for c, _, _ in pinned)
    sim.close()
    return {"value": 0.5 * (n_start + n_end) * steps / (t1 - t0), "unit": UNIT,
            "h2d_bytes_per_step": h2d / steps,
            "d2h_bytes_per_step": rho.nbytes + phi.nbytes + E.nbytes,
            "steps": steps, "note": "the settled particles loaded from pinned host memory "
                                    "(counted once per run, inside the timed region); rho, "
                                    "phi and E of every step read back into pinned memory "
                                    "(slpic_fields_async, a ring of two buffers), one "
                                    "synchronisation at the end"}


# ------------------------------------------------------------------ other workloads
def _gen_state(prob):
    from paper_1511_08225_gb300 import inputs
    return inputs.load_state(prob)


def run_batch(args):
    """Batched sheaths (slpic_create_batch): m independent 1D instances of uneven
    size, mass ratio and speed limit advanced by one set of batched kernels per
    step.  Inputs are generated in a spawn-started process pool before any GPU
    call."""
    import multiprocessing as mp
    from paper_1511_08225_gb300 import inputs
    probs = inputs.batch_problems(m=args.batch_m)
    ctx = mp.get_context("spawn")
    states = []
    with ctx.Pool(min(16, os.cpu_count() or 1)) as pool:
        states = pool.map(_gen_state, probs, chunksize=1)
    import torch
    from paper_1511_08225_gb300 import binding
    from paper_1511_08225_gb300 import build as pkg_build
    pkg_build.build()
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    b = binding.Batch(probs)
    binding.slpic_set_stream(b.h, stream.cuda_stream)
    for i, st in enumerate(states):
        b.load_state(i, st)
    n_load = sum(c.size for st in states for c, _, _ in st)
    del states
    b.prepare()

    def live():
        return sum(b.count(i, s) for i in range(len(probs)) for s in range(2))

    clocks = ClockSampler(0)
    clocks.start()
    b.step(args.warmup)
    tuning = binding.slpic_get_tuning(b.h)
    if args.autotune:  # outside the timed region; the trials advance the run
        tuning, _ = binding.slpic_autotune(b.h, steps_per_trial=16)
    b.synchronize()
    n0 = live()
    torch.cuda.synchronize()
    clocks.mark(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    b.step(args.steps)
    e1.record(stream)
    e1.synchronize()
    clocks.mark(False)
    ms = e0.elapsed_time(e1)
    b.synchronize()
    n1 = live()
    clocks.stop()
    n_mean = 0.5 * (n0 + n1)
    value = n_mean * args.steps / (ms * 1e-3)
    peak, peak_kind = hbm_peak()
    achieved = BYTES_PER_PARTICLE_STEP * n_mean / (ms / args.steps * 1e-3) / 1e9
    cells = [p["n_cells"] for p in probs]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "impl": "gb300",
        "config": {"workload": f"batched sheaths: {len(probs)} independent 1D3V instances, "
                               f"cells U{{512..8192}}, ppc U{{100..1000}}, m_i/m_e in "
                               f"{{1836, 73440}}, v0 log-uniform 0.01-0.5 v_te, dt = dx/v0; "
                               f"one set of batched kernels per step in a CUDA graph",
                   "instances": len(probs), "cells_total": int(sum(cells)),
                   "l2": "state far larger than L2"},
        "particles_at_load": int(n_load), "particles_timed_mean": n_mean,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": None, "kernel": "whole step",
                     "bytes_per_particle_step": BYTES_PER_PARTICLE_STEP,
                     "peak_source": f"{peak_kind} HBM copy bandwidth",
                     "note": "whole-step time (particles, iterative push, field) against "
                             "the particle kernel's algorithmic bytes: a lower bound",
                     "tuning": tuning, "autotuned": bool(args.autotune)},
        "gpu_launches": 3 * args.steps, "clocks": clocks.summary(),
    }
    print(json.dumps(line), flush=True)
    b.close()
    return 0


def run_2d(args):
    """2D3V plasma between absorbing plates (1024 x 1024 cells, 64 ppc/species by
    default): particle kernel + source + cooperative Jacobi-PCG per step."""
    import torch
    from paper_1511_08225_gb300 import binding2d, inputs
    from paper_1511_08225_gb300 import build as pkg_build
    prob = inputs.plasma2d_problem(nx=args.nx, ny=args.ny, ppc=args.ppc2d, v0=0.1,
                                   solver=args.solver)
    state = inputs.load_state2d(prob)
    pkg_build.build()
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    sim = binding2d.Simulation2D(prob)
    binding2d.slpic2d_set_stream(sim.h, stream.cuda_stream)
    t0 = time.perf_counter()
    sim.load_state(state)
    sim.prepare()
    prep_s = time.perf_counter() - t0
    d_prep = sim.diagnostics()
    n_load = sum(c.size for c, _, _ in state)

    def live():
        return sum(binding2d.slpic2d_particle_count(sim.h, s) for s in range(2))

    clocks = ClockSampler(0)
    clocks.start()
    sim.step(args.warmup)
    sim.synchronize()
    n0 = live()
    d0 = sim.diagnostics()
    binding2d.slpic2d_enable_kernel_timing(sim.h, True)
    torch.cuda.synchronize()
    clocks.mark(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sim.step(args.steps)
    e1.record(stream)
    e1.synchronize()
    clocks.mark(False)
    ms = e0.elapsed_time(e1)
    sim.synchronize()
    n1 = live()
    d1 = sim.diagnostics()
    pk, ik, fk, nrec = binding2d.slpic2d_kernel_times(sim.h)
    clocks.stop()
    n_mean = 0.5 * (n0 + n1)
    value = n_mean * args.steps / (ms * 1e-3)
    peak, peak_kind = hbm_peak()
    bpp = 48  # int32 cell + float4 + float vz, read once and written once
    achieved = bpp * n_mean / (pk * 1e-3) / 1e9
    cg_per_step = (d1["cg_iterations_total"] - d0["cg_iterations_total"]) / args.steps
    # CPU oracle: push + deposit of a particle subsample in the GPU's own field
    cpu = None
    if not args.no_cpu:
        from oracle import oracle as orc
        _, _, Ex, Ey = sim.fields()
        o = orc.OracleSim2D(prob)
        rng = np.random.default_rng(0)
        for s_, (c, off, v) in enumerate(state):
            idx = rng.choice(c.size, 20_000, replace=False)
            o.load_cells(s_, c[idx], off[idx], v[idx])
        o.Ex, o.Ey = Ex.astype(np.float64), Ey.astype(np.float64)
        t0 = time.perf_counter()
        k = 0
        while time.perf_counter() - t0 < args.cpu_budget and k < 200:
            o.push()
            o.deposit()
            k += 1
        dt_ = time.perf_counter() - t0
        cpu = {"value": 40_000 * k / dt_, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"{k} push+deposit passes of a 40,000-particle subsample in the GPU's "
                         f"field ({dt_:.1f} s, one thread); the oracle's direct 2D solve is "
                         f"O(nx^2 ny) and not part of the sample"}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "impl": "gb300",
        "config": {"workload": f"2D3V electrostatic SLPIC: {args.nx}x{args.ny} cells, dx=1 "
                               f"lambda_De, {args.ppc2d} ppc/species, periodic x, absorbing "
                               f"phi=0 plates in y, m_i/m_e=1836, Heaviside beta v0=0.1 v_te, "
                               f"dt=dx/v0, central LOSS_MATCHED source band; "
                               + ("Jacobi-PCG to 1e-8 relative residual, warm-started"
                                  if args.solver == "cg" else
                                  "direct FP64 solve: FFT along x, Thomas per mode along y"),
                   "solver": args.solver,
                   "l2": "state larger than L2"},
        "particles_at_load": int(n_load), "particles_timed_mean": n_mean,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": None,
                     "kernel": ("k_particles2d_tiles + k_hard2d (in-place steps; k_particles2d "
                                "every 16th)"),
                     "kernel_ms": pk, "inject_kernel_ms": ik, "field_kernel_ms": fk,
                     "inject_note": "source and bookkeeping, and the cell sort after the "
                                    "compacting step",
                     "iterative_pushes_last_step": d1["iterative_last"],
                     "bytes_per_particle_step": bpp,
                     "peak_source": f"{peak_kind} HBM copy bandwidth"},
        "field_solve": {"cg_iterations_per_step": cg_per_step,
                        "cg_rel_residual_last": d1["cg_rel_residual"],
                        "cold_start_iterations": d_prep["cg_iterations"],
                        "ms_per_step": fk, "load_and_first_solve_s": prep_s},
        "cpu_baseline": cpu, "gpu_launches": 3 * args.steps, "clocks": clocks.summary(),
    }
    print(json.dumps(line), flush=True)
    sim.close()
    return 0


def bf16_peak_tflops():
    """Dense BF16 tensor peak for a kernel timed alone: MEASURED_PEAKS.json's burst
    cuBLAS figure, else the fallback of 1,900 TFLOP/s."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            d = json.load(open(p))
            if d.get("bf16_tflops"):
                return float(d["bf16_tflops"]), "measured"
        except (ValueError, OSError):
            pass
    return 1900.0, "fallback"


def fp32_fma_peak_tflops():
    """FP32 FMA peak from unit counts: SMs x 128 FP32 lanes x 2 flops x the maximum
    SM clock (GB300: 152 x 128 x 2 x 2.07 GHz = 80.5 TFLOP/s)."""
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    mhz = 2070.0
    try:
        out = subprocess.run(["nvidia-smi", "--query-gpu=clocks.max.sm", "--format=csv,noheader,nounits",
                              "-i", "0"], capture_output=True, text=True, timeout=20).stdout.split()
        mhz = float(out[0]) if out else mhz
    except Exception:
        pass
    return sms * 128 * 2 * mhz * 1e6 / 1e12


def unet_macs(levels, base, H, W):
    """Multiply-adds of one forward pass (3x3 convs)."""
    from paper_1511_08225_gb300 import binding_unet
    tot = 0
    for k, (ci, co) in enumerate(binding_unet.layer_shapes(levels, base)):
        lvl = k if k < levels else (0 if k == 2 * levels - 1 else 2 * levels - 2 - k)
        tot += 9 * ci * co * (H >> lvl) * (W >> lvl)
    return tot


def run_unet_net(args):
    """The learned warm start's network alone: a tensor-core U-Net (4 levels, base
    channels --unet-base, BF16 weights, FP32 accumulation) on --nx x --ny images,
    batch 1, random data: W warm-up forward passes and Adam steps, then K forward
    passes and K training steps timed with CUDA events on the network's stream.  The
    forward's FLOPs against the measured BF16 tensor peak."""
    import torch
    from paper_1511_08225_gb300 import binding_unet
    from paper_1511_08225_gb300 import build as pkg_build
    pkg_build.build()
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    nx, ny, L, C = args.nx, args.ny, 4, args.unet_base
    net = binding_unet.UNet(L, C, ny, nx, max_batch=1, normalise=False, seed=1,
                            tensor_cores=not args.unet_cuda_cores)
    net.set_stream(stream.cuda_stream)
    g = torch.Generator(device="cuda").manual_seed(5)
    x = torch.randn(1, ny, nx, device="cuda", generator=g)
    t = torch.randn(1, ny, nx, device="cuda", generator=g)
    y = torch.zeros_like(x)
    torch.cuda.synchronize()
    for _ in range(args.warmup):
        net.forward(x, y)
        net.train_step(x, t, 1e-4)
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    ev[0].record(stream)
    for _ in range(args.steps):
        net.forward(x, y)
    ev[1].record(stream)
    for _ in range(args.steps):
        net.train_step(x, t, 1e-4)
    ev[2].record(stream)
    ev[2].synchronize()
    fwd_ms = ev[0].elapsed_time(ev[1]) / args.steps
    train_ms = ev[1].elapsed_time(ev[2]) / args.steps
    macs = unet_macs(L, C, ny, nx)
    fwd_tflops = 2 * macs / (fwd_ms * 1e-3) / 1e12
    peak, kind = bf16_peak_tflops()
    net.close()
    line = {
        "metric": "U-Net forward TFLOP/s (learned warm start's network), 1xGB300",
        "value": fwd_tflops, "unit": "TFLOP/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": fwd_ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
        "impl": "gb300",
        "config": {"workload": f"U-Net {L} levels, {C}..{C * 2 ** (L - 1)} channels, "
                               f"{nx}x{ny}, batch 1, random data", "macs": macs},
        "train_step_ms": train_ms,
        "train_step_tflops": 3 * 2 * macs / (train_ms * 1e-3) / 1e12,
        "roofline": {"bound": "tensor", "achieved": fwd_tflops, "peak": peak, "unit": "TFLOP/s",
                     "frac": fwd_tflops / peak, "traffic": None,
                     "kernel": "U-Net forward (k_conv_fwd_tc and the elementwise layers)",
                     "peak_source": f"{kind} dense BF16 (cuBLAS burst)"},
        "gpu_launches": None,
    }
    print(json.dumps(line), flush=True)
    return 0


def run_unet2d(args):
    """The 2D workload with the learned warm start of the CG: (rho, phi) pairs from a
    run of one seed, two U-Nets trained on them by the library (phi from rho, and the
    change of phi from the change of rho), then four identical copies of a run of
    another seed, timed with the CG started from the previous phi, the zero guess,
    the network's phi and the previous phi plus the network's change."""
    import torch
    from paper_1511_08225_gb300 import binding2d, binding_unet, inputs, warmstart
    from paper_1511_08225_gb300 import build as pkg_build
    pkg_build.build()
    torch.cuda.set_device(0)
    nx, ny = args.nx, args.ny
    prob = inputs.plasma2d_problem(nx=nx, ny=ny, ppc=args.ppc2d, v0=0.1, capacity_factor=2.0)
    t0 = time.perf_counter()
    # the pairs from a run of the direct solver (the same potential, 30x cheaper to make
    # when nx is a power of two); the timed runs below use the CG
    gen = dict(prob, solver="fft") if nx & (nx - 1) == 0 else prob
    # a large set (more than 512 pairs) is made on the device, change images only: the
    # network of the change mode alone is trained on it
    big = args.unet_pairs > 512
    if big:
        sets = [("delta", warmstart.collect_delta_images(gen, inputs.SEED + 1, args.unet_pairs,
                                                         every=2, skip=10))]
    else:
        pairs = warmstart.collect_pairs(gen, seeds=(inputs.SEED + 1,),
                                        pairs_per_seed=args.unet_pairs, every=2, skip=10,
                                        keep_prev=True)
        sets = [("direct", warmstart.images(pairs)), ("delta", warmstart.delta_images(pairs))]
        del pairs
    collect_s = time.perf_counter() - t0
    L, C = 4, args.unet_base
    nets, train_info = {}, {}
    for name, (x, t) in sets:
        if big:
            xd, td = x, t
            scale = warmstart.output_scale(x[:512].cpu().numpy(), t[:512].cpu().numpy())
        else:
            xd, td = torch.tensor(x, device="cuda"), torch.tensor(t, device="cuda")
            scale = warmstart.output_scale(x, t)
        net = binding_unet.UNet(L, C, ny, nx, max_batch=args.unet_batch, normalise=True,
                                out_scale=scale, seed=1, tensor_cores=not args.unet_cuda_cores)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        losses = warmstart.fit(net, xd, td, steps=args.unet_train_steps, batch=args.unet_batch,
                               lr=2e-3, log_every=max(args.unet_train_steps // 4, 1))
        torch.cuda.synchronize()
        train_info[name] = {"seconds": time.perf_counter() - t1, "loss_first": losses[0][1],
                            "loss_last": losses[-1][1]}
        nets[name] = net
        del xd, td, x, t
    sets = None
    fwd_net = nets.get("direct", nets["delta"])
    # the network's forward pass alone, CUDA events on its stream
    xin = torch.randn(1, ny, nx, device="cuda")
    yout = torch.zeros_like(xin)
    for _ in range(3):
        fwd_net.forward(xin, yout)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(10):
        fwd_net.forward(xin, yout)
    e1.record()
    e1.synchronize()
    fwd_ms = e0.elapsed_time(e1) / 10
    fwd_tflops = 2 * unet_macs(L, C, ny, nx) / (fwd_ms * 1e-3) / 1e12
    if args.unet_cuda_cores:
        peak, peak_src = fp32_fma_peak_tflops(), "FP32 FMA from unit counts: SMs x 128 lanes x 2 x max SM clock"
        bound, kern = "alu", "U-Net forward (k_conv_fwd, CUDA cores)"
    else:
        peak, kind = bf16_peak_tflops()
        peak_src = f"{kind} dense BF16 (cuBLAS burst)"
        bound, kern = "tensor", "U-Net forward (k_conv_fwd_tc, tcgen05)"

    state = inputs.load_state2d(prob)
    modes = (("prev", binding2d.SLPIC2D_WARM_PREV, None), ("zero", binding2d.SLPIC2D_WARM_ZERO, None))
    if "direct" in nets:
        modes += (("unet", binding2d.SLPIC2D_WARM_UNET, nets["direct"]),)
    modes += (("unet_delta", binding2d.SLPIC2D_WARM_UNET_DELTA, nets["delta"]),)
    clocks = ClockSampler(0)
    clocks.start()
    res = {}
    for name, mode, net in modes:
        stream = torch.cuda.Stream()
        sim = binding2d.Simulation2D(prob)
        binding2d.slpic2d_set_stream(sim.h, stream.cuda_stream)
        sim.load_state(state)
        sim.prepare()
        sim.step(args.warmup)
        sim.set_warm_start(mode, net)
        sim.step(1)  # the change mode's first step has no previous charge
        sim.synchronize()
        d0 = sim.diagnostics()
        n0 = sum(binding2d.slpic2d_particle_count(sim.h, s) for s in range(2))
        torch.cuda.synchronize()
        clocks.mark(True)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        sim.step(args.steps)
        b.record(stream)
        b.synchronize()
        clocks.mark(False)
        ms = a.elapsed_time(b)
        d1 = sim.diagnostics()
        n1 = sum(binding2d.slpic2d_particle_count(sim.h, s) for s in range(2))
        res[name] = {"ms_per_step": ms / args.steps,
                     "cg_iterations_per_step": (d1["cg_iterations_total"] - d0["cg_iterations_total"])
                     / args.steps,
                     "particle_steps_per_s": 0.5 * (n0 + n1) * args.steps / (ms * 1e-3),
                     "cg_rel_residual_last": d1["cg_rel_residual"]}
        sim.close()
    clocks.stop()
    for net in nets.values():
        net.close()
    best = res["unet_delta"]
    line = {
        "metric": METRIC, "value": best["particle_steps_per_s"], "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": best["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic", "impl": "gb300",
        "config": {"workload": f"2D3V electrostatic SLPIC with a learned CG warm start: {nx}x{ny} "
                               f"cells, {args.ppc2d} ppc/species (the plasma2d workload); U-Net "
                               f"{L} levels, {C}..{C << (L - 1)} channels, BF16 weights, FP32 "
                               f"accumulation, convolutions forward on "
                               f"{'CUDA cores' if args.unet_cuda_cores else 'tensor cores (BF16 operands)'}, trained on {args.unet_pairs} (rho, phi) pairs of "
                               f"one seed (every 2nd step after 10), {args.unet_train_steps} Adam "
                               f"steps of {args.unet_batch}; timed on another seed (CG to 1e-8); "
                               f"value is the previous-phi-plus-network-change mode",
                   "l2": "state larger than L2"},
        "warm_start": res,
        "cg_iterations_saved_vs_zero": 1 - best["cg_iterations_per_step"] / res["zero"]["cg_iterations_per_step"],
        "cg_iterations_saved_vs_prev": 1 - best["cg_iterations_per_step"] / res["prev"]["cg_iterations_per_step"],
        "unet": {"forward_ms": fwd_ms, "forward_tflops": fwd_tflops, "training": train_info,
                 "pair_collection_s": collect_s, "networks": sorted(nets),
                 "pairs": args.unet_pairs},
        "roofline": {"bound": bound, "achieved": fwd_tflops, "peak": peak, "unit": "TFLOP/s",
                     "frac": fwd_tflops / peak, "traffic": None, "kernel": kern,
                     "peak_source": peak_src},
        "cpu_baseline": None, "clocks": clocks.summary(),
        # per step in the change mode: particle, source, rho image, difference, the
        # network's forward (4L launches), guess, CG
        "gpu_launches": args.steps * (6 + 4 * L),
    }
    print(json.dumps(line), flush=True)
    return 0


def run_paper_sheath(args):
    """The paper's own benchmark (Sec. IV): the argon sheath filled from its wall
    source, run to steady state (24 us of plasma time) as plain PIC (beta = 1,
    dt = dx/(5 v_te)) and as SLPIC (v0 = 0.016 v_te, dt = dx/v0); the metric is
    the wall-time ratio, which the paper quotes as 160x.  Both runs are timed with
    CUDA events around the whole stepping; a second, sampled pass of each
    averages the profiles over the last third for the agreement figures."""
    import torch
    from paper_1511_08225_gb300 import binding, inputs
    from paper_1511_08225_gb300 import build as pkg_build
    pkg_build.build()
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    t_end = 9530.0
    res = {}
    for kind, name in ((inputs.BETA_ONE, "pic"), (inputs.BETA_HEAVISIDE, "slpic")):
        prob = inputs.paper_sheath_problem(kind=kind, ppc=args.ppc_sheath)
        n = int(round(t_end / prob["dt"]))
        sim = binding.Simulation(prob)
        binding.slpic_set_stream(sim.h, stream.cuda_stream)
        sim.load_state(inputs.empty_state(prob))
        sim.prepare()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.step(n)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        sim.synchronize()
        d = sim.diagnostics()
        sim.close()
        # sampled pass for the steady-state profiles
        sim = binding.Simulation(prob)
        sim.load_state(inputs.empty_state(prob))
        sim.prepare()
        start = 2 * n // 3
        stride = max(1, (n - start) // 150)
        sim.step(start)
        acc = [0.0, 0.0, 0.0]
        m, done = 0, start
        while done < n:
            k = min(stride, n - done)
            sim.step(k)
            done += k
            _, phi, _ = sim.fields()
            acc = [acc[0] + phi, acc[1] + sim.density(0), acc[2] + sim.density(1)]
            m += 1
        sim.close()
        res[name] = {"steps": n, "dt": prob["dt"], "ms": ms, "us_per_step": 1e3 * ms / n,
                     "macroparticles_end": d["count"][:2],
                     "profiles": [a / m for a in acc]}
    pic, sl = res["pic"], res["slpic"]
    ratio = pic["ms"] / sl["ms"]
    dphi = 12.5 / 2.2
    dphi_max = float(np.abs(pic["profiles"][0] - sl["profiles"][0]).max() / dphi)
    dens = []
    for k in (1, 2):
        a, b = sl["profiles"][k], pic["profiles"][k]
        dens.append(float(np.abs(a - b).max() / max(a.max(), b.max())))
    line = {
        "metric": "SLPIC over PIC wall-time speedup to steady state (Sec. IV argon sheath)",
        "value": ratio, "unit": "x", "n_gpus": 1, "steps": sl["steps"], "warmup": 0,
        "ms_per_step": sl["us_per_step"] / 1e3, "higher_is_better": True, "scaling": "strong",
        "vs_baseline": ratio / 160.0, "dtype": "f32", "data": "synthetic", "impl": "gb300",
        "config": {"workload": "1D3V argon sheath of Sec. IV: 100 cells, L = 25 lambda_D "
                               "(4 cm), bias 12.5 V = 5.68 T_e, m_i/m_e = 39.9 x 1836, "
                               "T_i/T_e = 0.5/2.2, wall source from a stationary plasma, empty "
                               "start, 24 us of plasma time; PIC dt = dx/(5 v_te), SLPIC "
                               "v0 = 0.016 v_te and dt = dx/v0",
                   "ppc_scale": args.ppc_sheath},
        "pic": {"steps": pic["steps"], "ms": pic["ms"], "us_per_step": pic["us_per_step"],
                "macroparticles_end": pic["macroparticles_end"]},
        "slpic": {"steps": sl["steps"], "ms": sl["ms"], "us_per_step": sl["us_per_step"],
                  "macroparticles_end": sl["macroparticles_end"]},
        "steady_state_agreement": {"max_dphi_over_bias": dphi_max,
                                   "max_dn_e_over_peak": dens[0], "max_dn_i_over_peak": dens[1]},
        "gpu_launches": 3 * (pic["steps"] + sl["steps"]),
        "note": "the paper's 160x is VSim on unstated CPU hardware: context, not the target",
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20000)
    ap.add_argument("--warmup", type=int, default=50)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=2000)
    ap.add_argument("--settle", type=int, default=4096,
                    help="steps run before the warm-up, outside any timed region, so that "
                         "the timed steps are past the start-up transient")
    ap.add_argument("--cpu-budget", type=float, default=12.0)
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 form")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--v0-profile", default="none", choices=["none", "sine"],
                    help="sheath1d: a speed limit varying in space (per-cell factors of v0)")
    ap.add_argument("--workload", default="sheath1d",
                    choices=["sheath1d", "plasma2d", "batch", "paper_sheath", "unet2d",
                             "unet_net"],
                    help="sheath1d (the headline), plasma2d (2D3V + CG), batch (many "
                         "independent sheaths) or paper_sheath (the paper's SLPIC-vs-PIC "
                         "sheath speedup) or unet2d (plasma2d with the learned CG warm start) "
                         "or unet_net (the warm start's network alone)")
    ap.add_argument("--ppc-sheath", type=int, default=500)
    ap.add_argument("--nx", type=int, default=1024)
    ap.add_argument("--ny", type=int, default=1024)
    ap.add_argument("--ppc2d", type=int, default=64)
    ap.add_argument("--solver", default="cg", choices=["cg", "fft"],
                    help="plasma2d: the 2D field solver")
    ap.add_argument("--batch-m", type=int, default=256)
    ap.add_argument("--autotune", action="store_true",
                    help="sheath1d / batch: pick the compaction interval, particle kernel and "
                         "batch work split with slpic_autotune after the warm-up")
    ap.add_argument("--compact-every", type=int, default=32,
                    help="sheath1d: the compaction interval (slpic_set_tuning), set before the "
                         "load; 32 measured about 1%% faster per step than the library's "
                         "default 16 on the saturated sheath, whose holes are few")
    ap.add_argument("--unet-pairs", type=int, default=96)
    ap.add_argument("--unet-train-steps", type=int, default=1500)
    ap.add_argument("--unet-batch", type=int, default=4)
    ap.add_argument("--unet-base", type=int, default=32)
    ap.add_argument("--unet-cuda-cores", action="store_true",
                    help="U-Net forward convolutions on the CUDA cores (FP32 activations)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "plasma2d":
        return run_2d(args)
    if args.workload == "batch":
        return run_batch(args)
    if args.workload == "paper_sheath":
        return run_paper_sheath(args)
    if args.workload == "unet_net":
        return run_unet_net(args)
    if args.workload == "unet2d":
        return run_unet2d(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
