"""GPU path vs the FP64 oracle, through the C ABI.

Bars (written into each test):
  * deposits: bit-exact int64 against the quantised rule;
  * fields: the FP64 solve within 1e-12 of the oracle's Thomas solve of the
    same charge (relative to max|phi|), E within FP32 rounding;
  * one push: |v_gpu - v_orc| <= 1e-5 |v| and positions within 1e-5 of the
    displacement plus 4 ulp of the FP32 in-cell offset;
  * sampled full-size step (test_gpu_fullsize): the same per-particle bars at
    4,096 cells and 8.2M particles in the launch configuration the benchmark
    times.
"""
import numpy as np
import pytest
import torch

from oracle import oracle as orc
from paper_1511_08225_gb300 import binding, inputs

from _match import key_of, match, periodic_diff
from _stepcheck import compare_step as _compare_step

pytestmark = pytest.mark.gpu

ONE, HEAV, REL = 0, 1, 2
TWO40 = float(2 ** 40)


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1511_08225_gb300 import build
    build.build()
    binding.load_library()


def _sim(prob, state):
    sim = binding.Simulation(prob)
    sim.load_state(state)
    sim.prepare()
    return sim


def _oracle(prob, state):
    o = orc.OracleSim(prob)
    for s, (c, off, v) in enumerate(state):
        o.load_cells(s, c, off, v)
    o.start()
    return o


def _problem(N=64, periodic=False, kind=HEAV, v0=0.3, dx=0.5, dt=None, phi_hi=0.0,
             ns=2, capacity=None):
    dt = dx / v0 if dt is None else dt
    sps = []
    for s in range(ns):
        q = -1.0 if s == 0 else 1.0
        m = 1.0 if s == 0 else 40.0 * (s + 1)
        sps.append({"name": f"s{s}", "q": q, "m": m, "w": 0.001 * (s + 1), "v0": v0,
                    "kind": kind, "T": 0.0, "capacity": capacity or 1 << 18})
    return {"n_cells": N, "dx": dx, "dt": dt, "periodic": periodic, "phi_lo": 0.0,
            "phi_hi": phi_hi, "eps0": 1.0, "seed": 11, "species": sps,
            "source": {"mode": binding.SLPIC_SRC_NONE}}


def _state(prob, n_per, seed=1, vscale=1.0, nonneutral=False):
    rng = inputs.make_rng(seed)
    out = []
    N = prob["n_cells"]
    for s, n in enumerate(n_per):
        cell, off = inputs.uniform_cells(rng, n, N, 0.0, N / 2 if (nonneutral and s == 0) else N)
        v = rng.normal(0.0, vscale / np.sqrt(prob["species"][s]["m"]), (n, 3)).astype(np.float32)
        out.append((cell, off, v))
    return out


# ------------------------------------------------------------------ deposit
@pytest.mark.parametrize("periodic", [False, True])
@pytest.mark.parametrize("kind", [ONE, HEAV, REL])
@pytest.mark.parametrize("n_per", [(0, 1), (1023, 1025), (100_003, 7), (300_000, 250_001)])
def test_deposit_bitexact(periodic, kind, n_per):
    prob = _problem(N=97, periodic=periodic, kind=kind, v0=0.4, capacity=max(n_per) + 1)
    st = _state(prob, n_per, seed=sum(n_per) + kind)
    sim = _sim(prob, st)
    for s, (c, o, v) in enumerate(st):
        ref = orc.deposit_q40(97, periodic, c, o, v, kind, np.float32(0.4))
        got = sim.charge_raw(s)
        assert np.array_equal(got, ref), f"species {s}"
    sim.close()


# ------------------------------------------------------------------ field solve
@pytest.mark.parametrize("periodic,phi_hi", [(False, 0.0), (False, 3.5), (True, 0.0)])
def test_field_solve_matches_thomas(periodic, phi_hi):
    prob = _problem(N=513, periodic=periodic, phi_hi=phi_hi)
    st = _state(prob, (60_000, 50_000), seed=3, nonneutral=True)
    sim = _sim(prob, st)
    rho_g, phi_g, E_g = sim.fields()
    rho = sum(sp["q"] * sp["w"] / prob["dx"] *
              orc.deposit_q40(513, periodic, c, o, v, HEAV, np.float32(sp["v0"])) / TWO40
              for sp, (c, o, v) in zip(prob["species"], st))
    np.testing.assert_allclose(rho_g, rho, rtol=1e-14, atol=1e-14 * np.abs(rho).max())
    phi = orc.poisson1d(rho, prob["dx"], periodic, 0.0, phi_hi, 1.0)
    E = orc.efield1d(phi, prob["dx"], periodic)
    scale = np.abs(phi).max()
    assert np.abs(phi_g - phi).max() <= 1e-12 * scale
    np.testing.assert_allclose(E_g, E.astype(np.float32), rtol=2e-7,
                               atol=1e-12 * np.abs(E).max() + 1e-30)
    sim.close()


# ------------------------------------------------------------------ one step
@pytest.mark.parametrize("kind", [ONE, HEAV, REL])
@pytest.mark.parametrize("periodic", [False, True])
def test_single_step_matches_oracle(kind, periodic):
    """Strong, non-uniform fields (half the electrons removed, biased plate):
    particles in both beta regimes, crossing v0, reversing, leaving walls."""
    v0 = 0.3
    prob = _problem(N=96, periodic=periodic, kind=kind, v0=v0, dx=0.5,
                    dt=0.5 / (v0 if kind != ONE else 4.0),
                    phi_hi=0.0 if periodic else 2.0)
    st = _state(prob, (40_000, 30_000), seed=5 + kind, vscale=1.0, nonneutral=True)
    gpu = _sim(prob, st)
    o = _oracle(prob, st)
    gpu.step(1)
    gpu.synchronize()
    o.step(1)
    stats = []
    _compare_step(prob, st, gpu, o, stats=stats)
    print("parity", kind, periodic, stats)
    d = gpu.diagnostics()
    for s in range(2):
        assert d["count"][s] == o.x[s].size or abs(d["count"][s] - o.x[s].size) <= 2
    gpu.close()


@pytest.mark.parametrize("n_per", [(1, 3), (7, 0), (151 * 4 + 3, 2), (4_099, 5),
                                   (1984 * 151 + 13, 1)])
def test_single_step_with_ragged_counts_matches_oracle(n_per):
    """The in-place particle kernel splits each species' slots over its CTAs in shares
    whose boundaries are multiples of 4, walked in tiles of 1,984: counts that leave most
    CTAs no slot, a CTA with fewer than 4 slots (no bulk copy of cells), tails of 1 to 3
    cells read one by one, and shares just over one whole tile.  Each is stepped once
    against the oracle (strong field, both beta regimes, a biased plate), and the deposit
    of the stepped particles is the oracle's rule on them, bit for bit."""
    v0 = 0.3
    prob = _problem(N=96, periodic=False, kind=HEAV, v0=v0, dx=0.5, dt=0.5 / v0, phi_hi=2.0,
                    capacity=max(n_per) + 64)
    st = _state(prob, n_per, seed=sum(n_per) + 17, vscale=1.0, nonneutral=True)
    gpu = _sim(prob, st)
    o = _oracle(prob, st)
    gpu.step(1)
    gpu.synchronize()
    o.step(1)
    _compare_step(prob, st, gpu, o)
    for s in range(2):
        c, off, v = gpu.particles(s)
        ref = orc.deposit_q40(96, False, c, off, v, HEAV, np.float32(v0))
        assert np.array_equal(gpu.charge_raw(s), ref), f"species {s}"
    gpu.close()


def test_slow_particles_are_plain_leapfrog_bitwise():
    """Heaviside beta with v0 above every speed: the GPU push is the beta = 1
    push bit for bit (Sec. II: SLPIC identical to PIC)."""
    # v0 = 5 with dt = 0.1 satisfies dt v0 <= dx; the speeds stay far below 5
    prob_a = _problem(N=64, periodic=True, kind=ONE, v0=5.0, dt=0.1)
    prob_b = _problem(N=64, periodic=True, kind=HEAV, v0=5.0, dt=0.1)
    st = _state(prob_a, (20_000, 20_000), seed=8, vscale=0.5)
    a, b = _sim(prob_a, st), _sim(prob_b, st)
    a.step(10)
    b.step(10)
    for s in range(2):
        ca, oa, va = a.particles(s)
        cb, ob, vb = b.particles(s)
        ia, ib = match(key_of(va), key_of(vb))
        assert ia.size == va.shape[0] == vb.shape[0]
        assert np.array_equal(ca[ia], cb[ib]) and np.array_equal(oa[ia], ob[ib])
        assert np.array_equal(va[ia], vb[ib])
        assert np.array_equal(a.charge_raw(s), b.charge_raw(s))
    a.close()
    b.close()


# ------------------------------------------------------------------ multi-step properties
def test_periodic_invariants_over_many_steps():
    """Periodic grid: macro counts never change, and every step's integer
    deposit totals sum_p rint(beta 2^40) over the GPU's own particles."""
    prob = _problem(N=128, periodic=True, kind=HEAV, v0=0.2, dx=0.5)
    st = _state(prob, (50_000, 50_000), seed=9)
    sim = _sim(prob, st)
    for _ in range(5):
        sim.step(4)
        for s in range(2):
            c, o, v = sim.particles(s)
            assert c.size == st[s][0].size
            v = v.astype(np.float32)
            s2 = (v[:, 0] * v[:, 0] + v[:, 1] * v[:, 1]) + v[:, 2] * v[:, 2]
            r = np.sqrt(s2)
            b = np.where(r <= np.float32(0.2), np.float32(1.0), np.float32(0.2) / r)
            qT = np.rint(b.astype(np.float32) * np.float32(TWO40)).astype(np.int64)
            assert int(sim.charge_raw(s).sum()) == int(qT.sum())
    sim.close()


def test_source_injection_matches_oracle():
    """RATE source: the same number of macroparticles per step, at the same
    FP32 positions (integer RNG + pinned FP32 ops), velocities to FP32 libm
    accuracy; the sheath problem's LOSS_MATCHED counts agree step by step."""
    prob = inputs.sheath_problem(n_cells=128, ppc=40, v0=0.2, source_mode=inputs.SRC_RATE,
                                 rate=3.0)
    st = inputs.load_state(prob)
    gpu = _sim(prob, st)
    o = _oracle(prob, st)
    gpu.step(1)
    o.step(1)
    for s in range(2):
        k = int(o.last_injected[s])
        assert k > 0
        c, off, v = gpu.particles(s)
        cg, og, vg = c[-k:], off[-k:], v[-k:]
        xo = o.x[s][-k:]
        xg = (cg.astype(np.float64) + og.astype(np.float64)) * prob["dx"]
        np.testing.assert_array_equal(xg, xo)  # injected positions are bit-exact
        np.testing.assert_allclose(vg, o.v[s][-k:], rtol=2e-6, atol=2e-6 * o.v[s][-k:].std())
    gpu.close()

    prob = inputs.sheath_problem(n_cells=128, ppc=40, v0=0.05)
    st = inputs.load_state(prob)
    gpu = _sim(prob, st)
    o = _oracle(prob, st)
    for _ in range(3):
        gpu.step(1)
        o.step(1)
        d = gpu.diagnostics()
        for s in range(2):
            assert abs(d["count"][s] - o.x[s].size) <= 2
    gpu.close()


@pytest.mark.parametrize("kind", [ONE, HEAV])
def test_wall_source_matches_oracle(kind):
    """Sec. IV wall source into an empty box: per step the same macroparticle
    counts as the oracle; the first step's particles at the oracle's positions
    (FP32 arithmetic on one side, FP64 on the other: a few 1e-6 of the distance
    moved, plus FP32 resolution of the position) and velocities to FP32 libm
    accuracy; the counts stay equal over later steps."""
    prob = inputs.paper_sheath_problem(kind=kind, ppc=200)
    # a denser source plasma, so that the slow ions enter in the first short PIC step
    prob["source"]["rate"] = 100.0
    st = inputs.empty_state(prob)
    gpu = _sim(prob, st)
    o = _oracle(prob, st)
    gpu.step(1)
    o.step(1)
    L = prob["n_cells"] * prob["dx"]
    for s in range(2):
        k = int(o.last_injected[s])
        assert k > 0
        c, off, v = gpu.particles(s)
        assert c.size == o.x[s].size == k
        xg = (c.astype(np.float64) + off.astype(np.float64)) * prob["dx"]
        moved = L - o.x[s]
        tol = 4e-6 * moved + 2.0 ** -24 * L * 2
        assert (np.abs(xg - o.x[s]) <= tol).all(), np.max(np.abs(xg - o.x[s]) - tol)
        np.testing.assert_allclose(v, o.v[s], rtol=4e-6, atol=4e-6 * np.abs(o.v[s]).max())
    injected = np.array([int(o.last_injected[s]) for s in range(2)])
    for _ in range(4):
        gpu.step(1)
        o.step(1)
        injected += o.last_injected
        d = gpu.diagnostics()
        for s in range(2):
            assert d["injected"][s] == injected[s]
            assert abs(d["count"][s] - o.x[s].size) <= 2
    gpu.close()


def test_speed_limit_raised_mid_run_matches_oracle():
    """A speed limit that changes in time (Sec. II, Summary): after 3 steps the
    timestep is halved and v0 doubled (in that order: dt v0 <= dx throughout;
    doubling v0 first is refused).  The next step, from the GPU's own state, agrees
    with the oracle under the new v0 and dt within the single-step bars."""
    v0 = 0.2
    prob = _problem(N=96, periodic=False, kind=HEAV, v0=v0, dx=0.5, phi_hi=1.0)
    st = _state(prob, (30_000, 20_000), seed=31, vscale=1.0, nonneutral=True)
    gpu = _sim(prob, st)
    gpu.step(3)
    with pytest.raises(binding.SlpicError) as ei:
        binding.slpic_set_speed_limit(gpu.h, 0, 0, 2 * v0)
    assert ei.value.code == binding.SLPIC_ERR_CFL
    binding.slpic_set_timestep(gpu.h, prob["dt"] / 2)
    for s in range(2):
        binding.slpic_set_speed_limit(gpu.h, 0, s, 2 * v0)
    new = dict(prob, dt=prob["dt"] / 2,
               species=[dict(sp, v0=2 * v0) for sp in prob["species"]])
    mid = [gpu.particles(s) for s in range(2)]
    # the oracle from the GPU's state: rho^3 and E^3 under the old v0 (as on the
    # GPU), then the new v0 and dt for the step
    old_prob = dict(prob, species=[dict(sp) for sp in prob["species"]])
    o = _oracle(old_prob, mid)
    o.dt = new["dt"]
    for sp in o.sp:
        sp["v0"] = 2 * v0
    gpu.step(1)
    o.step(1)
    stats = []
    _compare_step(new, mid, gpu, o, stats=stats)
    print("after the change", stats)
    gpu.close()


# ------------------------------------------------------------------ API behaviour
def test_checkpoint_restore_is_bitwise():
    prob = inputs.sheath_problem(n_cells=64, ppc=50, v0=0.1)
    st = inputs.load_state(prob)
    a = _sim(prob, st)
    a.step(5)
    blob = a.save()
    a.step(5)
    b = binding.Simulation(prob)
    b.restore(blob)
    b.step(5)
    for s in range(2):
        ca, oa, va = a.particles(s)
        cb, ob, vb = b.particles(s)
        ka, kb = key_of(va), key_of(vb)
        ia, ib = match(ka, kb)
        assert ia.size == ka.size == kb.size
        assert np.array_equal(ca[ia], cb[ib]) and np.array_equal(oa[ia], ob[ib])
        assert np.array_equal(a.charge_raw(s), b.charge_raw(s))
    np.testing.assert_array_equal(a.fields()[1], b.fields()[1])
    a.close()
    b.close()


def test_invalid_loads_are_rejected():
    prob = _problem(N=16)
    sim = binding.Simulation(prob)
    c = np.array([0, 16], np.int32)
    o = np.array([0.1, 0.2], np.float32)
    v = np.zeros((2, 3), np.float32)
    with pytest.raises(binding.SlpicError) as ei:
        sim.load(0, c, o, v)
    assert ei.value.code == binding.SLPIC_ERR_INVALID
    with pytest.raises(binding.SlpicError):
        sim.load(0, np.array([1], np.int32), np.array([1.0], np.float32), np.zeros((1, 3), np.float32))
    with pytest.raises(binding.SlpicError):
        sim.load(0, np.array([1], np.int32), np.array([0.5], np.float32),
                 np.array([[np.nan, 0, 0]], np.float32))
    assert sim.count(0) == 0
    sim.close()


def test_capacity_overflow_is_reported():
    prob = inputs.sheath_problem(n_cells=64, ppc=4, v0=0.1, source_mode=inputs.SRC_RATE,
                                 rate=50.0)
    for sp in prob["species"]:
        sp["capacity"] = 300
    sim = _sim(prob, inputs.load_state(prob))
    sim.step(20)
    with pytest.raises(binding.SlpicError) as ei:
        sim.synchronize()
    assert ei.value.code == binding.SLPIC_ERR_CAPACITY
    assert sim.count(1) <= 300
    sim.close()


def test_empty_species_and_device_load():
    import torch
    prob = _problem(N=32, periodic=True)
    st = _state(prob, (5000, 0), seed=2)
    a = _sim(prob, st)
    b = binding.Simulation(prob)
    c, o, v = st[0]
    binding.slpic_load_particles_dev(b.h, 0, 0, torch.from_numpy(c).cuda(),
                                     torch.from_numpy(o).cuda(), torch.from_numpy(v).cuda())
    b.prepare()
    for sim in (a, b):
        sim.step(3)
    assert a.count(1) == 0 and b.count(1) == 0
    ca, oa, va = a.particles(0)
    cb, ob, vb = b.particles(0)
    ia, ib = match(key_of(va), key_of(vb))
    assert ia.size == 5000
    assert np.array_equal(ca[ia], cb[ib]) and np.array_equal(va[ia], vb[ib])
    a.close()
    b.close()


def test_kernel_timing_records_both_kernels():
    prob = _problem(N=64)
    sim = _sim(prob, _state(prob, (10_000, 10_000)))
    sim.step(5)  # timed blocks start wherever the run is, not only at a cycle start
    binding.slpic_enable_kernel_timing(sim.h, 12)
    sim.step(30)  # two timed replays of 12 steps (the second crosses a compacting step),
    pm, hm, fm, n = binding.slpic_kernel_times(sim.h)  # then 6 untimed steps
    assert n == 12 and pm > 0 and hm > 0 and fm > 0
    assert binding.slpic_kernels_per_step(sim.h) == 3
    assert sim.diagnostics()["step"] == 35
    sim.close()


def test_kernel_spans_count_every_launch_of_the_steps():
    """slpic_kernel_spans: one launch of each kernel per step, device time > 0, and
    for a block of steps the summed spans fit inside the stream's elapsed time."""
    prob = _problem(N=64)
    sim = _sim(prob, _state(prob, (20_000, 20_000)))
    sim.step(3)
    sim.synchronize()
    ms0, n0 = binding.slpic_kernel_spans(sim.h)
    stream = torch.cuda.current_stream()
    binding.slpic_set_stream(sim.h, stream.cuda_stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sim.step(40)
    e1.record(stream)
    e1.synchronize()
    ms1, n1 = binding.slpic_kernel_spans(sim.h)
    assert list(n1 - n0) == [40, 40, 40]
    d = ms1 - ms0
    assert (d > 0).all()
    assert d.sum() <= e0.elapsed_time(e1) * 1.02  # two clocks: allow 2 %
    sim.close()
