"""A speed limit that varies in space (Sec. II), GPU path vs the FP64 oracle,
through the C ABI (slpic_set_speed_limit_profile).  Bars as in
test_gpu_parity: deposits bit-exact against the quantised rule with the limit
v0 lam_c of each particle's cell; one step within the per-particle bars; a
profile of ones bit for bit the uniform run (the profile variants of the kernels
run then); both particle kernels' profile variants bit for bit alike; the
steady free-streaming density of the oracle's pin reproduced."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1511_08225_gb300 import binding, inputs

from test_gpu_parity import _compare_step, _oracle, _problem, _sim, _state

pytestmark = pytest.mark.gpu

ONE, HEAV, REL = 0, 1, 2


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1511_08225_gb300 import build
    build.build()
    binding.load_library()


def _profile(N, seed, lo=0.3, hi=1.0):
    return np.random.default_rng(seed).uniform(lo, hi, N).astype(np.float32)


def _check_deposit(sim, prob, lam):
    """charge_raw of every species == the quantised rule on the GPU's own state."""
    for s, sp in enumerate(prob["species"]):
        c, o, v = sim.particles(s)
        ref = orc.deposit_q40(prob["n_cells"], prob["periodic"], c, o, v, int(sp["kind"]),
                              np.float32(sp["v0"]), lam)
        assert np.array_equal(sim.charge_raw(s), ref), f"species {s}"


@pytest.mark.parametrize("periodic", [False, True])
@pytest.mark.parametrize("kind", [HEAV, REL])
@pytest.mark.parametrize("n_per", [(0, 1), (1023, 1025), (200_003, 7)])
def test_profile_deposit_bitexact(periodic, kind, n_per):
    prob = _problem(N=97, periodic=periodic, kind=kind, v0=0.4, capacity=max(n_per) + 1)
    lam = _profile(97, 1 + kind)
    prob["v0_profile"] = lam
    st = _state(prob, n_per, seed=sum(n_per) + kind)
    sim = _sim(prob, st)
    for s, (c, o, v) in enumerate(st):
        ref = orc.deposit_q40(97, periodic, c, o, v, kind, np.float32(0.4), lam)
        assert np.array_equal(sim.charge_raw(s), ref), f"species {s}"
        # the uniform rule differs wherever a particle is present
        if c.size > 100:
            assert not np.array_equal(ref, orc.deposit_q40(97, periodic, c, o, v, kind,
                                                            np.float32(0.4)))
    sim.close()


@pytest.mark.parametrize("kind", [HEAV, REL])
@pytest.mark.parametrize("periodic", [False, True])
def test_single_step_with_profile_matches_oracle(kind, periodic):
    """The single-step case of test_gpu_parity (strong, non-uniform fields) with
    a random per-cell profile in [0.3, 1]: every particle's push takes the limit
    of its start cell, its deposit that of its end cell."""
    v0 = 0.3
    prob = _problem(N=96, periodic=periodic, kind=kind, v0=v0, dx=0.5, dt=0.5 / v0,
                    phi_hi=0.0 if periodic else 2.0)
    lam = _profile(96, 10 + kind)
    prob["v0_profile"] = lam
    st = _state(prob, (40_000, 30_000), seed=5 + kind, vscale=1.0, nonneutral=True)
    gpu = _sim(prob, st)
    o = _oracle(prob, st)
    gpu.step(1)
    o.step(1)
    stats = []
    _compare_step(prob, st, gpu, o, stats=stats, lam=lam)
    print("profile parity", kind, periodic, stats)
    _check_deposit(gpu, prob, lam)
    gpu.close()


def test_profile_over_many_steps_keeps_the_deposit_rule():
    """A sheath with its source, hard (iterative) pushes and compacting steps under
    a profile: after each burst of steps the deposit is the quantised rule on the
    GPU's own particles, and the diagnostics' physical weight uses each
    particle's own limit."""
    prob = inputs.sheath_problem(n_cells=512, ppc=100, v0=0.05, capacity_factor=2.0)
    N = prob["n_cells"]
    x = (np.arange(N) + 0.5) / N
    lam = (0.55 + 0.45 * np.cos(2 * np.pi * x) ** 2).astype(np.float32)
    prob = dict(prob, v0_profile=lam)
    st = inputs.load_state(prob)
    sim = _sim(prob, st)
    _check_deposit(sim, prob, lam)
    hard = 0
    for n in (1, 15, 17, 40):
        sim.step(n)
        _check_deposit(sim, prob, lam)
        d = sim.diagnostics()
        hard = sum(d["iterative"])
    assert hard > 0
    assert sim.diagnostics()["step"] == 73
    sim.close()


def test_profile_of_ones_is_bitwise_the_uniform_run():
    """lam = 1 everywhere gives v0 * 1 = v0 exactly, so the profile variants of
    the kernels must reproduce the uniform run bit for bit: particles as sets,
    deposits, fields, counters."""
    prob = inputs.sheath_problem(n_cells=512, ppc=200, v0=0.05, capacity_factor=2.0)
    st = inputs.load_state(prob)
    ref = _sim(prob, st)
    one = _sim(dict(prob, v0_profile=np.ones(prob["n_cells"])), st)
    from test_gpu_tuning import _same
    for n in (5, 40, 81):
        ref.step(n)
        one.step(n)
        _same(ref, one)
    ref.close()
    one.close()


@pytest.mark.parametrize("settings", [dict(particle_kernel=1), dict(compact_every=5)])
def test_profile_runs_alike_on_every_kernel(settings):
    """With a profile, the TMA-staged in-place kernel (the default), the per-warp
    one and any compaction interval give the same run bit for bit."""
    prob = inputs.sheath_problem(n_cells=512, ppc=200, v0=0.05, capacity_factor=2.0)
    N = prob["n_cells"]
    prob = dict(prob, v0_profile=_profile(N, 21, 0.4, 1.0))
    st = inputs.load_state(prob)
    a, b = _sim(prob, st), _sim(prob, st)
    binding.slpic_set_tuning(b.h, **settings)
    from test_gpu_tuning import _same
    for n in (7, 40, 66):
        a.step(n)
        b.step(n)
        _same(a, b)
    a.close()
    b.close()


def test_profile_set_mid_run_matches_oracle():
    """Set after 3 uniform steps (and cleared again): the next step from the GPU's
    own state agrees with the oracle under the profile."""
    v0 = 0.25
    prob = _problem(N=80, periodic=False, kind=HEAV, v0=v0, dx=0.5, phi_hi=1.0)
    st = _state(prob, (30_000, 20_000), seed=41, vscale=1.0, nonneutral=True)
    gpu = _sim(prob, st)
    gpu.step(3)
    lam = _profile(80, 7, 0.4, 1.0)
    binding.slpic_set_speed_limit_profile(gpu.h, lam)
    mid = [gpu.particles(s) for s in range(2)]
    o = _oracle(prob, mid)  # rho^3 and E^3 of the uniform limit, as on the GPU
    o.set_profile(lam)
    gpu.step(1)
    o.step(1)
    _compare_step(prob, mid, gpu, o, lam=lam)
    _check_deposit(gpu, prob, lam)
    binding.slpic_set_speed_limit_profile(gpu.h, None)
    gpu.step(2)
    _check_deposit(gpu, prob, None)
    gpu.close()


def test_profile_rejects_bad_input_and_keeps_the_cfl_bound():
    prob = _problem(N=40, periodic=False, kind=HEAV, v0=0.25, dx=0.5, dt=1.0)  # dt v0 = dx / 2
    sim = binding.Simulation(prob)
    for bad in (np.ones(39), np.r_[np.ones(39), 0.0], np.r_[np.ones(39), np.nan],
                np.r_[np.ones(39), -1.0], np.r_[np.ones(39), 1e-300]):
        with pytest.raises(binding.SlpicError) as ei:
            binding.slpic_set_speed_limit_profile(sim.h, bad)
        assert ei.value.code == binding.SLPIC_ERR_INVALID
    with pytest.raises(binding.SlpicError) as ei:  # 0.25 * 1.0 * 2.5 > 0.5
        binding.slpic_set_speed_limit_profile(sim.h, np.r_[np.ones(39), 2.5])
    assert ei.value.code == binding.SLPIC_ERR_CFL
    binding.slpic_set_speed_limit_profile(sim.h, np.r_[np.ones(39), 2.0])  # exactly dx
    with pytest.raises(binding.SlpicError) as ei:
        binding.slpic_set_timestep(sim.h, 1.5)
    assert ei.value.code == binding.SLPIC_ERR_CFL
    with pytest.raises(binding.SlpicError) as ei:
        binding.slpic_set_speed_limit(sim.h, 0, 0, 0.3)
    assert ei.value.code == binding.SLPIC_ERR_CFL
    binding.slpic_set_speed_limit_profile(sim.h, None)
    binding.slpic_set_speed_limit(sim.h, 0, 0, 0.3)
    sim.close()
    b = binding.Batch([prob, prob])
    with pytest.raises(binding.SlpicError) as ei:
        binding.slpic_set_speed_limit_profile(b.h, np.ones(40))
    assert ei.value.code == binding.SLPIC_ERR_INVALID
    b.close()


def test_steady_free_streaming_density_with_profile():
    """The oracle's steady-state pin on the GPU: E = 0 (q = 0), a wall source of
    density n_s; after the transient the time-averaged physical density is n_s/2
    with the uniform limit and with lam from 0.5 to 1 alike, while the
    macroparticle count grows as 1/lam."""
    N, dx, v0, n_s, w = 32, 0.5, 0.5, 5.0, 0.01
    lam = (0.5 + 0.5 * np.arange(N) / (N - 1)).astype(np.float32)

    def problem(profile):
        sp = {"name": "n", "q": 0.0, "m": 1.0, "w": w, "v0": v0, "kind": HEAV, "T": 1.0,
              "capacity": 1 << 16}
        p = {"n_cells": N, "dx": dx, "dt": dx / v0, "periodic": False, "phi_lo": 0.0,
             "phi_hi": 0.0, "eps0": 1.0, "seed": 7, "species": [sp],
             "source": {"mode": binding.SLPIC_SRC_WALL, "lo_cells": 0.0, "len_cells": 0.0,
                        "rate": n_s, "ref_species": 0}}
        if profile:
            p["v0_profile"] = lam
        return p

    out = {}
    for profile in (False, True):
        prob = problem(profile)
        sim = _sim(prob, inputs.empty_state(prob))
        sim.step(1000)
        dens = np.zeros(N + 1)
        count = np.zeros(N)
        for _ in range(600):
            sim.step(1)
            dens += sim.charge_raw(0) * (w / dx / 2.0 ** 40)
            count += np.bincount(sim.particles(0)[0], minlength=N)
        out[profile] = (dens / 600, count / 600)
        sim.close()
    inner = slice(1, N)
    for profile in (False, True):
        assert np.abs(out[profile][0][inner] / (n_s / 2) - 1.0).max() < 0.05, profile
    ratio = out[True][0][inner] / out[False][0][inner]
    assert np.abs(ratio - 1.0).max() < 0.02, ratio
    crat = out[True][1][:-1] / out[False][1][:-1]
    assert np.abs(crat * lam[:-1] - 1.0).max() < 0.06, crat
