"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test ties one oracle function to something other than itself: closed
forms, an independent integration route, invariants of the method, special
cases that reduce to plain PIC, or values printed in the paper.  All run on
the CPU in a few seconds.
"""
import math
import os

import numpy as np
import pytest

from oracle import oracle as orc
from paper_1511_08225_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
ONE, HEAV, REL = orc.BETA_ONE, orc.BETA_HEAVISIDE, orc.BETA_RELATIVISTIC


# ------------------------------------------------------------------ beta (Sec. II)
def test_beta_functions_limit_speed():
    """Eqs. (heavisideBeta)/(relativisticBeta): beta in (0,1], |beta v| <= v0,
    beta ~ 1 well below v0 and ~ v0/|v| well above it (Fig. 1's curves)."""
    v0 = 0.3
    for r in np.linspace(0.0, 20.0, 401):
        bh, br = orc.beta(HEAV, r, v0), orc.beta(REL, r, v0)
        assert 0.0 < bh <= 1.0 and 0.0 < br <= 1.0
        assert bh * r <= v0 * (1 + 1e-15) or r <= v0
        assert br * r < v0
        if r <= v0:
            assert bh == 1.0
        else:
            assert bh * r == pytest.approx(v0, rel=1e-15)
    assert orc.beta(REL, 0.0, v0) == 1.0
    assert orc.beta(REL, 1e4 * v0, v0) * 1e4 * v0 == pytest.approx(v0, rel=1e-8)
    assert orc.beta(ONE, 123.0, v0) == 1.0


# ------------------------------------------------------------------ the velocity integral
def _cases(n, seed=7):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        u = rng.normal(0, 1.0, 3) * rng.choice([0.01, 0.1, 1.0, 3.0])
        a = rng.normal(0, 1.0, 3) * rng.choice([1e-4, 1e-2, 0.3, 3.0])
        if rng.random() < 0.3:  # 1D-field cases (a along x)
            a[1:] = 0.0
        if rng.random() < 0.15:  # velocity parallel to a: speed passes through zero
            u = a / np.linalg.norm(a) * rng.normal(0, 1.0)
        v0 = rng.choice([0.01, 0.05, 0.2, 1.0])
        dt = rng.choice([0.2, 1.0, 10.0])
        out.append((u, a, dt, v0))
    return out


@pytest.mark.parametrize("kind", [HEAV, REL])
def test_beta_integral_matches_closed_form(kind):
    """tau* by quadrature on the velocity line vs bisection on the analytic
    antiderivative int sqrt(w^2+D) dw (independent derivation).  The closed
    form is a difference of two antiderivative values of size ~|u|^2/v0, so
    its own error is ~eps |u|^2 / (|a| v0 dt) relative; the tolerance adds
    that conditioning bound to 2e-9."""
    eps = np.finfo(float).eps
    for u, a, dt, v0 in _cases(300, seed=11 + kind):
        t_q = orc.beta_integral(kind, u, a, dt, v0)
        t_c = orc.beta_integral_closed(kind, u, a, dt, v0)
        assert 0.0 < t_q <= dt * (1 + 1e-15)
        cond = eps * (np.dot(u, u) + v0 * v0) / (np.linalg.norm(a) * v0 * dt)
        assert t_q == pytest.approx(t_c, rel=2e-9 + 50 * cond, abs=1e-13 * dt)


@pytest.mark.parametrize("kind", [HEAV, REL])
def test_beta_integral_matches_bruteforce_rk4(kind):
    """Brute-force RK4 of Eq. (LimPtclDyn) with 2e5 substeps: the velocity
    reached and int beta dt agree with v = u + a tau*."""
    for u, a, dt, v0 in _cases(12, seed=3 + kind):
        tau = orc.beta_integral(kind, u, a, dt, v0)
        out = orc.rk4_limited(kind, u, a, dt, v0, n_sub=200_000)
        vq = np.asarray(u) + np.asarray(a) * tau
        assert out[6] == pytest.approx(tau, rel=1e-7, abs=1e-12)
        np.testing.assert_allclose(out[:3], vq, rtol=1e-7, atol=1e-9 * (1 + np.abs(vq).max()))


def test_beta_one_is_plain_leapfrog_time():
    """beta == 1 (Sec. II): the integral is dt exactly, so the push is PIC's."""
    u, a = np.array([0.3, -2.0, 1.0]), np.array([5.0, 0.0, 0.0])
    assert orc.beta_integral(ONE, u, a, 0.37, 0.1) == 0.37


def test_heaviside_below_limit_is_exactly_pic():
    """Heaviside beta with v0 above every speed reached in the step: beta = 1
    all step (Sec. II, 'SLPIC becomes identical to PIC'), tau* = dt exactly."""
    u, a, dt = np.array([0.2, 0.1, -0.1]), np.array([0.05, 0.0, 0.0]), 2.0
    assert orc.beta_integral(HEAV, u, a, dt, v0=1.0) == dt


def test_zero_field_gives_beta_times_dt():
    """a = 0: v stays fixed, so int beta dt = beta(|u|) dt (free streaming)."""
    u = np.array([2.0, 0.0, 0.0])
    for kind, v0 in ((HEAV, 0.5), (REL, 0.5)):
        assert orc.beta_integral(kind, u, np.zeros(3), 3.0, v0) == pytest.approx(
            orc.beta(kind, 2.0, v0) * 3.0, rel=1e-15)


def test_fast_1d1v_particle_closed_form():
    """1D1V Heaviside, |v| > v0 all step, no reversal: d(v^2)/dt = 2 a v0 sgn(v),
    so v^2 changes linearly in t (derived from Eq. LimPtclDyn)."""
    u, a, dt, v0 = 1.5, 0.2, 4.0, 0.05
    v_end = math.sqrt(u * u + 2 * a * v0 * dt)
    vq = orc.push_velocity(HEAV, [u, 0, 0], [a, 0, 0], dt, v0)[0]
    assert vq == pytest.approx(v_end, rel=1e-13)


def test_paper_modified_midpoint_converges_to_integral():
    """Appendix A evaluates the integral by modified midpoint subdivided until
    1% convergence; tightening the tolerance converges to tau*."""
    for u, a, dt, v0 in _cases(40, seed=5):
        for kind in (HEAV, REL):
            exact = orc.beta_integral(kind, u, a, dt, v0)
            t1, n1 = orc.beta_integral_mmid(kind, u, a, dt, v0, 1e-2)
            t8, n8 = orc.beta_integral_mmid(kind, u, a, dt, v0, 1e-9)
            assert t1 == pytest.approx(exact, rel=3e-2)
            assert t8 == pytest.approx(exact, rel=1e-6)
            assert n8 >= n1


# ------------------------------------------------------------------ Poisson (Appendix A)
@pytest.mark.parametrize("N,dx", [(8, 0.5), (100, 0.04), (4096, 0.5)])
def test_poisson_dirichlet_uniform_rho_is_parabola(N, dx):
    """Uniform rho with phi = 0 walls: phi = rho x (L - x) / (2 eps0); the
    3-point stencil is exact on quadratics, so only roundoff remains."""
    rho = np.full(N + 1, 0.7)
    phi = orc.poisson1d(rho, dx, periodic=False, eps0=1.3)
    x = np.arange(N + 1) * dx
    ref = 0.7 * x * (N * dx - x) / (2 * 1.3)
    np.testing.assert_allclose(phi, ref, rtol=0, atol=1e-12 * ref.max() * N)


def test_poisson_dirichlet_bias_is_linear():
    """rho = 0 between plates at phi_lo, phi_hi (Sec. IV's biased plates):
    phi is the straight line and E is the uniform field -(phi_hi-phi_lo)/L."""
    N, dx = 100, 0.04
    phi = orc.poisson1d(np.zeros(N + 1), dx, False, phi_lo=0.0, phi_hi=12.5)
    np.testing.assert_allclose(phi, np.linspace(0.0, 12.5, N + 1), rtol=0, atol=1e-12)
    E = orc.efield1d(phi, dx, False)
    np.testing.assert_allclose(E, -12.5 / (N * dx), rtol=1e-12)


@pytest.mark.parametrize("m", [1, 3, 17])
def test_poisson_periodic_sinusoid_discrete_eigenvalue(m):
    """rho = sin(kx) + const on a periodic grid: the constant is removed
    (neutralising background) and phi = sin(kx) / (eps0 K^2), with
    K = (2/dx) sin(k dx / 2) the stencil's exact eigenvalue."""
    N, dx = 256, 0.5
    k = 2 * math.pi * m / (N * dx)
    x = np.arange(N) * dx
    phi = orc.poisson1d(np.sin(k * x) + 0.25, dx, periodic=True)
    K = 2.0 / dx * math.sin(k * dx / 2)
    np.testing.assert_allclose(phi, np.sin(k * x) / K ** 2, rtol=0, atol=1e-10)
    assert abs(phi.mean()) < 1e-12


def test_efield_centred_difference_of_linear_and_sine():
    N, dx = 64, 0.25
    x = np.arange(N) * dx
    k = 2 * math.pi / (N * dx)
    E = orc.efield1d(np.sin(k * x), dx, periodic=True)
    np.testing.assert_allclose(E, -np.cos(k * x) * math.sin(k * dx) / dx, atol=1e-13)


# ------------------------------------------------------------------ deposits
def test_q40_rule_single_particles():
    """The integer deposit rule on hand-checked particles: beta = 1 at rest,
    beta = 1/2 at |v| = 2 v0 (Heaviside), relativistic beta = 1/sqrt(2) at
    |v| = v0; offsets split qT into (1-d, d) parts exactly."""
    two40 = 2 ** 40
    acc = orc.deposit_q40(4, False, [1], [0.25], [[0, 0, 0]], HEAV, 0.5)
    assert acc.tolist() == [0, 3 * two40 // 4, two40 // 4, 0, 0]
    acc = orc.deposit_q40(4, False, [2], [0.5], [[0.6, 0.0, 0.8]], HEAV, 0.5)
    assert acc.tolist() == [0, 0, two40 // 4, two40 // 4, 0]
    acc = orc.deposit_q40(4, True, [3], [0.5], [[0.6, 0.0, 0.8]], HEAV, 0.5)
    assert acc.tolist() == [two40 // 4, 0, 0, two40 // 4]
    b = float(orc.beta_f32(REL, 1.0, 0.0, 0.0, 1.0))
    assert b == pytest.approx(1 / math.sqrt(2), rel=1e-7)


def test_q40_sum_equals_particle_total_and_fp64_deposit():
    """Integer sums are exact: sum_j acc_j = sum_p rint(beta 2^40); and the
    quantised deposit agrees with the FP64 deposit to FP32 rounding."""
    rng = inputs.make_rng(1)
    N = 37
    cell, off, v = inputs.random_state(rng, 5000, N, vscale=0.4)
    for periodic in (False, True):
        acc = orc.deposit_q40(N, periodic, cell, off, v, HEAV, 0.3)
        qT = [int(np.rint(np.float32(orc.beta_f32(HEAV, *vv, 0.3)) * np.float32(2 ** 40)))
              for vv in v]
        assert int(acc.sum()) == sum(qT)
        dens = np.zeros(N if periodic else N + 1)
        x = (cell.astype(np.float64) + off.astype(np.float64)) * 1.0
        orc.lib().orc_deposit1d(N, int(periodic), 1.0, x.size, orc._ptr(x),
                                orc._ptr(np.ascontiguousarray(v, dtype=np.float64)), None,
                                HEAV, 0.3, None, 1.0, orc._ptr(dens))
        np.testing.assert_allclose(acc / 2.0 ** 40, dens, rtol=1e-5, atol=1e-5)


# ------------------------------------------------------------------ whole steps
def _tiny_periodic(kind, v0, ppc=40, N=32, seed=3, T_e=1.0, load_kind=None):
    prob = inputs.periodic_problem(n_cells=N, dx=0.5, dt=0.2, ppc=ppc, v0=v0,
                                   kind=kind if load_kind is None else load_kind,
                                   seed=seed, T_e=T_e, T_i=T_e)
    st = inputs.load_state(prob)
    for sp in prob["species"]:
        sp["kind"] = kind
    sim = orc.OracleSim(prob)
    for s, (c, o, v) in enumerate(st):
        sim.load_cells(s, c, o, v)
    sim.start()
    return prob, sim


def test_heaviside_above_all_speeds_equals_plain_pic_bitwise():
    """Sec. II: with v0 above every particle speed, Heaviside SLPIC and PIC
    (beta == 1) are the same algorithm; the FP64 states agree bit for bit."""
    _, a = _tiny_periodic(ONE, 1e3, load_kind=ONE)
    _, b = _tiny_periodic(HEAV, 1e3, load_kind=ONE)
    a.step(15)
    b.step(15)
    for s in range(2):
        assert np.array_equal(a.x[s], b.x[s]) and np.array_equal(a.v[s], b.v[s])


def test_periodic_charge_and_count_conservation():
    """Periodic grid: the macro count never changes, and the deposited charge
    equals sum_p w beta(|v^{n+1/2}|) every step (Appendix A's rho)."""
    prob, sim = _tiny_periodic(HEAV, 0.2)
    n0 = [sim.x[s].size for s in range(2)]
    for _ in range(5):
        sim.step()
        d = sim.diagnostics()
        for s in range(2):
            assert sim.x[s].size == n0[s]
            assert sim.dens[s].sum() * sim.dx == pytest.approx(d["sum_wbeta"][s], rel=1e-12)


def test_beta_one_periodic_momentum_conserved():
    """beta == 1 with the same linear shape for gather and scatter, nodal
    centred E and a periodic grid: the total force sum_p q w E(x_p) vanishes,
    so sum_p m w v is constant to roundoff (Birdsall-Langdon momentum
    conservation, the plain-PIC limit of Sec. II)."""
    prob, sim = _tiny_periodic(ONE, 1.0)
    def mom():
        return sum(float(sp["m"]) * float(sp["w"]) * sim.v[s][:, 0].sum()
                   for s, sp in enumerate(prob["species"]))
    p0 = mom()
    scale = sum(float(sp["m"]) * float(sp["w"]) * np.abs(sim.v[s][:, 0]).sum()
                for s, sp in enumerate(prob["species"]))
    sim.step(20)
    assert abs(mom() - p0) <= 1e-12 * scale


def test_free_streaming_at_limited_speed():
    """Zero charge, hence zero field: each step moves x by beta(|v|) v_x dt,
    i.e. the speed along x is min(|v|, v0) * v_x/|v| (Sec. II, Eq. LimPtclDyn)."""
    prob = inputs.periodic_problem(n_cells=16, dx=1.0, dt=0.5, ppc=4, v0=0.7)
    for sp in prob["species"]:
        sp["q"] = 0.0
    rng = inputs.make_rng(2)
    sim = orc.OracleSim(prob)
    cell, off, v = inputs.random_state(rng, 64, 16, vscale=1.5)
    sim.load_cells(0, cell, off, v)
    sim.start()
    x0 = sim.x[0].copy()
    v64 = v.astype(np.float64)
    r = np.sqrt((v64 ** 2).sum(1))
    speed = np.minimum(r, 0.7) * v64[:, 0] / r
    sim.step(6)
    L = 16.0
    expect = np.mod(x0 + 6 * 0.5 * speed, L)
    d = (sim.x[0] - expect + L / 2) % L - L / 2
    assert np.abs(d).max() < 1e-12
    assert np.array_equal(sim.v[0], v64)


def test_cold_plasma_oscillates_at_leapfrog_plasma_frequency():
    """Cold electrons on a neutralising background, mode-1 displacement:
    beta = 1 below v0 (Sec. III: beta = 1 recovers omega = omega_p), and the
    leapfrog frequency is (2/dt) asin(omega_p dt / 2) = 1.001674 omega_p at
    dt = 0.2 (textbook leapfrog dispersion).  Measured from zero crossings of
    the mode amplitude; tolerance 1e-3, which excludes omega_p itself."""
    N, dx, dt, ppc = 256, 0.5, 0.2, 4
    L = N * dx
    prob = {"n_cells": N, "dx": dx, "dt": dt, "periodic": True, "phi_lo": 0.0,
            "phi_hi": 0.0, "eps0": 1.0, "seed": 1,
            "species": [{"name": "e", "q": -1.0, "m": 1.0, "w": dx / ppc, "v0": 10.0,
                         "kind": HEAV, "T": 0.0}],
            "source": {"mode": orc.SRC_NONE}}
    sim = orc.OracleSim(prob)
    x = (np.arange(N * ppc) + 0.5) * (L / (N * ppc))
    k = 2 * math.pi / L
    x = x + 0.01 * np.sin(k * x)
    sim.load(0, x, np.zeros((x.size, 3)))
    sim.start()
    amp = []
    for _ in range(160):
        # a displacement 0.01 sin(kx) perturbs the density as cos(kx)
        amp.append(float((sim.rho * np.cos(k * np.arange(N) * dx)).sum()))
        sim.step()
    amp = np.array(amp)
    zc = [i + amp[i] / (amp[i] - amp[i + 1]) for i in range(len(amp) - 1)
          if amp[i] * amp[i + 1] < 0]
    periods = 2 * np.diff(zc) * dt
    omega = 2 * math.pi / periods.mean()
    expect = 2 / dt * math.asin(dt / 2)
    assert omega == pytest.approx(expect, rel=1e-3)
    assert abs(omega - 1.0) > 1e-3


# ------------------------------------------------------------------ source
def test_splitmix64_published_vector():
    vals = [int(l) for l in open(os.path.join(GOLDEN, "splitmix64_seed1234567.txt"))
            if l.strip() and not l.startswith("#")]
    assert [orc.splitmix64_at(1234567, i) for i in range(5)] == vals


def test_injected_particles_are_physical_maxwellian_in_band():
    """Source particles: positions uniform in the band, each velocity component
    N(0, T/m) (a physical Maxwellian, the f-source equals the g-source)."""
    n = 200_000
    x = np.zeros(n)
    v = np.zeros((n, 3))
    orc.lib().orc_inject(5, 3, 1, n, np.float32(10.0), np.float32(4.0), 0.5, 0.3,
                         orc._ptr(x), orc._ptr(v))
    assert x.min() >= 5.0 and x.max() <= 7.0
    assert abs(x.mean() - 6.0) < 0.01
    np.testing.assert_allclose(v.std(axis=0), 0.3, rtol=0.01)
    np.testing.assert_allclose(v.mean(axis=0), 0.0, atol=0.003)


def test_loss_matched_injection_counts():
    """LOSS_MATCHED: the physical count of absorbed reference particles
    (w per macroparticle) re-enters as S/w_s macroparticles per species, with
    the fractional remainder carried over."""
    prob = inputs.sheath_problem(n_cells=64, ppc=10, v0=0.05)
    sim = orc.OracleSim(prob)
    we, wi = prob["species"][0]["w"], prob["species"][1]["w"]
    sim.last_absorbed[1] = [3, 4]
    k = sim.injection_counts()
    assert k[1] == 7
    assert k[0] == int(math.floor(7 * wi / we))
    assert sim.frac[0] == pytest.approx(7 * wi / we - k[0])


# ------------------------------------------------------------------ loader vs paper numbers
def test_maxwellian_speed_tails_match_paper_sec4():
    """Sec. IV: ~3% of a 3V Maxwellian exceed 3 v_te, < 0.002% exceed 5 v_te."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "maxwellian_tail_fractions.txt"))
            if l.strip() and not l.startswith("#")]
    rng = inputs.make_rng(9)
    v = inputs.g_velocities(rng, 2_000_000, 1.0, 1e9, inputs.BETA_ONE)
    r = np.sqrt((v ** 2).sum(1))
    for thr, frac, rel in rows:
        f = float((r > float(thr)).mean())
        if rel == "approx":
            assert f == pytest.approx(float(frac), rel=0.05)
        else:
            assert f < float(frac)


def test_g_load_weight_counts_physical_density():
    """A speed-limited load samples g0 = f0/beta; with w = n0 dx <1/beta>/ppc
    the physical density sum(w beta)/L equals n0 (f = beta g, Sec. II)."""
    rng = inputs.make_rng(4)
    v0 = 0.1
    sp = inputs.species("e", -1, 1, 1.0, v0, HEAV, ppc=1000, dx=0.5)
    v = inputs.g_velocities(rng, 400_000, 1.0, v0, HEAV)
    r = np.sqrt((v ** 2).sum(1))
    b = np.where(r <= v0, 1.0, v0 / r)
    dens = sp["w"] * b.sum() / (400_000 / 1000 * 0.5)
    assert dens == pytest.approx(1.0, rel=5e-3)
    # and the physical speed distribution is Maxwellian: <beta |v|^2> / <beta> = 3 T
    assert (b * r * r).sum() / b.sum() == pytest.approx(3.0, rel=1e-2)


# ------------------------------------------------------------------ wall source (Sec. IV)
def _wall_draw(kind, v0, n=200_000, vth=1.3, dt=0.7, dx=0.5, n_cells=40):
    x, v = np.zeros(n), np.zeros((n, 3))
    orc.lib().orc_inject_wall(7, 5, 1, n, n_cells, dx, dt, vth, kind, v0, orc._ptr(x),
                              orc._ptr(v))
    return x, v


@pytest.mark.parametrize("kind", [0, 1])
def test_wall_source_distribution(kind):
    """Flux-weighted half-Maxwellian through x = L: vx < 0 with |vx| Rayleigh
    (mean vth sqrt(pi/2), second moment 2 vth^2), vy and vz Maxwellian, and the
    distance moved since entry, L - x = u beta |vx| dt, with u uniform."""
    vth, dt, dx, N, v0 = 1.3, 0.7, 0.5, 40, 0.6
    x, v = _wall_draw(kind, v0, vth=vth, dt=dt, dx=dx, n_cells=N)
    L = N * dx
    assert (v[:, 0] < 0).all() and (x < L).all() and (x > 0).all()
    a = -v[:, 0]
    assert abs(a.mean() / (vth * np.sqrt(np.pi / 2)) - 1) < 0.01
    assert abs((a * a).mean() / (2 * vth * vth) - 1) < 0.01
    for k in (1, 2):
        assert abs(v[:, k].std() / vth - 1) < 0.01 and abs(v[:, k].mean()) < 0.01 * vth
    b = orc._beta_vec(kind, np.linalg.norm(v, axis=1), v0)
    u = (L - x) / (b * a * dt)
    assert u.max() <= 1.0 + 1e-12 and abs(u.mean() - 0.5) < 0.005
    assert abs(np.quantile(u, 0.25) - 0.25) < 0.005


def test_wall_source_counts_follow_the_flux():
    """Over K steps the macroparticles injected per species total
    floor(K n vth / sqrt(2 pi) dt / w) (the fraction is carried)."""
    prob = inputs.paper_sheath_problem(kind=inputs.BETA_ONE, ppc=20)
    o = orc.OracleSim(prob)
    o.start()
    tot = np.zeros(2, np.int64)
    K = 40
    for _ in range(K):
        o.push()
        o.inject()
        tot += o.last_injected
        o.deposit()
        o.solve()
        o.step_index += 1
    for s, sp in enumerate(prob["species"]):
        rate = np.sqrt(sp["T"] / sp["m"]) / np.sqrt(2 * np.pi) * prob["dt"] / sp["w"]
        assert abs(tot[s] - np.floor(K * rate)) <= 1


@pytest.mark.parametrize("kind", [inputs.BETA_ONE, inputs.BETA_HEAVISIDE])
def test_wall_source_fills_half_density(kind):
    """Neutral test particles (q = 0) entering from a stationary plasma of
    density 1 and leaving through the far plate stream across at the density of
    the half-Maxwellian that moves inwards: 1/2 everywhere.  For the speed-limited
    form this is the physical density sum w beta S / dx of the g-particles, so the
    check pins the flux, the half-Maxwellian and the g = f/beta weighting of the
    source (Sec. II) at once."""
    N, dx = 20, 1.0
    v0 = 0.5
    dt = 1.0 if kind == inputs.BETA_ONE else dx / v0
    sp = inputs.species("n", 0.0, 1.0, 1.0, v0, kind, ppc=100, dx=dx)
    sp["w"] = 0.5 * dx / 100
    sp["capacity"] = 100_000
    prob = {"n_cells": N, "dx": dx, "dt": dt, "periodic": False, "phi_lo": 0.0, "phi_hi": 0.0,
            "eps0": 1.0, "seed": 3, "species": [sp],
            "source": {"mode": inputs.SRC_WALL, "lo_cells": 0.0, "len_cells": 0.0, "rate": 1.0,
                       "ref_species": 0}}
    o = orc.OracleSim(prob)
    o.start()
    t_end = 1000.0
    n = int(t_end / dt)
    o.step(int(0.8 * n))
    acc, m = np.zeros(N + 1), 0
    for _ in range(n - int(0.8 * n)):
        o.step(1)
        acc += o.dens[0]
        m += 1
    prof = acc[1:N] / m
    assert abs(prof.mean() - 0.5) < 0.015, prof.mean()
    assert np.abs(prof - 0.5).max() < 0.08, prof


# ------------------------------------------------------------------ prescribed wave (Sec. V)
def test_prescribed_wave_frame_energy_is_conserved():
    """Test particles (beta = 1) in the travelling wave phi0 sin(k (x - vphi t)):
    in the wave frame the potential is static, so after the ramp
    (v - vphi)^2 / 2 + (q/m) phi(x, t) is a constant of each particle's motion; the
    leapfrog keeps it to O(dt^2).  A wrong sign of E, of the phase or of the wave
    speed breaks this by O(1)."""
    N, dx = 200, 0.5
    L = N * dx
    k = 2 * np.pi / L
    prob = inputs.periodic_problem(n_cells=N, dx=dx, dt=0.1, ppc=1, kind=inputs.BETA_ONE)
    prob["species"] = prob["species"][:1]
    prob["wave"] = {"phi0": 0.1, "k": k, "vphi": 1.0, "ramp": 0.0}
    o = orc.OracleSim(prob)
    rng = np.random.default_rng(2)
    n = 64
    x = rng.uniform(0, L, n)
    v = np.zeros((n, 3))
    v[:, 0] = 1.0 + rng.uniform(-0.8, 0.8, n)
    o.load(0, x, v)
    o.start()
    qm = prob["species"][0]["q"] / prob["species"][0]["m"]

    def energy():
        t = o.step_index * o.dt
        # v is v^{n-1/2}: compare at the same phase of the leapfrog each time
        return 0.5 * (o.v[0][:, 0] - 1.0) ** 2 + qm * 0.1 * np.sin(k * (o.x[0] - t))

    e0 = energy()
    for _ in range(40):
        o.step(50)
        assert np.abs(energy() - e0).max() < 0.02
    # and the field is the one prescribed
    t = o.step_index * o.dt
    xj = np.arange(N) * dx
    assert np.abs(o.E + 0.1 * k * np.cos(k * (xj - t))).max() < 1e-12
