"""Parity of the 2D CUDA path (include/slpic2d.h) with the FP64 oracle.

Bars: deposits bit-exact (the 2D quantised rule); the CG potential within
cond(A) * rtol of the oracle's direct solve, in at most twice the oracle's CG
iterations plus 50; one step's velocities within 1e-5 |v| of the oracle and positions
within the move that error causes (1e-5 beta |v| dt) plus 8 ulp of the FP32
offset, particles matched by vz (a has no z component, so vz is unchanged by
the push and identifies a particle on both sides)."""
import math

import numpy as np
import pytest

from oracle import oracle as orc
from paper_1511_08225_gb300 import binding2d, inputs

pytestmark = pytest.mark.gpu

TWO40 = 2.0 ** 40


def _unique_vz(state):
    """Make every vz bit pattern unique within a species (nudging repeats by one
    ulp), so vz can key the particle matching."""
    out = []
    for c, o, v in state:
        v = v.copy()
        bits = v[:, 2].view(np.uint32)
        _, first = np.unique(bits, return_index=True)
        dup = np.setdiff1d(np.arange(bits.size), first)
        for d in dup:
            x = v[d, 2]
            while True:
                x = np.nextafter(x, np.float32(np.inf), dtype=np.float32)
                if not np.any(v[:, 2].view(np.uint32) == np.float32(x).view(np.uint32)):
                    break
            v[d, 2] = x
        out.append((c, o, v))
    return out


def _prob(nx=32, ny=24, ppc=12, kind=inputs.BETA_HEAVISIDE, v0=0.35, dx=0.5, dt=None,
          source=inputs.SRC_NONE, rate=0.0, phi_hi=0.0, cg_rtol=1e-11):
    p = inputs.plasma2d_problem(nx=nx, ny=ny, dx=dx, v0=v0, ppc=ppc, kind=kind, dt=dt,
                                mass_ratio=25.0, T_i=0.5, source_mode=source, rate=rate,
                                cg_rtol=cg_rtol)
    p["phi_hi"] = phi_hi
    return p


def _nonneutral(state, frac=0.4, seed=1):
    """Drop part of the electrons in one half of the box: strong, non-uniform E."""
    rng = np.random.default_rng(seed)
    c, o, v = state[0]
    drop = (rng.random(c.size) < frac) & ((c % 1000) % 2 == 0)
    return [(c[~drop], o[~drop], v[~drop])] + list(state[1:])


def _sim(prob, st):
    g = binding2d.Simulation2D(prob)
    g.load_state(st)
    g.prepare()
    return g


def _oracle(prob, st):
    o = orc.OracleSim2D(prob)
    for s, (c, off, v) in enumerate(st):
        o.load_cells(s, c, off, v)
    o.start()
    return o


def _cond(ny):
    return 8.0 / (4.0 * math.sin(math.pi / (2 * ny)) ** 2)


@pytest.mark.parametrize("kind", [inputs.BETA_ONE, inputs.BETA_HEAVISIDE,
                                  inputs.BETA_RELATIVISTIC])
def test_deposit2d_bit_exact(kind):
    prob = _prob(nx=40, ny=30, ppc=20, kind=kind, v0=0.5, dt=0.5 if kind else 0.2)
    st = inputs.load_state2d(prob, seed=3 + kind)
    g = _sim(prob, st)
    for s, (c, o, v) in enumerate(st):
        ref = orc.deposit2d_q40(40, 30, c, o, v, kind, prob["species"][s]["v0"])
        got = g.charge_raw(s)
        assert np.array_equal(got, ref)
    g.close()


def test_cg_solve_matches_direct_solver():
    """The cooperative CG kernel (FP32 iterates, FP64 right-hand side, solution and
    true residual): the true residual meets rtol, the answer is the oracle's
    direct solve within cond(A) rtol, the iterations stay within twice the
    oracle's FP64 CG plus 50, and a solve warm-started from the answer takes 0
    iterations."""
    nx, ny, dx = 96, 72, 0.6
    prob = _prob(nx=nx, ny=ny, ppc=1, dx=dx, cg_rtol=1e-9)
    prob["phi_lo"], prob["phi_hi"] = 0.4, -0.2
    g = binding2d.Simulation2D(prob)
    rng = np.random.default_rng(5)
    rho = rng.normal(size=(ny + 1, nx))
    phi, it, res = g.solve_poisson(rho)
    exact = orc.poisson2d_direct(rho, dx, 0.4, -0.2)
    _, it_o, _ = orc.poisson2d_cg(rho, dx, None, 0.4, -0.2, rtol=1e-9)
    assert res <= 1e-9
    assert 0 < it <= 2 * it_o + 50, (it, it_o)
    assert np.abs(phi - exact).max() <= _cond(ny) * 1e-9 * np.abs(exact).max()
    assert np.all(phi[0] == 0.4) and np.all(phi[-1] == -0.2)
    _, it0, _ = g.solve_poisson(rho, exact)
    assert it0 == 0
    g.close()


def test_cg_reports_nonconvergence_and_stays_usable():
    prob = _prob(nx=64, ny=64, ppc=1, cg_rtol=1e-12)
    prob["cg_maxit"] = 3
    g = binding2d.Simulation2D(prob)
    rho = np.random.default_rng(1).normal(size=(65, 64))
    with pytest.raises(binding2d.SlpicError) as ei:
        g.solve_poisson(rho)
    assert ei.value.code == binding2d.binding.SLPIC_ERR_NOCONVERGE
    g.synchronize()  # the handle still works
    g.close()


def _compare_step2d(prob, st, g, o, rel=1e-5):
    dx, nx, ny = prob["dx"], prob["nx"], prob["ny"]
    Lx = nx * dx
    stats = []
    for s in range(len(st)):
        c, off, v = g.particles(s)
        kg = v[:, 2].astype(np.float32).view(np.uint32).astype(np.int64)
        ko = o.v[s][:, 2].astype(np.float32).view(np.uint32).astype(np.int64)
        og = np.argsort(kg)
        pos = np.searchsorted(kg[og], ko)
        pos = np.minimum(pos, kg.size - 1)
        found = kg[og][pos] == ko
        ia = np.nonzero(found)[0]
        ib = og[pos[found]]
        # survivors lost only within rounding of a plate
        miss = np.nonzero(~found)[0]
        if miss.size:
            yo = o.y[s][miss]
            assert (np.minimum(yo, ny * dx - yo) < 1e-4 * dx).all(), f"{miss.size} lost"
        extra = np.setdiff1d(np.arange(kg.size), ib)
        if extra.size:
            yg = (c[extra] // nx + off[extra, 1].astype(np.float64)) * dx
            assert (np.minimum(yg, ny * dx - yg) < 1e-4 * dx).all()
        xg = (c[ib] % nx + off[ib, 0].astype(np.float64)) * dx
        yg = (c[ib] // nx + off[ib, 1].astype(np.float64)) * dx
        vg = v[ib].astype(np.float64)
        vref = o.v[s][ia]
        vn = np.linalg.norm(vref, axis=1)
        dv = np.linalg.norm(vg - vref, axis=1)
        # the input speed bounds |v| from the other side
        cin, oin, vin = st[s]
        kin = vin[:, 2].view(np.uint32).astype(np.int64)
        oi = np.argsort(kin)
        vin_m = vin[oi[np.searchsorted(kin[oi], ko[ia])]].astype(np.float64)
        vnorm = np.maximum(vn, np.linalg.norm(vin_m, axis=1))
        assert (dv <= rel * vnorm + 1e-30).all(), \
            f"species {s}: worst dv/|v| {np.max(dv / np.maximum(vnorm, 1e-30)):.3e}"
        sp = prob["species"][s]
        b = orc._beta_vec(int(sp["kind"]), vn, float(sp["v0"]))
        tol = rel * b * vnorm * prob["dt"] + 8 * 2.0 ** -24 * dx
        ddx = (xg - o.x[s][ia] + 0.5 * Lx) % Lx - 0.5 * Lx
        ddy = yg - o.y[s][ia]
        assert (np.abs(ddx) <= tol).all(), f"species {s}: x error {np.max(np.abs(ddx) / tol):.2f} tol"
        assert (np.abs(ddy) <= tol).all(), f"species {s}: y error {np.max(np.abs(ddy) / tol):.2f} tol"
        stats.append((s, ia.size, float(np.max(dv / np.maximum(vnorm, 1e-30)))))
    return stats


@pytest.mark.parametrize("kind", [inputs.BETA_ONE, inputs.BETA_HEAVISIDE,
                                  inputs.BETA_RELATIVISTIC])
def test_single_step2d_matches_oracle(kind):
    """Non-neutral load and a biased plate: strong fields in both directions,
    particles in both beta regimes, some leaving through the plates."""
    v0 = 0.35
    prob = _prob(nx=48, ny=36, ppc=10, kind=kind, v0=v0, dx=0.5,
                 dt=0.5 / (v0 if kind != inputs.BETA_ONE else 4.0), phi_hi=1.5)
    st = _unique_vz(_nonneutral(inputs.load_state2d(prob, seed=11 + kind)))
    g = _sim(prob, st)
    o = _oracle(prob, st)
    # rho: the quantised deposit (FP32 beta and offsets) against the FP64 one; phi:
    # the CG answer against the direct solve of the GPU's own rho
    rho_g, phi_g, _, _ = g.fields()
    scale = sum(abs(prob["species"][s]["q"]) * o.dens[s] for s in range(2)).max()
    assert np.abs(rho_g - o.rho).max() <= 1e-6 * scale
    ref = orc.poisson2d_direct(rho_g, prob["dx"], prob["phi_lo"], prob["phi_hi"])
    assert np.abs(phi_g - ref).max() <= _cond(36) * 1e-11 * max(1.0, np.abs(ref).max())
    g.step(1)
    g.synchronize()
    o.step(1)
    stats = _compare_step2d(prob, st, g, o)
    print("parity2d", kind, stats)
    d = g.diagnostics()
    for s in range(2):
        assert abs(d["count"][s] - o.x[s].size) <= 2
        assert abs(d["absorbed"][s][0] + d["absorbed"][s][1] - o.flux[s].sum()) <= 2
    g.close()


def test_steps2d_deposit_totals_and_potential():
    """Over several steps (with one compacting step): every deposit totals
    sum_p rint(beta 2^40) over the GPU's own particles, and the GPU's potential
    solves Poisson for the GPU's own rho (oracle direct solve) within the CG
    bound."""
    prob = _prob(nx=40, ny=32, ppc=8, v0=0.3, dt=1.5, cg_rtol=1e-10)
    st = inputs.load_state2d(prob, seed=21)
    g = _sim(prob, st)
    for _ in range(3):
        g.step(6)  # 18 steps: crosses the compacting step at 15
        rho, phi, Ex, Ey = g.fields()
        for s in range(2):
            c, o, v = g.particles(s)
            b = np.array([orc.beta_f32(1, *vv, np.float32(0.3)) for vv in v], np.float32)
            qT = np.rint(b * np.float32(TWO40)).astype(np.int64)
            assert int(g.charge_raw(s).sum()) == int(qT.sum())
        ref = orc.poisson2d_direct(rho, prob["dx"])
        assert np.abs(phi - ref).max() <= _cond(32) * 1e-10 * max(1e-6, np.abs(ref).max())
        ex_o, ey_o = orc.efield2d(phi, prob["dx"])
        assert np.abs(Ex - ex_o).max() <= 1e-6 * max(1e-6, np.abs(ex_o).max())
        assert np.abs(Ey - ey_o).max() <= 1e-6 * max(1e-6, np.abs(ey_o).max())
    d = g.diagnostics()
    assert d["step"] == 18 and d["cg_iterations_total"] > 0
    g.close()


def test_source2d_matches_oracle_injection():
    """RATE source: the same macroparticle count per step as the oracle, at the
    same FP32 positions; velocities to FP32 libm accuracy."""
    prob = _prob(nx=32, ny=40, ppc=2, v0=0.3, dt=1.0, source=inputs.SRC_RATE, rate=150.0)
    st = inputs.load_state2d(prob, seed=4)
    st = [(c[:0], o[:0], v[:0]) for c, o, v in st]  # empty box: only the source
    g = _sim(prob, st)
    o = _oracle(prob, st)
    g.step(1)
    o.step(1)
    for s in range(2):
        c, off, v = g.particles(s)
        assert c.size == o.x[s].size > 0
        # injected at step 0; the oracle keeps them in order, the GPU too (no compaction)
        xg = (c % prob["nx"] + off[:, 0].astype(np.float64)) * prob["dx"]
        yg = (c // prob["nx"] + off[:, 1].astype(np.float64)) * prob["dx"]
        assert np.abs(xg - o.x[s]).max() <= 1e-6 and np.abs(yg - o.y[s]).max() <= 1e-6
        assert np.abs(v - o.v[s]).max() <= 1e-5 * max(1.0, np.abs(o.v[s]).max())
    g.close()


def test_load2d_rejects_bad_particles_and_capacity():
    prob = _prob(nx=16, ny=16, ppc=1)
    g = binding2d.Simulation2D(prob)
    with pytest.raises(binding2d.SlpicError):
        g.load(0, np.array([16 * 16], np.int32), np.zeros((1, 2), np.float32),
               np.zeros((1, 3), np.float32))
    with pytest.raises(binding2d.SlpicError):
        g.load(0, np.array([3], np.int32), np.array([[1.0, 0.0]], np.float32),
               np.zeros((1, 3), np.float32))
    cap = prob["species"][0]["capacity"]
    with pytest.raises(binding2d.SlpicError) as ei:
        g.load(0, np.zeros(cap + 1, np.int32), np.zeros((cap + 1, 2), np.float32),
               np.zeros((cap + 1, 3), np.float32))
    assert ei.value.code == binding2d.binding.SLPIC_ERR_CAPACITY
    g.close()


# ------------------------------------------------------------------ direct (FFT) solver
@pytest.mark.parametrize("nx,ny", [(64, 48), (128, 2), (2, 9), (1024, 33)])
def test_fft_solve_matches_direct_oracle(nx, ny):
    """SLPIC2D_SOLVER_FFT (radix-2 FFT along x, Thomas per mode along y, FP64)
    against the oracle's direct solve (plain DFT along x, Thomas per mode): biased
    plates, random rho, one interior row (ny = 2), a two-point period (nx = 2)."""
    prob = _prob(nx=nx, ny=ny, ppc=1, phi_hi=-0.7)
    prob["phi_lo"] = 0.3
    prob["solver"] = "fft"
    g = binding2d.Simulation2D(prob)
    rho = np.random.default_rng(nx + ny).normal(size=(ny + 1, nx))
    phi, it, res = g.solve_poisson(rho)
    exact = orc.poisson2d_direct(rho, prob["dx"], 0.3, -0.7)
    assert it == 0 and res <= 1e-13
    assert np.abs(phi - exact).max() <= 1e-12 * np.abs(exact).max()
    assert np.all(phi[0] == 0.3) and np.all(phi[-1] == -0.7)
    g.close()


def test_fft_solver_needs_a_power_of_two_period():
    prob = _prob(nx=48, ny=16, ppc=1)
    prob["solver"] = "fft"
    with pytest.raises(binding2d.SlpicError) as ei:
        binding2d.Simulation2D(prob)
    assert ei.value.code == binding2d.binding.SLPIC_ERR_INVALID


@pytest.mark.parametrize("kind", [inputs.BETA_ONE, inputs.BETA_HEAVISIDE])
def test_single_step2d_with_fft_solver_matches_oracle(kind):
    """The step of the parity test above with the direct solver: the potential is
    the direct solve of the GPU's own rho to roundoff, and the step matches the
    oracle's."""
    v0 = 0.35
    prob = _prob(nx=64, ny=36, ppc=10, kind=kind, v0=v0, dx=0.5,
                 dt=0.5 / (v0 if kind != inputs.BETA_ONE else 4.0), phi_hi=1.5)
    prob["solver"] = "fft"
    st = _unique_vz(_nonneutral(inputs.load_state2d(prob, seed=31 + kind)))
    g = _sim(prob, st)
    o = _oracle(prob, st)
    rho_g, phi_g, _, _ = g.fields()
    ref = orc.poisson2d_direct(rho_g, prob["dx"], prob["phi_lo"], prob["phi_hi"])
    assert np.abs(phi_g - ref).max() <= 1e-12 * max(1.0, np.abs(ref).max())
    g.step(1)
    g.synchronize()
    o.step(1)
    stats = _compare_step2d(prob, st, g, o)
    print("parity2d fft", kind, stats)
    d = g.diagnostics()
    assert d["cg_iterations"] == 0 and d["cg_rel_residual"] <= 1e-13
    for s in range(2):
        assert abs(d["count"][s] - o.x[s].size) <= 2
    g.close()


def test_fft_and_cg_steps_agree():
    """Twenty steps (a compacting step among them) with each solver from one load:
    the potentials agree to the CG's tolerance."""
    prob = _prob(nx=64, ny=40, ppc=8, v0=0.3, dt=1.5, cg_rtol=1e-12)
    st = inputs.load_state2d(prob, seed=41)
    pf = dict(prob, solver="fft")
    g1, g2 = _sim(prob, st), _sim(pf, st)
    g1.step(20)
    g2.step(20)
    p1, p2 = g1.fields()[1], g2.fields()[1]
    assert np.abs(p1 - p2).max() <= 1e-6 * max(1e-6, np.abs(p2).max())
    assert g2.diagnostics()["cg_iterations_total"] == 0
    g1.close()
    g2.close()


def test_particles_are_sorted_by_cell_after_load_and_compaction():
    """The counting sort by cell (after slpic2d_prepare and after every compacting
    step): particles come back in non-decreasing cell order, none lost."""
    prob = _prob(nx=32, ny=24, ppc=6, v0=0.3, dt=1.5)
    st = inputs.load_state2d(prob, seed=51)
    g = _sim(prob, st)
    for s in range(2):
        c, _, _ = g.particles(s)
        assert c.size == st[s][0].size and np.all(np.diff(c) >= 0)
        assert np.array_equal(np.sort(c), np.sort(st[s][0]))
    g.step(16)  # step 15 compacts, then sorts
    d = g.diagnostics()
    for s in range(2):
        c, _, _ = g.particles(s)
        assert c.size == d["count"][s] and np.all(np.diff(c) >= 0)
    g.close()


def test_tile_summed_deposit_is_the_per_particle_deposit():
    """The in-place step sums a chunk's charge in a window of nodes in shared memory
    (global atomics for what falls outside it) before adding it to the grid.  With
    the direct solver (exact to roundoff), the potential each step leaves equals the
    direct solve of the charge recomputed particle by particle (slpic2d_fields) at the
    same positions: a lost, doubled or misplaced sum would show at once.  On this
    narrow grid a chunk spans whole rows, so the windows are whole rows and the last
    column's cells take the global path."""
    prob = _prob(nx=64, ny=40, ppc=16, v0=0.3, dt=1.5, phi_hi=0.5)
    prob["solver"] = "fft"
    st = inputs.load_state2d(prob, seed=61)
    g = _sim(prob, st)
    for n in (1, 4, 16):  # the 16th step compacts and sorts again
        g.step(n)
        rho, phi, _, _ = g.fields()
        ref = orc.poisson2d_direct(rho, prob["dx"], prob["phi_lo"], prob["phi_hi"])
        assert np.abs(phi - ref).max() <= 1e-11 * max(1.0, np.abs(ref).max()), n
    g.close()


def test_sort_drops_holes_when_particles_are_added_later():
    """In-place steps leave holes; particles loaded afterwards are appended behind
    them; slpic2d_prepare sorts again: the holes go, the live particles stay."""
    prob = _prob(nx=32, ny=24, ppc=6, v0=0.3, dt=1.5)
    st = inputs.load_state2d(prob, seed=71)
    g = _sim(prob, st)
    g.step(5)  # in-place steps: absorbed particles leave holes
    d = g.diagnostics()
    before = [g.particles(s)[0].size for s in range(2)]
    assert before == d["count"][:2]
    extra = inputs.load_state2d(dict(prob, species=[dict(sp, ppc=1) for sp in prob["species"]]), seed=72)
    g.load_state(extra)
    g.prepare()
    for s in range(2):
        c, _, _ = g.particles(s)
        assert c.size == before[s] + extra[s][0].size
        assert np.all(c >= 0) and np.all(np.diff(c) >= 0)
    g.close()


def test_tile_windows_over_in_place_steps_match_per_particle_deposit():
    """The same bar on a wide grid, where a sorted chunk covers part of a row and its
    window a small box: over the in-place steps between two sorts (particles drift
    and the boxes grow), in a strong non-uniform field with absorbing plates and a
    biased plate, the step's summed deposit gives the potential of the charge
    recomputed particle by particle."""
    prob = _prob(nx=256, ny=48, ppc=20, v0=0.3, dt=1.5, phi_hi=0.5)
    prob["solver"] = "fft"
    st = _nonneutral(inputs.load_state2d(prob, seed=81), frac=0.5, seed=3)
    g = _sim(prob, st)
    for n in (1, 6, 8):  # after 1, 7 and 15 steps, all in place (the 16th compacts)
        g.step(n)
        rho, phi, _, _ = g.fields()
        ref = orc.poisson2d_direct(rho, prob["dx"], prob["phi_lo"], prob["phi_hi"])
        assert np.abs(phi - ref).max() <= 1e-11 * max(1.0, np.abs(ref).max()), n
    d = g.diagnostics()
    assert sum(d["absorbed"][0]) > 0
    g.close()


def test_2d_empty_species_and_a_single_particle():
    """Edge cases of the tile kernel and the sort: no electrons at all, and a single ion
    (one ragged chunk of one slot, its window a single cell's box), stepped across the
    sort step with the direct solver: the potential each step leaves is the direct solve
    of the charge recomputed from the particles, the counts are consistent and the ion
    stays the one particle."""
    prob = _prob(nx=32, ny=24, ppc=1, v0=0.3, dt=1.5)
    prob["solver"] = "fft"
    g = binding2d.Simulation2D(prob)
    g.load(0, np.zeros(0, np.int32), np.zeros((0, 2), np.float32), np.zeros((0, 3), np.float32))
    g.load(1, np.array([12 * 32 + 7], np.int32), np.array([[0.25, 0.5]], np.float32),
           np.array([[0.01, -0.02, 0.005]], np.float32))
    g.prepare()
    for n in (1, 15, 2):  # steps 1, 16 (the 16th sorts), 18
        g.step(n)
        rho, phi, _, _ = g.fields()
        ref = orc.poisson2d_direct(rho, prob["dx"], prob["phi_lo"], prob["phi_hi"])
        assert np.abs(phi - ref).max() <= 1e-11 * max(1.0, np.abs(ref).max()), n
        d = g.diagnostics()
        assert d["count"][0] == 0
        c, o, v = g.particles(1)
        live = c >= 0
        assert live.sum() + sum(d["absorbed"][1]) == 1
        assert d["count"][1] == live.sum()
    g.close()
