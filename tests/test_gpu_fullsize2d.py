"""Parity of the 2D path at its full size (1024 x 1024 cells, 64 particles per cell
and species: 134M particles), with the direct FFT solver, in the launch
configuration `bench.py --workload plasma2d --solver fft` times.

  * rho^0 and, after one step, rho^1: bit-exact against the 2D quantised rule over
    all particles;
  * phi^0 against the oracle's direct solve (DFT x Thomas) of the same charge,
    within cond(A) * 2e-15 of max|phi| (two direct FP64 solves of a system whose
    condition number is ~8.5e5 here);
  * one step of a random 20,000 particles per species from the rows 2..ny-3
    (which no particle leaves through a plate in one step), pushed one by one by
    the oracle with the oracle's E, against the same particles on the GPU: the
    single-step bars of test_gpu_2d.

Particle identity across the step: after prepare the particles are sorted by cell
and have no holes; the step keeps every particle in its slot, drops the absorbed
ones from the read-back and appends the source's.  Only row 0 can lose particles
ahead of the sampled rows (through y = 0), so a sampled slot i reads back at
i - d, d the count absorbed at y = 0, which vz (not changed by the push) confirms."""
import math

import numpy as np
import pytest

from oracle import oracle as orc
from paper_1511_08225_gb300 import binding2d, inputs

pytestmark = pytest.mark.gpu


def _cond(ny):
    return 8.0 / (4.0 * math.sin(math.pi / (2 * ny)) ** 2)


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1511_08225_gb300 import build
    build.build()
    binding2d.binding.load_library()


def test_full_size_2d_step_matches_oracle():
    nx = ny = 1024
    prob = inputs.plasma2d_problem(nx=nx, ny=ny, ppc=64, v0=0.1, solver="fft")
    dx, dt = prob["dx"], prob["dt"]
    Lx = nx * dx
    state = inputs.load_state2d(prob)
    g = binding2d.Simulation2D(prob)
    g.load_state(state)
    del state
    g.prepare()
    pre = [g.particles(s) for s in range(2)]
    for s, sp in enumerate(prob["species"]):
        c, o, v = pre[s]
        assert np.array_equal(g.charge_raw(s), orc.deposit2d_q40(
            nx, ny, c, o, v, int(sp["kind"]), np.float32(sp["v0"]))), f"species {s}: rho^0"
    rho_g, phi_g, _, _ = g.fields()
    phi = orc.poisson2d_direct(rho_g, dx, prob["phi_lo"], prob["phi_hi"])
    assert np.abs(phi_g - phi).max() <= _cond(ny) * 2e-15 * np.abs(phi).max()
    Ex, Ey = orc.efield2d(phi, dx)
    g.step(1)
    post = [g.particles(s) for s in range(2)]
    d_abs = g.diagnostics()["absorbed"]
    for s, sp in enumerate(prob["species"]):
        c, o, v = post[s]
        assert np.array_equal(g.charge_raw(s), orc.deposit2d_q40(
            nx, ny, c, o, v, int(sp["kind"]), np.float32(sp["v0"]))), f"species {s}: rho^1"
    g.close()

    rng = np.random.default_rng(0)
    ora = orc.OracleSim2D(prob)
    picks, shifts = [], []
    for s in range(2):
        c, o, v = pre[s]
        cy = c // nx
        mid = np.nonzero((cy >= 2) & (cy <= ny - 3))[0]
        idx = np.sort(rng.choice(mid, size=20_000, replace=False))
        d = int(d_abs[s][0])
        assert np.array_equal(post[s][2][idx - d, 2].view(np.uint32), v[idx, 2].view(np.uint32)), \
            f"species {s}: slot mapping"
        picks.append(idx)
        shifts.append(d)
        ora.load_cells(s, c[idx], o[idx], v[idx])
    ora.Ex, ora.Ey = Ex, Ey
    ora.push()
    for s, sp in enumerate(prob["species"]):
        assert ora.x[s].size == picks[s].size  # none of them can reach a plate
        c, o, v = post[s]
        j = picks[s] - shifts[s]
        xg = (c[j] % nx + o[j, 0].astype(np.float64)) * dx
        yg = (c[j] // nx + o[j, 1].astype(np.float64)) * dx
        vg = v[j].astype(np.float64)
        vref = ora.v[s]
        vin = pre[s][2][picks[s]].astype(np.float64)
        vnorm = np.maximum(np.linalg.norm(vref, axis=1), np.linalg.norm(vin, axis=1))
        dv = np.linalg.norm(vg - vref, axis=1)
        assert (dv <= 1e-5 * vnorm + 1e-30).all(), \
            f"species {s}: worst dv/|v| {np.max(dv / np.maximum(vnorm, 1e-30)):.3e}"
        b = orc._beta_vec(int(sp["kind"]), np.linalg.norm(vref, axis=1), float(sp["v0"]))
        tol = 1e-5 * b * vnorm * dt + 8 * 2.0 ** -24 * dx
        ddx = (xg - ora.x[s] + 0.5 * Lx) % Lx - 0.5 * Lx
        ddy = yg - ora.y[s]
        assert (np.abs(ddx) <= tol).all(), f"species {s}: x error {np.max(np.abs(ddx) / tol):.2f} tol"
        assert (np.abs(ddy) <= tol).all(), f"species {s}: y error {np.max(np.abs(ddy) / tol):.2f} tol"
        print(f"full size 2D, species {s}: {j.size} compared, worst dv/|v| "
              f"{np.max(dv / np.maximum(vnorm, 1e-30)):.2e}, absorbed at y=0: {shifts[s]}")
