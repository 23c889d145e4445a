"""The configured 1D sheath has no steady state under SLPIC: the oracle shows it on
a reduced grid.

The workload (Dirichlet phi = 0 plates, dx = lambda_D / 2, m_i/m_e = 73,440,
T_e/T_i = 10, Heaviside beta with v0 = 0.02 v_te, dt = dx / v0, a central source
band re-injecting the ions' losses) is run by the FP64 oracle on 1,024 cells (512
Debye lengths) from a quiet, symmetric, neutral load.  With the source the
potential runs away: within 40 steps (1,000 / omega_pe) max|phi| passes 100 T_e/e,
far above any sheath drop of the plasma (the textbook floating drop is about
5 T_e/e).  Without the source the same load stays below 10 T_e/e over those steps.
The source injects the physical Maxwellian at the physical rate, i.e. electron and
ion macroparticles in numbers that differ by the ratio of their g-weights (about
80 here), at independent positions of the band, so each step leaves local charges;
the physical charge of a speed-limited electron is w beta(|v|), which falls as the
electron gains energy in a potential well, so the response to such a charge
deepens the well instead of screening it until the slow g-particles catch up.  The
paper's own sheath (Sec. IV: 25 Debye lengths, wall source) settles, which
test_gpu_longrun.py checks against this oracle."""
import multiprocessing as mp

import numpy as np
import pytest


def _max_phi(args):
    src, nsteps = args
    from oracle import oracle as orc
    from paper_1511_08225_gb300 import inputs
    orc.build()
    mode = inputs.SRC_LOSS_MATCHED if src else inputs.SRC_NONE
    prob = inputs.sheath_problem(n_cells=1024, ppc=40, v0=0.02, source_mode=mode)
    st = inputs.quiet_symmetric_state(prob)
    o = orc.OracleSim(prob)
    for s, (c, off, v) in enumerate(st):
        o.load_cells(s, c, off, v)
    o.start()
    out = []
    for _ in range(nsteps):
        o.step(1)
        out.append(float(np.abs(o.phi).max()))
    return out


@pytest.fixture(scope="module")
def runs():
    with mp.get_context("spawn").Pool(2) as pool:
        return pool.map(_max_phi, [(True, 40), (False, 40)])


def test_quiet_symmetric_load_is_neutral():
    from paper_1511_08225_gb300 import inputs
    from oracle import oracle as orc
    prob = inputs.sheath_problem(n_cells=64, ppc=40, v0=0.02)
    st = inputs.quiet_symmetric_state(prob)
    o = orc.OracleSim(prob)
    for s, (c, off, v) in enumerate(st):
        o.load_cells(s, c, off, v)
        assert (v.astype(np.float64).reshape(-1, 40, 3).sum(1) == 0.0).all()
    o.start()
    # interior nodes neutral to rounding; the wall nodes carry half cells
    assert np.abs(o.rho[1:-1]).max() < 1e-12


def test_configured_sheath_runs_away_with_its_source(runs):
    with_src, _ = runs
    assert max(with_src) > 100.0


def test_same_load_without_source_stays_bounded(runs):
    _, without = runs
    assert max(without) < 10.0
