"""Long runs against the oracle: the steady profiles of the paper's argon sheath
(Sec. IV), from the library's mixed-precision step and from its plain FP64 form,
each as a seed ensemble compared with the FP64 oracle's ensemble
(``golden/paper_sheath_slpic_ensemble.txt``, 16 seeds, written by the oracle alone).

Every run fills the sheath from its wall source and averages phi(x), n_e(x) and
n_i(x) over the last third of the paper's 24 us (steps 407..610 of SLPIC with
v0 = 0.016 v_te, dt = dx / v0), and counts the physical flux of each species through
each plate over that window.  The library's runs use 16 other seeds, so the two
ensembles are independent samples of the same steady state.  The bar, for every
compared number (phi at the 99 interior nodes, n_e and n_i at the 101 nodes, the
three non-zero fluxes): |z| <= 5 with z the two-sample statistic of the means, and a
mean z^2 of at most 2.  No ion may leave through the source plate (x = L).  The
same comparison of a deliberately wrong oracle (beta dropped from the deposit) fails
it (tests/test_oracle_longrun.py)."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1511_08225_gb300 import binding, inputs

import _sheath_ensemble as ens

pytestmark = pytest.mark.gpu

N_SEEDS = 16
GPU_SEED0 = ens.BASE_SEED + 1000


def _mixed_run(seed, ppc):
    prob = inputs.paper_sheath_problem(kind=inputs.BETA_HEAVISIDE, ppc=ppc, seed=seed)
    sim = binding.Simulation(prob)
    sim.load_state(inputs.empty_state(prob))
    sim.prepare()
    n, start = ens.window(prob)
    sim.step(start)
    d0 = sim.diagnostics()
    acc = np.zeros((3, sim.nn))
    for _ in range(n - start):
        sim.step(1)
        _, phi, _ = sim.fields()
        acc[0] += phi
        acc[1] += sim.density(0)
        acc[2] += sim.density(1)
    d1 = sim.diagnostics()
    sim.close()
    t_win = (n - start) * prob["dt"]
    w = [sp["w"] for sp in prob["species"]]
    flux = np.array([(d1["absorbed"][s][k] - d0["absorbed"][s][k]) * w[s]
                     for s in (0, 1) for k in (0, 1)]) / t_win
    return acc / (n - start), flux


def _fp64_run(seed, ppc):
    """The plain FP64 form: phi from its own solve, the densities by depositing its
    FP64 particles with the oracle's FP64 cloud-in-cell rule (test side only)."""
    prob = inputs.paper_sheath_problem(kind=inputs.BETA_HEAVISIDE, ppc=ppc, seed=seed)
    g = binding.SimulationFP64(prob)
    g.prepare()
    n, start = ens.window(prob)
    g.step(start)
    dep = orc.OracleSim(prob)
    acc = np.zeros((3, g.nn))
    for _ in range(n - start):
        g.step(1)
        _, phi, _ = g.fields()
        for s in range(2):
            x, v = g.particles(s)
            dep.x[s], dep.v[s] = x, v
        dep.deposit()
        acc[0] += phi
        acc[1] += dep.dens[0]
        acc[2] += dep.dens[1]
    g.close()
    return acc / (n - start)


@pytest.fixture(scope="module")
def golden():
    return ens.read_golden()


def test_mixed_form_sheath_profiles_match_oracle_ensemble(golden):
    runs = [_mixed_run(GPU_SEED0 + k, golden["ppc"]) for k in range(N_SEEDS)]
    mine = ens.summarise([r[0] for r in runs], [r[1] for r in runs])
    zp, zf = ens.compare(mine, golden)
    # the plates hold their potentials (the stored file keeps 11 significant digits)
    assert np.allclose(mine["mean"][0, [0, -1]], golden["mean"][0, [0, -1]], rtol=0, atol=1e-9)
    assert np.abs(zp).max() <= ens.Z_MAX, f"profiles: max |z| = {np.abs(zp).max():.2f}"
    assert (zp ** 2).mean() <= ens.CHI2_MAX, f"profiles: mean z^2 = {(zp ** 2).mean():.2f}"
    assert np.abs(zf).max() <= ens.Z_MAX, f"fluxes: z = {zf}"
    # ions leave through the biased plate only
    assert mine["flux_mean"][3] == 0.0 and golden["flux_mean"][3] == 0.0


def test_fp64_form_sheath_profiles_match_oracle_ensemble(golden):
    """The plain FP64 form at the same accuracy bar: the comparison point of the
    metric reaches the same steady sheath as the oracle and the mixed form."""
    runs = [_fp64_run(GPU_SEED0 + 100 + k, golden["ppc"]) for k in range(N_SEEDS)]
    mine = ens.summarise(runs, np.zeros((N_SEEDS, 4)))
    zp, _ = ens.compare(mine, golden)
    assert np.abs(zp).max() <= ens.Z_MAX, f"profiles: max |z| = {np.abs(zp).max():.2f}"
    assert (zp ** 2).mean() <= ens.CHI2_MAX, f"profiles: mean z^2 = {(zp ** 2).mean():.2f}"
