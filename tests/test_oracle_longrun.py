"""The long-run comparison of the Sec. IV sheath has teeth, on the CPU.

The stored ensemble (golden/paper_sheath_slpic_ensemble.txt) holds the oracle's
time-averaged steady profiles over 16 seeds.  Here the oracle runs 4 further seeds
as it stands, which must pass the bar the GPU tests use (|z| <= 5 at every node,
mean z^2 <= 2), and 4 seeds with a planted mistake, which must fail it: the deposit
weighted by the g-weight alone, dropping beta (Sec. II: macroparticles sample
g = f / beta, so the physical charge is w beta per macroparticle)."""
import multiprocessing as mp
import os

import numpy as np
import pytest

import _sheath_ensemble as ens


@pytest.fixture(scope="module")
def runs():
    golden = ens.read_golden()
    seeds = [ens.BASE_SEED + 2000 + k for k in range(4)]
    jobs = [(s, golden["ppc"], None) for s in seeds] + \
           [(s, golden["ppc"], "g_deposit") for s in seeds]
    with mp.get_context("spawn").Pool(min(len(jobs), os.cpu_count() or 1)) as pool:
        res = pool.map(ens.oracle_run, jobs, chunksize=1)
    ok = ens.summarise([r[0] for r in res[:4]], [r[1] for r in res[:4]])
    bad = ens.summarise([r[0] for r in res[4:]], [r[1] for r in res[4:]])
    return golden, ok, bad


def test_golden_ensemble_is_sane(runs):
    golden, _, _ = runs
    assert golden["seeds"] == 16 and golden["mean"].shape == (3, 101)
    # the bias of Sec. IV at the plates, exactly
    assert golden["mean"][0, 0] == pytest.approx(-12.5 / 2.2, abs=1e-9)
    assert golden["mean"][0, -1] == 0.0
    # ions enter at the right plate and all leave through the left one: their flux
    # there is the one-sided flux n v_ti / sqrt(2 pi) of the source plasma (density 1)
    vti = np.sqrt((0.5 / 2.2) / ens_mass())
    assert golden["flux_mean"][2] == pytest.approx(vti / np.sqrt(2 * np.pi), rel=0.03)
    assert golden["flux_mean"][3] == 0.0


def ens_mass():
    from paper_1511_08225_gb300 import inputs
    return inputs.ARGON_MASS_RATIO


def test_further_oracle_seeds_pass_the_bar(runs):
    golden, ok, _ = runs
    zp, zf = ens.compare(ok, golden)
    assert np.abs(zp).max() <= ens.Z_MAX
    assert (zp ** 2).mean() <= ens.CHI2_MAX
    assert np.abs(zf).max() <= ens.Z_MAX


def test_planted_mistake_fails_the_bar(runs):
    golden, _, bad = runs
    zp, _ = ens.compare(bad, golden)
    assert np.abs(zp).max() > 4 * ens.Z_MAX
