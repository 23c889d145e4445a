"""Write the oracle's seed ensemble of the Sec. IV sheath's steady profiles.

    python tests/golden/make_paper_sheath_ensemble.py [--seeds 16] [--ppc 500]

Calls only the FP64 oracle (``oracle/``) and the seeded input generators.  For
each seed it runs the paper's collisionless argon sheath (Sec. IV: 100 cells of a
quarter Debye length, a 12.5 V / 2.2 eV bias, electrons and argon ions entering
through the right plate from a stationary plasma, an empty start) as SLPIC with
the paper's v0 = 0.016 v_te and dt = dx / v0, for the paper's 24 us (610 steps),
and averages over the last third of the run (every step of it):

    phi(x), the physical densities n_e(x) and n_i(x) (sum of w beta S / dx, nodal),

and counts the physical flux (absorbed macroparticles x w per unit time) of each
species through each plate over the same window.  The file holds, per node, the
ensemble mean and the standard deviation over seeds of these per-seed averages,
and the same two numbers for the four fluxes.  The GPU test compares its own
ensemble with them.
"""
from __future__ import annotations

import argparse
import multiprocessing as mp
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

sys.path.insert(0, os.path.dirname(HERE))
from _sheath_ensemble import BASE_SEED, oracle_run, window  # noqa: E402

OUT = os.path.join(HERE, "paper_sheath_slpic_ensemble.txt")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--seeds", type=int, default=16)
    ap.add_argument("--ppc", type=int, default=500)
    ap.add_argument("--workers", type=int, default=os.cpu_count() or 1)
    a = ap.parse_args()
    from oracle import oracle as orc
    from paper_1511_08225_gb300 import inputs
    orc.build()
    n, start = window(inputs.paper_sheath_problem(kind=inputs.BETA_HEAVISIDE))
    jobs = [(BASE_SEED + k, a.ppc, None) for k in range(a.seeds)]
    with mp.get_context("spawn").Pool(min(a.workers, a.seeds)) as pool:
        res = pool.map(oracle_run, jobs, chunksize=1)
    prof = np.stack([r[0] for r in res])   # (seeds, 3, nodes)
    flux = np.stack([r[1] for r in res])   # (seeds, 4)
    mean, std = prof.mean(0), prof.std(0, ddof=1)
    fm, fs = flux.mean(0), flux.std(0, ddof=1)
    with open(OUT, "w") as f:
        f.write("# Oracle (FP64 CPU) seed ensemble of the Sec. IV argon sheath, SLPIC:\n")
        f.write("# Werner et al., arXiv 1511.08225, Sec. IV (100 cells, dx = 0.25 lambda_D,\n")
        f.write("# phi(0) = -12.5/2.2, phi(L) = 0, wall source of density 1, m_i/m_e = 39.9 x 1836,\n")
        f.write("# T_i = 0.5/2.2, Heaviside beta, v0 = 0.016 v_te, dt = dx/v0, 610 steps = 24 us).\n")
        f.write("# Written by tests/golden/make_paper_sheath_ensemble.py "
                f"--seeds {a.seeds} --ppc {a.ppc}\n")
        f.write(f"# seeds {BASE_SEED}..{BASE_SEED + a.seeds - 1}; per-seed averages over steps "
                f"{start + 1}..{n} (every step); mean and sample std over seeds.\n")
        f.write(f"seeds {a.seeds}\nppc {a.ppc}\n")
        f.write("flux_mean " + " ".join(f"{x:.10e}" for x in fm) + "\n")
        f.write("flux_std " + " ".join(f"{x:.10e}" for x in fs) + "\n")
        f.write("# node phi_mean phi_std ne_mean ne_std ni_mean ni_std\n")
        for j in range(prof.shape[2]):
            f.write(f"{j} " + " ".join(f"{mean[k, j]:.10e} {std[k, j]:.10e}" for k in range(3))
                    + "\n")
    print(f"wrote {OUT}: {a.seeds} seeds, ppc {a.ppc}; fluxes {fm} +- {fs}")


if __name__ == "__main__":
    main()
