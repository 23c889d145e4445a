"""Seed ensembles of the Sec. IV sheath's steady profiles, and their comparison.

A run of the paper's argon sheath (Sec. IV) is reduced to its time averages over
the last third of the run to 24 us: phi(x), the physical densities n_e(x) and
n_i(x), and the physical flux of each species through each plate.  Two ensembles
of such averages (independent seeds) are compared node by node with a two-sample
z statistic, z = (mean_a - mean_b) / (s sqrt(1/n_a + 1/n_b)), s the pooled sample
standard deviation over seeds.  The stored oracle ensemble is
``golden/paper_sheath_slpic_ensemble.txt`` (written by
``golden/make_paper_sheath_ensemble.py``, which calls only the oracle).
"""
from __future__ import annotations

import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = os.path.join(HERE, "golden", "paper_sheath_slpic_ensemble.txt")
T_END = 9530.0  # 24 us in units of 1/omega_pe of the source plasma
BASE_SEED = 20151126
Z_MAX = 5.0      # largest |z| allowed over the ~300 compared numbers
CHI2_MAX = 2.0   # largest mean z^2 allowed


def window(prob):
    """(total steps, first averaged step): the last third of the run to T_END."""
    n = int(round(T_END / prob["dt"]))
    return n, 2 * n // 3


def read_golden(path=GOLDEN):
    """{'seeds', 'ppc', 'flux_mean', 'flux_std', 'mean' (3, nodes), 'std' (3, nodes)}
    with rows phi, n_e, n_i and fluxes [e at x=0, e at x=L, i at x=0, i at x=L]."""
    out, rows = {}, []
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        f = line.split()
        if f[0] in ("seeds", "ppc"):
            out[f[0]] = int(f[1])
        elif f[0] in ("flux_mean", "flux_std"):
            out[f[0]] = np.array([float(x) for x in f[1:]])
        else:
            rows.append([float(x) for x in f[1:]])
    a = np.array(rows)
    out["mean"] = a[:, 0::2].T.copy()
    out["std"] = a[:, 1::2].T.copy()
    return out


def summarise(profiles, fluxes):
    """Per-seed averages (seeds, 3, nodes) and fluxes (seeds, 4) -> ensemble."""
    p = np.asarray(profiles, dtype=np.float64)
    f = np.asarray(fluxes, dtype=np.float64)
    return {"seeds": p.shape[0], "mean": p.mean(0), "std": p.std(0, ddof=1),
            "flux_mean": f.mean(0), "flux_std": f.std(0, ddof=1)}


def _pooled_se(sa, sb, na, nb):
    """Standard error of mean_a - mean_b from the pooled standard deviation (both
    ensembles sample the same steady state under the hypothesis tested)."""
    s2 = ((na - 1) * sa ** 2 + (nb - 1) * sb ** 2) / (na + nb - 2)
    return np.sqrt(s2 * (1.0 / na + 1.0 / nb))


def compare(a, b):
    """z of every compared number: phi at the interior nodes (the plates' values are
    fixed), n_e and n_i at every node, and the three non-zero fluxes.  Returns
    (z of the profiles, z of the fluxes)."""
    na, nb = a["seeds"], b["seeds"]
    se = _pooled_se(a["std"], b["std"], na, nb)
    z = (a["mean"] - b["mean"]) / np.where(se > 0, se, np.inf)
    zp = np.concatenate([z[0, 1:-1], z[1], z[2]])
    fse = _pooled_se(a["flux_std"], b["flux_std"], na, nb)
    zf = (a["flux_mean"] - b["flux_mean"])[:3] / fse[:3]
    return zp, zf


def oracle_run(args):
    """One oracle seed of the sheath (spawn-pool job): (averages (3, nodes), fluxes
    (4,)).  args = (seed, ppc, planted), planted one of None or 'g_deposit' (the
    deposit weighted by the g-weight alone, dropping beta: a plausible mistake that
    the comparison must catch)."""
    seed, ppc, planted = args
    from oracle import oracle as orc
    from paper_1511_08225_gb300 import inputs
    orc.build()
    prob = inputs.paper_sheath_problem(kind=inputs.BETA_HEAVISIDE, ppc=ppc, seed=seed)
    o = orc.OracleSim(prob)
    if planted == "g_deposit":
        def deposit_g():
            L = orc.lib()
            o.dens = np.zeros((len(o.sp), o.nn))
            for s, sp in enumerate(o.sp):
                x = np.ascontiguousarray(o.x[s])
                v = np.ascontiguousarray(o.v[s])
                L.orc_deposit1d(o.N, int(o.periodic), o.dx, x.size, orc._ptr(x), orc._ptr(v),
                                None, orc.BETA_ONE, float(sp["v0"]), None, float(sp["w"]),
                                orc._ptr(o.dens[s]))
            o.rho = sum(float(sp["q"]) * o.dens[s] for s, sp in enumerate(o.sp))
        o.deposit = deposit_g
    o.start()
    n, start = window(prob)
    o.step(start)
    f0 = o.flux.copy()
    acc = np.zeros((3, o.nn))
    for _ in range(n - start):
        o.step(1)
        acc[0] += o.phi
        acc[1] += o.dens[0]
        acc[2] += o.dens[1]
    acc /= n - start
    t_win = (n - start) * prob["dt"]
    df = (o.flux - f0).astype(np.float64)
    w = [prob["species"][0]["w"], prob["species"][1]["w"]]
    flux = np.array([df[0, 0] * w[0], df[0, 1] * w[0], df[1, 0] * w[1], df[1, 1] * w[1]])
    return acc, flux / t_win
