"""One SLPIC step of the library against one step of the oracle, particle by
particle (tests only).  Particles are matched across the step by their (vy, vz)
bits, which a 1D push leaves unchanged (see _match.py)."""
import numpy as np

from oracle import oracle as orc

from _match import key_of, match, periodic_diff


def compare_step(prob, st, gpu, o, rel=1e-5, stats=None, lam=None, E=None):
    """The library's particles after one step (gpu) against the oracle's (o), both
    started from the FP32 state st, matched by (vy, vz).

    Velocity: |v_gpu - v_orc| <= rel |v|.  With E (the FP64 nodal field of the step)
    the bar adds the kick of the library's FP32 copy of that field: each node rounds
    to within 2^-24 of itself and the interpolation adds as much again, so the
    gathered acceleration is within 4 2^-24 (|E_c| + |E_c+1|) |q/m| of the oracle's,
    over at most dt of integral of beta; where the field nearly cancels at the
    particle this term, not the push, dominates.  Position: the move is
    beta(|v|) v_x dt, so a velocity error of rel |v| moves x by at most
    rel beta(|v|) |v| dt; the bar is that plus 8 ulp of the FP32 offset.
    lam: per-cell factors of v0 (beta then takes v0 lam[start cell])."""
    dx, N = prob["dx"], prob["n_cells"]
    L = N * dx
    for s in range(len(st)):
        c0, off0, v0in = st[s]
        x_in = (c0.astype(np.float64) + off0.astype(np.float64)) * dx
        c, off, v = gpu.particles(s)
        xo, vo = o.x[s], o.v[s]
        # survivors in the oracle, in input order (no injection here)
        ko = key_of(vo)
        kg = key_of(v)
        ia, ib = match(ko, kg)
        # every oracle survivor is found on the GPU except within rounding of a wall
        missing = np.setdiff1d(np.arange(ko.size), ia)
        extra = np.setdiff1d(np.arange(kg.size), ib)
        for idx, xs in ((missing, xo), ):
            if idx.size:
                near = np.minimum(xs[idx], L - xs[idx]) < 1e-5 * dx
                assert near.all(), f"species {s}: {idx.size} survivors lost"
        if extra.size:
            xg_extra = (c[extra] + off[extra].astype(np.float64)) * dx
            assert (np.minimum(xg_extra, L - xg_extra) < 1e-5 * dx).all()
        xg = (c[ib].astype(np.float64) + off[ib].astype(np.float64)) * dx
        vg = v[ib].astype(np.float64)
        vref = vo[ia]
        # input positions of the matched particles
        kin = key_of(v0in)
        ja, jb = match(ko[ia], kin)
        assert ja.size == ia.size
        xin = x_in[jb]
        vnorm = np.maximum(np.linalg.norm(vref, axis=1), np.linalg.norm(v0in[jb], axis=1))
        dv = np.linalg.norm(vg - vref, axis=1)
        field = 0.0
        if E is not None:
            ci = c0[jb].astype(np.int64)
            c1 = (ci + 1) % N if prob["periodic"] else ci + 1
            qm = abs(float(prob["species"][s]["q"]) / float(prob["species"][s]["m"]))
            field = 4.0 * 2.0 ** -24 * (np.abs(E[ci]) + np.abs(E[c1])) * qm * prob["dt"]
        assert (dv <= rel * vnorm + field + 1e-30).all(), \
            f"species {s}: worst dv/|v| {np.max(dv / np.maximum(vnorm, 1e-30)):.3e}"
        dxp = periodic_diff(xg, xo[ia], L) if prob["periodic"] else xg - xo[ia]
        sp = prob["species"][s]
        r = np.linalg.norm(vref, axis=1)
        v0p = float(sp["v0"]) if lam is None else \
            float(sp["v0"]) * np.asarray(lam, np.float64)[st[s][0][jb]]
        b = orc._beta_vec(int(sp["kind"]), r, v0p)
        tol = rel * b * r * prob["dt"] + 8 * 2.0 ** -24 * dx
        if stats is not None:
            stats.append({"species": s, "max_dv_rel": float(np.max(dv / np.maximum(vnorm, 1e-30))),
                          "max_dx_over_tol": float(np.max(np.abs(dxp) / tol)), "n": int(ia.size)})
        assert (np.abs(dxp) <= tol).all(), \
            f"species {s}: worst position error {np.max(np.abs(dxp) - tol):.3e} over tol"
