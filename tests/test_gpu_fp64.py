"""The plain FP64 form (include/slpic_fp64.h) against the FP64 oracle: both
compute in FP64, so the bars are tight -- fields to 1e-12 of their scale, one
step's velocities to 1e-9 |v| and positions to 1e-9 beta |v| dt (plus 1e-12 of
the domain), particles matched by (vy, vz), which a 1D push leaves unchanged."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1511_08225_gb300 import binding, inputs

from _match import match

pytestmark = pytest.mark.gpu

ONE, HEAV, REL = inputs.BETA_ONE, inputs.BETA_HEAVISIDE, inputs.BETA_RELATIVISTIC


def _key64(v):
    b = np.ascontiguousarray(np.asarray(v, np.float64)[:, 1:3]).view(np.uint64)
    return b[:, 0] ^ (b[:, 1] * np.uint64(0x9E3779B97F4A7C15))


def _setup(kind, periodic, seed=3):
    v0 = 0.3
    prob = inputs.periodic_problem(n_cells=96, ppc=200, v0=v0, kind=kind, dt=0.5 / 4.0) \
        if periodic else inputs.sheath_problem(n_cells=96, ppc=200, v0=v0, kind=kind,
                                               source_mode=inputs.SRC_NONE)
    if kind == ONE and not periodic:
        prob["dt"] = 0.5 / 4.0
    if not periodic:
        prob["phi_hi"] = 2.0
    st = inputs.load_state(prob, seed=seed)
    # a non-neutral start: strong, non-uniform fields
    c, o, v = st[0]
    keep = (np.arange(c.size) % 3 != 0) | (c < 48)
    st = [(c[keep], o[keep], v[keep])] + st[1:]
    g = binding.SimulationFP64(prob)
    orc_sim = orc.OracleSim(prob)
    for s, (c, o, v) in enumerate(st):
        g.load_cells(s, c, o, v)
        orc_sim.load_cells(s, c, o, v)
    g.prepare()
    orc_sim.start()
    return prob, st, g, orc_sim


@pytest.mark.parametrize("kind", [ONE, HEAV, REL])
@pytest.mark.parametrize("periodic", [False, True])
def test_fp64_form_fields_and_step_match_oracle(kind, periodic):
    prob, st, g, o = _setup(kind, periodic)
    rho, phi, E = g.fields()
    for a, b in ((rho, o.rho), (phi, o.phi), (E, o.E)):
        assert np.abs(a - b).max() <= 1e-12 * max(1.0, np.abs(b).max())
    g.step(1)
    o.step(1)
    L = prob["n_cells"] * prob["dx"]
    for s in range(2):
        x, v = g.particles(s)
        assert x.size == o.x[s].size
        ia, ib = match(_key64(o.v[s]), _key64(v))
        assert ia.size == x.size
        vo, xo = o.v[s][ia], o.x[s][ia]
        vg, xg = v[ib], x[ib]
        vn = np.linalg.norm(vo, axis=1)
        assert (np.linalg.norm(vg - vo, axis=1) <= 1e-9 * np.maximum(vn, 1e-12)).all()
        b = orc._beta_vec(int(prob["species"][s]["kind"]), vn, float(prob["species"][s]["v0"]))
        dxp = (xg - xo + 0.5 * L) % L - 0.5 * L if periodic else xg - xo
        assert (np.abs(dxp) <= 1e-9 * b * vn * prob["dt"] + 1e-12 * L).all()
    rho, phi, E = g.fields()
    assert np.abs(phi - o.phi).max() <= 1e-9 * max(1.0, np.abs(o.phi).max())
    g.close()


def test_fp64_form_source_counts_match_oracle():
    """LOSS_MATCHED source: the same macroparticle counts per step as the oracle
    (the counts follow from the absorbed particles and the carried fraction)."""
    prob = inputs.sheath_problem(n_cells=128, ppc=40, v0=0.2)
    st = inputs.load_state(prob)
    g = binding.SimulationFP64(prob)
    o = orc.OracleSim(prob)
    for s, (c, off, v) in enumerate(st):
        g.load_cells(s, c, off, v)
        o.load_cells(s, c, off, v)
    g.prepare()
    o.start()
    for _ in range(3):
        g.step(1)
        o.step(1)
        for s in range(2):
            assert abs(g.count(s) - o.x[s].size) <= 2
    g.close()
