"""Pins of the 2D oracle (no GPU): each check rests on something other than the
oracle itself -- discrete eigenfunctions, exact polynomial solutions, the
independent direct solver, brute-force RK4, exact integer identities."""
import math

import numpy as np
import pytest

from oracle import oracle as orc

TWO40 = 2.0 ** 40


def grid(nx, ny):
    j = np.arange(ny + 1)[:, None].astype(np.float64)
    i = np.arange(nx)[None, :].astype(np.float64)
    return i + 0 * j, j + 0 * i


@pytest.mark.parametrize("nx,ny,m,n,dx", [(32, 24, 3, 2, 0.7), (16, 40, 1, 7, 1.0),
                                          (64, 8, 31, 1, 0.25), (10, 10, 0, 3, 2.0)])
def test_poisson2d_discrete_eigenmodes(nx, ny, m, n, dx):
    """rho = cos/sin(2 pi m i/nx) sin(pi n j/ny) is an eigenvector of the 5-point
    operator with eigenvalue K^2 = (4/dx^2)(sin^2(pi m/nx) + sin^2(pi n/(2 ny))),
    so phi = rho / (eps0 K^2) exactly (plates at 0)."""
    i, j = grid(nx, ny)
    K2 = 4.0 / dx ** 2 * (math.sin(math.pi * m / nx) ** 2 + math.sin(math.pi * n / (2 * ny)) ** 2)
    for f in (np.sin, np.cos):
        rho = f(2 * np.pi * m * i / nx) * np.sin(np.pi * n * j / ny)
        if not np.abs(rho).max() > 0:
            continue
        phi = orc.poisson2d_direct(rho, dx, eps0=1.3)
        assert np.abs(phi - rho / (1.3 * K2)).max() <= 1e-12 * np.abs(rho / K2).max()


def test_poisson2d_quadratic_and_linear_exact():
    """Uniform rho between grounded plates: phi = rho y (Ly - y) / (2 eps0)
    (the stencil is exact on quadratics); no charge with plate potentials
    phi_lo, phi_hi: the linear profile."""
    nx, ny, dx = 12, 30, 0.5
    i, j = grid(nx, ny)
    y, Ly = j * dx, ny * dx
    phi = orc.poisson2d_direct(np.full((ny + 1, nx), 0.8), dx, eps0=2.0)
    assert np.abs(phi - 0.8 * y * (Ly - y) / 4.0).max() < 1e-12
    phi = orc.poisson2d_direct(np.zeros((ny + 1, nx)), dx, phi_lo=1.5, phi_hi=-0.5)
    assert np.abs(phi - (1.5 + (-2.0) * y / Ly)).max() < 1e-13


def test_poisson2d_cg_agrees_with_direct_solver():
    """CG reaches the requested relative residual and then agrees with the
    direct solve within cond(A) * rtol; warm-started from the solution it
    stops at once; a tighter rtol costs more iterations."""
    nx, ny, dx = 40, 28, 0.8
    rng = np.random.default_rng(3)
    rho = rng.normal(size=(ny + 1, nx))
    exact = orc.poisson2d_direct(rho, dx, 0.3, -0.1)
    phi, it8, res = orc.poisson2d_cg(rho, dx, None, 0.3, -0.1, rtol=1e-8)
    assert it8 > 0 and res <= 1e-8
    cond = 8.0 / (4.0 * math.sin(math.pi / (2 * ny)) ** 2)
    assert np.abs(phi - exact).max() <= cond * 1e-8 * np.abs(exact).max()
    _, it12, res12 = orc.poisson2d_cg(rho, dx, None, 0.3, -0.1, rtol=1e-12)
    assert it12 > it8 and res12 <= 1e-12
    _, it0, _ = orc.poisson2d_cg(rho, dx, exact, 0.3, -0.1, rtol=1e-8)
    assert it0 == 0
    # the reported residual is the true one: recompute b - A phi independently
    phi12, _, _ = orc.poisson2d_cg(rho, dx, None, 0.3, -0.1, rtol=1e-12)
    lap = (np.roll(phi12, 1, 1) + np.roll(phi12, -1, 1) - 4 * phi12)[1:-1] + \
        phi12[2:] + phi12[:-2]
    r = rho[1:-1] * dx * dx + lap
    b = rho[1:-1] * dx * dx
    b[0] += 0.3
    b[-1] += -0.1
    assert np.linalg.norm(r) / np.linalg.norm(b) <= 1.01e-12


def test_efield2d_exact_on_linear_and_sinusoid():
    nx, ny, dx = 16, 10, 0.5
    i, j = grid(nx, ny)
    Ex, Ey = orc.efield2d(2.0 - 0.7 * j * dx, dx)
    assert np.abs(Ex).max() == 0.0 and np.abs(Ey - 0.7).max() < 1e-14
    k = 2 * np.pi * 3 / (nx * dx)
    Ex, Ey = orc.efield2d(np.sin(k * i * dx), dx)
    assert np.abs(Ex + np.cos(k * i * dx) * np.sin(k * dx) / dx).max() < 1e-13
    assert np.abs(Ey).max() < 1e-15


def _q40_inputs(n, nx, ny, rng):
    cell = rng.integers(0, nx * ny, n).astype(np.int32)
    off = rng.random((n, 2)).astype(np.float32)
    v = rng.normal(0, 1, (n, 3)).astype(np.float32)
    return cell, off, v


def test_deposit2d_q40_rules():
    """Integer identities of the 2D quantised rule: the four node charges of a
    particle sum to qT = rint(beta 2^40); offsets (0, 0) put everything on the
    cell's own node; (1/2, 1/2) with beta = 1 gives 2^38 to each node; each
    node is within the FP32 rounding of its products (at most 4 terms of 2
    roundings each, 8 * 2^-24 beta 2^40) plus 4 units of the exact FP64
    bilinear weight."""
    nx, ny = 12, 9
    rng = np.random.default_rng(4)
    cell, off, v = _q40_inputs(3000, nx, ny, rng)
    for kind, v0 in ((0, 1.0), (1, 0.7), (2, 0.7)):
        acc = orc.deposit2d_q40(nx, ny, cell, off, v, kind, v0)
        b = np.array([orc.beta_f32(kind, *vv, v0) for vv in v], dtype=np.float32)
        qT = np.rint(b * np.float32(TWO40)).astype(np.int64)
        assert int(acc.sum()) == int(qT.sum())
        # per particle, against FP64 bilinear weights
        for p in range(0, 3000, 97):
            a1 = orc.deposit2d_q40(nx, ny, cell[p:p + 1], off[p:p + 1], v[p:p + 1], kind, v0)
            cx, cy = cell[p] % nx, cell[p] // nx
            fx, fy = float(off[p, 0]), float(off[p, 1])
            exact = {(cy, cx): (1 - fx) * (1 - fy), (cy, (cx + 1) % nx): fx * (1 - fy),
                     (cy + 1, cx): (1 - fx) * fy, (cy + 1, (cx + 1) % nx): fx * fy}
            for (jj, ii), wgt in exact.items():
                bound = 8 * 2.0 ** -24 * float(b[p]) * TWO40 + 4.0
                assert abs(a1[jj, ii] - float(b[p]) * wgt * TWO40) <= bound
    one = np.array([5], np.int32)
    a = orc.deposit2d_q40(nx, ny, one, np.zeros((1, 2), np.float32), np.zeros((1, 3), np.float32),
                          0, 1.0)
    assert a[0, 5] == 2 ** 40 and a.sum() == 2 ** 40
    a = orc.deposit2d_q40(nx, ny, one, np.full((1, 2), 0.5, np.float32),
                          np.zeros((1, 3), np.float32), 0, 1.0)
    assert a[0, 5] == a[0, 6] == a[1, 5] == a[1, 6] == 2 ** 38


def test_push2d_free_streaming_and_walls():
    """No field: x += beta(|v|) v dt exactly as written, x wraps, y beyond
    the plates is absorbed and counted per plate."""
    nx, ny, dx, dt, v0 = 10, 8, 1.0, 2.0, 0.4
    Ex = np.zeros((ny + 1, nx))
    x = np.array([0.5, 9.9, 3.0, 4.0])
    y = np.array([4.0, 4.0, 0.3, 7.9])
    v = np.array([[0.1, 0.0, 0.0], [0.3, 0.4, 0.0], [0.0, -0.5, 0.0], [0.0, 0.2, 0.0]])
    alive = np.ones(4, np.uint8)
    flux = np.zeros(2, np.int64)
    L = orc.lib()
    xx, yy, vv = x.copy(), y.copy(), v.copy()
    L.orc_push2d(nx, ny, dx, dt, orc._ptr(Ex), orc._ptr(Ex), 4, orc._ptr(xx), orc._ptr(yy),
                 orc._ptr(vv), orc._ptr(alive), 0.0, 1, v0, orc._ptr(flux))
    assert np.array_equal(vv, v)
    # particle 0: |v| < v0, beta = 1; particle 1: |v| = 0.5 > v0, beta = 0.8
    assert xx[0] == 0.5 + 0.1 * dt and yy[0] == 4.0
    assert abs(xx[1] - ((9.9 + 0.8 * 0.3 * dt) - 10.0)) < 1e-14
    assert abs(yy[1] - (4.0 + 0.8 * 0.4 * dt)) < 1e-15
    assert list(alive) == [1, 1, 0, 0] and list(flux) == [1, 1]


@pytest.mark.parametrize("kind", [1, 2])
def test_push2d_uniform_field_matches_rk4(kind):
    """A uniform field along an arbitrary direction: the oracle's new velocity
    equals brute-force RK4 of Eq. (LimPtclDyn) over one step to 1e-9."""
    nx, ny, dx, dt, v0 = 8, 8, 1.0, 2.0, 0.45
    ex, ey, qm = 0.13, -0.21, -1.0
    Ex = np.full((ny + 1, nx), ex)
    Ey = np.full((ny + 1, nx), ey)
    rng = np.random.default_rng(7 + kind)
    n = 6
    v = rng.normal(0, 0.6, (n, 3))
    x = rng.uniform(2, 6, n)
    y = rng.uniform(3, 5, n)
    alive = np.ones(n, np.uint8)
    flux = np.zeros(2, np.int64)
    vv = v.copy()
    orc.lib().orc_push2d(nx, ny, dx, dt, orc._ptr(Ex), orc._ptr(Ey), n, orc._ptr(x.copy()),
                         orc._ptr(y.copy()), orc._ptr(vv), orc._ptr(alive), qm, kind, v0,
                         orc._ptr(flux))
    a = np.array([qm * ex, qm * ey, 0.0])
    for p in range(n):
        ref = orc.rk4_limited(kind, v[p], a, dt, v0, n_sub=200_000)
        assert np.abs(vv[p] - ref[:3]).max() < 1e-9 * max(1.0, np.abs(ref[:3]).max())


def test_inject2d_positions_in_band_and_reproducible():
    """The 2D source: positions in the y band and over the whole x period, the
    same values for the same (seed, step, species), velocities Maxwellian."""
    L = orc.lib()
    n, nx, dx = 20000, 32, 0.5
    x, y, v = np.zeros(n), np.zeros(n), np.zeros((n, 3))
    L.orc_inject2d(11, 3, 1, n, np.float32(10.0), np.float32(4.0), nx, dx, 2.0,
                   orc._ptr(x), orc._ptr(y), orc._ptr(v))
    assert (y >= 10.0 * dx).all() and (y <= 14.0 * dx).all()
    assert (x >= 0).all() and (x < nx * dx).all()
    assert abs(x.mean() / (nx * dx) - 0.5) < 0.01
    assert abs(v.std(axis=0) / 2.0 - 1.0).max() < 0.03
    x2, y2, v2 = np.zeros(n), np.zeros(n), np.zeros((n, 3))
    L.orc_inject2d(11, 3, 1, n, np.float32(10.0), np.float32(4.0), nx, dx, 2.0,
                   orc._ptr(x2), orc._ptr(y2), orc._ptr(v2))
    assert np.array_equal(x, x2) and np.array_equal(y, y2) and np.array_equal(v, v2)


def test_oracle_sim2d_plain_pic_total_charge_is_conserved():
    """beta = 1 (plain PIC) with no particle reaching a plate: the bilinear
    deposit carries exactly w/dx^2 per particle, so sum(dens) dx^2 = N w."""
    from paper_1511_08225_gb300 import inputs
    prob = inputs.plasma2d_problem(nx=16, ny=16, ppc=4, kind=inputs.BETA_ONE, v0=1.0, dt=0.1,
                                   source_mode=inputs.SRC_NONE)
    st = inputs.load_state2d(prob)
    sim = orc.OracleSim2D(prob)
    for s, (c, o, v) in enumerate(st):
        keep = (c // 16 >= 2) & (c // 16 <= 13)
        sim.load_cells(s, c[keep], o[keep], v[keep] * 0.1)
    sim.start()
    n0 = [sim.x[s].size for s in range(2)]
    sim.step(3)
    for s in range(2):
        assert sim.x[s].size == n0[s]
        w = prob["species"][s]["w"]
        assert abs(sim.dens[s].sum() * prob["dx"] ** 2 - n0[s] * w) < 1e-9 * n0[s] * w
