"""The GPU path against the paper's speed-limited plasma frequency (Sec. III): the
warm-plasma oscillation of test_oracle_dispersion, through the C ABI, with four
times as many velocity groups (the quiet start's spread shrinks with them)."""
import math

import numpy as np
import pytest
from scipy import optimize

from paper_1511_08225_gb300 import binding

from test_oracle_dispersion import REL, _beta, slpic_omega

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1511_08225_gb300 import build
    build.build()
    binding.load_library()


def _fit_omega(amp, dt, w_guess, skip):
    t = np.arange(amp.size) * dt

    def model(t, A, om, ph, g, C):
        return A * np.cos(om * t + ph) * np.exp(g * t) + C

    best = None
    for ph in np.linspace(0.0, 2 * math.pi, 8, endpoint=False):
        try:
            p, _ = optimize.curve_fit(model, t[skip:], amp[skip:],
                                      p0=[np.abs(amp).max(), w_guess, ph, 0.0, 0.0],
                                      maxfev=20000)
        except RuntimeError:
            continue
        r = float(((model(t[skip:], *p) - amp[skip:]) ** 2).sum())
        if best is None or r < best[0]:
            best = (r, p)
    assert best is not None
    return abs(best[1][1])


@pytest.mark.parametrize("seed", [1, 2])
def test_warm_plasma_frequency_on_the_gpu(seed):
    N, dx, dt, M, v0, steps = 64, 0.5, 1.0, 1024, 0.2, 300
    L = N * dx
    k = 2 * math.pi / L
    w_th, w0 = slpic_omega(k, v0)
    vs = np.linspace(-12.0, 12.0, 400001)
    cdf = np.cumsum(np.exp(-0.5 * vs ** 2) * np.sqrt(vs ** 2 + v0 ** 2))
    cdf /= cdf[-1]
    vq = np.interp((np.arange(M) + 0.5) / M, cdf, vs)
    rng = np.random.default_rng(seed)
    x = np.tile((np.arange(N) + 0.5) * dx, M) + np.repeat(rng.uniform(-0.5, 0.5, M), N) * dx
    v = np.repeat(vq, N)
    x = np.mod(x + 0.05 * np.sin(k * x), L)
    w = L / _beta(v, v0).sum()
    xi = x / dx
    cell = np.minimum(np.floor(xi).astype(np.int32), N - 1)
    off = np.clip((xi - cell).astype(np.float32), 0.0, np.nextafter(np.float32(1), np.float32(0)))
    vel = np.zeros((v.size, 3), np.float32)
    vel[:, 0] = v
    prob = {"n_cells": N, "dx": dx, "dt": dt, "periodic": True, "phi_lo": 0.0, "phi_hi": 0.0,
            "eps0": 1.0, "seed": 1,
            "species": [{"name": "e", "q": -1.0, "m": 1.0, "w": w, "v0": v0, "kind": REL,
                         "T": 0.0, "capacity": v.size + 64}],
            "source": {"mode": binding.SLPIC_SRC_NONE}}
    sim = binding.Simulation(prob)
    sim.load_state([(cell, off, vel)])
    sim.prepare()
    proj = np.cos(k * np.arange(N) * dx)
    amp = []
    for _ in range(steps):
        amp.append(float((sim.fields()[0] * proj).sum()))
        sim.step(1)
    sim.close()
    omega = _fit_omega(np.array(amp), dt, w_th, int(2 * math.pi / w_th / dt))
    print(f"seed {seed}: omega {omega:.5f}, relation {w_th:.5f} (k -> 0: {w0:.5f}), "
          f"ratio {omega / w_th:.4f}")
    assert omega == pytest.approx(w_th, rel=0.03)
