"""Why the previous step's potential barely warm-starts the 2D CG, with the FP64 oracle.

The charge of a particle plasma is a smooth part plus shot noise (64 particles per
cell: 1/8 relative per cell), and from one step to the next a fraction of that
noise renews.  The residual the previous potential leaves is the Poisson image of
that renewed noise, about 0.4 of ||b|| and white, so the CG still has to converge
from nearly the start: the oracle's FP64 CG (no mixed precision involved) saves
only a few per cent of its iterations at 256^2.  When the same charge changes
smoothly instead, the previous potential leaves 3e-4 of ||b|| and the CG needs a
thirtieth of the iterations.  The learned guess of the library's 2D path is judged
against this baseline."""
import numpy as np
import pytest

from oracle import oracle as orc


def _charges(n=256, seed=0):
    rng = np.random.default_rng(seed)
    y = np.linspace(0, 1, n + 1)[:, None]
    x = np.linspace(0, 1, n, endpoint=False)[None, :]
    smooth = 0.05 * np.sin(np.pi * y) * (1 + 0.3 * np.cos(2 * np.pi * x))
    noise = rng.normal(0, 0.125, (n + 1, n))
    prev = smooth + noise
    noisy = smooth * 1.001 + 0.9 * noise + np.sqrt(1 - 0.81) * rng.normal(0, 0.125, (n + 1, n))
    calm = smooth * 1.001 + noise
    for r in (prev, noisy, calm):
        r[0] = r[-1] = 0.0  # the plate rows
    return prev, noisy, calm


@pytest.fixture(scope="module")
def runs():
    orc.build()
    prev, noisy, calm = _charges()
    phi_prev, _, _ = orc.poisson2d_cg(prev, 1.0, rtol=1e-12)
    out = {}
    for name, rho in (("noisy", noisy), ("calm", calm)):
        _, it_zero, _ = orc.poisson2d_cg(rho, 1.0, rtol=1e-8)
        _, it_prev, _ = orc.poisson2d_cg(rho, 1.0, phi0=phi_prev, rtol=1e-8)
        _, _, r0 = orc.poisson2d_cg(rho, 1.0, phi0=phi_prev, rtol=1e-8, maxit=0)
        out[name] = (it_zero, it_prev, r0)
    return out


def test_renewed_shot_noise_leaves_the_warm_start_far_from_the_answer(runs):
    it_zero, it_prev, r0 = runs["noisy"]
    assert 0.2 < r0 < 0.8
    assert it_prev > 0.85 * it_zero  # saves less than 15 %


def test_a_smooth_change_is_what_the_warm_start_saves(runs):
    it_zero, it_prev, r0 = runs["calm"]
    assert r0 < 1e-3
    assert it_prev < 0.1 * it_zero
