"""The learned warm start of the 2D CG: a U-Net trained on the GPU, by the
library's own kernels, on (rho, phi) pairs that 2D runs generate, then used as
the CG's initial guess.  The CG to the same residual stays the judge: the answer
does not change; the iterations do.

Workload: the 2D plasma of the throughput benchmark at 64 x 64 cells (periodic
x, absorbing phi = 0 plates in y, central source band, m_i/m_e = 1836, Heaviside
beta, v0 = 0.1, dt = dx / v0), 16 particles per cell and species.  Training
pairs: three seeds, 60 pairs each, one every 3 steps after 20 steps.  Held out:
a fourth seed."""
import numpy as np
import pytest

from paper_1511_08225_gb300 import binding2d, binding_unet, inputs, warmstart

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N = 64


def _prob(seed=inputs.SEED):
    return inputs.plasma2d_problem(nx=N, ny=N, ppc=16, seed=seed, cg_rtol=1e-8, capacity_factor=4.0)


@pytest.fixture(scope="module")
def trained():
    prob = _prob()
    train = warmstart.collect_pairs(prob, seeds=(101, 102, 103), pairs_per_seed=60, every=3,
                                    skip=20)
    held = warmstart.collect_pairs(prob, seeds=(104,), pairs_per_seed=12, every=3, skip=20,
                                   keep_prev=True)
    x, t = warmstart.images(train)
    c = warmstart.output_scale(x, t)
    net = binding_unet.UNet(4, 16, N, N, max_batch=16, normalise=True, out_scale=c, seed=1)
    xd = torch.tensor(x, device="cuda")
    td = torch.tensor(t, device="cuda")
    losses = warmstart.fit(net, xd, td, steps=1500, batch=16, lr=2e-3, log_every=500)
    yield {"prob": prob, "net": net, "held": held, "losses": losses}
    net.close()


def _net_guess(net, rho):
    x = torch.tensor(warmstart.rho_image(rho)[None], device="cuda")
    y = torch.zeros_like(x)
    net.forward(x, y)
    return warmstart.guess_from_image(y[0].cpu().numpy().astype(np.float64))


def test_training_lowers_the_loss(trained):
    losses = trained["losses"]
    assert losses[-1][1] < 0.2 * losses[0][1], losses


def test_learned_guess_saves_cg_iterations(trained):
    """Held-out pairs: iterations of the standalone CG (rtol 1e-8) from the zero
    guess, from the previous step's phi, and from the network's guess; the three
    solutions agree to the solver's tolerance."""
    g = binding2d.Simulation2D(trained["prob"])
    held = trained["held"]
    its = {"zero": [], "prev": [], "unet": []}
    for rho, phi_prev in zip(held["rho"], held["phi_prev"]):
        p0, i0, r0 = g.solve_poisson(rho)
        p1, i1, r1 = g.solve_poisson(rho, phi_prev)
        p2, i2, r2 = g.solve_poisson(rho, _net_guess(trained["net"], rho))
        for r in (r0, r1, r2):
            assert r <= 1e-8
        scale = np.abs(p0).max()
        assert np.abs(p2 - p0).max() <= 1e-5 * scale
        assert np.abs(p1 - p0).max() <= 1e-5 * scale
        its["zero"].append(i0)
        its["prev"].append(i1)
        its["unet"].append(i2)
    g.close()
    mean = {k: float(np.mean(v)) for k, v in its.items()}
    print("CG iterations (mean over held-out pairs):", mean)
    assert mean["unet"] < 0.85 * mean["zero"], mean


def test_in_step_warm_start_modes_agree(trained):
    """Three copies of one run, the CG started each step from the previous phi,
    from the zero guess and from the network: the same fields to the solver's
    tolerance, and the learned guess needs fewer iterations than the zero one."""
    prob = _prob(seed=105)
    st = inputs.load_state2d(prob)
    sims, its = [], []
    for mode in (binding2d.SLPIC2D_WARM_PREV, binding2d.SLPIC2D_WARM_ZERO,
                 binding2d.SLPIC2D_WARM_UNET):
        g = binding2d.Simulation2D(prob)
        g.load_state(st)
        g.prepare()
        g.set_warm_start(mode, trained["net"] if mode == binding2d.SLPIC2D_WARM_UNET else None)
        total = 0
        for _ in range(4):
            g.step(1)
            total += g.diagnostics()["cg_iterations"]
        its.append(total)
        sims.append(g)
    phis = [s.fields()[1] for s in sims]
    scale = np.abs(phis[0]).max()
    for p in phis[1:]:
        assert np.abs(p - phis[0]).max() <= 1e-4 * scale
    assert its[2] < its[1], its
    for s in sims:
        s.close()


def test_warm_start_rejects_a_network_of_the_wrong_grid():
    g = binding2d.Simulation2D(_prob())
    net = binding_unet.UNet(2, 4, N, 2 * N)
    with pytest.raises(binding2d.SlpicError) as ei:
        g.set_warm_start(binding2d.SLPIC2D_WARM_UNET, net)
    assert ei.value.code == binding2d.binding.SLPIC_ERR_INVALID
    with pytest.raises(binding2d.SlpicError):
        g.set_warm_start(binding2d.SLPIC2D_WARM_UNET, None)
    g.set_warm_start(binding2d.SLPIC2D_WARM_ZERO)
    net.close()
    g.close()
