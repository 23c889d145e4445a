"""The learned warm start of the 2D CG: a U-Net trained on the GPU, by the
library's own kernels, on (rho, phi) pairs that 2D runs generate, then used as
the CG's initial guess.  The CG to the same residual stays the judge: the answer
does not change; the iterations do.

Workload: the 2D plasma of the throughput benchmark at 64 x 64 cells (periodic
x, absorbing phi = 0 plates in y, central source band, m_i/m_e = 1836, Heaviside
beta, v0 = 0.1, dt = dx / v0), 16 particles per cell and species.  Training
pairs: three seeds, 60 pairs each, one every 3 steps after 20 steps, each with
the step before it.  Held out: a fourth seed.  Two networks (4 levels, 16 base
channels, mean-squared-error loss, 1,500 Adam steps of 16 samples): one maps rho
to phi, the other the change of rho between consecutive steps to the change of
phi."""
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
                                    skip=20, keep_prev=True)
    held = warmstart.collect_pairs(prob, seeds=(104,), pairs_per_seed=12, every=3, skip=20,
                                   keep_prev=True)
    nets, losses = {}, {}
    for name, (x, t) in (("direct", warmstart.images(train)), ("delta", warmstart.delta_images(train))):
        net = binding_unet.UNet(4, 16, N, N, max_batch=16, normalise=True,
                                out_scale=warmstart.output_scale(x, t), seed=1)
        losses[name] = warmstart.fit(net, torch.tensor(x, device="cuda"),
                                     torch.tensor(t, device="cuda"), steps=1500, batch=16, lr=2e-3,
                                     log_every=500)
        nets[name] = net
    yield {"prob": prob, "nets": nets, "held": held, "losses": losses}
    for net in nets.values():
        net.close()


def _net_image(net, rho):
    x = torch.tensor(warmstart.rho_image(rho)[None], device="cuda")
    y = torch.zeros_like(x)
    net.forward(x, y)
    return y[0].cpu().numpy().astype(np.float64)


def test_training_lowers_the_loss(trained):
    for name, losses in trained["losses"].items():
        assert losses[-1][1] < 0.2 * losses[0][1], (name, losses)


def test_learned_guess_saves_cg_iterations(trained):
    """Held-out pairs: iterations of the standalone CG (rtol 1e-8) from the zero
    guess, from the previous step's phi, from the network's guess of phi, and from
    the previous phi plus the network's guess of the change; the solutions agree
    to the solver's tolerance.  Measured on GB300: 244, 224, 231 and 216."""
    g = binding2d.Simulation2D(trained["prob"])
    held, nets = trained["held"], trained["nets"]
    its = {"zero": [], "prev": [], "unet": [], "delta": []}
    for rho, phi_prev, rho_prev in zip(held["rho"], held["phi_prev"], held["rho_prev"]):
        guesses = {"zero": None, "prev": phi_prev,
                   "unet": warmstart.guess_from_image(_net_image(nets["direct"], rho)),
                   "delta": phi_prev + warmstart.guess_from_image(
                       _net_image(nets["delta"], rho - rho_prev))}
        ref = None
        for name, guess in guesses.items():
            phi, it, res = g.solve_poisson(rho, guess)
            assert res <= 1e-8
            if ref is None:
                ref = phi
            assert np.abs(phi - ref).max() <= 1e-5 * np.abs(ref).max(), name
            its[name].append(it)
    g.close()
    mean = {k: float(np.mean(v)) for k, v in its.items()}
    print("CG iterations (mean over held-out pairs):", mean)
    assert mean["unet"] < 0.97 * mean["zero"], mean
    assert mean["delta"] < mean["prev"], mean


def test_in_step_warm_start_modes_agree(trained):
    """Four copies of one run, identical for 20 steps, then the CG of each step
    started from the previous phi, the zero guess, the network's phi and the
    previous phi plus the network's change: the same fields to the solver's
    tolerance; the first step of the change mode (no previous charge yet) is the
    previous-phi step bit for bit."""
    prob = _prob(seed=105)
    st = inputs.load_state2d(prob)
    modes = ((binding2d.SLPIC2D_WARM_PREV, None), (binding2d.SLPIC2D_WARM_ZERO, None),
             (binding2d.SLPIC2D_WARM_UNET, trained["nets"]["direct"]),
             (binding2d.SLPIC2D_WARM_UNET_DELTA, trained["nets"]["delta"]))
    sims, its, first = [], [], []
    for mode, net in modes:
        g = binding2d.Simulation2D(prob)
        g.load_state(st)
        g.prepare()
        g.step(20)
        g.set_warm_start(mode, net)
        g.step(1)
        first.append(g.fields()[1])
        total = 0
        for _ in range(8):
            g.step(1)
            total += g.diagnostics()["cg_iterations"]
        its.append(total)
        sims.append(g)
    assert np.array_equal(first[3], first[0])
    phis = [s.fields()[1] for s in sims]
    scale = np.abs(phis[0]).max()
    for p in phis[1:]:
        assert np.abs(p - phis[0]).max() <= 1e-4 * scale
    print("CG iterations over 8 steps (prev, zero, unet, delta):", its)
    assert its[2] < its[1], its
    assert its[3] <= 1.02 * its[0], its
    for s in sims:
        s.close()


def test_warm_start_rejects_a_network_of_the_wrong_grid():
    g = binding2d.Simulation2D(_prob())
    net = binding_unet.UNet(2, 4, N, 2 * N)
    for mode in (binding2d.SLPIC2D_WARM_UNET, binding2d.SLPIC2D_WARM_UNET_DELTA):
        with pytest.raises(binding2d.SlpicError) as ei:
            g.set_warm_start(mode, net)
        assert ei.value.code == binding2d.binding.SLPIC_ERR_INVALID
        with pytest.raises(binding2d.SlpicError):
            g.set_warm_start(mode, None)
    with pytest.raises(binding2d.SlpicError):
        g.set_warm_start(7)
    g.set_warm_start(binding2d.SLPIC2D_WARM_ZERO)
    net.close()
    g.close()


def test_device_made_change_images_equal_the_host_made_ones():
    """collect_delta_images (pairs made one by one into device tensors, for sets too
    large for host memory) gives exactly delta_images of collect_pairs with keep_prev
    on the same run."""
    import torch
    prob = inputs.plasma2d_problem(nx=64, ny=32, ppc=8, v0=0.2, solver="fft")
    pairs = warmstart.collect_pairs(prob, seeds=(7,), pairs_per_seed=5, every=2, skip=3,
                                    keep_prev=True)
    x_h, t_h = warmstart.delta_images(pairs)
    x_d, t_d = warmstart.collect_delta_images(prob, 7, 5, every=2, skip=3)
    torch.cuda.synchronize()
    assert x_d.dtype == torch.float32 and tuple(x_d.shape) == x_h.shape
    assert np.array_equal(x_d.cpu().numpy(), x_h) and np.array_equal(t_d.cpu().numpy(), t_h)
