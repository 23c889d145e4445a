"""Pins of the U-Net oracle (no GPU), each resting on something other than the
oracle: a library correlation, adjoint identities, bfloat16 values worked out by
hand, and central finite differences of the loss for parameters of every layer
(2-level, 8-channel nets at 32 x 32 among them)."""
import numpy as np
import pytest
from scipy import signal

from oracle import unet


def test_conv_single_channel_is_a_2d_correlation():
    rng = np.random.default_rng(1)
    x = rng.normal(size=(1, 9, 11))
    w = rng.normal(size=(1, 1, 3, 3))
    b = np.array([0.3])
    y = unet.conv(x, w, b)
    ref = signal.correlate2d(x[0], w[0, 0], mode="same", boundary="fill", fillvalue=0.0) + 0.3
    assert np.abs(y[0] - ref).max() < 1e-12


def test_conv_channels_add_up():
    rng = np.random.default_rng(2)
    x = rng.normal(size=(3, 6, 6))
    w = rng.normal(size=(2, 3, 3, 3))
    b = rng.normal(size=2)
    y = unet.conv(x, w, b)
    for o in range(2):
        ref = b[o] + sum(signal.correlate2d(x[c], w[o, c], mode="same") for c in range(3))
        assert np.abs(y[o] - ref).max() < 1e-12


def test_pool_and_up_backward_are_adjoints():
    """<up(a), B> = <a, up^T(B)> and <pool(A), b> = <A, pool^T(b)>."""
    rng = np.random.default_rng(3)
    a, B = rng.normal(size=(2, 4, 5)), rng.normal(size=(2, 8, 10))
    assert np.isclose((unet.up(a) * B).sum(), (a * unet.up_backward(B)).sum())
    assert np.isclose((unet.pool(B) * a).sum(), (B * unet.pool_backward(a)).sum())
    assert np.allclose(unet.pool(unet.up(a)), a)


def test_bf16_rounding():
    """8 significant bits, round to nearest, ties to even."""
    vals = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, 1.0 + 2 ** -7, -2.5 + 2 ** -9,
                     3.0e-3], np.float32)
    out = unet.bf16(vals)
    assert out[0] == 1.0
    assert out[1] == 1.0                      # halfway: to the even 1.0
    assert out[2] == 1.0 + 2 ** -6            # halfway: to the even 1 + 2^-6
    assert out[3] == 1.0 + 2 ** -7            # representable
    assert out[4] == -2.5                     # below half an ulp (2^-7 at 2.5)
    assert abs(out[5] / 3.0e-3 - 1) < 2 ** -8


def test_layer_shapes():
    assert unet.layer_shapes(2, 8) == [(1, 8), (8, 16), (24, 8), (8, 1)]
    assert unet.layer_shapes(4, 32)[3] == (128, 256)
    assert unet.layer_shapes(4, 32)[4] == (256 + 128, 128)


@pytest.mark.parametrize("levels,base,n", [(2, 8, 32), (3, 4, 16), (1, 3, 8)])
def test_gradients_match_finite_differences(levels, base, n):
    rng = np.random.default_rng(levels + base)
    params = unet.init_params(levels, base, seed=4)
    # nonzero biases so every ReLU sees both signs
    params = [(w, rng.normal(0, 0.1, b.shape)) for w, b in params]
    x = rng.normal(size=(n, n))
    t = rng.normal(size=(n, n))
    y, cache = unet.forward(params, x, levels)
    loss, dy = unet.mse(y, t)
    grads = unet.backward(params, cache, dy, levels)
    h = 1e-6
    for k, ((w, b), (dw, db)) in enumerate(zip(params, grads)):
        for idx in [tuple(rng.integers(0, s) for s in w.shape) for _ in range(3)]:
            wp = [(ww.copy(), bb.copy()) for ww, bb in params]
            wp[k][0][idx] += h
            lp = unet.mse(unet.forward(wp, x, levels)[0], t)[0]
            wp[k][0][idx] -= 2 * h
            lm = unet.mse(unet.forward(wp, x, levels)[0], t)[0]
            fd = (lp - lm) / (2 * h)
            assert abs(fd - dw[idx]) <= 1e-5 * max(abs(fd), 1e-3), (k, idx, fd, dw[idx])
        j = int(rng.integers(0, b.size))
        wp = [(ww.copy(), bb.copy()) for ww, bb in params]
        wp[k][1][j] += h
        lp = unet.mse(unet.forward(wp, x, levels)[0], t)[0]
        wp[k][1][j] -= 2 * h
        lm = unet.mse(unet.forward(wp, x, levels)[0], t)[0]
        assert abs((lp - lm) / (2 * h) - db[j]) <= 1e-5 * max(abs(db[j]), 1e-3)


def test_energy_loss_is_the_sum_over_grid_edges():
    """Discrete Green identity: e . A e is the sum over all grid edges of the
    squared difference across the edge, the edges to the plates (held at zero)
    included, and the periodic edge in x too."""
    rng = np.random.default_rng(9)
    y, t = rng.normal(size=(6, 5)), rng.normal(size=(6, 5))
    loss, _ = unet.energy(y, t)
    e = y - t
    e[0] = 0.0
    full = np.zeros((8, 5))          # plate row, rows 0..5 (row 0 zeroed), plate row
    full[1:7] = e
    s = ((full[1:] - full[:-1]) ** 2).sum()          # vertical edges, both plates
    s += ((e - np.roll(e, -1, axis=1)) ** 2)[1:].sum()   # horizontal, periodic, interior rows
    # row 0 is a plate: its vertical edge to row 1 counts once, as above
    assert loss * e.size == pytest.approx(s, rel=1e-12)
    assert loss > 0


def test_energy_gradient_matches_finite_differences():
    rng = np.random.default_rng(10)
    y, t = rng.normal(size=(5, 4)), rng.normal(size=(5, 4))
    _, g = unet.energy(y, t)
    h = 1e-6
    for idx in [(0, 1), (1, 0), (4, 3), (2, 2)]:
        yp, ym = y.copy(), y.copy()
        yp[idx] += h
        ym[idx] -= h
        fd = (unet.energy(yp, t)[0] - unet.energy(ym, t)[0]) / (2 * h)
        assert fd == pytest.approx(g[idx], abs=1e-8)
    assert np.all(g[0] == 0.0)


def test_bf16_activation_mode_rounds_every_conv_input():
    """The tensor-core precision: every conv input the cache keeps is a bfloat16
    value, the output stays within the rounding's bound of the FP64 forward, and
    the rounding is really applied (the two differ)."""
    levels, base, n = 3, 4, 16
    rng = np.random.default_rng(11)
    params = [(unet.bf16(w), rng.normal(0, 0.1, b.shape)) for w, b in unet.init_params(levels, base, 5)]
    x = rng.normal(size=(n, n))
    y64, _ = unet.forward(params, x, levels)
    y16, cache = unet.forward(params, x, levels, act_bf16=True)
    for a in cache["in"]:
        assert np.array_equal(unet.bf16(a), a)
    rel = np.abs(y16 - y64).max() / np.abs(y64).max()
    assert 1e-6 < rel < 3e-2, rel
    # the backward pass takes the rounded inputs: its weight gradient of the
    # output conv is the correlation of the rounded d_0 with dy
    dy = rng.normal(size=(n, n))
    g = unet.backward(params, cache, dy, levels)
    dw_ref = np.einsum("hw,chw->c", dy, cache["in"][-1])  # centre tap, no shift
    assert np.allclose(g[-1][0][0, :, 1, 1], dw_ref, rtol=1e-12, atol=1e-12)
    # with the tensor-core rounding of output gradients: the bias gradients take dy
    # unrounded, the weight gradients the rounded one (close, not equal)
    g16 = unet.backward(params, cache, dy, levels, act_bf16=True)
    assert np.array_equal(g16[-1][1], g[-1][1])
    dw16 = np.einsum("hw,chw->c", unet.bf16(dy), cache["in"][-1])
    assert np.allclose(g16[-1][0][0, :, 1, 1], dw16, rtol=1e-12, atol=1e-12)
    for k in (0, -1):
        rel = np.abs(g16[k][0] - g[k][0]).max() / np.abs(g[k][0]).max()
        assert 0 < rel < 3e-2, (k, rel)
