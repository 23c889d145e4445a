"""The U-Net's CUDA forward, backward and Adam step against the FP64 oracle
(oracle/unet.py) on the same seeded inputs, through the C ABI.

The GPU multiplies by BF16 copies of the FP32 weights and accumulates in FP32;
the oracle is given the same BF16-rounded weights and runs in FP64, so the
difference is FP32 accumulation alone: the bar is 1e-3 of each tensor's largest
entry, tighter than the 1e-2 a BF16 network calls for."""
import numpy as np
import pytest

from oracle import unet as ounet
from paper_1511_08225_gb300 import binding_unet

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-3


def _params(levels, base, seed):
    rng = np.random.default_rng(seed)
    return [(np.float32(w), np.float32(rng.normal(0, 0.1, b.shape)))
            for w, b in ounet.init_params(levels, base, seed=seed)]


def _bf(params):
    return [(ounet.bf16(w), b.astype(np.float64)) for w, b in params]


def _tc_available():
    return torch.cuda.is_available() and torch.cuda.get_device_capability(0)[0] >= 10


def _dev(a):
    return torch.tensor(np.ascontiguousarray(a, dtype=np.float32), device="cuda")


def _oracle_grads(params, xs, ts, levels, energy=False, act_bf16=False):
    """Summed over the samples, for the mean over all samples and pixels."""
    pb = _bf(params)
    count = xs.size
    grads = None
    loss = 0.0
    for x, t in zip(xs, ts):
        y, cache = ounet.forward(pb, x.astype(np.float32).astype(np.float64), levels,
                                 act_bf16=act_bf16)
        if energy:
            lk, dy = ounet.energy(y, t)
            loss += lk * y.size
            dy = dy * (y.size / count)
        else:
            r = y - t
            loss += float((r * r).sum())
            dy = 2.0 * r / count
        g = ounet.backward(pb, cache, dy, levels, act_bf16=act_bf16)
        grads = g if grads is None else [(a + c, b + d) for (a, b), (c, d) in zip(grads, g)]
    return loss / count, grads


@pytest.mark.parametrize("levels,base,n,nb", [(2, 8, 32, 2), (3, 4, 16, 3), (1, 3, 8, 1),
                                              (4, 8, 40, 2)])
def test_forward_matches_oracle(levels, base, n, nb):
    params = _params(levels, base, seed=levels * 10 + base)
    rng = np.random.default_rng(7)
    xs = rng.normal(size=(nb, n, n))
    net = binding_unet.UNet(levels, base, n, n, max_batch=nb, normalise=False)
    net.set_params(params)
    y = torch.zeros((nb, n, n), device="cuda")
    net.forward(_dev(xs), y)
    got = y.cpu().numpy()
    for k in range(nb):
        ref = ounet.forward(_bf(params), xs[k], levels)[0]
        assert np.abs(got[k] - ref).max() <= TOL * np.abs(ref).max(), k
    net.close()


def test_forward_scaling_is_per_sample_rms():
    """With normalisation: y_n = s_n * c * net(x_n / s_n), s_n the RMS of x_n; an
    all-zero sample gives net(0) * c."""
    levels, base, n = 3, 4, 16
    params = _params(levels, base, seed=3)
    rng = np.random.default_rng(8)
    xs = np.stack([rng.normal(size=(n, n)) * 40.0, np.zeros((n, n)), rng.normal(size=(n, n)) * 1e-3])
    c = 2.5
    net = binding_unet.UNet(levels, base, n, n, max_batch=3, normalise=True, out_scale=c)
    net.set_params(params)
    y = torch.zeros((3, n, n), device="cuda")
    net.forward(_dev(xs), y)
    got = y.cpu().numpy()
    for k in range(3):
        x32 = xs[k].astype(np.float32).astype(np.float64)
        s = np.sqrt((x32 ** 2).mean()) or 1.0
        ref = s * c * ounet.forward(_bf(params), x32 / s, levels)[0]
        assert np.abs(got[k] - ref).max() <= TOL * np.abs(ref).max(), k
    net.close()


@pytest.mark.parametrize("levels,base,n,nb", [(2, 8, 32, 2), (3, 4, 16, 3), (1, 3, 8, 2)])
def test_gradients_match_oracle(levels, base, n, nb):
    params = _params(levels, base, seed=levels + base)
    rng = np.random.default_rng(levels * base)
    xs, ts = rng.normal(size=(nb, n, n)), rng.normal(size=(nb, n, n))
    net = binding_unet.UNet(levels, base, n, n, max_batch=nb, normalise=False)
    net.set_params(params)
    loss, grads = net.gradients(_dev(xs), _dev(ts))
    ref_loss, ref = _oracle_grads(params, xs, ts, levels)
    assert loss == pytest.approx(ref_loss, rel=1e-5)
    for k, ((dw, db), (rw, rb)) in enumerate(zip(grads, ref)):
        assert np.abs(dw - rw).max() <= TOL * np.abs(rw).max(), ("W", k)
        assert np.abs(db - rb).max() <= TOL * max(np.abs(rb).max(), 1e-12), ("b", k)
    # the parameters are left alone
    for (w, b), (w2, b2) in zip(params, net.params()):
        assert np.array_equal(w, w2) and np.array_equal(b, b2)
    net.close()


@pytest.mark.parametrize("levels,base,n,nb", [(2, 8, 32, 2), (3, 4, 16, 1)])
def test_energy_loss_gradients_match_oracle(levels, base, n, nb):
    params = _params(levels, base, seed=5 + levels)
    rng = np.random.default_rng(20 + levels)
    xs, ts = rng.normal(size=(nb, n, n)), rng.normal(size=(nb, n, n))
    net = binding_unet.UNet(levels, base, n, n, max_batch=nb, normalise=False,
                            loss=binding_unet.SLPIC_UNET_LOSS_ENERGY)
    net.set_params(params)
    loss, grads = net.gradients(_dev(xs), _dev(ts))
    ref_loss, ref = _oracle_grads(params, xs, ts, levels, energy=True)
    assert loss == pytest.approx(ref_loss, rel=1e-5)
    for k, ((dw, db), (rw, rb)) in enumerate(zip(grads, ref)):
        assert np.abs(dw - rw).max() <= TOL * np.abs(rw).max(), ("W", k)
        assert np.abs(db - rb).max() <= TOL * max(np.abs(rb).max(), 1e-12), ("b", k)
    net.close()


# ---------------------------------------------------------------- tensor cores
@pytest.mark.parametrize("levels,base,n,nb", [(2, 8, 32, 2), (3, 4, 16, 3), (4, 8, 40, 2),
                                              (1, 3, 8, 1), (4, 32, 64, 1)])
def test_tensor_core_forward_matches_oracle(levels, base, n, nb):
    """tcgen05 implicit-GEMM convolutions (BF16 operands, FP32 accumulation in
    tensor memory) against the oracle with every conv input rounded to BF16: a
    ragged last pixel tile (40 x 40), a grid smaller than one tile (8 x 8), 3 and
    256 output channels.  The bar is 1e-2 of the largest output: a
    conv input whose FP32 and FP64 values straddle a BF16 rounding boundary rounds
    differently on the two sides, and with 256 channels a few hundred of the
    ~700k activations do.  The mean error is less than half that against the
    FP32-input oracle, so the tensor-core path is the one that ran."""
    assert _tc_available()
    params = _params(levels, base, seed=levels * 7 + base)
    rng = np.random.default_rng(17)
    xs = rng.normal(size=(nb, n, n))
    net = binding_unet.UNet(levels, base, n, n, max_batch=nb, normalise=False, tensor_cores=True)
    net.set_params(params)
    y = torch.zeros((nb, n, n), device="cuda")
    net.forward(_dev(xs), y)
    got = y.cpu().numpy()
    for k in range(nb):
        x64 = xs[k].astype(np.float32).astype(np.float64)
        ref = ounet.forward(_bf(params), x64, levels, act_bf16=True)[0]
        ref32 = ounet.forward(_bf(params), x64, levels)[0]
        err = np.abs(got[k] - ref)
        assert err.max() <= 1e-2 * np.abs(ref).max(), (k, err.max())
        assert err.mean() < 0.5 * np.abs(got[k] - ref32).mean(), k
    net.close()


@pytest.mark.parametrize("levels,base,n,nb", [(2, 8, 32, 2), (3, 4, 16, 1), (4, 32, 32, 1)])
def test_tensor_core_gradients_match_oracle(levels, base, n, nb):
    """Forward and input-gradient convolutions on the tensor cores; (4, 32, 32) has a
    transposed conv of 384 output channels, done in two slices."""
    params = _params(levels, base, seed=31 + levels)
    rng = np.random.default_rng(32 + levels)
    xs, ts = rng.normal(size=(nb, n, n)), rng.normal(size=(nb, n, n))
    net = binding_unet.UNet(levels, base, n, n, max_batch=nb, normalise=False, tensor_cores=True)
    net.set_params(params)
    loss, grads = net.gradients(_dev(xs), _dev(ts))
    ref_loss, ref = _oracle_grads(params, xs, ts, levels, act_bf16=True)
    assert loss == pytest.approx(ref_loss, rel=1e-3)
    for k, ((dw, db), (rw, rb)) in enumerate(zip(grads, ref)):
        assert np.abs(dw - rw).max() <= 1e-2 * np.abs(rw).max(), ("W", k)
        assert np.abs(db - rb).max() <= 1e-2 * max(np.abs(rb).max(), 1e-12), ("b", k)
    net.close()


def test_tensor_core_training_repacks_weights_after_each_step():
    """Two Adam steps, then the forward pass: the output matches the oracle at the
    parameters the library now holds (the packed tensor-core weights follow)."""
    levels, base, n = 2, 8, 32
    params = _params(levels, base, seed=41)
    rng = np.random.default_rng(42)
    xs, ts = rng.normal(size=(2, n, n)), rng.normal(size=(2, n, n))
    net = binding_unet.UNet(levels, base, n, n, max_batch=2, normalise=False, tensor_cores=True)
    net.set_params(params)
    for _ in range(2):
        net.train_step(_dev(xs), _dev(ts), 1e-2)
    now = net.params()
    y = torch.zeros((2, n, n), device="cuda")
    net.forward(_dev(xs), y)
    ref = ounet.forward(_bf(now), xs[0].astype(np.float32).astype(np.float64), levels,
                        act_bf16=True)[0]
    assert np.abs(y[0].cpu().numpy() - ref).max() <= 2e-3 * np.abs(ref).max()
    net.close()


def test_two_adam_steps_match_the_textbook_update():
    """Adam (Kingma & Ba, 2015), b1 = 0.9, b2 = 0.999, eps = 1e-8, on two
    different batches: the moments and the bias corrections of both steps."""
    levels, base, n = 2, 4, 16
    params = _params(levels, base, seed=11)
    rng = np.random.default_rng(12)
    batches = [(rng.normal(size=(2, n, n)), rng.normal(size=(2, n, n))) for _ in range(2)]
    lr, b1, b2, eps = 1e-3, 0.9, 0.999, 1e-8
    net = binding_unet.UNet(levels, base, n, n, max_batch=2, normalise=False)
    net.set_params(params)
    ref = [(w.astype(np.float64), b.astype(np.float64)) for w, b in params]
    m = [(np.zeros_like(w), np.zeros_like(b)) for w, b in ref]
    v = [(np.zeros_like(w), np.zeros_like(b)) for w, b in ref]
    for step, (xs, ts) in enumerate(batches, start=1):
        before = net.params()
        net.train_step(_dev(xs), _dev(ts), lr)
        after = net.params()
        cur = [(np.float32(w), np.float32(b)) for w, b in ref]
        _, g = _oracle_grads(cur, xs, ts, levels)
        new_ref = []
        for k in range(len(ref)):
            pair = []
            for a in range(2):
                m[k][a][...] = b1 * m[k][a] + (1 - b1) * g[k][a]
                v[k][a][...] = b2 * v[k][a] + (1 - b2) * g[k][a] ** 2
                vh = v[k][a] / (1 - b2 ** step)
                delta = -lr * (m[k][a] / (1 - b1 ** step)) / (np.sqrt(vh) + eps)
                got = after[k][a].astype(np.float64) - before[k][a]
                sel = np.sqrt(vh) > 1e-2 * np.sqrt(vh).max()
                assert np.abs(got - delta)[sel].max() <= 1e-2 * lr, (step, k, a)
                assert np.abs(got).max() <= lr * 1.001 * (1 + (step > 1)), (step, k, a)
                pair.append(ref[k][a] + delta)
            new_ref.append(tuple(pair))
        ref = new_ref
    net.close()


def test_training_fits_a_fixed_linear_map():
    """A property at any size: Adam on the GPU's own gradients drives the loss of a
    fixed smooth target (a blurred copy of the input) down tenfold."""
    levels, base, n, nb = 3, 8, 32, 8
    rng = np.random.default_rng(5)
    net = binding_unet.UNet(levels, base, n, n, max_batch=nb, normalise=False, seed=2)
    xs = torch.tensor(rng.normal(size=(64, n, n)), dtype=torch.float32, device="cuda")
    k = torch.tensor([[1.0, 2.0, 1.0], [2.0, 4.0, 2.0], [1.0, 2.0, 1.0]], device="cuda") / 16
    ts = torch.nn.functional.conv2d(xs[:, None], k[None, None], padding=1)[:, 0].contiguous()
    first = net.train_step(xs[:nb].contiguous(), ts[:nb].contiguous(), 2e-3, want_loss=True)
    last = None
    for it in range(400):
        j = (it * nb) % 64
        last = net.train_step(xs[j:j + nb].contiguous(), ts[j:j + nb].contiguous(), 2e-3,
                              want_loss=(it == 399))
    assert last < 0.1 * first, (first, last)
    net.close()


# ---------------------------------------------------------------- against the plain oracle
@pytest.mark.parametrize("levels,base,n,nb", [(2, 8, 32, 2), (3, 4, 16, 3), (4, 8, 40, 2),
                                              (1, 3, 8, 1), (4, 32, 64, 1)])
def test_tensor_core_forward_within_bf16_bar_of_plain_oracle(levels, base, n, nb):
    """The tensor-core forward against the plain FP64 oracle, which rounds nothing but
    the weights (the BF16 weights are the network's parameters as stored): within
    1e-2 of the largest output, the bar a BF16 network is held to.  The BF16-input
    oracle mode above states where the kernels round; this bar does not depend on
    that mode."""
    assert _tc_available()
    params = _params(levels, base, seed=levels * 7 + base)
    rng = np.random.default_rng(17)
    xs = rng.normal(size=(nb, n, n))
    net = binding_unet.UNet(levels, base, n, n, max_batch=nb, normalise=False, tensor_cores=True)
    net.set_params(params)
    y = torch.zeros((nb, n, n), device="cuda")
    net.forward(_dev(xs), y)
    got = y.cpu().numpy()
    for k in range(nb):
        ref = ounet.forward(_bf(params), xs[k].astype(np.float32).astype(np.float64), levels)[0]
        assert np.abs(got[k] - ref).max() <= 1e-2 * np.abs(ref).max(), k
    net.close()


@pytest.mark.parametrize("levels,base,n,nb", [(2, 8, 32, 2), (3, 4, 16, 1), (4, 32, 32, 1)])
def test_tensor_core_gradients_against_plain_oracle(levels, base, n, nb):
    """Loss and parameter gradients of the tensor-core path against the plain FP64
    oracle's (BF16 weights, nothing else rounded).  BF16 activations alone move a
    small random network's weight gradients: by up to ~14 % of a layer's largest
    entry at (3, 4, 16), oracle against oracle, through flipped ReLU masks and
    cancelling sums.  So the bar is that deviation, measured here by the oracle
    alone (its BF16-operand mode against its plain mode), plus 1e-2 of the layer's
    largest entry, and every layer's gradient must point the same way as the plain
    one (cosine >= 0.99)."""
    params = _params(levels, base, seed=31 + levels)
    rng = np.random.default_rng(32 + levels)
    xs, ts = rng.normal(size=(nb, n, n)), rng.normal(size=(nb, n, n))
    net = binding_unet.UNet(levels, base, n, n, max_batch=nb, normalise=False, tensor_cores=True)
    net.set_params(params)
    loss, grads = net.gradients(_dev(xs), _dev(ts))
    ref_loss, ref = _oracle_grads(params, xs, ts, levels, act_bf16=False)
    _, ref16 = _oracle_grads(params, xs, ts, levels, act_bf16=True)
    assert loss == pytest.approx(ref_loss, rel=1e-2)
    for k, ((dw, db), (rw, rb), (qw, qb)) in enumerate(zip(grads, ref, ref16)):
        assert np.abs(dw - rw).max() <= np.abs(qw - rw).max() + 1e-2 * np.abs(rw).max(), ("W", k)
        cos = float((dw.astype(np.float64) * rw).sum() /
                    np.sqrt((dw.astype(np.float64) ** 2).sum() * (rw * rw).sum()))
        assert cos >= 0.99, ("W", k, cos)
        assert np.abs(db - rb).max() <= np.abs(qb - rb).max() + \
            1e-2 * max(np.abs(rb).max(), 1e-12), ("b", k)
    net.close()
