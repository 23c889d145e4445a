"""FP64 reference of the small convolutional U-Net that warm-starts the 2D CG.

TEST INFRASTRUCTURE, like the rest of ``oracle/``: only the tests, the smoke check
and the benchmark's CPU legs use it; the CUDA library has its own kernels.

The paper has no learned part.  The network follows the plain U-Net pattern
(Ronneberger et al., 2015) at the size the 2D CG needs, written out step by step
in numpy so that a reader can check every layer and every gradient:

  level l = 0..L-1 has C_l = C * 2^l channels.
  encoder:  e_0 = relu(conv(x)),  e_l = relu(conv(pool(e_{l-1})))    (l >= 1)
  decoder:  d_{L-1} = e_{L-1},
            d_l = relu(conv(concat(up(d_{l+1}), e_l)))             (l = L-2..0)
  output:   y = conv(d_0)                                          (1 channel)

conv: 3x3, zero padding, stride 1, with bias.  pool: 2x2 average.  up: nearest
neighbour x2.  concat: channels of up(d_{l+1}) first, then e_l.  Tensors are
(channels, H, W); weights (c_out, c_in, 3, 3).  The loss is the mean squared
error.  Gradients are formed by hand, layer by layer, in reverse.
"""
from __future__ import annotations

import numpy as np


def layer_shapes(levels: int, base: int):
    """(c_in, c_out) of every conv, in parameter order: encoder 0..L-1, decoder
    L-2..0, output."""
    ch = [base * 2 ** l for l in range(levels)]
    shapes = [(1, ch[0])] + [(ch[l - 1], ch[l]) for l in range(1, levels)]
    shapes += [(ch[l + 1] + ch[l], ch[l]) for l in range(levels - 2, -1, -1)]
    shapes.append((ch[0], 1))
    return shapes


def init_params(levels: int, base: int, seed: int = 0):
    """He-normal weights, zero biases: a list of (W, b)."""
    rng = np.random.default_rng(seed)
    out = []
    for ci, co in layer_shapes(levels, base):
        w = rng.normal(0.0, np.sqrt(2.0 / (9 * ci)), (co, ci, 3, 3))
        out.append((w, np.zeros(co)))
    return out


def bf16(a):
    """Round to bfloat16 (nearest, ties to even) and back: the precision of the
    GPU's weights."""
    a = np.asarray(a, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


# ------------------------------------------------------------------ layers
def conv(x, w, b):
    """3x3 convolution with zero padding: y[o,i,j] = b[o] + sum_{c,di,dj}
    w[o,c,di,dj] x[c, i+di-1, j+dj-1]."""
    c, h, wd = x.shape
    xp = np.zeros((c, h + 2, wd + 2))
    xp[:, 1:-1, 1:-1] = x
    y = np.zeros((w.shape[0], h, wd)) + b[:, None, None]
    for di in range(3):
        for dj in range(3):
            y += np.einsum("oc,chw->ohw", w[:, :, di, dj], xp[:, di:di + h, dj:dj + wd])
    return y


def conv_backward(x, w, dy):
    """Gradients of conv: (dx, dw, db)."""
    c, h, wd = x.shape
    xp = np.zeros((c, h + 2, wd + 2))
    xp[:, 1:-1, 1:-1] = x
    dxp = np.zeros_like(xp)
    dw = np.zeros_like(w)
    for di in range(3):
        for dj in range(3):
            dw[:, :, di, dj] = np.einsum("ohw,chw->oc", dy, xp[:, di:di + h, dj:dj + wd])
            dxp[:, di:di + h, dj:dj + wd] += np.einsum("oc,ohw->chw", w[:, :, di, dj], dy)
    return dxp[:, 1:-1, 1:-1], dw, dy.sum(axis=(1, 2))


def pool(x):
    c, h, w = x.shape
    return x.reshape(c, h // 2, 2, w // 2, 2).mean(axis=(2, 4))


def pool_backward(dy):
    return np.repeat(np.repeat(dy, 2, axis=1), 2, axis=2) * 0.25


def up(x):
    return np.repeat(np.repeat(x, 2, axis=1), 2, axis=2)


def up_backward(dy):
    c, h, w = dy.shape
    return dy.reshape(c, h // 2, 2, w // 2, 2).sum(axis=(2, 4))


# ------------------------------------------------------------------ network
def forward(params, x, levels: int, act_bf16: bool = False):
    """y and the cache the backward pass needs.  x: (H, W), H and W divisible by
    2^(levels-1).  With act_bf16 every conv's input is rounded to bfloat16 first
    (the precision of tensor-core operands); the cache keeps the rounded inputs,
    so the weight gradients multiply by them, and the input gradients pass the
    rounding through unchanged."""
    rnd = (lambda a: bf16(a)) if act_bf16 else (lambda a: a)
    cache = {"in": [], "pre": []}
    k = 0
    h = x[None].astype(np.float64)
    enc = []
    for l in range(levels):
        if l > 0:
            h = pool(h)
        h = rnd(h)
        cache["in"].append(h)
        z = conv(h, *params[k])
        cache["pre"].append(z)
        h = np.maximum(z, 0.0)
        enc.append(h)
        k += 1
    d = enc[-1]
    for l in range(levels - 2, -1, -1):
        cat = rnd(np.concatenate([up(d), enc[l]], axis=0))
        cache["in"].append(cat)
        z = conv(cat, *params[k])
        cache["pre"].append(z)
        d = np.maximum(z, 0.0)
        k += 1
    d = rnd(d)
    cache["in"].append(d)
    y = conv(d, *params[k])
    return y[0], cache


def backward(params, cache, dy, levels: int, act_bf16: bool = False):
    """Parameter gradients [(dW, db)] for the loss gradient dy = dL/dy (H, W).  With
    act_bf16 (tensor-core operands) each conv's input and weight gradients are formed
    from its output gradient rounded to bfloat16; the bias gradients from it
    unrounded."""
    def cb(x, w, gz):
        gx, dw, db = conv_backward(x, w, gz)
        if act_bf16:
            gx, dw, _ = conv_backward(x, w, bf16(gz))
        return gx, dw, db

    grads = [None] * len(params)
    k = len(params) - 1
    g, dw, db = cb(cache["in"][k], params[k][0], dy[None])
    grads[k] = (dw, db)
    d_enc = [np.zeros_like(cache["pre"][l]) for l in range(levels)]
    g_d = g  # gradient at the output of the current decoder level (d_l)
    for l in range(0, levels - 1):
        k -= 1
        gz = g_d * (cache["pre"][k] > 0)
        gc, dw, db = cb(cache["in"][k], params[k][0], gz)
        grads[k] = (dw, db)
        c_up = cache["in"][k].shape[0] - d_enc[l].shape[0]
        d_enc[l] += gc[c_up:]
        g_d = up_backward(gc[:c_up])  # gradient at d_{l+1}
    # g_d is now the gradient at d_{L-1} = e_{L-1}
    d_enc[levels - 1] += g_d
    for l in range(levels - 1, -1, -1):
        k = l
        gz = d_enc[l] * (cache["pre"][k] > 0)
        gi, dw, db = cb(cache["in"][k], params[k][0], gz)
        grads[k] = (dw, db)
        if l > 0:
            d_enc[l - 1] += pool_backward(gi)
    return grads


def mse(y, t):
    """Mean squared error and its gradient."""
    r = y - t
    return float((r * r).mean()), 2.0 * r / r.size


def energy(y, t):
    """Energy-norm loss of the error e = y - t on the 2D solver's grid, for one
    (H, W) image: rows are y (row 0 a plate, the other plate just past row H-1,
    both held at zero), columns x (periodic).  e is zeroed on row 0 (the plate's
    value is not the network's), and
        L = (e . A e) / (H W),  A e = 4 e - e(x+1) - e(x-1) - e(y+1) - e(y-1)
    (the 5-point operator of the field solve, zero outside rows 0..H-1); the
    gradient is 2 A e / (H W), zero on row 0.  Returns (L, dL/dy)."""
    e = np.array(y - t, dtype=np.float64)
    e[0] = 0.0
    ep = np.zeros((e.shape[0] + 1, e.shape[1]))
    ep[:-1] = e
    ae = 4 * e - np.roll(e, 1, axis=1) - np.roll(e, -1, axis=1) - ep[1:] - np.roll(ep, 1, axis=0)[:-1]
    ae[0] = 0.0
    n = e.size
    return float((e * ae).sum() / n), 2.0 * ae / n
