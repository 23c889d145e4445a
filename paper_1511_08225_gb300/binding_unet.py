"""Thin ctypes binding of the U-Net entry points of libslpic.so
(include/slpic_unet.h), same names.

Argument marshalling only: the forward pass, the gradients and the Adam step run
in the library's kernels; there is no CPU fallback.  x, y and t are torch CUDA
tensors (float32, contiguous, (nb, H, W)) or raw device pointers.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import binding
from .binding import SLPIC_OK, SlpicError

SLPIC_UNET_LOSS_MSE, SLPIC_UNET_LOSS_ENERGY = 0, 1

#: every function declared in include/slpic_unet.h
EXPORTS_UNET = (
    "slpic_unet_create", "slpic_unet_destroy", "slpic_unet_last_error", "slpic_unet_set_stream",
    "slpic_unet_param_count", "slpic_unet_set_params", "slpic_unet_get_params",
    "slpic_unet_forward", "slpic_unet_gradients", "slpic_unet_train_step",
    "slpic_unet_reset_optimizer",
)


class slpic_unet_config(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int32), ("base", ctypes.c_int32),
                ("height", ctypes.c_int32), ("width", ctypes.c_int32),
                ("max_batch", ctypes.c_int32), ("normalise", ctypes.c_int32),
                ("loss", ctypes.c_int32), ("tensor_cores", ctypes.c_int32),
                ("out_scale", ctypes.c_double), ("adam_beta1", ctypes.c_double),
                ("adam_beta2", ctypes.c_double), ("adam_eps", ctypes.c_double),
                ("seed", ctypes.c_uint64)]


_ready = False


def load_library() -> ctypes.CDLL:
    global _ready
    L = binding.load_library()
    if _ready:
        return L
    P, I, I32, I64, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    sig = {
        "slpic_unet_create": (I, [ctypes.POINTER(slpic_unet_config), ctypes.POINTER(P)]),
        "slpic_unet_destroy": (I, [P]),
        "slpic_unet_last_error": (ctypes.c_char_p, [P]),
        "slpic_unet_set_stream": (I, [P, P]),
        "slpic_unet_param_count": (I, [P, ctypes.POINTER(I64)]),
        "slpic_unet_set_params": (I, [P, P]),
        "slpic_unet_get_params": (I, [P, P]),
        "slpic_unet_forward": (I, [P, I32, P, P]),
        "slpic_unet_gradients": (I, [P, I32, P, P, ctypes.POINTER(D), P]),
        "slpic_unet_train_step": (I, [P, I32, P, P, D, ctypes.POINTER(D)]),
        "slpic_unet_reset_optimizer": (I, [P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _ready = True
    return L


def _check(h, rc: int, where: str):
    if rc != SLPIC_OK:
        msg = (load_library().slpic_unet_last_error(h) if h else b"invalid configuration") or b""
        raise SlpicError(rc, where, msg.decode())


def _dev(a) -> ctypes.c_void_p:
    """Device pointer of a torch CUDA tensor (float32, contiguous) or an int."""
    if isinstance(a, int):
        return ctypes.c_void_p(a)
    if not (a.is_cuda and a.is_contiguous() and str(a.dtype) == "torch.float32"):
        raise ValueError("expected a contiguous float32 CUDA tensor")
    return ctypes.c_void_p(a.data_ptr())


def slpic_unet_create(cfg: slpic_unet_config):
    h = ctypes.c_void_p()
    _check(None, load_library().slpic_unet_create(ctypes.byref(cfg), ctypes.byref(h)),
           "slpic_unet_create")
    return h


def slpic_unet_destroy(h):
    load_library().slpic_unet_destroy(h)


def slpic_unet_set_stream(h, stream: int):
    _check(h, load_library().slpic_unet_set_stream(h, ctypes.c_void_p(stream)),
           "slpic_unet_set_stream")


def slpic_unet_param_count(h) -> int:
    n = ctypes.c_int64()
    _check(h, load_library().slpic_unet_param_count(h, ctypes.byref(n)), "slpic_unet_param_count")
    return n.value


def slpic_unet_set_params(h, params: np.ndarray):
    params = np.ascontiguousarray(params, dtype=np.float32)
    _check(h, load_library().slpic_unet_set_params(h, params.ctypes.data_as(ctypes.c_void_p)),
           "slpic_unet_set_params")


def slpic_unet_get_params(h) -> np.ndarray:
    out = np.zeros(slpic_unet_param_count(h), np.float32)
    _check(h, load_library().slpic_unet_get_params(h, out.ctypes.data_as(ctypes.c_void_p)),
           "slpic_unet_get_params")
    return out


def slpic_unet_forward(h, nb: int, x, y):
    _check(h, load_library().slpic_unet_forward(h, nb, _dev(x), _dev(y)), "slpic_unet_forward")


def slpic_unet_gradients(h, nb: int, x, t, want_grads: bool = True):
    """(loss, grads or None) for nb samples."""
    loss = ctypes.c_double()
    g = np.zeros(slpic_unet_param_count(h), np.float32) if want_grads else None
    gp = g.ctypes.data_as(ctypes.c_void_p) if want_grads else None
    _check(h, load_library().slpic_unet_gradients(h, nb, _dev(x), _dev(t), ctypes.byref(loss), gp),
           "slpic_unet_gradients")
    return loss.value, g


def slpic_unet_train_step(h, nb: int, x, t, lr: float, want_loss: bool = False):
    loss = ctypes.c_double()
    _check(h, load_library().slpic_unet_train_step(h, nb, _dev(x), _dev(t), float(lr),
                                                   ctypes.byref(loss) if want_loss else None),
           "slpic_unet_train_step")
    return loss.value if want_loss else None


def slpic_unet_reset_optimizer(h):
    _check(h, load_library().slpic_unet_reset_optimizer(h), "slpic_unet_reset_optimizer")


def layer_shapes(levels: int, base: int):
    """(c_in, c_out) of every conv in parameter order (encoder, decoder, output)."""
    ch = [base << l for l in range(levels)]
    shapes = [(1, ch[0])] + [(ch[l - 1], ch[l]) for l in range(1, levels)]
    shapes += [(ch[l + 1] + ch[l], ch[l]) for l in range(levels - 2, -1, -1)]
    return shapes + [(ch[0], 1)]


def split_params(flat: np.ndarray, levels: int, base: int):
    """The flat parameter array as a list of (W (c_out, c_in, 3, 3), b (c_out,))."""
    out, k = [], 0
    for ci, co in layer_shapes(levels, base):
        w = flat[k:k + co * ci * 9].reshape(co, ci, 3, 3)
        k += co * ci * 9
        out.append((w, flat[k:k + co]))
        k += co
    assert k == flat.size
    return out


def join_params(params) -> np.ndarray:
    return np.concatenate([np.concatenate([np.ravel(w), np.ravel(b)]) for w, b in params]).astype(
        np.float32)


class UNet:
    """Owning wrapper around one slpic_unet handle."""

    def __init__(self, levels: int, base: int, height: int, width: int, max_batch: int = 1,
                 normalise: bool = True, out_scale: float = 1.0, seed: int = 0,
                 loss: int = SLPIC_UNET_LOSS_MSE, tensor_cores: bool = False):
        c = slpic_unet_config()
        c.levels, c.base, c.height, c.width = levels, base, height, width
        c.max_batch, c.normalise, c.out_scale, c.seed = max_batch, int(normalise), out_scale, seed
        c.loss = loss
        c.tensor_cores = int(tensor_cores)
        self.cfg = c
        self.levels, self.base = levels, base
        self.h = slpic_unet_create(c)

    def close(self):
        if self.h:
            slpic_unet_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream: int):
        slpic_unet_set_stream(self.h, stream)

    def params(self):
        return split_params(slpic_unet_get_params(self.h), self.levels, self.base)

    def set_params(self, params):
        slpic_unet_set_params(self.h, join_params(params))

    def forward(self, x, y):
        slpic_unet_forward(self.h, int(x.shape[0]) if x.dim() == 3 else 1, x, y)

    def gradients(self, x, t):
        nb = int(x.shape[0]) if x.dim() == 3 else 1
        loss, g = slpic_unet_gradients(self.h, nb, x, t)
        return loss, split_params(g, self.levels, self.base)

    def train_step(self, x, t, lr: float, want_loss: bool = False):
        nb = int(x.shape[0]) if x.dim() == 3 else 1
        return slpic_unet_train_step(self.h, nb, x, t, lr, want_loss)

    def reset_optimizer(self):
        slpic_unet_reset_optimizer(self.h)
