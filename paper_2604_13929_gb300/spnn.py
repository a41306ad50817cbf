"""Thin ctypes binding of libspnn, the fluence surrogate (argument marshalling only).

Every layer, loss, optimiser and data step runs in the CUDA library; this
module converts torch CUDA tensors to device pointers and raises on error
codes.  There is no CPU fallback: if ``libspnn.so`` has not been built,
:func:`load` raises, and without a GPU the calls return ``SPNN_ECUDA``.

Function names follow include/spnn.h.  Tensors are torch CUDA tensors:
activations ``torch.bfloat16`` in chunk planes, shape (C/8, B, D, H, W, 8)
(see :func:`to_planes` / :func:`from_planes`), weights and gradients
``torch.float32``.  Streams default to torch's current stream.
"""
from __future__ import annotations

import ctypes
import math
import os
import threading

import numpy as np

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "_lib", "libspnn.so")
HEADER = os.path.join(os.path.dirname(PKG), "include", "spnn.h")

SPNN_OK, SPNN_EINVAL, SPNN_ENOMEM, SPNN_ECUDA = 0, -1, -2, -3
CONV3, DOWN, UP = 0, 1, 2
PACK_FWD, PACK_DGRAD = 0, 1
KIND = {"conv3": CONV3, "down": DOWN, "up": UP}
N_FEATURES = 16
LAYER_NAMES = ("e0a", "e0b", "d1", "e1a", "e1b", "d2", "e2a", "e2b", "d3", "b1", "b2",
               "u2", "c2a", "c2b", "u1", "c1a", "c1b", "u0", "c0a", "c0b")

_lock = threading.Lock()
_lib = None
_P = ctypes.c_void_p
_I = ctypes.c_int


class SpnnError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"spnn error {code}: {msg}")
        self.code = code


def load():
    """Load libspnn.so (built by ``paper_2604_13929_gb300.build``)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run `python -m paper_2604_13929_gb300.build`")
        lib = ctypes.CDLL(LIB_PATH)
        sig = {
            "spnn_last_error": (ctypes.c_char_p, []),
            "spnn_version": (_I, []),
            "spnn_status": (_I, [_P]),
            "spnn_set_option": (_I, [_I, _I]),
            "spnn_packed_elems": (ctypes.c_size_t, [_I, _I, _I]),
            "spnn_pack_weights": (_I, [_I, _I, _I, _I, _P, _P, _P]),
            "spnn_layer_forward": (_I, [_I, _I, _I, _I, _I, _P, _I, _P, _I, _P, _P, _I, _I, _P, _P, _P, _P,
                                        _P]),
            "spnn_layer_dgrad": (_I, [_I, _I, _I, _I, _I, _P, _I, _P, _I, _I, _P, _P, _P, _P, _P, _P, _P]),
            "spnn_layer_wgrad": (_I, [_I, _I, _I, _I, _I, _P, _I, _P, _I, _P, _I, _P, _P, _P]),
            "spnn_pack_input": (_I, [_P, _P, _I, _I, _I, _I, _P, _P]),
            "spnn_log_fluence": (_I, [_P, _P, _I, _I, _I, _I, ctypes.c_float, _P, _P]),
            "spnn_phase_profiles": (_I, [_P, _P, _I, _I, _I, _I, _P, _P]),
            "spnn_unet_create": (_P, [_I, _I, _I]),
            "spnn_unet_destroy": (None, [_P]),
            "spnn_unet_param_count": (ctypes.c_size_t, [_P]),
            "spnn_unet_set_params": (_I, [_P, _P]),
            "spnn_unet_get_params": (_I, [_P, _P]),
            "spnn_unet_get_grads": (_I, [_P, _P]),
            "spnn_unet_forward": (_I, [_P, _P, _I, _P, _P]),
            "spnn_unet_backward": (_I, [_P, _P, _I, _P, _P]),
            "spnn_unet_adam": (_I, [_P, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float, _P]),
            "spnn_unet_copy_activation": (_I, [_P, _I, _I, _P, _P]),
            "spnn_unet_layer_shape": (_I, [_P, _I, ctypes.POINTER(_I), ctypes.POINTER(_I)]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def declared_symbols():
    """Function names declared in include/spnn.h."""
    import re
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"\b(spnn_\w+)\s*\(", txt)) - {"spnn_unet_t"})


def to_planes(x):
    """(B, D, H, W, C) tensor -> contiguous chunk planes (C/8, B, D, H, W, 8)."""
    B, D, H, W, C = x.shape
    return x.reshape(B, D, H, W, C // 8, 8).permute(4, 0, 1, 2, 3, 5).contiguous()


def from_planes(x):
    """Chunk planes (C/8, B, D, H, W, 8) -> (B, D, H, W, C)."""
    C8, B, D, H, W, _ = x.shape
    return x.permute(1, 2, 3, 4, 0, 5).reshape(B, D, H, W, C8 * 8)


def planes_empty(B, D, H, W, C, dtype=None):
    import torch
    return torch.zeros((C // 8, B, D, H, W, 8), dtype=dtype or torch.bfloat16, device="cuda")


def _channels(t):
    return 0 if t is None else t.shape[0] * 8


def _check(rc: int):
    if rc != SPNN_OK:
        raise SpnnError(rc, load().spnn_last_error().decode())


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


# ------------------------------------------------------------ C-named calls --

def spnn_status(stream=None):
    _check(load().spnn_status(_stream(stream)))


OPT = {"conv_subtiles": 1, "conv_planes": 2, "stage_kb": 3, "wgrad_halo": 4, "conv_full_halo": 5,
       "rows_persistent": 7, "loss_fluence_weight": 8}


def spnn_set_option(key, value: int):
    _check(load().spnn_set_option(OPT.get(key, key), int(value)))


def spnn_packed_elems(kind: int, cin: int, cout: int) -> int:
    return int(load().spnn_packed_elems(kind, cin, cout))


def spnn_pack_weights(kind, cin, cout, which, w, packed, stream=None):
    _check(load().spnn_pack_weights(kind, cin, cout, which, _ptr(w), _ptr(packed), _stream(stream)))


def spnn_layer_forward(kind, grid, x0, x1, packed, bias, cout, relu, y, head_w=None, head_b=None,
                       head_out=None, stream=None):
    B, D, H, W = grid
    c0, c1 = _channels(x0), _channels(x1)
    _check(load().spnn_layer_forward(kind, B, D, H, W, _ptr(x0), c0, _ptr(x1), c1, _ptr(packed), _ptr(bias),
                                     cout, int(relu), _ptr(y), _ptr(head_w), _ptr(head_b), _ptr(head_out),
                                     _stream(stream)))


def spnn_layer_dgrad(kind, grid, dy, packed, c0, c1, dx0, addend0=None, mask0=None, dx1=None, addend1=None,
                     mask1=None, stream=None):
    B, D, H, W = grid
    _check(load().spnn_layer_dgrad(kind, B, D, H, W, _ptr(dy), _channels(dy), _ptr(packed), c0, c1, _ptr(dx0),
                                   _ptr(addend0), _ptr(mask0), _ptr(dx1), _ptr(addend1), _ptr(mask1),
                                   _stream(stream)))


def spnn_layer_wgrad(kind, grid, x0, x1, dy, dw, db=None, stream=None):
    B, D, H, W = grid
    c0, c1 = _channels(x0), _channels(x1)
    _check(load().spnn_layer_wgrad(kind, B, D, H, W, _ptr(x0), c0, _ptr(x1), c1, _ptr(dy), _channels(dy),
                                   _ptr(dw), _ptr(db), _stream(stream)))


def spnn_pack_input(mask, optics, x, stream=None):
    B, D, H, W = mask.shape
    _check(load().spnn_pack_input(_ptr(mask), _ptr(optics), B, D, H, W, _ptr(x), _stream(stream)))


def spnn_log_fluence(raw, n_photons, out, floor=1e-6, stream=None):
    B, D, H, W = raw.shape
    _check(load().spnn_log_fluence(_ptr(raw), _ptr(n_photons), B, D, H, W, float(floor), _ptr(out),
                                   _stream(stream)))


def spnn_phase_profiles(log_phi, mask, prof, stream=None):
    B, D, H, W = log_phi.shape
    _check(load().spnn_phase_profiles(_ptr(log_phi), _ptr(mask), B, D, H, W, _ptr(prof), _stream(stream)))


# ------------------------------------------------------------------ network --

class UNet:
    """Owner of one spnn_unet handle (flat FP32 parameter vector, see spnn.h)."""

    def __init__(self, c0: int, n: int, max_batch: int):
        self.c0, self.n, self.max_batch = c0, n, max_batch
        self._h = load().spnn_unet_create(c0, n, max_batch)
        if not self._h:
            raise SpnnError(SPNN_EINVAL, load().spnn_last_error().decode())
        self.param_count = int(load().spnn_unet_param_count(self._h))

    def close(self):
        if self._h:
            load().spnn_unet_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, flat: np.ndarray):
        a = np.ascontiguousarray(flat, dtype=np.float32)
        assert a.size == self.param_count
        _check(load().spnn_unet_set_params(self._h, a.ctypes.data_as(ctypes.c_void_p)))

    def get_params(self) -> np.ndarray:
        a = np.empty(self.param_count, dtype=np.float32)
        _check(load().spnn_unet_get_params(self._h, a.ctypes.data_as(ctypes.c_void_p)))
        return a

    def get_grads(self) -> np.ndarray:
        a = np.empty(self.param_count, dtype=np.float32)
        _check(load().spnn_unet_get_grads(self._h, a.ctypes.data_as(ctypes.c_void_p)))
        return a

    def forward(self, x, pred, stream=None):
        """x: input features in chunk planes (2, B, n, n, n, 8); pred FP32 (B, n, n, n)."""
        _check(load().spnn_unet_forward(self._h, _ptr(x), pred.shape[0], _ptr(pred), _stream(stream)))

    def backward(self, target, loss=None, stream=None):
        _check(load().spnn_unet_backward(self._h, _ptr(target), target.shape[0], _ptr(loss), _stream(stream)))

    def adam(self, lr, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
        _check(load().spnn_unet_adam(self._h, lr, beta1, beta2, eps, _stream(stream)))

    def activation(self, layer: int, batch: int, stream=None):
        """Copy of a layer's BF16 output in chunk planes (C/8, batch, e, e, e, 8)."""
        import torch
        e, c = _I(), _I()
        _check(load().spnn_unet_layer_shape(self._h, layer, ctypes.byref(e), ctypes.byref(c)))
        out = torch.empty((c.value // 8, batch, e.value, e.value, e.value, 8), dtype=torch.bfloat16,
                          device="cuda")
        _check(load().spnn_unet_copy_activation(self._h, layer, batch, _ptr(out), _stream(stream)))
        return out


def layer_table(c0: int):
    """(name, kind, input channels, output channels) of the library's U-Net in
    forward order (the table compiled into libspnn; its parameter count is
    checked against spnn_unet_param_count by the tests)."""
    c1, c2, c3 = 2 * c0, 4 * c0, 8 * c0
    return [("e0a", "conv3", N_FEATURES, c0), ("e0b", "conv3", c0, c0), ("d1", "down", c0, c1),
            ("e1a", "conv3", c1, c1), ("e1b", "conv3", c1, c1), ("d2", "down", c1, c2),
            ("e2a", "conv3", c2, c2), ("e2b", "conv3", c2, c2), ("d3", "down", c2, c3),
            ("b1", "conv3", c3, c3), ("b2", "conv3", c3, c3), ("u2", "up", c3, c2),
            ("c2a", "conv3", 2 * c2, c2), ("c2b", "conv3", c2, c2), ("u1", "up", c2, c1),
            ("c1a", "conv3", 2 * c1, c1), ("c1b", "conv3", c1, c1), ("u0", "up", c1, c0),
            ("c0a", "conv3", 2 * c0, c0), ("c0b", "conv3", c0, c0)]


def init_params(c0: int, seed: int) -> np.ndarray:
    """He-normal initial weights (std sqrt(2 / fan_in), fan_in = taps x input
    channels, or input channels for the transposed 2x2x2 layers), zero biases,
    head weights of std sqrt(1 / c0): the flat FP32 vector of spnn.h."""
    rng = np.random.default_rng(seed)
    parts = []
    for _, kind, ci, co in layer_table(c0):
        taps = 27 if kind == "conv3" else 8
        fan_in = ci if kind == "up" else taps * ci
        parts += [rng.standard_normal(taps * ci * co) * math.sqrt(2.0 / fan_in), np.zeros(co)]
    parts += [rng.standard_normal(c0) * math.sqrt(1.0 / c0), np.zeros(1)]
    return np.concatenate(parts).astype(np.float32)


def flatten_params(params: dict, c0: int) -> np.ndarray:
    """Oracle-style {name: (W, b)} -> the library's flat FP32 vector."""
    parts = []
    for name in LAYER_NAMES:
        w, b = params[name]
        parts += [np.asarray(w, dtype=np.float64).ravel(), np.asarray(b, dtype=np.float64).ravel()]
    hw, hb = params["head"]
    parts += [np.asarray(hw, dtype=np.float64).ravel(), np.asarray(hb, dtype=np.float64).reshape(1)]
    return np.concatenate(parts)


def unflatten_params(flat: np.ndarray, table, c0: int) -> dict:
    """The library's flat vector -> {name: (W, b)} for a layer table
    [(name, kind, cin, cout, relu), ...]."""
    out, off = {}, 0
    taps = {"conv3": 27, "down": 8, "up": 8}
    for name, kind, ci, co, _ in table:
        n = taps[kind] * ci * co
        out[name] = (flat[off:off + n].reshape(taps[kind], ci, co).astype(np.float64),
                     flat[off + n:off + n + co].astype(np.float64))
        off += n + co
    out["head"] = (flat[off:off + c0].astype(np.float64), np.array(float(flat[off + c0])))
    return out
