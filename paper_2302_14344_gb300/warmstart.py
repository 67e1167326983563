"""Python binding of the warm-start network (include/warmstart.h): argument marshalling only.

Every call goes to a C function of libsubadmm of the same name; the arithmetic runs in the
library's kernels.  Device arrays are torch CUDA tensors (float32, contiguous), passed by
pointer.
"""
from __future__ import annotations

import ctypes as C
from typing import Optional, Sequence

import numpy as np

from . import subadmm as _sa

VP = C.c_void_p
PF = C.POINTER(C.c_float)
PI = C.POINTER(C.c_int)

EXPORTS = ("wsn_create", "wsn_destroy", "wsn_last_error", "wsn_num_params", "wsn_shape",
           "wsn_workspace_generation",
           "wsn_set_params",
           "wsn_get_params", "wsn_set_normalization", "wsn_get_normalization",
           "wsn_fit_normalization", "wsn_forward", "wsn_forward_layers", "wsn_fused_error",
           "wsn_gradients", "wsn_train_step")

_sigs = {
    "wsn_create": (C.c_int, [C.c_int, C.c_int, PI, C.POINTER(VP)]),
    "wsn_destroy": (None, [VP]),
    "wsn_last_error": (C.c_char_p, [VP]),
    "wsn_num_params": (C.c_longlong, [VP]),
    "wsn_shape": (C.c_int, [VP, PI]),
    "wsn_workspace_generation": (C.c_longlong, [VP]),
    "wsn_set_params": (C.c_int, [VP, PF]),
    "wsn_get_params": (C.c_int, [VP, PF]),
    "wsn_set_normalization": (C.c_int, [VP, PF, PF, PF]),
    "wsn_get_normalization": (C.c_int, [VP, PF, PF, PF]),
    "wsn_fit_normalization": (C.c_int, [VP, VP, C.c_longlong, VP, C.c_int, VP]),
    "wsn_forward": (C.c_int, [VP, VP, C.c_longlong, C.c_int, VP, VP]),
    "wsn_forward_layers": (C.c_int, [VP, VP, C.c_longlong, C.c_int, VP, VP]),
    "wsn_fused_error": (C.c_int, [VP, PI]),
    "wsn_gradients": (C.c_int, [VP, VP, C.c_longlong, VP, VP, C.c_int, VP, VP, VP]),
    "wsn_train_step": (C.c_int, [VP, VP, C.c_longlong, VP, VP, C.c_int, C.c_float, VP, VP]),
}
_lib = None


def lib():
    global _lib
    if _lib is None:
        L = _sa.load()
        for name, (res, args) in _sigs.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _fp(a: np.ndarray):
    return a.ctypes.data_as(PF)


def _dev(t) -> int:
    assert t.is_cuda and t.dtype.itemsize == 4 and t.is_contiguous()
    return t.data_ptr()


class Network:
    """A fully connected GELU network on one GPU (widths `sizes`, input first)."""

    def __init__(self, sizes: Sequence[int], device: int = 0, stream: int = 0):
        self.sizes = list(sizes)
        self.stream = stream
        h = VP()
        arr = (C.c_int * len(sizes))(*sizes)
        rc = lib().wsn_create(device, len(sizes) - 1, arr, C.byref(h))
        if rc < 0:
            raise _sa.SimError(rc, "wsn_create failed")
        self.h = h

    def _check(self, rc: int) -> int:
        if rc < 0:
            msg = lib().wsn_last_error(self.h)
            raise _sa.SimError(rc, msg.decode() if msg else "error")
        return rc

    def close(self):
        if self.h:
            lib().wsn_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def num_params(self) -> int:
        return int(lib().wsn_num_params(self.h))

    def set_params(self, flat: np.ndarray) -> None:
        a = np.ascontiguousarray(flat, dtype=np.float32)
        assert a.size == self.num_params
        self._check(lib().wsn_set_params(self.h, _fp(a)))

    def get_params(self) -> np.ndarray:
        a = np.zeros(self.num_params, dtype=np.float32)
        self._check(lib().wsn_get_params(self.h, _fp(a)))
        return a

    def set_normalization(self, mean_in, std_in, scale_out) -> None:
        m = np.ascontiguousarray(mean_in, dtype=np.float32)
        s = np.ascontiguousarray(std_in, dtype=np.float32)
        o = np.ascontiguousarray(scale_out, dtype=np.float32)
        self._check(lib().wsn_set_normalization(self.h, _fp(m), _fp(s), _fp(o)))

    def get_normalization(self):
        m = np.zeros(self.sizes[0], np.float32)
        s = np.zeros(self.sizes[0], np.float32)
        o = np.zeros(self.sizes[-1], np.float32)
        self._check(lib().wsn_get_normalization(self.h, _fp(m), _fp(s), _fp(o)))
        return m, s, o

    def fit_normalization(self, x, t) -> None:
        self._check(lib().wsn_fit_normalization(self.h, _dev(x), x.shape[1], _dev(t), x.shape[0],
                                                VP(self.stream)))

    def forward(self, x, y) -> None:
        self._check(lib().wsn_forward(self.h, _dev(x), x.shape[1], x.shape[0], _dev(y),
                                      VP(self.stream)))

    def forward_layers(self, x, y) -> None:
        """The layer-by-layer inference (any shape)."""
        self._check(lib().wsn_forward_layers(self.h, _dev(x), x.shape[1], x.shape[0], _dev(y),
                                             VP(self.stream)))

    def fused_error(self) -> int:
        out = (C.c_int * 1)()
        self._check(lib().wsn_fused_error(self.h, out))
        return int(out[0])

    def gradients(self, x, t, mask, grad, loss=None) -> None:
        self._check(lib().wsn_gradients(self.h, _dev(x), x.shape[1], _dev(t), _dev(mask),
                                        x.shape[0], _dev(grad),
                                        None if loss is None else _dev(loss), VP(self.stream)))

    def train_step(self, x, t, mask, lr: float, loss=None) -> None:
        self._check(lib().wsn_train_step(self.h, _dev(x), x.shape[1], _dev(t), _dev(mask),
                                         x.shape[0], lr, None if loss is None else _dev(loss),
                                         VP(self.stream)))


def split_params(flat: np.ndarray, sizes: Sequence[int]):
    """The flat parameter vector as [(W_l, b_l)] (layout of wsn_set_params)."""
    out, off = [], 0
    for a, b in zip(sizes[:-1], sizes[1:]):
        W = flat[off:off + a * b].reshape(a, b)
        off += a * b
        out.append((W, flat[off:off + b]))
        off += b
    return out


def join_params(params) -> np.ndarray:
    return np.concatenate([np.concatenate([W.ravel(), b.ravel()]) for W, b in params])
