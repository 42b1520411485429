"""Python binding of include/lb_mlp.h (argument marshalling only)."""
from __future__ import annotations

import ctypes as C

import numpy as np

from .lb import LB_OK, LbError, _TorchAllocator, library

_sig_done = False


def _lib():
    global _sig_done
    L = library()
    if not _sig_done:
        vp, fp = C.c_void_p, C.c_void_p
        sig = {
            "lb_mlp_create": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_ulonglong, vp, vp,
                                        C.POINTER(vp)]),
            "lb_mlp_destroy": (None, [vp]),
            "lb_mlp_num_params": (C.c_long, [vp]),
            "lb_mlp_get_params": (C.c_int, [vp, C.c_int, fp]),
            "lb_mlp_set_params": (C.c_int, [vp, C.c_int, fp]),
            "lb_mlp_set_data": (C.c_int, [vp, C.c_int, fp, fp]),
            "lb_mlp_gradients": (C.c_int, [vp, C.c_int, fp, C.POINTER(C.c_float)]),
            "lb_mlp_train": (C.c_int, [vp, C.c_int, C.c_float, C.c_float, C.c_float, fp]),
            "lb_mlp_predict": (C.c_int, [vp, C.c_int, fp, fp, fp, fp]),
            "lb_mlp_last_error": (C.c_char_p, [vp]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _sig_done = True
    return L


def exported_symbols():
    return ["lb_mlp_create", "lb_mlp_destroy", "lb_mlp_num_params", "lb_mlp_get_params", "lb_mlp_set_params",
            "lb_mlp_set_data", "lb_mlp_gradients", "lb_mlp_train", "lb_mlp_predict", "lb_mlp_last_error"]


def _f32(a, shape=None):
    out = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    if shape is not None and out.shape != shape:
        raise ValueError(f"expected {shape}, got {out.shape}")
    return out


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


class MLP:
    """Ensemble of members 4 -> H -> H -> out on the current CUDA device."""

    def __init__(self, n_in=4, n_hidden=256, n_out=64, members=5, max_batch=4096, seed=0, stream=None):
        import torch
        L = _lib()
        self.n_in, self.n_hidden, self.n_out, self.members = n_in, n_hidden, n_out, members
        dev = torch.cuda.current_device()
        self._stream = stream if stream is not None else torch.cuda.current_stream(dev)
        self._alloc = _TorchAllocator(dev)
        h = C.c_void_p()
        st = L.lb_mlp_create(n_in, n_hidden, n_out, members, max_batch, seed, C.byref(self._alloc.struct),
                             C.c_void_p(self._stream.cuda_stream), C.byref(h))
        if st != LB_OK:
            raise LbError(st, L.lb_mlp_last_error(None).decode(errors="replace"))
        self.h = h
        self.P = L.lb_mlp_num_params(h)

    def _check(self, st):
        if st != LB_OK:
            raise LbError(st, _lib().lb_mlp_last_error(self.h).decode(errors="replace"))

    def close(self):
        if getattr(self, "h", None) is not None:
            _lib().lb_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def get_params(self, k):
        out = np.empty(self.P, dtype=np.float32)
        self._check(_lib().lb_mlp_get_params(self.h, k, _ptr(out)))
        return out

    def set_params(self, k, p):
        self._check(_lib().lb_mlp_set_params(self.h, k, _ptr(_f32(p, (self.P,)))))

    def set_data(self, x, y):
        x = _f32(x)
        y = _f32(y)
        self._check(_lib().lb_mlp_set_data(self.h, x.shape[0], _ptr(x), _ptr(y)))

    def gradients(self, k):
        g = np.empty(self.P, dtype=np.float32)
        loss = C.c_float()
        self._check(_lib().lb_mlp_gradients(self.h, k, _ptr(g), C.byref(loss)))
        return loss.value, g

    def train(self, steps, lr=3e-3, lr_min=3e-5, wd=1e-5):
        losses = np.empty(self.members, dtype=np.float32)
        self._check(_lib().lb_mlp_train(self.h, int(steps), lr, lr_min, wd, _ptr(losses)))
        return losses

    def predict(self, x, members=False):
        x = _f32(x)
        n = x.shape[0]
        mean = np.empty((n, self.n_out), dtype=np.float32)
        sd = np.empty((n, self.n_out), dtype=np.float32)
        mem = np.empty((self.members, n, self.n_out), dtype=np.float32) if members else None
        self._check(_lib().lb_mlp_predict(self.h, n, _ptr(x), _ptr(mean), _ptr(sd), _ptr(mem)))
        return (mean, sd, mem) if members else (mean, sd)
