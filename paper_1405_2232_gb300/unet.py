"""ctypes binding of the warm-start network C ABI (include/unet.h).

Argument marshalling only: the network's forward and backward passes, Adam
and the handoff run in the CUDA library (liblbgb.so, loaded through
``lb.load``).  Device arrays are anything exposing ``data_ptr()`` (torch
tensors) or raw integer addresses; host arrays are float32 numpy arrays.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import lb

UN_LEVELS, UN_IN, UN_IN_PAD, UN_OUT, UN_LAYERS = 4, 3, 32, 2, 15
UN_T_X0, UN_T_A, UN_T_CAT, UN_T_P, UN_T_C, UN_T_D0 = 0, 10, 30, 40, 50, 60
UN_T_UP, UN_T_SKIP, UN_T_GRAD = 70, 80, 100

EXPORTED = ["un_param_count", "un_layer_info", "un_create", "un_set_params", "un_get_params",
            "un_get_grads", "un_forward", "un_loss_grad", "un_adam_step", "un_train_step",
            "un_get_tensor", "un_synchronize", "un_free", "un_warm_fields"]


class un_config(ctypes.Structure):
    _fields_ = [("H", ctypes.c_int32), ("W", ctypes.c_int32), ("max_batch", ctypes.c_int32),
                ("base", ctypes.c_int32)]


_bound = False


def load():
    """The library with the un_* signatures declared."""
    global _bound
    lib = lb.load()
    if _bound:
        return lib
    C = ctypes.POINTER(un_config)
    vp = ctypes.c_void_p
    fp = ctypes.POINTER(ctypes.c_float)
    dp = ctypes.POINTER(ctypes.c_double)
    i32, i64, st, dbl = ctypes.c_int32, ctypes.c_int64, ctypes.c_int, ctypes.c_double
    sig = {
        "un_param_count": (i64, [C]),
        "un_layer_info": (st, [C, i32, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i32),
                               ctypes.POINTER(i64)]),
        "un_create": (st, [C, vp, ctypes.POINTER(vp)]),
        "un_set_params": (st, [vp, vp, i64]),
        "un_get_params": (st, [vp, fp, i64]),
        "un_get_grads": (st, [vp, fp, i64]),
        "un_forward": (st, [vp, i32, vp, vp]),
        "un_loss_grad": (st, [vp, i32, vp, vp, dp]),
        "un_adam_step": (st, [vp, dbl, dbl, dbl, dbl]),
        "un_train_step": (st, [vp, i32, vp, vp, dbl, dp]),
        "un_get_tensor": (st, [vp, i32, fp, i64]),
        "un_synchronize": (st, [vp]),
        "un_free": (st, [vp]),
        "un_warm_fields": (st, [i32, i32, i32, vp, dbl, dbl, dbl, vp, vp, vp, vp, vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _bound = True
    return lib


def config(H, W, max_batch, base=32) -> un_config:
    return un_config(int(H), int(W), int(max_batch), int(base))


def param_count(cfg: un_config) -> int:
    return int(load().un_param_count(ctypes.byref(cfg)))


def layer_table(cfg: un_config):
    """[(cin_stored, cout, ksize, offset)] in the flat parameter order."""
    out = []
    for k in range(UN_LAYERS):
        ci, co, ks = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        off = ctypes.c_int64()
        lb._check(load().un_layer_info(ctypes.byref(cfg), k, ctypes.byref(ci), ctypes.byref(co),
                                       ctypes.byref(ks), ctypes.byref(off)))
        out.append((ci.value, co.value, ks.value, off.value))
    return out


def _f32(a, n):
    a = np.ascontiguousarray(a, dtype=np.float32).reshape(-1)
    if a.size != n:
        raise ValueError(f"expected {n} values, got {a.size}")
    return a


class UNet:
    """Owner of one network (frees it on close / garbage collection)."""

    def __init__(self, H, W, max_batch, base=32, stream=None):
        self.cfg = config(H, W, max_batch, base)
        self.n = param_count(self.cfg)
        self.net = ctypes.c_void_p()
        lb._check(load().un_create(ctypes.byref(self.cfg), lb._stream(stream), ctypes.byref(self.net)))

    def set_params(self, params):
        if hasattr(params, "data_ptr"):
            lb._check(load().un_set_params(self.net, lb._addr(params), self.n))
        else:
            p = _f32(params, self.n)
            lb._check(load().un_set_params(self.net, p.ctypes.data_as(ctypes.c_void_p), self.n))

    def params(self):
        out = np.empty(self.n, dtype=np.float32)
        lb._check(load().un_get_params(self.net, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), self.n))
        return out

    def grads(self):
        out = np.empty(self.n, dtype=np.float32)
        lb._check(load().un_get_grads(self.net, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), self.n))
        return out

    def forward(self, d_in, d_out, N):
        lb._check(load().un_forward(self.net, int(N), lb._addr(d_in), lb._addr(d_out)))

    def loss_grad(self, d_in, d_target, N, want_loss=True):
        loss = ctypes.c_double()
        lb._check(load().un_loss_grad(self.net, int(N), lb._addr(d_in), lb._addr(d_target),
                                      ctypes.byref(loss) if want_loss else None))
        return loss.value if want_loss else None

    def adam_step(self, lr, beta1=0.9, beta2=0.999, eps=1e-8):
        lb._check(load().un_adam_step(self.net, float(lr), float(beta1), float(beta2), float(eps)))

    def train_step(self, d_in, d_target, N, lr, want_loss=True):
        loss = ctypes.c_double()
        lb._check(load().un_train_step(self.net, int(N), lb._addr(d_in), lb._addr(d_target), float(lr),
                                       ctypes.byref(loss) if want_loss else None))
        return loss.value if want_loss else None

    def tensor(self, tid, shape):
        out = np.empty(shape, dtype=np.float32)
        lb._check(load().un_get_tensor(self.net, int(tid), out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                       out.size))
        return out

    def synchronize(self):
        lb._check(load().un_synchronize(self.net))

    def close(self):
        if self.net is not None and self.net.value:
            lb._check(load().un_free(self.net))
        self.net = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def warm_fields(N, H, W, d_pred, norm, d_rho0, d_T0, d_rho, d_T, rho_floor=1e-4, stream=None):
    """Handoff: network prediction -> mass- and energy-matched FP64 rho, T (device)."""
    lb._check(load().un_warm_fields(int(N), int(H), int(W), lb._addr(d_pred), norm["rho_dev_scale"],
                                    float(rho_floor), norm["t_dev_scale"],
                                    lb._addr(d_rho0), lb._addr(d_T0), lb._addr(d_rho), lb._addr(d_T),
                                    lb._stream(stream)))
