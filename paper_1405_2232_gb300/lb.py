"""ctypes binding of the C ABI in include/lb.h (liblbgb.so).

Argument marshalling only: every step of the method runs in the CUDA
library.  The names mirror the C functions (lb_init, lb_step, lb_moments,
lb_totals, lb_free, ...).  Host arrays are float64 numpy arrays; device
arrays are anything exposing ``data_ptr()`` (torch tensors) or raw integer
addresses; streams are ``torch.cuda.Stream`` objects or raw ``cudaStream_t``
integers.

The library is loaded from ``paper_1405_2232_gb300/_build/liblbgb.so``.  If
it is missing, importing this module raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

LB_OK, LB_ERR_ARG, LB_ERR_CUDA, LB_ERR_OOM = 0, 1, 2, 3
LB_ERR_NONFINITE, LB_ERR_PSI_DOMAIN, LB_ERR_TIMEOUT, LB_ERR_UNSUPPORTED = 4, 5, 6, 7
LB_ERR_NOT_CONVERGED = 8
LB_EOS_CS, LB_EOS_VDW, LB_EOS_IDEAL = 0, 1, 2
LB_THERMAL_EQ7, LB_THERMAL_EQ24, LB_THERMAL_FD26, LB_THERMAL_FD26_PRINTED = 0, 1, 2, 3
LB_PREC_FP64, LB_PREC_FP32, LB_PREC_FP16_DEV, LB_PREC_BF16_DEV = 0, 1, 2, 3
LB_WALLS_PERIODIC, LB_WALLS_CAVITY, LB_WALLS_CHANNEL = 0, 1, 2
LB_TOTALS_N = 5
LB_TUNE_N = 5
LB_BATCH_TUNE_N = 4
LB_HALO_ROWS = 2

PRECISIONS = {"fp64": LB_PREC_FP64, "fp32": LB_PREC_FP32, "fp16": LB_PREC_FP16_DEV,
              "bf16": LB_PREC_BF16_DEV}


class LbError(RuntimeError):
    """A non-zero lb_status; ``status`` holds the code."""

    def __init__(self, status: int, msg: str):
        super().__init__(f"lb status {status}: {msg}")
        self.status = status


class lb_params(ctypes.Structure):
    """Mirror of ``lb_params`` (field order and types as in include/lb.h)."""

    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
        ("eos", ctypes.c_int32), ("thermal", ctypes.c_int32),
        ("precision", ctypes.c_int32), ("psi_uses_local_T", ctypes.c_int32),
        ("tile_x", ctypes.c_int32), ("tile_y", ctypes.c_int32),
        ("tau_f", ctypes.c_double), ("tau_g", ctypes.c_double),
        ("G", ctypes.c_double), ("beta", ctypes.c_double),
        ("a", ctypes.c_double), ("b", ctypes.c_double), ("R", ctypes.c_double),
        ("cv", ctypes.c_double), ("T_psi", ctypes.c_double),
        ("rho0", ctypes.c_double), ("T0", ctypes.c_double),
        ("walls", ctypes.c_int32), ("adiabatic_bottom", ctypes.c_int32),
        ("T_hot", ctypes.c_double), ("T_cold", ctypes.c_double), ("g_grav", ctypes.c_double),
        ("T_in", ctypes.c_double), ("T_w", ctypes.c_double), ("U_in", ctypes.c_double),
        ("init_balanced", ctypes.c_int32),
        ("halo_rows", ctypes.c_int32),
    ]


_lib = None

#: Every symbol include/lb.h declares (checked by the CPU test-suite).
EXPORTED = [
    "lb_params_default", "lb_init", "lb_init_device", "lb_step", "lb_synchronize",
    "lb_moments", "lb_moments_device", "lb_get_populations", "lb_set_populations",
    "lb_totals", "lb_state_size", "lb_save_state", "lb_load_state", "lb_time",
    "lb_get_params", "lb_free", "lb_last_error", "lb_version", "lb_field_totals_noalloc",
    "lb_set_wait_limit", "lb_halo_bytes", "lb_halo_pack", "lb_halo_unpack",
    "lb_batch_init", "lb_batch_step", "lb_batch_check", "lb_batch_run", "lb_batch_fields",
    "lb_batch_time", "lb_batch_free", "lb_tune_candidate", "lb_autotune",
    "lb_batch_set_chunk_rows", "lb_batch_chunk_rows", "lb_batch_autotune", "lb_batch_restart",
]


def library_path() -> str:
    return _build.LIB


def load(path: str | None = None):
    """Load liblbgb.so (building it first if the sources are newer)."""
    global _lib
    if _lib is not None:
        return _lib
    if path is None:
        path = _build.build()
    if not os.path.exists(path):
        raise ImportError(f"CUDA library not found at {path}")
    lib = ctypes.CDLL(path)
    P = ctypes.POINTER(lb_params)
    vp = ctypes.c_void_p
    dp = ctypes.POINTER(ctypes.c_double)
    st = ctypes.c_int
    sig = {
        "lb_params_default": (None, [P]),
        "lb_init": (st, [P, dp, dp, vp, ctypes.POINTER(vp)]),
        "lb_init_device": (st, [P, vp, vp, vp, ctypes.POINTER(vp)]),
        "lb_step": (st, [vp, ctypes.c_int64]),
        "lb_synchronize": (st, [vp]),
        "lb_moments": (st, [vp, dp, dp, dp, dp]),
        "lb_moments_device": (st, [vp, vp, vp, vp, vp]),
        "lb_get_populations": (st, [vp, dp, dp]),
        "lb_set_populations": (st, [vp, dp, dp]),
        "lb_totals": (st, [vp, dp]),
        "lb_state_size": (st, [vp, ctypes.POINTER(ctypes.c_size_t)]),
        "lb_save_state": (st, [vp, vp]),
        "lb_load_state": (st, [vp, vp]),
        "lb_time": (ctypes.c_int64, [vp]),
        "lb_set_wait_limit": (st, [vp, ctypes.c_int64]),
        "lb_halo_bytes": (st, [vp, ctypes.POINTER(ctypes.c_size_t)]),
        "lb_halo_pack": (st, [vp, ctypes.c_int32, vp]),
        "lb_halo_unpack": (st, [vp, ctypes.c_int32, vp]),
        "lb_get_params": (st, [vp, P]),
        "lb_free": (st, [vp]),
        "lb_last_error": (ctypes.c_char_p, []),
        "lb_version": (ctypes.c_char_p, []),
        "lb_field_totals_noalloc": (st, [ctypes.c_int32, ctypes.c_int32, ctypes.c_double, vp, vp,
                                         vp, vp, vp, vp, ctypes.c_int64, vp, vp]),
        "lb_batch_init": (st, [P, ctypes.c_int32, ctypes.POINTER(dp), ctypes.POINTER(dp), vp,
                               ctypes.POINTER(vp)]),
        "lb_batch_step": (st, [vp, ctypes.c_int64]),
        "lb_batch_check": (st, [vp, dp, dp, dp, ctypes.POINTER(ctypes.c_int32)]),
        "lb_batch_run": (st, [vp, ctypes.c_double, ctypes.c_int64, ctypes.c_int64,
                              ctypes.POINTER(ctypes.c_int64), dp, ctypes.POINTER(ctypes.c_int32)]),
        "lb_batch_fields": (st, [vp, ctypes.c_int32, dp, dp]),
        "lb_batch_time": (ctypes.c_int64, [vp]),
        "lb_batch_free": (st, [vp]),
        "lb_tune_candidate": (st, [ctypes.c_int32, ctypes.POINTER(ctypes.c_int32),
                                   ctypes.POINTER(ctypes.c_int32)]),
        "lb_autotune": (st, [P, ctypes.c_int32, vp, P, dp]),
        "lb_batch_set_chunk_rows": (st, [vp, ctypes.c_int32]),
        "lb_batch_chunk_rows": (ctypes.c_int32, [vp]),
        "lb_batch_autotune": (st, [vp, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32), dp]),
        "lb_batch_restart": (st, [vp, ctypes.c_int32, vp, vp, ctypes.c_int32]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(status: int):
    if status != LB_OK:
        raise LbError(status, load().lb_last_error().decode())


def _host(a, shape=None, writable=False):
    a = np.ascontiguousarray(a, dtype=np.float64) if not writable else a
    if shape is not None and a.shape != shape:
        raise ValueError(f"expected shape {shape}, got {a.shape}")
    if writable and not (a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]):
        raise ValueError("output arrays must be C-contiguous float64")
    return a


def _dptr(a) -> ctypes.POINTER(ctypes.c_double):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _addr(x):
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return ctypes.c_void_p(x.data_ptr())
    return ctypes.c_void_p(int(x))


def _stream(s):
    if s is None:
        return None
    if hasattr(s, "cuda_stream"):
        return ctypes.c_void_p(s.cuda_stream)
    return ctypes.c_void_p(int(s))


def lb_params_default(**overrides) -> lb_params:
    p = lb_params()
    load().lb_params_default(ctypes.byref(p))
    for k, v in overrides.items():
        if k == "precision" and isinstance(v, str):
            v = PRECISIONS[v]
        setattr(p, k, v)
    return p


def lb_init(p: lb_params, rho0, T0, stream=None) -> ctypes.c_void_p:
    rho0 = _host(rho0, (p.ny, p.nx))
    T0 = _host(T0, (p.ny, p.nx))
    ctx = ctypes.c_void_p()
    _check(load().lb_init(ctypes.byref(p), _dptr(rho0), _dptr(T0), _stream(stream),
                          ctypes.byref(ctx)))
    return ctx


def lb_init_device(p: lb_params, d_rho0, d_T0, stream=None) -> ctypes.c_void_p:
    ctx = ctypes.c_void_p()
    _check(load().lb_init_device(ctypes.byref(p), _addr(d_rho0), _addr(d_T0), _stream(stream),
                                 ctypes.byref(ctx)))
    return ctx


def lb_step(ctx, n: int = 1):
    _check(load().lb_step(ctx, int(n)))


def lb_synchronize(ctx):
    _check(load().lb_synchronize(ctx))


def lb_get_params(ctx) -> lb_params:
    p = lb_params()
    _check(load().lb_get_params(ctx, ctypes.byref(p)))
    return p


def lb_moments(ctx):
    """Host (rho, ux, uy, T), each float64 [ny, nx]."""
    p = lb_get_params(ctx)
    outs = [np.empty((p.ny, p.nx)) for _ in range(4)]
    _check(load().lb_moments(ctx, *[_dptr(o) for o in outs]))
    return tuple(outs)


def lb_moments_device(ctx, d_rho=None, d_ux=None, d_uy=None, d_T=None):
    _check(load().lb_moments_device(ctx, _addr(d_rho), _addr(d_ux), _addr(d_uy), _addr(d_T)))


def lb_get_populations(ctx):
    """Pre-collision (f, g) at time t, float64 [9, ny, nx] each."""
    p = lb_get_params(ctx)
    f = np.empty((9, p.ny, p.nx))
    g = np.empty((9, p.ny, p.nx))
    _check(load().lb_get_populations(ctx, _dptr(f), _dptr(g)))
    return f, g


def lb_set_populations(ctx, f, g):
    p = lb_get_params(ctx)
    f = _host(f, (9, p.ny, p.nx))
    g = _host(g, (9, p.ny, p.nx))
    _check(load().lb_set_populations(ctx, _dptr(f), _dptr(g)))


def lb_totals(ctx) -> np.ndarray:
    """[mass, energy, px, py, residual] (FP64, deterministic device reduction)."""
    out = np.zeros(LB_TOTALS_N)
    _check(load().lb_totals(ctx, _dptr(out)))
    return out


def lb_save_state(ctx) -> bytes:
    n = ctypes.c_size_t()
    _check(load().lb_state_size(ctx, ctypes.byref(n)))
    buf = ctypes.create_string_buffer(n.value)
    _check(load().lb_save_state(ctx, ctypes.cast(buf, ctypes.c_void_p)))
    return buf.raw


def lb_load_state(ctx, blob: bytes):
    n = ctypes.c_size_t()
    _check(load().lb_state_size(ctx, ctypes.byref(n)))
    if len(blob) != n.value:
        raise ValueError(f"state blob has {len(blob)} bytes, expected {n.value}")
    buf = ctypes.create_string_buffer(blob, len(blob))
    _check(load().lb_load_state(ctx, ctypes.cast(buf, ctypes.c_void_p)))


def lb_time(ctx) -> int:
    return int(load().lb_time(ctx))


def lb_set_wait_limit(ctx, cycles: int):
    """Limit (SM clock cycles, 0 = default) of the strip kernels' bounded waits."""
    _check(load().lb_set_wait_limit(ctx, int(cycles)))


def lb_halo_bytes(ctx) -> int:
    n = ctypes.c_size_t()
    _check(load().lb_halo_bytes(ctx, ctypes.byref(n)))
    return n.value


def lb_halo_pack(ctx, face: int, d_buf):
    """Owned edge rows (face 0: first, 1: last) into the device buffer d_buf."""
    _check(load().lb_halo_pack(ctx, int(face), _addr(d_buf)))


def lb_halo_unpack(ctx, face: int, d_buf):
    """Device buffer d_buf into the ghost rows (face 0: lower, 1: upper)."""
    _check(load().lb_halo_unpack(ctx, int(face), _addr(d_buf)))


def lb_free(ctx):
    if ctx is not None:
        _check(load().lb_free(ctx))


def _check_noalloc_args(nx, ny, fields, d_out, stream):
    """The C entry point takes raw device addresses and trusts their sizes, so
    the binding checks every tensor first: float64, C-contiguous, large enough
    for the nx*ny sites (d_out: LB_TOTALS_N values), on a CUDA device, all on
    the stream's device.  Raises LbError(LB_ERR_ARG) otherwise."""
    n = int(nx) * int(ny)

    def bad(msg):
        raise LbError(LB_ERR_ARG, msg)

    named = [(k, v) for k, v in fields if v is not None] + [("d_out", d_out)]
    for name, t in named:
        if not hasattr(t, "data_ptr") or not hasattr(t, "dtype"):
            bad(f"{name}: a torch tensor is required")
        if str(t.dtype) != "torch.float64":
            bad(f"{name}: float64 required, got {t.dtype}")
        if not t.is_contiguous():
            bad(f"{name}: must be contiguous")
        need = LB_TOTALS_N if name == "d_out" else n
        if t.numel() < need:
            bad(f"{name}: {t.numel()} elements, at least {need} required")
    for name, t in named:
        if not t.is_cuda:
            bad(f"{name}: must be a CUDA tensor")
    devs = {t.device.index for _, t in named}
    if stream is not None and hasattr(stream, "device"):
        devs.add(stream.device.index)
    if len(devs) > 1:
        bad(f"tensors and stream on different devices: {sorted(devs)}")


def lb_field_totals_noalloc(nx, ny, cv, d_rho, d_ux, d_uy, d_T, d_out, d_ref_rho=None,
                            d_ref_T=None, K=0, stream=None):
    """Totals of device fields without any device allocation (see include/lb.h);
    d_out receives [mass, energy, px, py, residual] on the device.  Every
    tensor is checked (dtype, layout, size, device) before the call."""
    _check_noalloc_args(nx, ny, [("d_rho", d_rho), ("d_ux", d_ux), ("d_uy", d_uy), ("d_T", d_T),
                                 ("d_ref_rho", d_ref_rho), ("d_ref_T", d_ref_T)], d_out, stream)
    _check(load().lb_field_totals_noalloc(int(nx), int(ny), float(cv), _addr(d_rho), _addr(d_ux),
                                          _addr(d_uy), _addr(d_T), _addr(d_ref_rho),
                                          _addr(d_ref_T), int(K), _addr(d_out), _stream(stream)))


def lb_last_error() -> str:
    return load().lb_last_error().decode()


def lb_version() -> str:
    return load().lb_version().decode()


def lb_batch_init(params, rhos, Ts, stream=None, device_inputs=False):
    """params: sequence of lb_params; rhos, Ts: float64 fields per domain (host
    arrays, or device addresses / tensors with device_inputs=True)."""
    n = len(params)
    arr = (lb_params * n)(*params)
    if device_inputs:
        addr = lambda a: ctypes.cast(_addr(a), ctypes.POINTER(ctypes.c_double))
        rp = (ctypes.POINTER(ctypes.c_double) * n)(*[addr(r) for r in rhos])
        tp = (ctypes.POINTER(ctypes.c_double) * n)(*[addr(t) for t in Ts])
    else:
        rhos = [_host(r, (p.ny, p.nx)) for r, p in zip(rhos, params)]
        Ts = [_host(t, (p.ny, p.nx)) for t, p in zip(Ts, params)]
        rp = (ctypes.POINTER(ctypes.c_double) * n)(*[_dptr(r) for r in rhos])
        tp = (ctypes.POINTER(ctypes.c_double) * n)(*[_dptr(t) for t in Ts])
    b = ctypes.c_void_p()
    _check(load().lb_batch_init(arr, n, rp, tp, _stream(stream), ctypes.byref(b)))
    return b


def lb_batch_step(b, n=1):
    _check(load().lb_batch_step(b, int(n)))


def lb_batch_check(b, n):
    """(residual, mass, energy, status) arrays of length n."""
    r, m, e = np.zeros(n), np.zeros(n), np.zeros(n)
    stt = np.zeros(n, dtype=np.int32)
    _check(load().lb_batch_check(b, _dptr(r), _dptr(m), _dptr(e),
                                 stt.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))))
    return r, m, e, stt


def lb_batch_run(b, n, tol, K=100, max_steps=10 ** 6):
    """Run to residual < tol; returns (steps, residual, status) arrays."""
    steps = np.zeros(n, dtype=np.int64)
    resid = np.zeros(n)
    stt = np.zeros(n, dtype=np.int32)
    _check(load().lb_batch_run(b, float(tol), int(K), int(max_steps),
                               steps.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _dptr(resid),
                               stt.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))))
    return steps, resid, stt


def lb_batch_restart(b, d, rho, T, init_balanced=0, shape=None):
    """Restart domain d from fields rho, T: host float64 arrays [ny, nx] (shape
    checked when given), or device tensors / addresses."""
    if isinstance(rho, np.ndarray):
        rho, T = _host(rho, shape), _host(T, shape)
        _check(load().lb_batch_restart(b, int(d), rho.ctypes.data_as(ctypes.c_void_p),
                                       T.ctypes.data_as(ctypes.c_void_p), int(init_balanced)))
    else:
        _check(load().lb_batch_restart(b, int(d), _addr(rho), _addr(T), int(init_balanced)))


def lb_batch_fields(b, d, nx, ny):
    rho = np.empty((ny, nx))
    T = np.empty((ny, nx))
    _check(load().lb_batch_fields(b, int(d), _dptr(rho), _dptr(T)))
    return rho, T


def lb_batch_time(b) -> int:
    return int(load().lb_batch_time(b))


def lb_tune_candidate(k: int):
    """(tile_x, tile_y) of step shape k (tile_y == 0: strip kernel)."""
    tx, ty = ctypes.c_int32(), ctypes.c_int32()
    _check(load().lb_tune_candidate(int(k), ctypes.byref(tx), ctypes.byref(ty)))
    return tx.value, ty.value


def lb_autotune(p: lb_params, steps: int, stream=None):
    """Time every valid step shape for p; returns (best params, ms per step per shape)."""
    best = lb_params()
    ms = np.full(LB_TUNE_N, np.nan)
    _check(load().lb_autotune(ctypes.byref(p), int(steps), _stream(stream), ctypes.byref(best),
                              _dptr(ms)))
    return best, ms


def lb_batch_set_chunk_rows(b, rows: int):
    _check(load().lb_batch_set_chunk_rows(b, int(rows)))


def lb_batch_chunk_rows(b) -> int:
    return int(load().lb_batch_chunk_rows(b))


def lb_batch_autotune(b, steps: int):
    """Time the row-chunk heights; returns (chosen height, ms per step per height)."""
    rows = ctypes.c_int32()
    ms = np.full(LB_BATCH_TUNE_N, np.nan)
    _check(load().lb_batch_autotune(b, int(steps), ctypes.byref(rows), _dptr(ms)))
    return rows.value, ms


def lb_batch_free(b):
    if b is not None:
        _check(load().lb_batch_free(b))


class Batch:
    """Owner of one batch of independent domains (see lb_batch_* in include/lb.h)."""

    def __init__(self, params, rhos, Ts, stream=None, device_inputs=False):
        self.params = list(params)
        self.n = len(self.params)
        self.b = lb_batch_init(self.params, rhos, Ts, stream, device_inputs)

    def step(self, n=1):
        lb_batch_step(self.b, n)
        return self

    def check(self):
        return lb_batch_check(self.b, self.n)

    def run(self, tol, K=100, max_steps=10 ** 6):
        return lb_batch_run(self.b, self.n, tol, K, max_steps)

    def fields(self, d):
        p = self.params[d]
        return lb_batch_fields(self.b, d, p.nx, p.ny)

    def restart(self, d, rho, T, init_balanced=0):
        """Restart domain d from the fields rho, T (see lb_batch_restart)."""
        p = self.params[d]
        lb_batch_restart(self.b, d, rho, T, init_balanced, shape=(p.ny, p.nx))

    @property
    def time(self):
        return lb_batch_time(self.b)

    @property
    def chunk_rows(self):
        return lb_batch_chunk_rows(self.b)

    @chunk_rows.setter
    def chunk_rows(self, rows):
        lb_batch_set_chunk_rows(self.b, rows)

    def autotune(self, steps=20):
        return lb_batch_autotune(self.b, steps)

    def close(self):
        if self.b is not None:
            lb_batch_free(self.b)
            self.b = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Lattice:
    """Convenience owner of one context (frees it on close / garbage collection)."""

    def __init__(self, rho, T, stream=None, device_inputs=False, **params):
        """rho, T: initial density and temperature fields [ny, nx] (host float64
        arrays, or device arrays with device_inputs=True); params: lb_params fields."""
        self.params = lb_params_default(**params)
        if device_inputs:
            self.ctx = lb_init_device(self.params, rho, T, stream)
        else:
            self.ctx = lb_init(self.params, rho, T, stream)

    def step(self, n=1):
        lb_step(self.ctx, n)
        return self

    def synchronize(self):
        lb_synchronize(self.ctx)

    def moments(self):
        return lb_moments(self.ctx)

    def populations(self):
        return lb_get_populations(self.ctx)

    def set_populations(self, f, g):
        lb_set_populations(self.ctx, f, g)

    def totals(self):
        return lb_totals(self.ctx)

    @property
    def time(self):
        return lb_time(self.ctx)

    def close(self):
        if self.ctx is not None:
            lb_free(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
