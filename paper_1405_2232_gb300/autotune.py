"""Autotuned step shapes and batch work-list granularity, with a JSON cache.

The timing itself is native (``lb_autotune`` and ``lb_batch_autotune`` in the
library, CUDA events on the device); this module only keys, stores and
reuses the winners.

A single-lattice tuning is keyed by the device name, storage precision,
temperature treatment (Eq. 7 or Eq. 24), force form (beta = 0, 1 or mixed,
Eq. 2 / Eq. 4), the lattice's size class (nx and ny rounded up to powers of
two) and whether nx meets the strip kernel's 16-byte row rule.  A batch
tuning is keyed by the device, precision, treatment, force form, the number
of domains and the total site count (both rounded up to powers of two).

The cache is a flat JSON object ``{key: entry}``; it is written atomically
(temporary file + rename).  Its default path is ``$LBGB_TUNE_CACHE`` or
``~/.cache/lbgb/autotune.json``.
"""
from __future__ import annotations

import json
import math
import os
import tempfile

from . import lb

STRIP_HALO = {lb.LB_PREC_FP64: 2, lb.LB_PREC_FP32: 4, lb.LB_PREC_FP16_DEV: 8, lb.LB_PREC_BF16_DEV: 8}
PREC_NAMES = {v: k for k, v in lb.PRECISIONS.items()}


def default_cache_path() -> str:
    return os.environ.get("LBGB_TUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "lbgb", "autotune.json"))


def _pow2(n: int) -> int:
    return 1 << max(0, math.ceil(math.log2(max(1, int(n)))))


def force_form(beta: float) -> str:
    return "b0" if beta == 0.0 else ("b1" if beta == 1.0 else "bmix")


TREATMENTS = {lb.LB_THERMAL_EQ7: "eq7", lb.LB_THERMAL_EQ24: "eq24", lb.LB_THERMAL_FD26: "fd26",
              lb.LB_THERMAL_FD26_PRINTED: "fd26p"}
BOUNDARIES = {lb.LB_WALLS_PERIODIC: "periodic", lb.LB_WALLS_CAVITY: "cavity", lb.LB_WALLS_CHANNEL: "channel"}


def tune_key(p, device_name: str) -> str:
    aligned = "a" if p.nx % STRIP_HALO[p.precision] == 0 else "u"
    return "|".join([device_name, PREC_NAMES[p.precision], TREATMENTS[p.thermal], BOUNDARIES[p.walls],
                     force_form(p.beta), f"{_pow2(p.nx)}x{_pow2(p.ny)}{aligned}"])


def batch_key(params, device_name: str) -> str:
    p = params[0]
    sites = sum(q.nx * q.ny for q in params)
    return "|".join([device_name, "batch", PREC_NAMES[p.precision], TREATMENTS[p.thermal],
                     force_form(p.beta), f"n{_pow2(len(params))}", f"s{_pow2(sites)}"])


def default_steps(sites: int) -> int:
    """About 2e9 site updates per shape, 4..200 steps (even)."""
    s = int(2e9 / max(1, sites))
    return max(4, min(200, s - s % 2))


def _device_name() -> str:
    import torch
    return torch.cuda.get_device_name(torch.cuda.current_device()).replace("|", "/")


class TuneCache:
    """A JSON file of tuning results."""

    def __init__(self, path: str | None = None):
        self.path = path or default_cache_path()
        self.data = {}
        if os.path.exists(self.path):
            try:
                with open(self.path) as fh:
                    d = json.load(fh)
                if isinstance(d, dict):
                    self.data = d
            except (OSError, ValueError):
                self.data = {}

    def get(self, key):
        return self.data.get(key)

    def put(self, key, entry):
        self.data[key] = entry
        os.makedirs(os.path.dirname(os.path.abspath(self.path)), exist_ok=True)
        fd, tmp = tempfile.mkstemp(dir=os.path.dirname(os.path.abspath(self.path)), suffix=".tmp")
        with os.fdopen(fd, "w") as fh:
            json.dump(self.data, fh, indent=1, sort_keys=True)
        os.replace(tmp, self.path)


def tuned_params(p, cache: TuneCache | None = None, steps: int | None = None,
                 device_name: str | None = None, timer=None):
    """p with tile_x/tile_y set to the fastest step shape (cached per key).

    ``timer(p, steps) -> (best_params, ms_per_shape)`` defaults to lb.lb_autotune."""
    cache = cache or TuneCache()
    key = tune_key(p, device_name or _device_name())
    hit = cache.get(key)
    out = lb.lb_params()
    ctypes_copy(out, p)
    if hit is None:
        timer = timer or lb.lb_autotune
        best, ms = timer(p, steps or default_steps(p.nx * p.ny))
        hit = {"tile_x": int(best.tile_x), "tile_y": int(best.tile_y),
               "ms_per_step": [None if math.isnan(v) else float(v) for v in ms],
               "shapes": [list(lb.lb_tune_candidate(k)) for k in range(len(ms))]}
        cache.put(key, hit)
    out.tile_x, out.tile_y = hit["tile_x"], hit["tile_y"]
    return out


def tuned_batch(batch, cache: TuneCache | None = None, steps: int = 20,
                device_name: str | None = None, timer=None) -> int:
    """Set the batch's row-chunk height to the fastest (cached per key); returns it.

    ``timer(batch, steps) -> (rows, ms_per_height)`` defaults to Batch.autotune."""
    cache = cache or TuneCache()
    key = batch_key(batch.params, device_name or _device_name())
    hit = cache.get(key)
    if hit is None:
        rows, ms = (timer or (lambda b, s: b.autotune(s)))(batch, steps)
        hit = {"chunk_rows": int(rows),
               "ms_per_step": [None if math.isnan(v) else float(v) for v in ms]}
        cache.put(key, hit)
    else:
        batch.chunk_rows = hit["chunk_rows"]
    return hit["chunk_rows"]


def ctypes_copy(dst, src):
    for name, _ in src._fields_:
        setattr(dst, name, getattr(src, name))
    return dst
