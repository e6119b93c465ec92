"""Host logic of the autotuner: cache keys, the JSON cache, the shape list and
argument checks of the native entry points (no GPU needed)."""
import ctypes
import json
import math

import numpy as np
import pytest

from paper_1405_2232_gb300 import autotune as A
from paper_1405_2232_gb300 import lb


@pytest.fixture(scope="module")
def lib():
    return lb.load()


def test_shape_list(lib):
    shapes = [lb.lb_tune_candidate(k) for k in range(lb.LB_TUNE_N)]
    assert shapes == [(256, 0), (128, 0), (32, 8), (32, 16), (64, 4)]
    with pytest.raises(lb.LbError):
        lb.lb_tune_candidate(lb.LB_TUNE_N)


def test_autotune_argument_checks(lib):
    p = lb.lb_params_default(nx=64, ny=64)
    best = lb.lb_params()
    assert lib.lb_autotune(ctypes.byref(p), 0, None, ctypes.byref(best), None) == lb.LB_ERR_ARG
    assert lib.lb_autotune(None, 4, None, ctypes.byref(best), None) == lb.LB_ERR_ARG
    assert lib.lb_batch_autotune(None, 4, None, None) == lb.LB_ERR_ARG
    assert lib.lb_batch_set_chunk_rows(None, 64) == lb.LB_ERR_ARG
    assert lib.lb_batch_chunk_rows(None) == -1


def test_keys_separate_what_changes_the_choice():
    base = dict(nx=300, ny=200, precision="fp32")
    k0 = A.tune_key(lb.lb_params_default(**base), "GB300")
    assert k0 == A.tune_key(lb.lb_params_default(nx=500, ny=256, precision="fp32"), "GB300")
    differ = [dict(base, precision="fp64"), dict(base, thermal=lb.LB_THERMAL_EQ7),
              dict(base, thermal=lb.LB_THERMAL_FD26), dict(base, thermal=lb.LB_THERMAL_FD26_PRINTED),
              dict(base, walls=lb.LB_WALLS_CAVITY), dict(base, walls=lb.LB_WALLS_CHANNEL),
              dict(base, beta=1.3), dict(base, beta=0.0), dict(base, nx=600),
              dict(base, ny=257), dict(base, nx=302)]  # 302: not a multiple of 4
    keys = {A.tune_key(lb.lb_params_default(**d), "GB300") for d in differ}
    assert len(keys) == len(differ) and k0 not in keys
    assert A.tune_key(lb.lb_params_default(**base), "other") != k0


def test_cache_round_trip(tmp_path):
    calls = []

    def timer(p, steps):
        calls.append((p.nx, steps))
        best = A.ctypes_copy(lb.lb_params(), p)
        best.tile_x, best.tile_y = 32, 16
        return best, np.array([1.0, 0.9, 0.8, 0.5, np.nan])

    path = str(tmp_path / "sub" / "tune.json")
    p = lb.lb_params_default(nx=96, ny=64, precision="fp32", tau_f=0.7)
    q = A.tuned_params(p, A.TuneCache(path), device_name="dev", timer=timer)
    assert (q.tile_x, q.tile_y, q.tau_f, q.nx) == (32, 16, 0.7, 96)
    assert calls == [(96, A.default_steps(96 * 64))]
    # a fresh cache object reads the file; the timer is not called again
    q2 = A.tuned_params(p, A.TuneCache(path), device_name="dev", timer=timer)
    assert (q2.tile_x, q2.tile_y) == (32, 16) and len(calls) == 1
    d = json.load(open(path))
    (entry,) = d.values()
    assert entry["ms_per_step"][4] is None and entry["shapes"][3] == [32, 16]
    # the caller's params are not modified
    assert (p.tile_x, p.tile_y) == (0, 0)


def test_batch_cache_round_trip(tmp_path):
    class FakeBatch:
        def __init__(self):
            self.params = [lb.lb_params_default(nx=64, ny=64), lb.lb_params_default(nx=128, ny=96)]
            self.chunk_rows = 64

    path = str(tmp_path / "tune.json")
    n = []

    def timer(b, steps):
        n.append(steps)
        b.chunk_rows = 32
        return 32, np.array([2.0, 1.0, 1.5, 3.0])

    b = FakeBatch()
    assert A.tuned_batch(b, A.TuneCache(path), device_name="dev", timer=timer) == 32
    b2 = FakeBatch()
    assert A.tuned_batch(b2, A.TuneCache(path), device_name="dev", timer=timer) == 32
    assert b2.chunk_rows == 32 and n == [20]


def test_corrupt_cache_is_ignored(tmp_path):
    path = tmp_path / "tune.json"
    path.write_text("{not json")
    assert A.TuneCache(str(path)).data == {}


def test_default_steps():
    assert A.default_steps(4096 * 4096) == 118
    assert A.default_steps(64 * 64) == 200
    assert A.default_steps(10 ** 10) == 4
    assert all(A.default_steps(s) % 2 == 0 for s in (3, 1000, 123457, 10 ** 8))
