"""Warm-start network boundary on the host: exported symbols, the parameter
layout against the oracle's architecture, argument checks (no GPU needed)."""
import ctypes
import re
from pathlib import Path

import pytest

from oracle import unet as U
from paper_1405_2232_gb300 import lb
from paper_1405_2232_gb300 import unet as N

ROOT = Path(__file__).resolve().parents[1]


def test_header_symbols_are_exported():
    lib = N.load()
    text = (ROOT / "include" / "unet.h").read_text()
    declared = set(re.findall(r"\b(un_[a-z_]+)\s*\(", text))
    assert declared == set(N.EXPORTED)
    for name in declared:
        assert hasattr(lib, name), name


@pytest.mark.parametrize("base", [32, 64])
def test_layer_table_matches_oracle(base):
    cfg = N.config(64, 64, 2, base)
    arch = U.architecture(base=base)
    assert N.param_count(cfg) == U.param_count(arch)
    off = 0
    for (name, ci, co, k, _), (ci2, co2, k2, off2) in zip(arch, N.layer_table(cfg)):
        assert (ci, co, k, off) == (ci2, co2, k2, off2), name
        off += co * k * k * ci + co


@pytest.mark.parametrize("H,W,batch,base", [(60, 64, 1, 32), (64, 12, 1, 32), (64, 64, 0, 32),
                                             (64, 64, 1, 48), (0, 64, 1, 32)])
def test_invalid_configs_rejected(H, W, batch, base):
    lib = N.load()
    cfg = N.config(H, W, batch, base)
    net = ctypes.c_void_p()
    assert lib.un_create(ctypes.byref(cfg), None, ctypes.byref(net)) == lb.LB_ERR_ARG
    assert net.value is None
    assert lib.un_param_count(ctypes.byref(cfg)) == -1


def test_unsupported_width_and_null_arguments():
    lib = N.load()
    cfg = N.config(64, 64, 1, 96)
    net = ctypes.c_void_p()
    assert lib.un_create(ctypes.byref(cfg), None, ctypes.byref(net)) == lb.LB_ERR_UNSUPPORTED
    assert lib.un_forward(None, 1, None, None) == lb.LB_ERR_ARG
    assert lib.un_adam_step(None, 1e-3, 0.9, 0.999, 1e-8) == lb.LB_ERR_ARG
    assert lib.un_warm_fields(0, 8, 8, None, 0, 0, 0, None, None, None, None, None) == lb.LB_ERR_ARG
    assert lib.un_free(None) == lb.LB_OK
