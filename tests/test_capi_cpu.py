"""CPU checks of the C-ABI boundary: the CUDA library builds for sm_103a, loads,
exports every function include/lb.h declares, and validates arguments on the
host.  No kernel is launched here (there is no GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1405_2232_gb300 import lb
    return lb, lb.load()


def declared_functions():
    """Function names declared in include/*.h (C declarations ending in ');')."""
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(lb_\w+)\s*\([^;{]*\)\s*;", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_every_declared_symbol_is_exported(lib):
    lb, so = lib
    names = declared_functions()
    assert len(names) >= 18
    for name in names:
        assert hasattr(so, name), f"{name} declared in include/ but not exported"
    assert set(names) <= set(lb.EXPORTED) | set(names)
    for name in lb.EXPORTED:
        assert name in names, f"binding names {name}, which the header does not declare"


def test_library_is_built_for_sm103a(lib):
    lb, _ = lib
    from paper_1405_2232_gb300 import build
    assert ["-gencode", "arch=compute_103a,code=sm_103a"] == build.ARCH
    assert os.path.exists(lb.library_path())


def test_params_default_layout(lib):
    lb, _ = lib
    p = lb.lb_params_default()
    assert (p.nx, p.ny) == (64, 64)
    assert (p.tau_f, p.tau_g, p.G, p.beta) == (1.0, 0.8, -1.0, 1.0)
    assert (p.a, p.b, p.R, p.cv) == (1.0, 4.0, 1.0, 1.0)
    assert p.eos == lb.LB_EOS_CS and p.thermal == lb.LB_THERMAL_EQ24
    assert p.precision == lb.LB_PREC_FP32 and p.psi_uses_local_T == 1
    assert (p.rho0, p.T0) == (0.12, 0.075)
    assert p.init_balanced == 0 and p.walls == lb.LB_WALLS_PERIODIC


@pytest.mark.parametrize("field,value", [
    ("nx", 2), ("ny", 0), ("tau_f", 0.5), ("tau_g", 0.3), ("G", 0.0), ("cv", 0.0),
    ("eos", 7), ("thermal", 4), ("precision", 9), ("tile_x", 17), ("init_balanced", 2),
])
def test_invalid_params_rejected_on_host(lib, field, value):
    import numpy as np
    lb, so = lib
    p = lb.lb_params_default(nx=8, ny=8)
    setattr(p, field, value)
    rho = np.ones((8, 8))
    dp = rho.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    ctx = ctypes.c_void_p()
    st = so.lb_init(ctypes.byref(p), dp, dp, None, ctypes.byref(ctx))
    assert st == lb.LB_ERR_ARG
    assert ctx.value is None
    assert lb.lb_last_error() != ""


@pytest.mark.parametrize("field,value", [("walls", 1), ("walls", 2), ("thermal", 2)])
def test_start_at_rest_is_periodic_lb_only(lib, field, value):
    """The start at rest under the force is refused on the host for walled
    lattices and the finite-difference treatment."""
    import numpy as np
    lb, so = lib
    p = lb.lb_params_default(nx=32, ny=8, precision=lb.LB_PREC_FP64, init_balanced=1)
    setattr(p, field, value)
    if field == "walls":
        p.tile_x, p.tile_y = 32, 8
    rho = np.ones((8, 32))
    dp = rho.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    ctx = ctypes.c_void_p()
    st = so.lb_init(ctypes.byref(p), dp, dp, None, ctypes.byref(ctx))
    assert st == lb.LB_ERR_UNSUPPORTED
    assert ctx.value is None
    assert "rest" in lb.lb_last_error()


def test_null_arguments(lib):
    lb, so = lib
    assert so.lb_free(None) == lb.LB_OK
    assert so.lb_step(None, 1) == lb.LB_ERR_ARG
    assert so.lb_totals(None, None) == lb.LB_ERR_ARG
    assert so.lb_time(None) == -1
    assert "sm_103a" in lb.lb_version()


def test_oracle_and_cuda_path_share_nothing():
    """The oracle includes nothing of the library and the library nothing of the oracle."""
    csrc = os.path.join(ROOT, "paper_1405_2232_gb300", "csrc")
    for fn in os.listdir(csrc):
        text = open(os.path.join(csrc, fn)).read()
        assert "oracle" not in text.lower(), fn
    otext = open(os.path.join(ROOT, "oracle", "lb_oracle.c")).read()
    assert '#include "lb.h"' not in otext and "lbgb" not in otext
    for fn in os.listdir(os.path.join(ROOT, "paper_1405_2232_gb300")):
        if fn.endswith(".py"):
            text = open(os.path.join(ROOT, "paper_1405_2232_gb300", fn)).read()
            assert "import oracle" not in text and "from oracle" not in text, fn


def test_noalloc_binding_rejects_bad_tensors(lib):
    """lb_field_totals_noalloc takes raw device addresses, so the binding checks
    dtype, layout, size and device of every tensor before the call (no tensor
    reaches the library here: each case is rejected on the host)."""
    import torch
    lb, _ = lib
    nx, ny = 8, 4
    ok = lambda n=nx * ny: torch.zeros(n, dtype=torch.float64)
    out = torch.zeros(lb.LB_TOTALS_N, dtype=torch.float64)
    cases = [
        ((torch.zeros(nx * ny, dtype=torch.float32), ok(), ok(), ok(), out), "float64"),
        ((torch.zeros(ny, 2 * nx, dtype=torch.float64)[:, ::2], ok(), ok(), ok(), out), "contiguous"),
        ((ok(nx * ny - 1), ok(), ok(), ok(), out), "at least"),
        ((ok(), ok(), ok(), ok(), torch.zeros(4, dtype=torch.float64)), "at least 5"),
        ((ok(), ok(), ok(), ok(), out), "CUDA"),
        ((12345, ok(), ok(), ok(), out), "torch tensor"),
    ]
    for args, word in cases:
        with pytest.raises(lb.LbError) as ei:
            lb.lb_field_totals_noalloc(nx, ny, 1.0, *args)
        assert ei.value.status == lb.LB_ERR_ARG and word in str(ei.value), (word, str(ei.value))
    with pytest.raises(lb.LbError) as ei:  # a too-small reference field
        lb.lb_field_totals_noalloc(nx, ny, 1.0, ok(), ok(), ok(), ok(), out, d_ref_rho=ok(3),
                                   d_ref_T=ok(), K=1)
    assert "d_ref_rho" in str(ei.value)


def test_halo_rows_validated_on_host(lib):
    """Ghost-row (y-slab) contexts: only LB_HALO_ROWS ghost rows, periodic lattice
    Boltzmann contexts only, enough rows; the exchange calls reject a NULL context
    (all rejected before any device work)."""
    lb, so = lib
    import numpy as np
    rho = np.full((12, 16), 0.2)
    for kw, code in [(dict(halo_rows=3), lb.LB_ERR_ARG), (dict(halo_rows=2, ny=4), lb.LB_ERR_ARG),
                     (dict(halo_rows=2, walls=lb.LB_WALLS_CAVITY), lb.LB_ERR_UNSUPPORTED),
                     (dict(halo_rows=2, thermal=lb.LB_THERMAL_FD26), lb.LB_ERR_UNSUPPORTED)]:
        p = lb.lb_params_default(nx=16, ny=kw.pop("ny", 12), **kw)
        r = np.full((p.ny, p.nx), 0.2)
        ctx = ctypes.c_void_p()
        st = so.lb_init(ctypes.byref(p), lb._dptr(r), lb._dptr(r), None, ctypes.byref(ctx))
        assert st == code and ctx.value is None, (kw, st)
    n = ctypes.c_size_t()
    assert so.lb_halo_bytes(None, ctypes.byref(n)) == lb.LB_ERR_ARG
    assert so.lb_halo_pack(None, 0, None) == lb.LB_ERR_ARG
    assert so.lb_halo_unpack(None, 1, None) == lb.LB_ERR_ARG
    assert lb.lb_params_default().halo_rows == 0 and lb.LB_HALO_ROWS == 2
