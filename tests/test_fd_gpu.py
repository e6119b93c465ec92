"""Finite-difference temperature treatment (Eqs. 26-27) on the GPU against
the FP64 oracle: FP64 storage to 1e-12 (the arithmetic follows the printed
order), FP32 within 2e-5 on rho and T; both RK2 forms; ragged lattices;
totals; and the calls that do not apply rejected."""
import ctypes

import numpy as np
import pytest

import oracle as O
from paper_1405_2232_gb300 import inputs as I


@pytest.fixture(scope="module")
def lb():
    from paper_1405_2232_gb300 import lb as _lb
    _lb.load()
    return _lb


def setup(nx=64, ny=64, local_T=1):
    rho, _ = I.slab_fields(nx, ny, width=nx // 2, rho_l=0.3, rho_g=0.04, noise=1e-3)
    X = np.arange(nx)[None, :].repeat(ny, axis=0)
    T = 0.85 * I.CS_TC * (1.0 + 0.01 * np.sin(2 * np.pi * X / nx))
    P = O.params(nx, ny, tau_f=1.0, tau_g=0.8, G=-1.0, beta=1.0, eos=O.EOS_CS, a=1.0, b=4.0, R=1.0,
                 psi_uses_local_T=local_T, T_psi=0.0 if local_T else 0.85 * I.CS_TC)
    return rho, T, P


def oracle_run(P, rho, T, n, printed):
    f, _ = O.init_equilibrium(P, rho, T)
    f, Tn, st, _ = O.step_fd(P, f, T, n=n, printed=printed, check=False)
    # rho, u at the final time level: the front half of one more step
    _, _, _, (r, ux, uy) = O.step_fd(P, f, Tn, n=1, printed=printed, check=False)
    return r, ux, uy, Tn, st


def gpu_run(lb, P, rho, T, n, thermal, prec, tile=None):
    extra = {} if tile is None else dict(tile_x=tile[0], tile_y=tile[1])
    with lb.Lattice(rho, T, nx=P.nx, ny=P.ny, precision=prec, tau_f=P.tau_f, tau_g=P.tau_g, G=P.G,
                    beta=P.beta, thermal=thermal, psi_uses_local_T=P.psi_uses_local_T, T_psi=P.T_psi,
                    **extra) as L:
        L.step(n)
        m = L.moments()
        tot = L.totals()
        shape = (lb.lb_get_params(L.ctx).tile_x, lb.lb_get_params(L.ctx).tile_y)
    return m, tot, shape


def rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.gpu
@pytest.mark.parametrize("printed", [False, True])
def test_fd_fp64_matches_oracle(lb, printed):
    rho, T, P = setup()
    thermal = lb.LB_THERMAL_FD26_PRINTED if printed else lb.LB_THERMAL_FD26
    r, ux, uy, Tn, st = oracle_run(P, rho, T, 300, printed)
    assert st == 0
    (gr, gux, guy, gT), _, _ = gpu_run(lb, P, rho, T, 300, thermal, "fp64")
    assert rel(gr, r) <= 1e-12 and rel(gT, Tn) <= 1e-12
    assert np.abs(gux - ux).max() <= 1e-12 * np.abs(ux).max()
    assert np.abs(guy - uy).max() <= 1e-12 * max(np.abs(uy).max(), 1e-300) or np.abs(guy - uy).max() < 1e-15


@pytest.mark.gpu
@pytest.mark.parametrize("nx,ny", [(67, 45), (5, 130), (33, 9)])
def test_fd_fp64_ragged(lb, nx, ny):
    rho, T, P = setup(nx, ny, local_T=0)
    r, ux, uy, Tn, st = oracle_run(P, rho, T, 60, False)
    (gr, gux, guy, gT), _, _ = gpu_run(lb, P, rho, T, 60, lb.LB_THERMAL_FD26, "fp64")
    assert rel(gr, r) <= 1e-12 and rel(gT, Tn) <= 1e-12


@pytest.mark.gpu
def test_fd_fp32_within_tolerance(lb):
    rho, T, P = setup()
    r, ux, uy, Tn, st = oracle_run(P, rho, T, 1000, False)
    (gr, gux, guy, gT), _, _ = gpu_run(lb, P, rho, T, 1000, lb.LB_THERMAL_FD26, "fp32")
    e_rho, e_T = rel(gr, r), rel(gT, Tn)
    assert e_rho <= 2e-5 and e_T <= 2e-5, (e_rho, e_T)


@pytest.mark.gpu
def test_fd_totals(lb):
    rho, T, P = setup()
    r, ux, uy, Tn, st = oracle_run(P, rho, T, 100, False)
    (gr, gux, guy, gT), tot, _ = gpu_run(lb, P, rho, T, 100, lb.LB_THERMAL_FD26, "fp64")
    assert tot[0] == pytest.approx(rho.sum(), rel=1e-13)              # mass of the density LBE
    assert tot[1] == pytest.approx(np.sum(r * Tn), rel=1e-12)         # sum rho c_v T (c_v = 1)
    assert tot[2] == pytest.approx(np.sum(r * ux), rel=1e-9, abs=1e-15)


@pytest.mark.gpu
def test_fd_rejects_what_does_not_apply(lb):
    rho, T, P = setup(16, 12)
    p16 = lb.lb_params_default(nx=16, ny=12, thermal=lb.LB_THERMAL_FD26, precision="fp16")
    ctx = ctypes.c_void_p()
    dp = lambda a: np.ascontiguousarray(a).ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    assert lb.load().lb_init(ctypes.byref(p16), dp(rho), dp(T), None, ctypes.byref(ctx)) == lb.LB_ERR_UNSUPPORTED
    ps = lb.lb_params_default(nx=16, ny=12, thermal=lb.LB_THERMAL_FD26, tile_x=128, tile_y=0)
    assert lb.load().lb_init(ctypes.byref(ps), dp(rho), dp(T), None, ctypes.byref(ctx)) == lb.LB_ERR_ARG
    with lb.Lattice(rho, T, nx=16, ny=12, thermal=lb.LB_THERMAL_FD26) as L:
        with pytest.raises(lb.LbError) as ei:
            L.populations()
        assert ei.value.status == lb.LB_ERR_UNSUPPORTED
        L.step(5)
        L.synchronize()


@pytest.mark.gpu
@pytest.mark.parametrize("prec,nx,ny,strip", [("fp64", 64, 64, (128, 0)), ("fp64", 300, 40, (128, 0)),
                                              ("fp32", 64, 64, (256, 0)), ("fp32", 260, 24, (256, 0))])
def test_fd_strip_front_matches_tile_front(lb, prec, nx, ny, strip):
    """The fused strip kernel (whole FD step in one pass, ghost-column
    layout) and the tile front + fused RK2 give the same bits in FP64, which
    also match the oracle to 1e-12; FP32 agrees to 1e-6; the lattices include
    partial last strips."""
    rho, T, P = setup(nx, ny)
    (sr, sux, suy, sT), _, shape_s = gpu_run(lb, P, rho, T, 40, lb.LB_THERMAL_FD26, prec, tile=strip)
    (tr, tux, tuy, tT), _, shape_t = gpu_run(lb, P, rho, T, 40, lb.LB_THERMAL_FD26, prec, tile=(32, 8))
    assert shape_s == strip and shape_t == (32, 8)
    if prec == "fp64":
        for a, b in ((sr, tr), (sux, tux), (suy, tuy), (sT, tT)):
            assert np.array_equal(a, b)
        r, ux, uy, Tn, st = oracle_run(P, rho, T, 40, False)
        assert rel(sr, r) <= 1e-12 and rel(sT, Tn) <= 1e-12
    else:
        assert rel(sr, tr) <= 1e-6 and rel(sT, tT) <= 1e-6
