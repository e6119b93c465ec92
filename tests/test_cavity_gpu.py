"""Natural-convection cavity (Sec. III B) on the GPU: FP64 bit for bit with the
oracle's cavity step (walls, buoyancy, both temperature treatments, partial
tiles), FP32 within rounding, and Table II at Ra = 10^3 and 10^4."""
import numpy as np
import pytest

import oracle as O


@pytest.fixture(scope="module")
def lb():
    from paper_1405_2232_gb300 import lb as _lb
    _lb.load()
    return _lb


def oracle_cavity(nx, ny, thermal, g_grav, T_hot=1.03, T_cold=0.97):
    P, Cv = O.cavity_setup(1e3, nx, thermal=thermal, T_hot=T_hot, T_cold=T_cold)
    P.ny = ny
    Cv.g_grav = g_grav
    return P, Cv


def gpu_cavity(lb, P, Cv, prec, rho=None, T=None):
    rho = np.ones((P.ny, P.nx)) if rho is None else rho
    T = np.ones((P.ny, P.nx)) if T is None else T
    return lb.Lattice(rho, T, nx=P.nx, ny=P.ny, precision=prec, tau_f=P.tau_f, tau_g=P.tau_g, G=P.G,
                      beta=P.beta, eos=lb.LB_EOS_IDEAL, a=0.0, b=0.0, R=P.R, cv=P.cv, thermal=P.thermal,
                      psi_uses_local_T=1, walls=lb.LB_WALLS_CAVITY, T_hot=Cv.T_hot, T_cold=Cv.T_cold,
                      g_grav=Cv.g_grav)


@pytest.mark.gpu
@pytest.mark.parametrize("thermal", [O.THERMAL_EQ24, O.THERMAL_EQ7])
@pytest.mark.parametrize("nx,ny", [(37, 21), (64, 64)])
def test_cavity_fp64_bit_identical(lb, thermal, nx, ny):
    P, Cv = oracle_cavity(nx, ny, thermal, 2e-3)
    f0, g0 = O.init_equilibrium(P, np.ones((ny, nx)), np.ones((ny, nx)))
    f_ref, g_ref, st = O.step_cavity(P, Cv, f0, g0, n=300, threads=8, check=False)
    with gpu_cavity(lb, P, Cv, "fp64") as L:
        assert (lb.lb_get_params(L.ctx).tile_x, lb.lb_get_params(L.ctx).tile_y) == (32, 8)
        L.step(300)
        f, g = L.populations()
    assert np.array_equal(f, f_ref) and np.array_equal(g, g_ref)


@pytest.mark.gpu
def test_cavity_fp32_within_rounding(lb):
    P, Cv = oracle_cavity(48, 40, O.THERMAL_EQ24, 2e-3)
    f0, g0 = O.init_equilibrium(P, np.ones((40, 48)), np.ones((40, 48)))
    f_ref, g_ref, _ = O.step_cavity(P, Cv, f0, g0, n=2000, threads=8)
    r_ref, _, _, T_ref, _, _ = O.moments(P, f_ref, g_ref)
    with gpu_cavity(lb, P, Cv, "fp32") as L:
        L.step(2000)
        r, ux, uy, T = L.moments()
    assert np.abs(r - r_ref).max() < 2e-5 and np.abs(T - T_ref).max() < 2e-5


def _run_to_steady(lb, P, Cv, prec, seg, max_steps, rel=2e-5):
    """Steps until the flux Nusselt number changes by less than rel over a segment."""
    with gpu_cavity(lb, P, Cv, prec) as L:
        prev, steps = None, 0
        while steps < max_steps:
            L.step(seg)
            steps += seg
            f, g = L.populations()
            nu = O.nusselt_hot_flux(P, Cv, f, g)
            if prev is not None and abs(nu - prev) < rel * abs(nu):
                break
            prev = nu
        T = L.moments()[3]
    return nu, O.nusselt_hot(P, Cv, T), steps


@pytest.mark.gpu
@pytest.mark.parametrize("Ra,Lc,nu24_paper,nu7_paper", [(1e3, 100, 1.118, 4.884), (1e4, 150, 2.246, 8.431)])
def test_cavity_table2(lb, Ra, Lc, nu24_paper, nu7_paper):
    """Table II: Eq. (24) reproduces the benchmark Nusselt number; Eq. (7)
    shows the steep wall gradient of the forcing-term effect."""
    P, Cv = O.cavity_setup(Ra, Lc, thermal=O.THERMAL_EQ24)
    nu24, nu24_grad, steps = _run_to_steady(lb, P, Cv, "fp64", 20000, 600000)
    print(f"Ra={Ra:g} L={Lc}: Eq.24 Nu(flux)={nu24:.4f} Nu(grad)={nu24_grad:.4f} after {steps} steps")
    assert nu24 == pytest.approx(nu24_paper, rel=0.01)
    assert nu24_grad == pytest.approx(nu24_paper, rel=0.035)
    P7, Cv7 = O.cavity_setup(Ra, Lc, thermal=O.THERMAL_EQ7)
    nu7, nu7_grad, steps7 = _run_to_steady(lb, P7, Cv7, "fp64", 20000, 200000, rel=1e-3)
    print(f"Ra={Ra:g} L={Lc}: Eq.7 Nu(flux)={nu7:.4f} Nu(grad)={nu7_grad:.4f} after {steps7} steps")
    # the paper: Eq. (7) is off by more than 250% at Ra = 10^4
    assert nu7_grad > 3.5 * nu24_paper
    if Ra == 1e3:
        assert nu7_grad == pytest.approx(nu7_paper, rel=0.1)
    # the energy that actually crosses the wall is small: lambda_eff of Eq. (23) ~ 0
    assert nu7 < 0.5 * nu24


def gpu_fd_cavity(lb, P, Cv, prec, printed=False):
    thermal = lb.LB_THERMAL_FD26_PRINTED if printed else lb.LB_THERMAL_FD26
    return lb.Lattice(np.ones((P.ny, P.nx)), np.ones((P.ny, P.nx)), nx=P.nx, ny=P.ny, precision=prec,
                      tau_f=P.tau_f, tau_g=P.tau_g, G=P.G, beta=P.beta, eos=lb.LB_EOS_IDEAL, a=0.0, b=0.0,
                      R=P.R, cv=P.cv, thermal=thermal, psi_uses_local_T=1, walls=lb.LB_WALLS_CAVITY,
                      T_hot=Cv.T_hot, T_cold=Cv.T_cold, g_grav=Cv.g_grav)


@pytest.mark.gpu
@pytest.mark.parametrize("printed", [False, True])
@pytest.mark.parametrize("nx,ny", [(37, 21), (64, 64)])
def test_cavity_fd_fp64_bit_identical(lb, printed, nx, ny):
    """The hybrid scheme (Eqs. 26-27) in the cavity: tile front with the wall
    rules, both RK2 stages with the reflected ghosts; FP64 bit for bit with
    the oracle's FD cavity step."""
    P, Cv = oracle_cavity(nx, ny, O.THERMAL_EQ24, 2e-3)
    f0, _ = O.init_equilibrium(P, np.ones((ny, nx)), np.ones((ny, nx)))
    f, T, st, _ = O.step_fd_cavity(P, Cv, f0, np.ones((ny, nx)), n=200, printed=printed, threads=8)
    _, _, _, (r, ux, uy) = O.step_fd_cavity(P, Cv, f, T, n=1, printed=printed, check=False)
    with gpu_fd_cavity(lb, P, Cv, "fp64", printed) as L:
        L.step(200)
        gr, gux, guy, gT = L.moments()
    assert np.array_equal(gr, r) and np.array_equal(gT, T)
    assert np.abs(gux - ux).max() <= 1e-14 and np.abs(guy - uy).max() <= 1e-14


@pytest.mark.gpu
@pytest.mark.parametrize("Ra,Lc,nu_paper", [(1e3, 100, 1.118), (1e4, 150, 2.242)])
def test_cavity_fd_table2(lb, Ra, Lc, nu_paper):
    """Table II, finite-difference column."""
    P, Cv = O.cavity_setup(Ra, Lc)
    with gpu_fd_cavity(lb, P, Cv, "fp64") as L:
        prev, steps = None, 0
        while steps < 600000:
            L.step(20000)
            steps += 20000
            rho, _, _, T = L.moments()
            nu = O.nusselt_hot_wall(P, Cv, T)
            if prev is not None and abs(nu - prev) < 2e-5 * abs(nu):
                break
            prev = nu
    nu_f = O.nusselt_hot_wall(P, Cv, T, rho)
    print(f"Ra={Ra:g} L={Lc}: FD Nu(wall gradient)={nu:.4f} Nu(wall flux)={nu_f:.4f} "
          f"Nu(3-point)={O.nusselt_hot(P, Cv, T):.4f} after {steps} steps")
    # the conductive wall flux lambda(rho) dT/dx, as the LB energy flux through
    # the wall links: Table II's FD column to 0.1%; the bare wall gradient
    # (like the LB gradient Nusselt number) within 3%
    assert nu_f == pytest.approx(nu_paper, rel=0.01)
    assert nu == pytest.approx(nu_paper, rel=0.03)
