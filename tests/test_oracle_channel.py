"""The oracle's plate channel (Sec. III A) pinned to what the paper and the
mathematics fix: a uniform state at rest (inlet, outlet and plates at one
temperature, no inflow) stays put; with inflow and no heating the fully
developed flow is plane Poiseuille flow carrying the inlet flux; with the
plates cooling the flow the thermally fully developed Nusselt numbers are the
analytical 7.54 (Case A, both plates at T_w) and 4.86 (Case B, lower plate
adiabatic) quoted with Table I (the paper's corrected LB gives 7.51, 4.91)."""
import numpy as np
import pytest

import oracle as O

NU_ANALYTICAL = {"A": 7.54, "B": 4.86}  # Table I, analytical [28]


def _start(P):
    return O.init_equilibrium(P, np.ones((P.ny, P.nx)), np.ones((P.ny, P.nx)))


def test_uniform_state_at_rest_is_steady():
    P, Ch = O.channel_setup(24, 10, "A", T_in=1.0, T_w=1.0, U_in=0.0)
    f0, g0 = _start(P)
    f, g, st = O.step_channel(P, Ch, f0, g0, n=50)
    assert st == O.OK
    assert np.abs(f - f0).max() < 1e-15 and np.abs(g - g0).max() < 1e-15


def test_isothermal_inflow_is_poiseuille():
    P, Ch = O.channel_setup(120, 20, "A", T_in=1.0, T_w=1.0)
    f, g = _start(P)
    f, g, _ = O.step_channel(P, Ch, f, g, n=12000, threads=8)
    rho, ux, uy, T, _, _ = O.moments(P, f, g)
    col = ux[:, 80]
    H = P.ny
    y = np.arange(H) + 0.5                  # distance from the lower plate (halfway walls)
    mean = col.mean()
    parab = 6.0 * mean * y * (H - y) / H**2
    assert np.abs(col - parab).max() < 0.02 * col.max()
    assert (rho[:, 80] * ux[:, 80]).sum() == pytest.approx(H * Ch.U_in * rho[:, 0].mean(), rel=0.03)
    assert np.abs(uy[:, 80]).max() < 1e-3 * Ch.U_in


@pytest.mark.parametrize("case", ["A", "B"])
def test_table1_fully_developed_nusselt(case):
    P, Ch = O.channel_setup(250, 30, case)
    f, g = _start(P)
    f, g, _ = O.step_channel(P, Ch, f, g, n=20000, threads=8)
    rho, ux, uy, T, _, _ = O.moments(P, f, g)
    nus = [O.channel_nusselt(P, Ch, g, rho, ux, T, x) for x in range(100, 201, 20)]
    assert np.ptp(nus) < 0.02 * np.mean(nus)              # fully developed: flat in x
    assert np.mean(nus) == pytest.approx(NU_ANALYTICAL[case], rel=0.04), nus


@pytest.mark.parametrize("case", ["A", "B"])
def test_fd_table1_fully_developed_nusselt(case):
    """The hybrid scheme (Eqs. 26-27) in the channel (ghosts reflected about
    the plate and inlet temperatures): Table I's FD column (7.51, 4.91) and
    the analytical values, on 150 x 20."""
    P, Ch = O.channel_setup(150, 20, case)
    f, _ = _start(P)
    T = np.ones((P.ny, P.nx))
    f, T, st, _ = O.step_fd_channel(P, Ch, f, T, n=10000, threads=8)
    assert st == O.OK
    _, _, _, (rho, ux, uy) = O.step_fd_channel(P, Ch, f, T, n=1, check=False)
    nus = [O.channel_nusselt_wall(P, Ch, rho, ux, T, x) for x in range(60, 121, 15)]
    assert np.ptp(nus) < 0.01 * np.mean(nus)
    assert np.mean(nus) == pytest.approx(NU_ANALYTICAL[case], rel=0.02), nus


def test_eq7_lateral_conduction_vanishes():
    """Why Eq. (7) under-reads the plate channel (Sec. III A; the paper's
    Fig. 1 has it high).  Eq. (23): Eq. (7) solves the temperature equation
    with the flux lambda grad T + vartheta T F, vartheta = lambda / p,
    p = rho c_s^2, so across the channel lambda_eff,y = lambda (1 + c) with
    c = T F_y / (p dT/dy).  With the ideal EOS the pseudopotential force is
    F = -grad(rho R T - rho c_s^2) (the text after Eq. 4), and a developed
    channel flow is in lateral balance of the total pressure rho R T, so
    F_y = c_s^2 d rho/dy = -c_s^2 rho (dT/dy) / T and c = -1: heat is not
    conducted across the flow at all.  Checked on the developed state of both
    treatments (the momentum balance does not depend on the thermal
    equation), and the consequence for Eq. (7): a plate Nusselt number far
    below Eq. (24)'s."""
    import os
    nx, ny = 120, 20
    out = {}
    for th in (O.THERMAL_EQ7, O.THERMAL_EQ24):
        P, Ch = O.channel_setup(nx, ny, "A", thermal=th)
        f, g = O.init_equilibrium(P, np.ones((ny, nx)), np.ones((ny, nx)))
        f, g, _ = O.step_channel(P, Ch, f, g, n=20000, threads=os.cpu_count() or 1)
        rho, ux, uy, T, Fx, Fy = O.moments(P, f, g)
        dT = 0.5 * (T[2:, :] - T[:-2, :])  # d/dy at rows 1 .. ny - 2
        c = T[1:-1, :] * Fy[1:-1, :] / (rho[1:-1, :] * (1.0 / 3.0) * dT)  # p = rho c_s^2, c_s^2 = 1/3
        # interior rows with a clear gradient, away from the plates (the
        # moment routine's force is periodic, the channel's clamped) and from
        # the channel's centre line (dT/dy = 0), in the developed half
        rows = [r - 1 for r in (2, 3, 4, 5, ny - 6, ny - 5, ny - 4, ny - 3)]
        sel = c[rows][:, nx // 2: 3 * nx // 4]
        assert np.abs(sel + 1.0).max() < 0.01, sel
        out[th] = O.channel_nusselt_grad(P, Ch, rho, ux, T, nx // 2)
    assert out[O.THERMAL_EQ7] < 0.2 * out[O.THERMAL_EQ24], out
