"""Thermal flow between parallel plates (Sec. III A) on the GPU: FP64 bit for
bit with the oracle's channel step (plates, inlet, outlet; both temperature
treatments; Cases A and B), and Table I on the paper's 500 x 60 lattice."""
import numpy as np
import pytest

import oracle as O


@pytest.fixture(scope="module")
def lb():
    from paper_1405_2232_gb300 import lb as _lb
    _lb.load()
    return _lb


def gpu_channel(lb, P, Ch, prec):
    return lb.Lattice(np.ones((P.ny, P.nx)), np.ones((P.ny, P.nx)), nx=P.nx, ny=P.ny, precision=prec,
                      tau_f=P.tau_f, tau_g=P.tau_g, G=P.G, beta=P.beta, eos=lb.LB_EOS_IDEAL, a=0.0, b=0.0,
                      R=P.R, cv=P.cv, thermal=P.thermal, psi_uses_local_T=1, walls=lb.LB_WALLS_CHANNEL,
                      adiabatic_bottom=Ch.adiabatic_bottom, T_in=Ch.T_in, T_w=Ch.T_w, U_in=Ch.U_in)


@pytest.mark.gpu
@pytest.mark.parametrize("thermal", [O.THERMAL_EQ24, O.THERMAL_EQ7])
@pytest.mark.parametrize("case,nx,ny", [("A", 64, 24), ("B", 77, 19)])
def test_channel_fp64_bit_identical(lb, thermal, case, nx, ny):
    P, Ch = O.channel_setup(nx, ny, case, thermal=thermal)
    f0, g0 = O.init_equilibrium(P, np.ones((ny, nx)), np.ones((ny, nx)))
    f_ref, g_ref, _ = O.step_channel(P, Ch, f0, g0, n=300, threads=8, check=False)
    with gpu_channel(lb, P, Ch, "fp64") as L:
        L.step(300)
        f, g = L.populations()
    assert np.array_equal(f, f_ref) and np.array_equal(g, g_ref)


@pytest.mark.gpu
def test_channel_fp32_within_rounding(lb):
    P, Ch = O.channel_setup(96, 24, "A")
    f0, g0 = O.init_equilibrium(P, np.ones((24, 96)), np.ones((24, 96)))
    f_ref, g_ref, _ = O.step_channel(P, Ch, f0, g0, n=2000, threads=8)
    r_ref, ux_ref, _, T_ref, _, _ = O.moments(P, f_ref, g_ref)
    with gpu_channel(lb, P, Ch, "fp32") as L:
        L.step(2000)
        r, ux, uy, T = L.moments()
    assert np.abs(r - r_ref).max() < 2e-5 and np.abs(T - T_ref).max() < 2e-5
    # (the oracle's moments take the periodic force, so u is compared off the
    # inlet and outlet columns)
    assert np.abs(ux - ux_ref)[:, 1:-1].max() < 1e-4 * np.abs(ux_ref).max()


TABLE_I = {"A": (7.51, 7.54), "B": (4.91, 4.86)}  # (corrected LB Eq. (24), analytical [28])


@pytest.mark.gpu
@pytest.mark.parametrize("case", ["A", "B"])
def test_channel_table1(lb, case):
    """Table I: thermally fully developed Nusselt numbers on 500 x 60."""
    P, Ch = O.channel_setup(500, 60, case)
    with gpu_channel(lb, P, Ch, "fp64") as L:
        prev, steps = None, 0
        while steps < 300000:
            L.step(20000)
            steps += 20000
            f, g = L.populations()
            rho, ux, uy, T = L.moments()
            nus = np.array([O.channel_nusselt(P, Ch, g, rho, ux, T, x) for x in range(300, 401, 25)])
            if prev is not None and np.abs(nus - prev).max() < 1e-4 * nus.mean():
                break
            prev = nus
    grads = [O.channel_nusselt_grad(P, Ch, rho, ux, T, x) for x in range(300, 401, 25)]
    print(f"case {case}: Nu(x = 300..400) = {np.round(nus, 3)} (gradient {np.round(grads, 3)}) after {steps} steps")
    lb_paper, analytical = TABLE_I[case]
    assert np.ptp(nus) < 0.01 * nus.mean()
    assert nus.mean() == pytest.approx(analytical, rel=0.02)
    assert nus.mean() == pytest.approx(lb_paper, rel=0.02)
    # Eq. (7) deviates (the forcing-term effect): report it, and check it differs
    P7, Ch7 = O.channel_setup(500, 60, case, thermal=O.THERMAL_EQ7)
    with gpu_channel(lb, P7, Ch7, "fp64") as L:
        L.step(steps)
        f, g = L.populations()
        rho, ux, uy, T = L.moments()
    nus7 = [O.channel_nusselt(P7, Ch7, g, rho, ux, T, x) for x in range(300, 401, 25)]
    grads7 = [O.channel_nusselt_grad(P7, Ch7, rho, ux, T, x) for x in range(300, 401, 25)]
    print(f"case {case}: Eq.7 Nu(x) = {np.round(nus7, 3)} (gradient {np.round(grads7, 3)})")
    assert abs(np.mean(nus7) - nus.mean()) > 0.2 * nus.mean()


def gpu_fd_channel(lb, P, Ch, prec, printed=False):
    thermal = lb.LB_THERMAL_FD26_PRINTED if printed else lb.LB_THERMAL_FD26
    return lb.Lattice(np.ones((P.ny, P.nx)), np.ones((P.ny, P.nx)), nx=P.nx, ny=P.ny, precision=prec,
                      tau_f=P.tau_f, tau_g=P.tau_g, G=P.G, beta=P.beta, eos=lb.LB_EOS_IDEAL, a=0.0, b=0.0,
                      R=P.R, cv=P.cv, thermal=thermal, psi_uses_local_T=1, walls=lb.LB_WALLS_CHANNEL,
                      adiabatic_bottom=Ch.adiabatic_bottom, T_in=Ch.T_in, T_w=Ch.T_w, U_in=Ch.U_in)


@pytest.mark.gpu
@pytest.mark.parametrize("printed", [False, True])
@pytest.mark.parametrize("case,nx,ny", [("A", 64, 24), ("B", 77, 19)])
def test_channel_fd_fp64_bit_identical(lb, printed, case, nx, ny):
    P, Ch = O.channel_setup(nx, ny, case)
    f0, _ = O.init_equilibrium(P, np.ones((ny, nx)), np.ones((ny, nx)))
    f, T, st, _ = O.step_fd_channel(P, Ch, f0, np.ones((ny, nx)), n=200, printed=printed, threads=8)
    _, _, _, (r, ux, uy) = O.step_fd_channel(P, Ch, f, T, n=1, printed=printed, check=False)
    with gpu_fd_channel(lb, P, Ch, "fp64", printed) as L:
        L.step(200)
        gr, gux, guy, gT = L.moments()
    assert np.array_equal(gr, r) and np.array_equal(gT, T)
    assert np.abs(gux - ux).max() <= 1e-14 and np.abs(guy - uy).max() <= 1e-14


@pytest.mark.gpu
@pytest.mark.parametrize("case", ["A", "B"])
def test_channel_fd_table1(lb, case):
    """Table I, finite-difference column, on 500 x 60."""
    P, Ch = O.channel_setup(500, 60, case)
    with gpu_fd_channel(lb, P, Ch, "fp64") as L:
        prev, steps = None, 0
        while steps < 300000:
            L.step(20000)
            steps += 20000
            rho, ux, uy, T = L.moments()
            nus = np.array([O.channel_nusselt_wall(P, Ch, rho, ux, T, x) for x in range(300, 401, 25)])
            if prev is not None and np.abs(nus - prev).max() < 1e-4 * nus.mean():
                break
            prev = nus
    print(f"case {case}: FD Nu(x = 300..400) = {np.round(nus, 3)} after {steps} steps")
    fd_paper = {"A": 7.51, "B": 4.91}[case]
    analytical = TABLE_I[case][1]
    assert np.ptp(nus) < 0.01 * nus.mean()
    assert nus.mean() == pytest.approx(analytical, rel=0.02)
    # (Case B: the paper's FD value sits 1% above the analytical one, ours 1% below)
    assert nus.mean() == pytest.approx(fd_paper, rel=0.025)
