"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

Nothing here compares the oracle with itself: each test checks a moment
identity, a closed form, a published constant, a textbook decay rate, an
exact invariant, or a Chapman-Enskog prediction of the paper (Eq. 23 and
Eq. A11).  A plausible slip in the oracle (a dropped term, a wrong sign or
index, a transposed operand, tau in place of 1/tau) fails at least one.
"""
import numpy as np
import pytest

import oracle as O
from paper_1405_2232_gb300 import inputs as I

# D2Q9 velocities in the numbering of the oracle (reading of Sec. II A)
E = np.array([[0, 0], [1, 0], [0, 1], [-1, 0], [0, -1], [1, 1], [-1, 1], [-1, -1], [1, -1]],
             dtype=np.float64)
CS2 = 1.0 / 3.0


def moments_of(p):
    m0 = p.sum()
    m1 = E.T @ p
    m2 = np.einsum("ia,ib,i->ab", E, E, p)
    return m0, m1, m2


# --------------------------------------------------------------------- #
# Equilibrium, forcing term and correction term: exact moment identities
# --------------------------------------------------------------------- #
@pytest.mark.parametrize("rho,ux,uy", [(1.0, 0.0, 0.0), (0.35, 0.03, -0.07), (0.03, -0.1, 0.05)])
def test_feq_moments(rho, ux, uy):
    """Sec. II A: f^eq carries rho, rho u and rho cs^2 I + rho u u."""
    m0, m1, m2 = moments_of(O.feq(rho, ux, uy))
    u = np.array([ux, uy])
    assert m0 == pytest.approx(rho, rel=1e-15)
    np.testing.assert_allclose(m1, rho * u, rtol=0, atol=1e-16)
    np.testing.assert_allclose(m2, rho * CS2 * np.eye(2) + rho * np.outer(u, u), rtol=0,
                               atol=2e-16)


@pytest.mark.parametrize("tau", [0.6, 1.0, 1.7])
def test_forcing_term_moments(tau):
    """Eq. (1) forcing term (scheme of Ref. [21]): sum F_i = 0,
    sum e_i F_i = (1 - 1/(2 tau)) F, sum e_i e_i F_i = (1 - 1/(2 tau)) (uF + Fu)."""
    u = np.array([0.04, -0.02])
    F = np.array([1.3e-3, 2.1e-3])
    m0, m1, m2 = moments_of(O.forcing_term(tau, u[0], u[1], F[0], F[1]))
    pre = 1.0 - 1.0 / (2.0 * tau)
    assert abs(m0) < 1e-18
    np.testing.assert_allclose(m1, pre * F, rtol=1e-14, atol=0)
    np.testing.assert_allclose(m2, pre * (np.outer(u, F) + np.outer(F, u)), rtol=0, atol=1e-18)


@pytest.mark.parametrize("tau_g,cv,T", [(0.8, 1.0, 0.08), (1.3, 2.0, 1.0)])
def test_correction_term_identities(tau_g, cv, T):
    """Eq. (25) and the identities printed after it: sum C_i = 0,
    sum e_i C_i = (1 - 0.5/tau_g) c_v T F, sum e_i e_i C_i = 0."""
    F = np.array([-3.0e-3, 1.7e-3])
    m0, m1, m2 = moments_of(O.correction_term(tau_g, cv, T, F[0], F[1]))
    assert abs(m0) < 1e-18
    np.testing.assert_allclose(m1, (1.0 - 0.5 / tau_g) * cv * T * F, rtol=1e-14)
    np.testing.assert_allclose(m2, np.zeros((2, 2)), atol=1e-19)


# --------------------------------------------------------------------- #
# Equations of state
# --------------------------------------------------------------------- #
def test_vdw_critical_point_closed_form():
    """vdW EOS of Sec. III: T_c = 8a/(27 b R), rho_c = 1/(3b)."""
    a, b, R = 9.0 / 49.0, 2.0 / 21.0, 1.0
    P = O.params(8, 8, eos=O.EOS_VDW, a=a, b=b, R=R)
    Tc, rhoc = O.critical_point(P)
    assert Tc == pytest.approx(8 * a / (27 * b * R), rel=1e-9)
    assert rhoc == pytest.approx(1.0 / (3.0 * b), rel=1e-4)
    assert O.p_eos(P, 1.0 / (3 * b), 8 * a / (27 * b * R)) == pytest.approx(a / (27 * b * b),
                                                                             rel=1e-12)


def test_cs_critical_point_published():
    """Carnahan-Starling critical point, T_c = 0.3773 a/(bR), rho_c = 0.5218/(b/4)/4
    (the constants published with the CS pseudopotential EOS), and the constant the
    input recipes use."""
    P = O.params(8, 8, eos=O.EOS_CS, a=1.0, b=4.0, R=1.0)
    Tc, rhoc = O.critical_point(P)
    assert Tc == pytest.approx(0.3773 / 4.0, rel=2e-4)
    assert rhoc == pytest.approx(0.5218 / 4.0, rel=2e-4)
    assert I.CS_TC == pytest.approx(Tc, rel=1e-9)
    assert I.CS_RHOC == pytest.approx(rhoc, rel=1e-4)


def test_cs_virial_coefficients():
    """Hard-sphere part of CS: Z = 1 + 4 eta + 10 eta^2 + 18 eta^3 + 28 eta^4 + ...
    (B_n = n^2 + n - 2), a pin independent of how the EOS is coded."""
    P = O.params(8, 8, eos=O.EOS_CS, a=0.0, b=4.0, R=1.0)
    T = 0.7
    for eta in (1e-2, 5e-3):
        rho = 4.0 * eta / 4.0  # eta = b rho / 4 with b = 4
        Z = O.p_eos(P, rho, T) / (rho * T)
        c4 = (Z - 1 - 4 * eta - 10 * eta ** 2 - 18 * eta ** 3) / eta ** 4
        assert c4 == pytest.approx(28.0, rel=0.05)


def test_vdw_and_ideal_low_density_limits():
    P = O.params(8, 8, eos=O.EOS_VDW, a=0.0, b=0.5, R=2.0)
    rho, T = 1e-3, 0.3
    Z = O.p_eos(P, rho, T) / (rho * 2.0 * T)
    assert (Z - 1.0) / rho == pytest.approx(0.5, rel=1e-3)  # second virial coefficient b
    Pi = O.params(8, 8, eos=O.EOS_IDEAL, R=0.25)
    assert O.p_eos(Pi, 2.0, 3.0) == 1.5
    # psi^2 = 2 (p - rho cs^2) / G  (Sec. II A); sign follows G
    assert O.psi_sq(Pi, 3.0, 1.0) == pytest.approx(2 * (0.75 - 1.0) / -1.0, rel=1e-15)


# --------------------------------------------------------------------- #
# Force stencil, Eqs. (2)-(4)
# --------------------------------------------------------------------- #
def _force(P, rho, T):
    f, g = O.init_equilibrium(P, rho, T)
    m = O.moments(P, f, g)
    return m[4], m[5]


@pytest.mark.parametrize("axis", [0, 1])
def test_force_closed_form_beta0(axis):
    """Eq. (4) with beta = 0 on rho = rho0 (1 + eps sin kx), ideal EOS (Sec. III):
    F_x = -(RT - cs^2) rho0 eps sin(k) cos(kx), and F_y = 0 exactly."""
    L, rho0, eps, R, T0 = 48, 0.7, 0.02, 0.9, 1.0
    nx, ny = (L, 5) if axis == 0 else (5, L)
    P = O.params(nx, ny, G=1.0, beta=0.0, eos=O.EOS_IDEAL, R=R)
    rho, T = I.sinusoid_fields(nx, ny, rho0, T0, eps, mode=2, axis=axis)
    Fx, Fy = _force(P, rho, T)
    k = 2 * np.pi * 2 / L
    ref = -(R * T0 - CS2) * rho0 * eps * np.sin(k) * np.cos(k * np.arange(L))
    if axis == 0:
        np.testing.assert_allclose(Fx, ref[None, :] * np.ones((ny, 1)), atol=1e-15)
        assert np.all(Fy == 0.0)
    else:
        np.testing.assert_allclose(Fy, ref[:, None] * np.ones((1, nx)), atol=1e-15)
        assert np.all(Fx == 0.0)


def test_force_closed_form_diagonal():
    """Diagonal pattern rho = rho0 (1 + eps sin k(x+y)) tests w(2) = 1/12:
    F_x = F_y = -(RT - cs^2) rho0 eps cos(phi) [(2/3) sin k + (1/6) sin 2k]."""
    L, rho0, eps, R, T0 = 32, 0.5, 0.01, 0.8, 1.0
    P = O.params(L, L, G=1.0, beta=0.0, eos=O.EOS_IDEAL, R=R)
    y, x = np.mgrid[0:L, 0:L]
    k = 2 * np.pi / L
    rho = rho0 * (1 + eps * np.sin(k * (x + y)))
    T = np.full((L, L), T0)
    Fx, Fy = _force(P, np.ascontiguousarray(rho), T)
    ref = -(R * T0 - CS2) * rho0 * eps * np.cos(k * (x + y)) * (2 / 3 * np.sin(k) + np.sin(2 * k) / 6)
    np.testing.assert_allclose(Fx, ref, atol=1e-15)
    np.testing.assert_allclose(Fy, ref, atol=1e-15)


def test_force_taylor_limit_eq3():
    """Eq. (3): the Eq. (2) force minus -G[grad(psi^2)/2 + psi grad(lap psi)/6] is
    O(k^5): the gap falls 32x each time the wavelength doubles."""
    sp = pytest.importorskip("sympy")
    xs = sp.symbols("x")
    errs = []
    for L in (16, 32, 64):
        k = 2 * sp.pi / L
        psi = sp.sqrt((1 + sp.Rational(1, 20) * sp.sin(k * xs)) / 3)
        Fx_s = -(sp.Rational(1, 2) * sp.diff(psi ** 2, xs) + sp.Rational(1, 6) * psi * sp.diff(psi, xs, 3))
        ref = sp.lambdify(xs, Fx_s, "numpy")(np.arange(L, dtype=float))
        # ideal EOS, G = 1, R T = 1/2: psi^2 = 2 rho (1/2 - 1/3) = rho/3
        P = O.params(L, 3, G=1.0, beta=1.0, eos=O.EOS_IDEAL, R=0.5)
        rho, T = I.sinusoid_fields(L, 3, 1.0, 1.0, 0.05)
        Fx, _ = _force(P, rho, T)
        errs.append(np.abs(Fx[1] - ref).max())
    assert errs[0] / errs[1] == pytest.approx(32.0, rel=0.05)
    assert errs[1] / errs[2] == pytest.approx(32.0, rel=0.05)


def test_mixed_force_linear_in_beta():
    """Eq. (4) is linear in beta between Eq. (2) (beta = 1) and the psi^2 form (beta = 0)."""
    L = 24
    rho, T = I.sinusoid_fields(L, L, 0.9, 1.0, 0.1, mode=1, axis=0)
    rho = np.ascontiguousarray(rho + 0.05 * np.sin(2 * np.pi * np.arange(L) / L)[:, None])
    F = {}
    for beta in (0.0, 0.3, 1.0):
        P = O.params(L, L, G=1.0, beta=beta, eos=O.EOS_IDEAL, R=0.6)
        F[beta] = _force(P, rho, T)
    for c in range(2):
        np.testing.assert_allclose(F[0.3][c], 0.7 * F[0.0][c] + 0.3 * F[1.0][c], atol=1e-16)
    # Eq. (2)/(4) both approximate -grad(p_EOS - rho cs^2) (Sec. II A)
    assert np.abs(F[1.0][0] - F[0.0][0]).max() < 0.02 * np.abs(F[0.0][0]).max()


# --------------------------------------------------------------------- #
# Whole step: invariants
# --------------------------------------------------------------------- #
def c1_params(thermal=O.THERMAL_EQ24, **kw):
    return O.params(64, 64, tau_f=1.0, tau_g=0.8, G=-1.0, beta=1.0, eos=O.EOS_CS, a=1.0,
                    b=4.0, R=1.0, thermal=thermal, **kw)


def test_uniform_state_stays_uniform():
    """Uniform rho, T, u = 0: F vanishes exactly (pair differences are 0) and every
    site stays bitwise equal to every other; rho and T move by rounding only."""
    P = O.params(16, 12, thermal=O.THERMAL_EQ7)
    rho, T = I.uniform_fields(16, 12, 0.2, 0.8 * I.CS_TC)
    f, g = O.init_equilibrium(P, rho, T)
    f2, g2, _ = O.step(P, f, g, n=50)
    for p in (f2, g2):
        assert np.all(p == p[:, :1, :1])
    r, ux, uy, T2, Fx, Fy = O.moments(P, f2, g2)
    assert np.all(Fx == 0) and np.all(Fy == 0) and np.all(ux == 0) and np.all(uy == 0)
    assert np.abs(r - 0.2).max() < 1e-15 and np.abs(T2 / T - 1).max() < 1e-14


@pytest.mark.parametrize("thermal", [O.THERMAL_EQ7, O.THERMAL_EQ24])
def test_conservation(thermal):
    """Eq. (13)/(A5) and sum C_i = 0: mass sum f, energy sum g and (periodic,
    pair-antisymmetric force) momentum are conserved up to rounding."""
    P = c1_params(thermal, psi_uses_local_T=0, T_psi=0.85 * I.CS_TC)
    rho, T = I.slab_fields(64, 64)
    f, g = O.init_equilibrium(P, rho, T)
    t0 = O.totals(P, f, g)
    f2, g2, _ = O.step(P, f, g, n=200)
    t1 = O.totals(P, f2, g2)
    assert abs(t1[0] / t0[0] - 1) < 1e-13
    assert abs(t1[1] / t0[1] - 1) < 1e-13
    assert abs(t1[2]) < 1e-13 * t0[0] and abs(t1[3]) < 1e-13 * t0[0]


def test_translation_invariance():
    """Shifting the initial field periodically shifts the result bit for bit."""
    P = c1_params()
    rho, T = I.slab_fields(64, 64)
    f, g = O.init_equilibrium(P, rho, T)
    fa, ga, _ = O.step(P, f, g, n=30)
    sh = (5, -7)
    fb, gb, _ = O.step(P, np.roll(f, sh, axis=(1, 2)), np.roll(g, sh, axis=(1, 2)), n=30)
    assert np.array_equal(np.roll(fa, sh, axis=(1, 2)), fb)
    assert np.array_equal(np.roll(ga, sh, axis=(1, 2)), gb)


def test_G_drops_out():
    """With psi from the EOS, G psi(x) psi(y) = -2 sqrt(A_x A_y) for G < 0: the force,
    hence the whole run, does not depend on G (to rounding)."""
    rho, T = I.slab_fields(64, 64)
    out = []
    for G in (-1.0, -2.5):
        P = O.params(64, 64, G=G, thermal=O.THERMAL_EQ24)
        f, g = O.init_equilibrium(P, rho, T)
        f2, g2, _ = O.step(P, f, g, n=40)
        out.append(O.moments(P, f2, g2))
    # rounding differences grow in the violent start-up transient; a force that
    # depended on G would differ at O(1)
    for a, b in zip(out[0][:4], out[1][:4]):
        np.testing.assert_allclose(a, b, rtol=0, atol=1e-8 * np.abs(a).max())


def test_cv_scaling_exact():
    """g, g^eq and C_i all scale with c_v, so c_v = 2 gives bit-identical T and f."""
    rho, T = I.slab_fields(64, 64)
    out = []
    for cv in (1.0, 2.0):
        P = O.params(64, 64, cv=cv, thermal=O.THERMAL_EQ24)
        f, g = O.init_equilibrium(P, rho, T)
        f2, g2, _ = O.step(P, f, g, n=40)
        out.append((f2, g2, O.moments(P, f2, g2)[3]))
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(2.0 * out[0][1], out[1][1])
    assert np.array_equal(out[0][2], out[1][2])


# --------------------------------------------------------------------- #
# Textbook LB behaviour with the force switched off (R T = cs^2 exactly)
# --------------------------------------------------------------------- #
def _force_free(L, tau_f, tau_g):
    return O.params(L, 3, tau_f=tau_f, tau_g=tau_g, G=1.0, beta=0.0, eos=O.EOS_IDEAL, R=1.0,
                    psi_uses_local_T=0, T_psi=1.0 / 3.0)


def test_shear_wave_decay_viscosity():
    """BGK of Eq. (1): a shear wave decays as exp(-nu k^2 t), nu = (tau_f - 1/2) cs^2."""
    L, tau, U, n = 64, 0.8, 1e-3, 200
    P = _force_free(L, tau, 0.7)
    k = 2 * np.pi / L
    f = np.zeros((9, 3, L))
    for x in range(L):
        f[:, :, x] = O.feq(1.0, 0.0, U * np.sin(k * x))[:, None]
    f2, g2, _ = O.step(P, f, f.copy(), n=n)
    uy = O.moments(P, f2, g2)[2][1]
    amp = 2.0 / L * np.sum(uy * np.sin(k * np.arange(L)))
    assert amp / U == pytest.approx(np.exp(-(tau - 0.5) / 3 * k * k * n), rel=2e-3)


def test_thermal_diffusion_decay():
    """Eq. (7) at rest: a temperature wave decays as exp(-kappa k^2 t) with
    kappa = lambda/(rho c_v) = (tau_g - 1/2) cs^2 (Eq. 23 with F = 0)."""
    L, tau_g, dT, n = 64, 0.9, 1e-3, 200
    P = _force_free(L, 1.0, tau_g)
    k = 2 * np.pi / L
    T = 1.0 + dT * np.sin(k * np.arange(L))[None, :] * np.ones((3, 1))
    f, g = O.init_equilibrium(P, np.ones((3, L)), np.ascontiguousarray(T))
    f2, g2, _ = O.step(P, f, g, n=n)
    Tn = O.moments(P, f2, g2)[3][1]
    amp = 2.0 / L * np.sum((Tn - 1.0) * np.sin(k * np.arange(L)))
    assert amp / dT == pytest.approx(np.exp(-(tau_g - 0.5) / 3 * k * k * n), rel=2e-3)


def test_centre_of_mass_moves_with_momentum():
    """Streaming f_i(x + e_i) <- f*_i(x) moves the centre of mass by exactly the
    total post-collision momentum / mass each step (force-free: = sum e_i f_i)."""
    L = 64
    P = O.params(L, L, G=1.0, beta=0.0, eos=O.EOS_IDEAL, R=1.0, psi_uses_local_T=0,
                 T_psi=1.0 / 3.0)
    y, x = np.mgrid[0:L, 0:L]
    bump = np.exp(-((x - 32) ** 2 + (y - 30) ** 2) / 20.0)
    rho = 1.0 + 0.5 * bump
    f = np.zeros((9, L, L))
    # the velocity is confined to the bump, so nothing crosses the periodic seam
    for yy in range(L):
        for xx in range(L):
            f[:, yy, xx] = O.feq(rho[yy, xx], 0.05 * bump[yy, xx], -0.03 * bump[yy, xx])
    g = f.copy()
    for _ in range(3):
        mass = f.sum()
        cx, cy = (f.sum(0) * x).sum() / mass, (f.sum(0) * y).sum() / mass
        px = (E[:, 0, None, None] * f).sum()
        py = (E[:, 1, None, None] * f).sum()
        f, g, _ = O.step(P, f, g, n=1)
        cx2, cy2 = (f.sum(0) * x).sum() / mass, (f.sum(0) * y).sum() / mass
        assert cx2 - cx == pytest.approx(px / mass, rel=1e-10)
        assert cy2 - cy == pytest.approx(py / mass, rel=1e-10)


# --------------------------------------------------------------------- #
# Chapman-Enskog predictions of the paper
# --------------------------------------------------------------------- #
def _ce_setup(thermal):
    L, T0, R = 128, 1.0, 0.5
    P = O.params(L, 3, tau_f=1.0, tau_g=0.8, G=1.0, beta=0.0, eos=O.EOS_IDEAL, R=R,
                 thermal=thermal)
    rho, T = I.sinusoid_fields(L, 3, 1.0, T0, 1e-3)
    f, g = O.init_equilibrium(P, rho, T)
    f, g, _ = O.step(P, f, g, n=10)
    rho, ux, uy, T, Fx, Fy = O.moments(P, f, g)
    f2, g2, _ = O.step(P, f, g, n=1)
    T2 = O.moments(P, f2, g2)[3]
    dTdt = (T2 - T)[1]
    divF = ((np.roll(Fx, -1, 1) - np.roll(Fx, 1, 1)) / 2.0)[1]
    pred = (0.8 - 0.5) * T[1] * divF / rho[1]
    return dTdt, pred


def test_eq7_temperature_drift_matches_eq23():
    """Eq. (23): with Eq. (7) a uniform-T, non-uniform-rho state heats and cools at
    dT/dt = (tau_g - 1/2) T div(F) / rho (the div(theta T F) term, theta = lambda/p)."""
    dTdt, pred = _ce_setup(O.THERMAL_EQ7)
    assert np.abs(dTdt - pred).max() < 0.05 * np.abs(pred).max()


def test_eq24_removes_drift():
    """Eq. (24)/(A11): the corrected equation has no such drift (>= 30x smaller)."""
    dTdt, pred = _ce_setup(O.THERMAL_EQ24)
    assert np.abs(dTdt).max() < np.abs(pred).max() / 30.0


def _slab_steady(thermal):
    nx, ny = 64, 4
    T0 = 0.85 * I.CS_TC
    rho0, Tf = I.slab_fields(nx, ny, noise=0.0)
    P = O.params(nx, ny, thermal=thermal, psi_uses_local_T=0, T_psi=T0)
    f, g = O.init_equilibrium(P, rho0, Tf)
    f, g, _ = O.step(P, f, g, n=12000)
    rho, ux, uy, T, Fx, Fy = O.moments(P, f, g)
    return rho0, Tf, rho, T


def test_eq7_steady_state_rhoT_uniform():
    """Eq. (23) at rest with F = grad(rho cs^2): the flux theta (p grad T + T F) =
    theta grad(pT) vanishes only if rho T is uniform: T follows 1/rho across the slab."""
    rho0, T0, rho, T = _slab_steady(O.THERMAL_EQ7)
    rT = rho * T
    assert (rT.max() - rT.min()) / rT.mean() < 0.01
    assert rT.mean() == pytest.approx((rho0 * T0).sum() / rho0.size, rel=0.01)
    assert T.max() / T.min() > 5.0  # far from uniform temperature


def test_eq24_steady_state_T_uniform():
    """Eq. (A11) at rest: lambda grad T = 0, so T is uniform and equals
    sum(rho T)_0 / sum(rho_0) (energy conservation)."""
    rho0, T0, rho, T = _slab_steady(O.THERMAL_EQ24)
    assert (T.max() - T.min()) / T.mean() < 2e-3
    assert T.mean() == pytest.approx((rho0 * T0).sum() / rho0.sum(), rel=1e-3)
    assert rho.max() / rho.min() > 5.0  # two phases are present


def test_eq7_with_local_T_leaves_psi_domain():
    """With psi(rho, T) and Eq. (7), the spurious heating of the vapour drives
    p_EOS above rho cs^2 (psi^2 < 0 for G < 0) within tens of steps on the 64x64
    slab; Eq. (24) stays in the domain."""
    rho, T = I.slab_fields(64, 64)
    P7 = c1_params(O.THERMAL_EQ7)
    f, g = O.init_equilibrium(P7, rho, T)
    f, g, st = O.step(P7, f, g, n=100, check=False)
    assert st == O.ERR_PSI_DOMAIN
    P24 = c1_params(O.THERMAL_EQ24)
    f, g = O.init_equilibrium(P24, rho, T)
    f, g, st = O.step(P24, f, g, n=100, check=False)
    assert st == O.OK


# --------------------------------------------------------------------- #
# Helpers used by the GPU parity checks
# --------------------------------------------------------------------- #
def test_step_sites_agrees_with_full_step():
    """The per-site recomputation used for sampled checks of big lattices gives the
    same values as the full step at every sampled site (incl. the periodic seams)."""
    P = O.params(20, 13, thermal=O.THERMAL_EQ24)
    rho, T = I.slab_fields(20, 13, width=8, noise=1e-2)
    f, g = O.init_equilibrium(P, rho, T)
    f, g, _ = O.step(P, f, g, n=5)
    f2, g2, _ = O.step(P, f, g, n=1)
    sites = np.array([0, 19, 20 * 12, 20 * 13 - 1, 137, 55])
    sf, sg = O.step_sites(P, f, g, sites)
    np.testing.assert_array_equal(sf, f2.reshape(9, -1)[:, sites].T)
    np.testing.assert_array_equal(sg, g2.reshape(9, -1)[:, sites].T)


def test_residual_closed_form():
    n = 100
    r0 = np.ones(n)
    r1 = np.ones(n) * 1.001
    T0 = np.full(n, 2.0)
    T1 = T0 + 1e-4
    r = O.residual(r0, T0, r1, T1, 10)
    assert r == pytest.approx(0.001 / 1.001 / 10, rel=1e-12)
