"""Pins of the finite-difference temperature treatment (Eqs. 26-27) in the oracle.

On Fourier modes the isotropic central stencils have closed-form eigenvalues
(gradient along an axis: i sin k; Laplacian of a mode along x: 2 (cos k - 1);
along the diagonal: (8 (cos k - 1) + (cos 2k - 1)) / 3), the two RK2 forms
have closed-form amplification factors (Heun 1 + z + z^2/2, the printed form
1 + z + z^2/4), and a uniform field is invariant.  A dropped term, a wrong
sign, a wrong weight or a transposed index fails one of these."""
import numpy as np
import pytest

import oracle as O
from paper_1405_2232_gb300 import inputs as I


def P(nx=32, ny=24, tau_g=0.9, **kw):
    return O.params(nx, ny, tau_f=1.0, tau_g=tau_g, G=-1.0, beta=1.0, eos=O.EOS_CS, a=1.0, b=4.0, R=1.0, **kw)


def grid(p):
    return np.meshgrid(np.arange(p.nx), np.arange(p.ny))


def test_uniform_temperature_is_steady():
    p = P()
    r = np.random.default_rng(1)
    T = np.full((p.ny, p.nx), 0.08)
    rho = 0.1 + r.random((p.ny, p.nx))
    ux, uy = r.standard_normal((2, p.ny, p.nx)) * 0.01
    assert np.all(O.fd_rhs(p, T, rho, ux, uy) == 0.0)
    assert np.array_equal(O.fd_rk2(p, T, rho, ux, uy), T)


@pytest.mark.parametrize("m", [1, 3, 7])
def test_laplacian_eigenvalue_along_x(m):
    p = P()
    X, Y = grid(p)
    k = 2 * np.pi * m / p.nx
    T = 0.08 + 1e-3 * np.cos(k * X)
    z = np.zeros_like(T)
    chi = (p.tau_g - 0.5) / 3.0
    K = O.fd_rhs(p, T, np.full_like(T, 0.2), z, z)
    assert np.allclose(K, chi * 2.0 * (np.cos(k) - 1.0) * 1e-3 * np.cos(k * X), rtol=0, atol=1e-16)


def test_laplacian_eigenvalue_along_diagonal():
    p = P(nx=24, ny=24)
    X, Y = grid(p)
    k = 2 * np.pi * 2 / 24
    T = 0.08 + 1e-3 * np.cos(k * (X + Y))
    z = np.zeros_like(T)
    chi = (p.tau_g - 0.5) / 3.0
    lam = (8.0 * (np.cos(k) - 1.0) + (np.cos(2 * k) - 1.0)) / 3.0
    K = O.fd_rhs(p, T, np.full_like(T, 0.2), z, z)
    assert np.allclose(K, chi * lam * 1e-3 * np.cos(k * (X + Y)), rtol=0, atol=1e-16)


def test_advection_uses_the_central_gradient():
    p = P()
    X, Y = grid(p)
    k = 2 * np.pi * 2 / p.ny
    T = 0.08 + 1e-3 * np.sin(k * Y)
    U = 0.05
    K_adv = O.fd_rhs(p, T, np.full_like(T, 0.2), np.zeros_like(T), np.full_like(T, U))
    chi = (p.tau_g - 0.5) / 3.0
    lam = 2.0 * (np.cos(k) - 1.0)
    expect = -U * 1e-3 * np.sin(k) * np.cos(k * Y) + chi * lam * 1e-3 * np.sin(k * Y)
    assert np.allclose(K_adv, expect, rtol=0, atol=1e-16)


def test_variable_conductivity_term():
    """chi grad rho . grad T / rho with rho and T modes along x."""
    p = P()
    X, Y = grid(p)
    q, k = 2 * np.pi * 1 / p.nx, 2 * np.pi * 2 / p.nx
    rho = 0.2 * (1 + 0.1 * np.sin(q * X))
    T = 0.08 + 1e-3 * np.sin(k * X)
    z = np.zeros_like(T)
    chi = (p.tau_g - 0.5) / 3.0
    grad_rho = 0.02 * np.sin(q) * np.cos(q * X)
    grad_T = 1e-3 * np.sin(k) * np.cos(k * X)
    lap_T = 2.0 * (np.cos(k) - 1.0) * 1e-3 * np.sin(k * X)
    expect = chi * (lap_T + grad_rho * grad_T / rho)
    assert np.allclose(O.fd_rhs(p, T, rho, z, z), expect, rtol=0, atol=1e-16)


@pytest.mark.parametrize("printed", [False, True])
def test_rk2_amplification(printed):
    p = P(tau_g=1.1)
    X, Y = grid(p)
    k = 2 * np.pi * 5 / p.nx
    T = 0.08 + 1e-3 * np.cos(k * X)
    z = np.zeros_like(T)
    zeta = (p.tau_g - 0.5) / 3.0 * 2.0 * (np.cos(k) - 1.0)
    G = 1 + zeta + zeta * zeta * (0.25 if printed else 0.5)
    Tn = O.fd_rk2(p, T, np.full_like(T, 0.2), z, z, printed=printed)
    assert np.allclose(Tn - 0.08, G * 1e-3 * np.cos(k * X), rtol=0, atol=5e-16)


def test_full_step_on_a_uniform_density():
    """Uniform rho (no force, u = 0): f stays at rest, a T mode decays by G per step."""
    p = P(nx=32, ny=8, tau_g=0.8, psi_uses_local_T=0, T_psi=0.85 * I.CS_TC)
    X, Y = grid(p)
    k = 2 * np.pi / p.nx
    rho0 = np.full((p.ny, p.nx), 0.2)
    T0 = 0.08 + 1e-3 * np.cos(k * X)
    f, _ = O.init_equilibrium(p, rho0, T0)
    f1, T1, st, (rho, ux, uy) = O.step_fd(p, f, T0, n=3)
    assert st == 0 and np.allclose(f1, f, rtol=0, atol=1e-16)
    zeta = (p.tau_g - 0.5) / 3.0 * 2.0 * (np.cos(k) - 1.0)
    G = 1 + zeta + 0.5 * zeta * zeta
    assert np.allclose(T1 - 0.08, G ** 3 * 1e-3 * np.cos(k * X), rtol=0, atol=1e-16)


def test_full_step_conserves_mass_and_matches_the_lb_f_update():
    """The f half of the FD step is the f half of the LB step with the same psi."""
    rho0, T0 = I.slab_fields(24, 20, width=10, rho_l=0.3, rho_g=0.04, noise=1e-3)
    # psi from a fixed T: the f update is the same arithmetic, bit for bit
    p = P(nx=24, ny=20, psi_uses_local_T=0, T_psi=0.085)
    f, g = O.init_equilibrium(p, rho0, T0)
    f_lb, _, _ = O.step(p, f, g, n=1, check=False)
    f_fd, T_fd, st, _ = O.step_fd(p, f, T0, n=1, check=False)
    assert np.array_equal(f_lb, f_fd)
    # psi from the local T: the LB recovers T = sum g / (rho c_v) up to rounding
    p = P(nx=24, ny=20, psi_uses_local_T=1)
    f_lb, _, _ = O.step(p, f, g, n=1, check=False)
    f_fd, _, _, _ = O.step_fd(p, f, T0, n=1, check=False)
    assert np.allclose(f_lb, f_fd, rtol=1e-13, atol=0)
    f5, T5, st, _ = O.step_fd(p, f, T0, n=20, check=False)
    assert f5.sum() == pytest.approx(f.sum(), rel=1e-13)
