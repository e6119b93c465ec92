"""Pins of the oracle's start at rest under the force (``init_balanced``).

The paper states no initial condition.  With the forcing scheme of Eq. (1)
the velocity of a state is u = (sum_i e_i f_i + F/2) / rho, so a state at
rest carries sum_i e_i f_i = -F/2; the start f = f^eq(rho0, -F/(2 rho0)),
g = c_v T0 f^eq(rho0, -F/(2 rho0)) is that state.  The pins below check it
against what that definition fixes, through the oracle's moment routine
(which recomputes rho, T and F from the populations): zero velocity, the
given rho0 and T0, the plain equilibrium where F = 0, and a smaller impulse
than the plain start from fields near a steady state.  CPU only.
"""
import numpy as np
import pytest

import oracle as O
from paper_1405_2232_gb300 import inputs as I


def _slab(nx, ny, T_over=0.75):
    rg, rl = I.coexistence_densities(T_over)
    rho, _ = I.slab_fields(nx, ny, width=2 * (nx // 5), rho_l=rl, rho_g=rg, noise=0.0)
    return rho, np.full((ny, nx), T_over * I.CS_TC)


def _droplet(nx, ny):
    rho, T = I.droplet_fields(nx, ny, min(nx, ny) / 4, rho_l=0.3, rho_g=0.05, T_lo=0.85, T_hi=0.9)
    return rho, T


CASES = [
    # (name, params kwargs, field builder)
    ("slab_mixed_beta_T_psi", dict(beta=1.3, psi_uses_local_T=0, T_psi=0.75 * I.CS_TC), lambda: _slab(37, 29)),
    ("droplet_beta1_local_T", dict(beta=1.0, psi_uses_local_T=1), lambda: _droplet(41, 33)),
    ("droplet_mixed_local_T", dict(beta=1.2, psi_uses_local_T=1), lambda: _droplet(40, 36)),
    ("slab_beta0", dict(beta=0.0, psi_uses_local_T=0, T_psi=0.75 * I.CS_TC), lambda: _slab(30, 20)),
]


def _params(shape, kw):
    ny, nx = shape
    return O.params(nx, ny, tau_f=0.9, tau_g=0.8, G=-1.0, eos=O.EOS_CS, a=1.0, b=4.0, R=1.0, **kw)


@pytest.mark.parametrize("name,kw,fields", CASES, ids=[c[0] for c in CASES])
def test_balanced_start_is_at_rest(name, kw, fields):
    """u = (sum e_i f_i + F/2)/rho vanishes: the first moment of f^eq(rho, v)
    is rho v, and v = -F/(2 rho)."""
    rho0, T0 = fields()
    P = _params(rho0.shape, kw)
    f, g, st = O.init_balanced(P, rho0, T0)
    assert st == O.OK
    rho, ux, uy, T, Fx, Fy = O.moments(P, f, g)
    scale = max(np.abs(Fx / rho).max(), np.abs(Fy / rho).max()) / 2.0
    assert scale > 1e-3, "the fields must carry a force for this pin to mean anything"
    assert np.abs(ux).max() <= 1e-12 * scale
    assert np.abs(uy).max() <= 1e-12 * scale
    # the plain start is not at rest: it moves with F/(2 rho)
    fp, gp = O.init_equilibrium(P, rho0, T0)
    _, uxp, uyp, _, _, _ = O.moments(P, fp, gp)
    assert np.abs(uxp - Fx / (2.0 * rho)).max() <= 1e-12 * scale
    assert np.abs(uyp - Fy / (2.0 * rho)).max() <= 1e-12 * scale


@pytest.mark.parametrize("name,kw,fields", CASES, ids=[c[0] for c in CASES])
def test_balanced_start_keeps_rho_and_T(name, kw, fields):
    """sum_i f^eq_i(rho, v) = rho and sum_i c_v T f^eq_i = rho c_v T for any v."""
    rho0, T0 = fields()
    P = _params(rho0.shape, kw)
    f, g, _ = O.init_balanced(P, rho0, T0)
    rho, _, _, T, _, _ = O.moments(P, f, g)
    assert np.abs(rho - rho0).max() <= 4e-16 * rho0.max()
    assert np.abs(T - T0).max() <= 4e-15 * T0.max()


def test_balanced_start_with_cv():
    """g scales with c_v and T does not (c_v = 2 against c_v = 1)."""
    rho0, T0 = _droplet(24, 24)
    P1 = _params(rho0.shape, dict(beta=1.0, psi_uses_local_T=1))
    P2 = O.params(24, 24, tau_f=0.9, tau_g=0.8, G=-1.0, beta=1.0, psi_uses_local_T=1, cv=2.0)
    f1, g1, _ = O.init_balanced(P1, rho0, T0)
    f2, g2, _ = O.init_balanced(P2, rho0, T0)
    assert np.array_equal(f1, f2)
    assert np.allclose(g2, 2.0 * g1, rtol=1e-15, atol=0)


def test_balanced_start_of_uniform_state_is_plain_equilibrium():
    """With uniform rho and T the pair sums of Eq. (2)/(4) vanish exactly, so
    the start is f^eq(rho, 0) bit for bit."""
    rho0 = np.full((16, 20), 0.2)
    T0 = np.full((16, 20), 0.08)
    for beta in (0.0, 1.0, 1.3):
        P = O.params(20, 16, tau_f=1.0, tau_g=0.8, G=-1.0, beta=beta, psi_uses_local_T=1)
        f, g, st = O.init_balanced(P, rho0, T0)
        fp, gp = O.init_equilibrium(P, rho0, T0)
        assert st == O.OK
        assert np.array_equal(f, fp) and np.array_equal(g, gp)


def test_balanced_start_reports_psi_domain():
    """beta != 0 needs psi^2 >= 0; a density where p_EOS > rho c_s^2 (G < 0)
    is reported, as the step reports it."""
    rho0 = np.full((12, 12), 0.2)
    rho0[5, 5] = 0.9
    T0 = np.full((12, 12), 0.09)
    P = O.params(12, 12, tau_f=1.0, tau_g=0.8, G=-1.0, beta=1.0, psi_uses_local_T=1)
    _, _, st = O.init_balanced(P, rho0, T0)
    assert st == O.ERR_PSI_DOMAIN


def test_balanced_start_launches_a_smaller_impulse():
    """The purpose of the start: fields near a steady state (a slab relaxed
    for 1500 steps) restarted at rest stay nearly at rest, while the plain
    equilibrium kicks every interface with F/(2 rho).  After five steps the
    largest velocity of the balanced restart is at least 20x smaller."""
    rho0, T0 = _slab(48, 8, T_over=0.8)
    P = _params(rho0.shape, dict(beta=1.3, psi_uses_local_T=0, T_psi=0.8 * I.CS_TC))
    f, g = O.init_equilibrium(P, rho0, T0)
    f, g, _ = O.step(P, f, g, n=1500)
    rho, _, _, T, _, _ = O.moments(P, f, g)
    fb, gb, _ = O.init_balanced(P, rho, T)
    fp, gp = O.init_equilibrium(P, rho, T)
    fb, gb, _ = O.step(P, fb, gb, n=5)
    fp, gp, _ = O.step(P, fp, gp, n=5)
    ub = np.abs(O.moments(P, fb, gb)[1]).max()
    up = np.abs(O.moments(P, fp, gp)[1]).max()
    assert ub < 0.05 * up
