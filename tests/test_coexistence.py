"""Coexistence densities of the Carnahan-Starling EOS (Maxwell construction).

The stored table of the input generator must equal what oracle/coexistence.py
computes, and every row must satisfy the two Maxwell conditions when they are
re-evaluated independently: equal pressures from the oracle's EOS, and zero
area between the isotherm and the coexistence pressure, integrated here with
the trapezoid rule in specific volume on a fine grid."""
import numpy as np
import pytest

import oracle as O
from oracle import coexistence as C
from paper_1405_2232_gb300 import inputs as I


@pytest.fixture(scope="module")
def P():
    return O.params(8, 8, eos=O.EOS_CS, a=1.0, b=4.0, R=1.0)


def test_table_is_what_the_generator_writes():
    rows = C.cs_table()
    assert len(rows) == len(I.COEXISTENCE_CS) == 36
    for (t, g, l), (t2, g2, l2) in zip(rows, I.COEXISTENCE_CS):
        assert t == t2 and g == pytest.approx(g2, rel=1e-12) and l == pytest.approx(l2, rel=1e-12)


@pytest.mark.parametrize("k", [0, 10, 20, 30, 35])
def test_maxwell_conditions(P, k):
    t, g, l = I.COEXISTENCE_CS[k]
    T = t * I.CS_TC
    pg, pl = O.p_eos(P, g, T), O.p_eos(P, l, T)
    assert pg == pytest.approx(pl, rel=1e-9)
    v = np.geomspace(1.0 / l, 1.0 / g, 200001)
    pv = np.array([O.p_eos(P, 1.0 / x, T) for x in v])
    area = np.trapezoid(pv - pg, v)
    scale = np.trapezoid(np.abs(pv - pg), v)
    assert abs(area) < 1e-6 * scale


def test_order_and_approach_to_the_critical_point():
    t = np.array([r[0] for r in I.COEXISTENCE_CS])
    g = np.array([r[1] for r in I.COEXISTENCE_CS])
    l = np.array([r[2] for r in I.COEXISTENCE_CS])
    assert np.all(np.diff(g) > 0) and np.all(np.diff(l) < 0) and np.all(g < I.CS_RHOC) and np.all(l > I.CS_RHOC)
    # mean-field approach: (rho_l - rho_g)^2 roughly linear in (1 - T/T_c) near T_c
    d2 = (l - g) ** 2
    slope_hi = (d2[-1] - d2[-2]) / (t[-2] - t[-1])
    slope_lo = (d2[-5] - d2[-6]) / (t[-6] - t[-5])
    assert slope_hi == pytest.approx(slope_lo, rel=0.1)


def test_interpolation():
    g, l = I.coexistence_densities(0.805)
    r0, r1 = I.COEXISTENCE_CS[20], I.COEXISTENCE_CS[21]
    assert g == pytest.approx(0.5 * (r0[1] + r1[1])) and l == pytest.approx(0.5 * (r0[2] + r1[2]))
    with pytest.raises(ValueError):
        I.coexistence_densities(0.59)
