"""Liquid-vapour coexistence densities of the EOS (test infrastructure).

Maxwell's equal-area construction for the equation of state the oracle
evaluates (or_p_eos): at temperature T the coexisting densities rho_g < rho_l
satisfy p(rho_g) = p(rho_l) = p* and, in specific volume v = 1/rho,
integral_{v_l}^{v_g} (p(v) - p*) dv = 0, i.e.
integral_{rho_g}^{rho_l} (p(rho) - p*) / rho^2 drho = 0.

Running ``python -m oracle.coexistence`` prints the table that the seeded
input generator (paper_1405_2232_gb300/inputs.py, COEXISTENCE_CS) stores
for the Carnahan-Starling EOS with a = 1, b = 4, R = 1.
"""
from __future__ import annotations

import warnings

import numpy as np
from scipy.integrate import quad
from scipy.optimize import brentq

from . import p_eos, params, critical_point, EOS_CS


def spinodal(P, T, lo=1e-6, hi=None):
    """Densities where dp/drho = 0 at T (below T_c): (rho_s1, rho_s2)."""
    hi = hi or 0.999 * 4.0 / P.b
    rs = np.linspace(lo, hi, 4001)
    dp = np.array([p_eos(P, r + 1e-7, T) - p_eos(P, r - 1e-7, T) for r in rs])
    idx = np.flatnonzero(np.sign(dp[:-1]) != np.sign(dp[1:]))
    f = lambda r: p_eos(P, r + 1e-7, T) - p_eos(P, r - 1e-7, T)
    return brentq(f, rs[idx[0]], rs[idx[0] + 1]), brentq(f, rs[idx[1]], rs[idx[1] + 1])


def maxwell(P, T):
    """(rho_g, rho_l, p*) at T < T_c."""
    s1, s2 = spinodal(P, T)
    p_lo = max(p_eos(P, s2, T), 1e-300)
    p_hi = p_eos(P, s1, T)

    def roots(ps):
        lo = min(1e-12, ps / (10.0 * P.R * T))  # p ~ rho R T at low density
        g = brentq(lambda r: p_eos(P, r, T) - ps, lo, s1, xtol=1e-300, rtol=1e-14)
        l = brentq(lambda r: p_eos(P, r, T) - ps, s2, 0.999 * 4.0 / P.b, xtol=1e-300, rtol=1e-14)
        return g, l

    def area(ps):
        g, l = roots(ps)
        with warnings.catch_warnings():
            warnings.simplefilter("ignore")  # quad reports round-off at the requested 1e-13
            return quad(lambda r: (p_eos(P, r, T) - ps) / (r * r), g, l, limit=200, epsabs=0, epsrel=1e-13)[0]

    ps = brentq(area, p_lo * (1 + 1e-9) + 1e-30, p_hi * (1 - 1e-9), xtol=1e-300, rtol=1e-14)
    g, l = roots(ps)
    return g, l, ps


def cs_table(t_lo=0.60, t_hi=0.95, dt=0.01):
    P = params(8, 8, eos=EOS_CS, a=1.0, b=4.0, R=1.0)
    Tc, _ = critical_point(P)
    out = []
    for k in range(int(round((t_hi - t_lo) / dt)) + 1):
        t = round(t_lo + k * dt, 10)
        g, l, _ = maxwell(P, t * Tc)
        out.append((t, g, l))
    return out


if __name__ == "__main__":
    for t, g, l in cs_table():
        print(f"    ({t:.2f}, {g:.10e}, {l:.10e}),")
