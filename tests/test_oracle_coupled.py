"""Why the batched sweep runs with psi from the domain's T0 (passive temperature).

With psi(rho, T) of the local temperature and the corrected thermal LBE
(Eq. 24), a flat slab at the coexistence densities develops a period-two
(odd-even in x) mode of the velocity that grows exponentially and saturates
at |u| ~ 0.2-0.4, dissolving the slab; with Eq. (7) the same start leaves the
psi domain within a few hundred steps (the spurious heating of Eq. (23)).
With psi from T0 the odd-even amplitude stays at the few-1e-3 level of the
interfaces' Guo velocity F/(2 rho).  The growth does not depend on beta
(Eq. 2 and the mixed Eq. 4 alike), so it is the coupled scheme's own
behaviour, not a reading of the force; measured on the oracle over
T/T_c = 0.85, 0.92, tau_f = 0.6, 1.0, beta = 1, 1.3: growth rate 3.8e-4 ..
1.6e-3 per step (e-folding 600 - 2,600 steps), faster for deeper quenches
and smaller tau_f.  These tests keep that evidence: one case each way."""
import numpy as np
import pytest

import oracle as O
from paper_1405_2232_gb300 import inputs as I


def staggered_amplitude(m):
    """Half the difference of the mean x-velocity on even and odd columns."""
    ux = m[1]
    return abs(ux[:, 0::2].mean() - ux[:, 1::2].mean()) / 2


def slab_run(coupled, thermal, beta, steps, every=500, Tr=0.85, tau_f=1.0):
    rg, rl = I.coexistence_densities(Tr)
    rho, _ = I.slab_fields(48, 8, width=24, rho_l=rl, rho_g=rg, noise=0.0)
    T = np.full((8, 48), Tr * I.CS_TC)
    P = O.params(48, 8, tau_f=tau_f, tau_g=0.8, G=-1.0, beta=beta, eos=O.EOS_CS, a=1.0, b=4.0, R=1.0,
                 thermal=thermal, psi_uses_local_T=1 if coupled else 0, T_psi=Tr * I.CS_TC)
    f, g = O.init_equilibrium(P, rho, T)
    amps = []
    for _ in range(steps // every):
        f, g, st = O.step(P, f, g, n=every, check=False)
        if st:
            return amps, st
        amps.append(staggered_amplitude(O.moments(P, f, g)))
    return amps, O.OK


@pytest.mark.parametrize("beta", [1.0, 1.3])
def test_coupled_eq24_slab_grows_an_odd_even_mode(beta):
    passive, st_p = slab_run(False, O.THERMAL_EQ24, beta, 6000)
    coupled, st_c = slab_run(True, O.THERMAL_EQ24, beta, 6000)
    assert st_p == O.OK and st_c == O.OK
    assert max(passive) < 1e-2 and passive[-1] < 1.2 * passive[0]
    assert coupled[-1] > 0.1 and coupled[-1] > 10 * coupled[0]


def test_coupled_eq7_slab_leaves_the_psi_domain():
    amps, st = slab_run(True, O.THERMAL_EQ7, 1.3, 2000, every=100)
    assert st == O.ERR_PSI_DOMAIN and len(amps) < 5
