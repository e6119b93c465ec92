"""How strongly the 64x64 slab workload amplifies rounding (oracle only, CPU).

The GPU parity tolerances are set from the dynamics, not by guesswork: a
relative perturbation of FP32 size (6e-8) of the initial populations,
propagated by the FP64 oracle itself, moves rho, u and T by at most ~2e-6
(max-norm, u measured against max|u| over both components) after 1000
steps.  The amplification is benign (about 10x), so the FP32 path can be
held to 2e-5 on every field.
"""
import numpy as np

import oracle as O
from paper_1405_2232_gb300 import inputs as I


def test_fp32_sized_perturbation_stays_small():
    rho, T = I.slab_fields(64, 64)
    P = O.params(64, 64, thermal=O.THERMAL_EQ24)
    f, g = O.init_equilibrium(P, rho, T)
    rng = np.random.default_rng(7)
    fp = f * (1 + 6e-8 * rng.uniform(-1, 1, f.shape))
    gp = g * (1 + 6e-8 * rng.uniform(-1, 1, g.shape))
    fa, ga, _ = O.step(P, f, g, n=1000, threads=4)
    fb, gb, _ = O.step(P, fp, gp, n=1000, threads=4)
    ma, mb = O.moments(P, fa, ga), O.moments(P, fb, gb)
    e_rho = np.abs(ma[0] - mb[0]).max() / np.abs(ma[0]).max()
    e_T = np.abs(ma[3] - mb[3]).max() / np.abs(ma[3]).max()
    umax = max(np.abs(ma[1]).max(), np.abs(ma[2]).max())
    e_u = max(np.abs(ma[1] - mb[1]).max(), np.abs(ma[2] - mb[2]).max()) / umax
    assert max(e_rho, e_u, e_T) < 5e-6
    assert max(e_rho, e_u, e_T) > 6e-8  # the perturbation is felt, not lost
