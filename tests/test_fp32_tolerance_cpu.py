"""Where the FP32 velocity bound of the GPU parity test comes from.

The FP32 path stores populations in FP32 and computes psi, the force and the
collision in FP32.  After 1000 steps of the 64x64 slab the GPU meets 2e-5 on
rho and T, but its velocity error is 4e-5 to 7e-5, so the parity test bounds u
by 1e-4 instead.  This file shows, on the CPU and without the GPU path, that
the 2e-5 target on u is below what FP32 arithmetic supports on this workload
while FP32 storage alone stays within it:

  a float32 model of the step (the same formulas as the FP32 kernel: pair
  sums of the force stencil, the even and odd parts of f^eq and F_i shared by
  opposite directions, mass and energy closed through the rest populations)
  is run with each stage -- storage, psi, force, collision -- in float64 or
  float32.  In float64 throughout it reproduces the FP64 oracle (1e-10), which
  pins the model; FP32 storage with float64 arithmetic gives e_u below 2e-5;
  the FP32 collision alone (the precision every storage mode collides in)
  already exceeds 2e-5; everything in float32 stays below 1e-4 on u and 2e-5
  on rho and T.

The velocity is small (max|u| = 0.014 in this start-up transient) and is set
by the balance of the pseudopotential force and the pressure, so rounding of
psi or of the collision at the 1e-7 level shows up in u amplified ~100x.
Error metric: e_phi = max|d phi| / max|phi_oracle|, u over both components.
"""
import numpy as np
import pytest

import oracle as O
from paper_1405_2232_gb300 import inputs as I

EX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
EY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])
WT = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
F32, F64 = np.float32, np.float64


def model_step(P, f, g, t_store, t_psi, t_force, t_coll):
    """One step from pre-collision (f, g) [9, ny, nx]; each stage in its type.
    beta = 1 (Eq. 2), Carnahan-Starling EOS, Eq. (24) when P.thermal == 1."""
    # moments and psi (Sec. II A)
    fp, gp = f.astype(t_psi), g.astype(t_psi)
    rho, e = fp[0].copy(), gp[0].copy()
    for i in range(1, 9):
        rho = rho + fp[i]
        e = e + gp[i]
    T = e / (rho * t_psi(P.cv))
    Te = T if P.psi_uses_local_T else t_psi(P.T_psi)
    eta = t_psi(P.b) * rho / t_psi(4)
    num = 1 + eta * (1 + eta * (1 - eta))
    d = 1 - eta
    p = rho * t_psi(P.R) * Te * num / (d * d * d) - t_psi(P.a) * rho * rho
    psi = np.sqrt((p - rho * t_psi(1 / 3)) * t_psi(2 / P.G))
    # Eq. (2) as antisymmetric pair sums
    ps = psi.astype(t_force)
    E, Wv = np.roll(ps, -1, 1), np.roll(ps, 1, 1)
    N, S = np.roll(ps, -1, 0), np.roll(ps, 1, 0)
    NE, NW, SE, SW = np.roll(N, -1, 1), np.roll(N, 1, 1), np.roll(S, -1, 1), np.roll(S, 1, 1)
    w1, w2 = t_force(1 / 3), t_force(1 / 12)
    d1, d2, d3 = NE - SW, SE - NW, NW - SE
    Fx = -t_force(P.G) * (ps * (w1 * (E - Wv) + w2 * (d1 + d2)))
    Fy = -t_force(P.G) * (ps * (w1 * (N - S) + w2 * (d1 + d3)))
    # collision: Eq. (1) with F_i, Eq. (7) / (24)
    t = t_coll
    fc, gc, Fx, Fy = f.astype(t), g.astype(t), Fx.astype(t), Fy.astype(t)
    rho, e = fc[0].copy(), gc[0].copy()
    for i in range(1, 9):
        rho = rho + fc[i]
        e = e + gc[i]
    mx = (fc[1] - fc[3]) + ((fc[5] - fc[7]) + (fc[8] - fc[6]))
    my = (fc[2] - fc[4]) + ((fc[5] - fc[7]) + (fc[6] - fc[8]))
    inv = t(1) / rho
    ux, uy = (mx + t(0.5) * Fx) * inv, (my + t(0.5) * Fy) * inv
    cvT = t(P.cv) * (e / (rho * t(P.cv)))
    omf, omg = t(1 / P.tau_f), t(1 / P.tau_g)
    guo, corr = t(1 - 0.5 / P.tau_f), t(1 - 0.5 / P.tau_g)
    base = t(1) - t(1.5) * (ux * ux + uy * uy)
    uF3 = t(3) * (ux * Fx + uy * Fy)
    of, og = np.empty_like(fc), np.empty_like(gc)
    for i, k in ((1, 3), (2, 4), (5, 7), (8, 6)):
        w = t(WT[i])
        eu = t(EX[i]) * ux + t(EY[i]) * uy
        eF = t(EX[i]) * Fx + t(EY[i]) * Fy
        rw = rho * w
        fe, fo = rw * (base + t(4.5) * eu * eu), t(3) * rw * eu
        Fe, Fo = guo * w * (t(9) * eu * eF - uF3), t(3) * guo * w * eF
        of[i] = fc[i] + omf * ((fe + fo) - fc[i]) + (Fe + Fo)
        of[k] = fc[k] + omf * ((fe - fo) - fc[k]) + (Fe - Fo)
        gi = gc[i] + omg * (cvT * (fe + fo) - gc[i])
        gk = gc[k] + omg * (cvT * (fe - fo) - gc[k])
        if P.thermal == O.THERMAL_EQ24:
            Co = t(3) * corr * w * cvT * eF
            gi, gk = gi + Co, gk - Co
        og[i], og[k] = gi, gk
    sf, sg = of[1].copy(), og[1].copy()
    for i in range(2, 9):
        sf = sf + of[i]
        sg = sg + og[i]
    of[0], og[0] = rho - sf, e - sg
    # storage rounding, then streaming (an exact move)
    of = of.astype(t_store).astype(F64)
    og = og.astype(t_store).astype(F64)
    for i in range(9):
        of[i] = np.roll(of[i], (EY[i], EX[i]), (0, 1))
        og[i] = np.roll(og[i], (EY[i], EX[i]), (0, 1))
    return of, og


@pytest.fixture(scope="module")
def slab():
    rho, T = I.slab_fields(64, 64, width=32)
    P = O.params(64, 64, tau_f=1.0, tau_g=0.8, G=-1.0, beta=1.0, eos=O.EOS_CS, a=1.0, b=4.0,
                 R=1.0, cv=1.0, thermal=O.THERMAL_EQ24)
    f, g = O.init_equilibrium(P, rho, T)
    fr, gr, st = O.step(P, f, g, n=1000)
    assert st == O.OK
    return P, f, g, O.moments(P, fr, gr)


def errors(P, f, g, ref, types, n=1000):
    ff = f.astype(types[0]).astype(F64)
    gg = g.astype(types[0]).astype(F64)
    for _ in range(n):
        ff, gg = model_step(P, ff, gg, *types)
    m = O.moments(P, ff, gg)
    e_rho = np.abs(m[0] - ref[0]).max() / np.abs(ref[0]).max()
    du = max(np.abs(m[1] - ref[1]).max(), np.abs(m[2] - ref[2]).max())
    e_u = du / max(np.abs(ref[1]).max(), np.abs(ref[2]).max())
    e_T = np.abs(m[3] - ref[3]).max() / np.abs(ref[3]).max()
    return e_rho, e_u, e_T


def test_model_in_float64_is_the_oracle(slab):
    P, f, g, ref = slab
    assert max(errors(P, f, g, ref, (F64, F64, F64, F64))) < 1e-10


def test_fp32_storage_alone_meets_2e5_on_u(slab):
    P, f, g, ref = slab
    e_rho, e_u, e_T = errors(P, f, g, ref, (F32, F64, F64, F64))
    print(f"FP32 storage, FP64 arithmetic: e_rho={e_rho:.2e} e_u={e_u:.2e} e_T={e_T:.2e}")
    assert e_u < 2e-5 and e_rho < 2e-5 and e_T < 2e-5


def test_fp32_collision_alone_exceeds_2e5_on_u(slab):
    P, f, g, ref = slab
    e_rho, e_u, e_T = errors(P, f, g, ref, (F64, F64, F64, F32))
    print(f"FP32 collision only: e_rho={e_rho:.2e} e_u={e_u:.2e} e_T={e_T:.2e}")
    assert e_u > 2e-5


def test_fp32_throughout_within_parity_bounds(slab):
    """The bounds the GPU parity test applies to the FP32 path: rho and T within
    2e-5, u within 1e-4 (the float32 model has no fused multiply-adds; the
    GPU's own e_u, 4e-5 to 7e-5, is of the same size)."""
    P, f, g, ref = slab
    e_rho, e_u, e_T = errors(P, f, g, ref, (F32, F32, F32, F32))
    print(f"FP32 throughout: e_rho={e_rho:.2e} e_u={e_u:.2e} e_T={e_T:.2e}")
    assert 2e-5 < e_u < 1e-4 and e_rho < 2e-5 and e_T < 2e-5
