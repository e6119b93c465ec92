"""GPU parity: the CUDA path, called through the C ABI, against the FP64 oracle
on the same seeded inputs.

Tolerances (max-norm errors e_phi = max|d phi| / max|phi_oracle| per field):
  * FP64 storage: the FP64 path evaluates the printed formulas in their order
    without contraction, so populations must match the oracle BIT FOR BIT
    (hence e = 0 <= 1e-12) after 1000 steps.
  * FP32 storage, one step from a shared state: populations within 2e-6 of
    their plane's maximum; moments within 1e-5 (the velocity is a difference
    of populations divided by rho, so one FP32 ulp of the populations of the
    vapour, rho ~ 0.02, is ~4e-6 of max|u|).
  * FP32 storage after 1000 steps of the 64x64 slab: rho and T within 2e-5,
    u within 1e-4 (measured on the GPU: e_u between 4e-5 and 7e-5, depending on
    the fused multiply-adds the compiler forms in a given build).  The 2e-5 target on u
    is not met: FP32 arithmetic cannot meet it on this workload.  A float32
    model of the step (tests/test_fp32_tolerance_cpu.py) shows FP32 storage
    alone gives e_u = 8e-6, the FP32 collision alone 3.8e-5 and FP32
    throughout 7.7e-5 (u, max 0.014, is a small balance of force and pressure,
    so 1e-7 roundings of psi or the collision appear ~100x larger in it).
    u is measured against max|u| over both components.
  * 16-bit deviation storage, one step: each moving population within half an
    ulp of its stored deviation plus the FP32 step error (bound derived per
    element); the rest population, an FP32 deviation that closes the site's
    mass and energy, within the sum of the others' bounds.  Mass and energy
    drift by FP32 roundings only (1e-6 after 400 steps of a 256^2 quench).
"""
import numpy as np
import pytest

import oracle as O
from paper_1405_2232_gb300 import inputs as I

pytestmark = pytest.mark.gpu

C1 = dict(nx=64, ny=64, tau_f=1.0, tau_g=0.8, G=-1.0, beta=1.0, a=1.0, b=4.0, R=1.0, cv=1.0)
# the spinodal quench (T = 0.75 T_c) runs the mixed force Eq. (4) with beta = 1.3:
# with Eq. (2) its vapour density falls below zero within ~200 steps
SPIN_BETA = 1.3


@pytest.fixture(scope="module")
def lb():
    import torch  # noqa: F401  (initialises CUDA in this process)
    from paper_1405_2232_gb300 import lb as _lb
    _lb.load()
    return _lb


def emax(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def field_errors(gpu, ref):
    """(e_rho, e_u, e_T) between (rho, ux, uy, T) tuples."""
    e_rho = emax(gpu[0], ref[0])
    du = max(np.abs(gpu[1] - ref[1]).max(), np.abs(gpu[2] - ref[2]).max())
    umax = max(np.abs(ref[1]).max(), np.abs(ref[2]).max())
    return e_rho, float(du / umax), emax(gpu[3], ref[3])


def oracle_params(thermal, psi_local=1, T_psi=0.0, **kw):
    d = dict(C1)
    d.update(kw)
    return O.params(d["nx"], d["ny"], tau_f=d["tau_f"], tau_g=d["tau_g"], G=d["G"],
                    beta=d["beta"], eos=d.get("eos", O.EOS_CS), a=d["a"], b=d["b"], R=d["R"],
                    cv=d["cv"], thermal=thermal, psi_uses_local_T=psi_local, T_psi=T_psi)


def gpu_lattice(lb, rho, T, thermal, precision, psi_local=1, T_psi=0.0, **kw):
    d = dict(C1)
    d.update(kw)
    d.update(thermal=thermal, precision=lb.PRECISIONS[precision], psi_uses_local_T=psi_local,
             T_psi=T_psi)
    d["nx"], d["ny"] = rho.shape[1], rho.shape[0]
    return lb.Lattice(rho, T, **d)


_cache = {}


def oracle_run(thermal, n, psi_local=1, shape=(64, 64), **kw):
    key = (thermal, n, psi_local, shape, tuple(sorted(kw.items())))
    if key not in _cache:
        ny, nx = shape
        rho, T = I.slab_fields(nx, ny, width=min(32, nx // 2))
        P = oracle_params(thermal, psi_local, 0.85 * I.CS_TC, nx=nx, ny=ny, **kw)
        f, g = O.init_equilibrium(P, rho, T)
        f, g, st = O.step(P, f, g, n=n, check=False)
        _cache[key] = (rho, T, P, f, g, st, O.moments(P, f, g)[:4])
    return _cache[key]


# ------------------------------------------------------------------ FP64
@pytest.mark.parametrize("thermal,psi_local", [(O.THERMAL_EQ24, 1), (O.THERMAL_EQ7, 0)])
def test_fp64_bit_identical_1000_steps(lb, thermal, psi_local):
    """64x64 CS slab + noise (seed 1), 1000 steps: populations equal bit for bit."""
    rho, T, P, f_ref, g_ref, st, m_ref = oracle_run(thermal, 1000, psi_local)
    assert st == O.OK
    with gpu_lattice(lb, rho, T, thermal, "fp64", psi_local, 0.85 * I.CS_TC) as L:
        L.step(1000)
        f, g = L.populations()
        m = L.moments()
    assert np.array_equal(f, f_ref) and np.array_equal(g, g_ref)
    e = field_errors(m, m_ref)
    assert max(e) <= 1e-12, e


def test_fp64_eq7_local_T_reports_psi_domain_at_same_step(lb):
    """Eq. (7) with psi(rho, T): the oracle leaves the psi domain at step k; the GPU
    reports LB_ERR_PSI_DOMAIN in the same step and not before."""
    rho, T = I.slab_fields(64, 64)
    P = oracle_params(O.THERMAL_EQ7)
    f, g = O.init_equilibrium(P, rho, T)
    k = 0
    while True:
        f, g, st = O.step(P, f, g, n=1, check=False)
        k += 1
        if st:
            break
        assert k < 200
    assert st == O.ERR_PSI_DOMAIN
    with gpu_lattice(lb, rho, T, O.THERMAL_EQ7, "fp64") as L:
        L.step(k - 1)
        L.synchronize()  # no error before step k
        L.step(1)
        with pytest.raises(lb.LbError) as ei:
            L.synchronize()
        assert ei.value.status == lb.LB_ERR_PSI_DOMAIN


@pytest.mark.parametrize("shape", [(45, 67), (130, 5), (3, 3), (9, 33), (8, 64), (17, 200)])
def test_fp64_ragged_and_small_lattices(lb, shape):
    """Lattices that leave ragged tiles, a single partial tile, the 3x3 minimum."""
    ny, nx = shape
    rho, T = I.slab_fields(nx, ny, width=max(2, nx // 2), noise=1e-3)
    P = oracle_params(O.THERMAL_EQ24, nx=nx, ny=ny)
    f0, g0 = O.init_equilibrium(P, rho, T)
    f_ref, g_ref, st = O.step(P, f0, g0, n=40, check=False)
    with gpu_lattice(lb, rho, T, O.THERMAL_EQ24, "fp64") as L:
        L.step(40)
        f, g = L.populations()
    assert np.array_equal(f, f_ref, equal_nan=True) and np.array_equal(g, g_ref, equal_nan=True)


@pytest.mark.parametrize("case", ["vdw_eq2", "ideal_beta0", "ideal_mixed", "passive_T", "cv2"])
def test_fp64_other_eos_and_force_forms(lb, case):
    """vdW EOS, Eq. (4) with beta = 0 and beta = 0.3, passive T, c_v = 2."""
    nx, ny = 48, 40
    if case == "vdw_eq2":
        kw = dict(eos=O.EOS_VDW, a=9.0 / 49.0, b=2.0 / 21.0, R=1.0, G=-1.0, beta=1.0)
        Tc = 8 * kw["a"] / (27 * kw["b"])
        rho, T = I.droplet_fields(nx, ny, 10, rho_l=5.0, rho_g=2.0, Tc=Tc, T_lo=0.9, T_hi=0.9)
        psi_local, T_psi = 1, 0.0
    elif case in ("ideal_beta0", "ideal_mixed"):
        kw = dict(eos=O.EOS_IDEAL, a=0.0, b=0.0, R=0.5, G=1.0,
                  beta=0.0 if case == "ideal_beta0" else 0.3)
        rho, T = I.sinusoid_fields(nx, ny, 1.0, 1.0, 0.05, mode=2, axis=0)
        T = T * (1.0 + 0.01 * np.sin(2 * np.pi * np.arange(ny) / ny))[:, None]
        psi_local, T_psi = 1, 0.0
    elif case == "passive_T":
        kw = {}
        rho, T = I.slab_fields(nx, ny, width=20)
        psi_local, T_psi = 0, 0.85 * I.CS_TC
    else:
        kw = dict(cv=2.0)
        rho, T = I.slab_fields(nx, ny, width=20)
        psi_local, T_psi = 1, 0.0
    for thermal in (O.THERMAL_EQ7, O.THERMAL_EQ24):
        pl, tp = psi_local, T_psi
        if thermal == O.THERMAL_EQ7 and case in ("vdw_eq2", "cv2"):
            # Eq. (7) with psi(rho, T) leaves the psi domain here: run T passively
            pl, tp = 0, float(T.mean())
        P = oracle_params(thermal, pl, tp, nx=nx, ny=ny, **kw)
        f0, g0 = O.init_equilibrium(P, rho, T)
        f_ref, g_ref, st = O.step(P, f0, g0, n=60, check=False)
        assert st == O.OK
        with gpu_lattice(lb, rho, T, thermal, "fp64", pl, tp, **kw) as L:
            L.step(60)
            f, g = L.populations()
        assert np.array_equal(f, f_ref), case
        assert np.array_equal(g, g_ref), case


@pytest.mark.parametrize("tile", [(32, 8), (32, 16), (64, 4), (128, 0), (0, 0)])
def test_fp64_tiles_identical(lb, tile):
    rho, T, P, f_ref, g_ref, st, m_ref = oracle_run(O.THERMAL_EQ24, 100)
    with gpu_lattice(lb, rho, T, O.THERMAL_EQ24, "fp64", tile_x=tile[0], tile_y=tile[1]) as L:
        L.step(100)
        f, g = L.populations()
    assert np.array_equal(f, f_ref) and np.array_equal(g, g_ref)


def test_fp64_totals_and_residual(lb):
    """FP64 totals (deterministic device reduction) against the oracle's compensated sums;
    the residual against the oracle's residual between the two snapshot times."""
    rho, T, P, f_ref, g_ref, st, m_ref = oracle_run(O.THERMAL_EQ24, 300)
    rho_a, T_a, P_a, f_a, g_a, _, m_a = oracle_run(O.THERMAL_EQ24, 200)
    t_ref = O.totals(P, f_ref, g_ref)
    t0 = O.totals(P, *O.init_equilibrium(P, rho, T))
    with gpu_lattice(lb, rho, T, O.THERMAL_EQ24, "fp64") as L:
        L.step(200)
        L.totals()
        L.step(100)
        tot = L.totals()
    assert tot[0] == pytest.approx(t_ref[0], rel=1e-14)
    assert tot[1] == pytest.approx(t_ref[1], rel=1e-14)
    assert abs(tot[2] - t_ref[2]) < 1e-14 * t_ref[0] and abs(tot[3] - t_ref[3]) < 1e-14 * t_ref[0]
    assert tot[0] == pytest.approx(t0[0], rel=1e-13) and tot[1] == pytest.approx(t0[1], rel=1e-13)
    r_ref = O.residual(m_a[0], m_a[3], m_ref[0], m_ref[3], 100)
    assert tot[4] == pytest.approx(r_ref, rel=1e-9)


# ------------------------------------------------------------------ FP32
def test_fp32_one_step_from_shared_state(lb):
    """From the oracle state at step 500 rounded to FP32, one GPU FP32 step against one
    oracle step from the same (rounded) state."""
    rho, T, P, f5, g5, st, _ = oracle_run(O.THERMAL_EQ24, 500)
    f32 = f5.astype(np.float32).astype(np.float64)
    g32 = g5.astype(np.float32).astype(np.float64)
    f_ref, g_ref, _ = O.step(P, f32, g32, n=1)
    with gpu_lattice(lb, rho, T, O.THERMAL_EQ24, "fp32") as L:
        L.set_populations(f32, g32)
        f0, g0 = L.populations()
        assert np.array_equal(f0, f32) and np.array_equal(g0, g32)
        L.step(1)
        f, g = L.populations()
        m = L.moments()
    for i in range(9):
        assert emax(f[i], f_ref[i]) < 2e-6, i
        assert emax(g[i], g_ref[i]) < 2e-6, i
    e = field_errors(m, O.moments(P, f_ref, g_ref)[:4])
    assert e[0] < 2e-6 and e[2] < 2e-6 and e[1] < 1e-5, e


@pytest.mark.parametrize("thermal,psi_local", [(O.THERMAL_EQ24, 1), (O.THERMAL_EQ7, 0)])
def test_fp32_1000_steps(lb, thermal, psi_local):
    rho, T, P, f_ref, g_ref, st, m_ref = oracle_run(thermal, 1000, psi_local)
    with gpu_lattice(lb, rho, T, thermal, "fp32", psi_local, 0.85 * I.CS_TC) as L:
        L.step(1000)
        m = L.moments()
    e_rho, e_u, e_T = field_errors(m, m_ref)
    print(f"FP32 1000 steps thermal={thermal}: e_rho={e_rho:.3e} e_u={e_u:.3e} e_T={e_T:.3e}")
    assert e_rho <= 2e-5 and e_T <= 2e-5 and e_u <= 1e-4, (e_rho, e_u, e_T)


def test_fp32_eq7_local_T_first_steps(lb):
    """Eq. (7) with psi(rho, T) until just before it leaves the psi domain."""
    rho, T, P, f_ref, g_ref, st, m_ref = oracle_run(O.THERMAL_EQ7, 25)
    assert st == O.OK
    with gpu_lattice(lb, rho, T, O.THERMAL_EQ7, "fp32") as L:
        L.step(25)
        m = L.moments()
    e = field_errors(m, m_ref)
    assert e[0] <= 2e-5 and e[2] <= 2e-5 and e[1] <= 1e-4, e


@pytest.mark.parametrize("shape,tile", [((17, 130), (128, 0)), ((33, 260), (128, 0)),
                                        ((8, 4), (128, 0)), ((5, 6), (128, 0)),
                                        ((64, 64), (128, 0)), ((17, 131), (128, 0)),
                                        ((9, 67), (128, 0)), ((6, 5), (128, 0))])
def test_fp64_strip_kernel_ragged(lb, shape, tile):
    """Strip kernel on partial strips, one-strip lattices and few-row chunks: still bit
    for bit with the oracle (the periodic ghost columns at both ends of every row)."""
    ny, nx = shape
    rho, T = I.slab_fields(nx, ny, width=max(2, nx // 2), noise=1e-3)
    P = oracle_params(O.THERMAL_EQ24, nx=nx, ny=ny)
    f0, g0 = O.init_equilibrium(P, rho, T)
    f_ref, g_ref, st = O.step(P, f0, g0, n=25, check=False)
    with gpu_lattice(lb, rho, T, O.THERMAL_EQ24, "fp64", tile_x=tile[0], tile_y=tile[1]) as L:
        assert lb.lb_get_params(L.ctx).tile_y == 0
        L.step(25)
        f, g = L.populations()
    assert np.array_equal(f, f_ref, equal_nan=True) and np.array_equal(g, g_ref, equal_nan=True)


@pytest.mark.parametrize("shape", [(24, 200), (9, 130), (16, 4)])
def test_fp64_strip_set_populations_then_step(lb, shape):
    """Populations written through lb_set_populations (which also writes the
    strip layout's ghost columns) step on bit for bit with the oracle."""
    ny, nx = shape
    rho, T = I.slab_fields(nx, ny, width=max(2, nx // 2), noise=1e-3)
    P = oracle_params(O.THERMAL_EQ24, nx=nx, ny=ny)
    f0, g0 = O.init_equilibrium(P, rho, T)
    f1, g1, _ = O.step(P, f0, g0, n=20, check=False)
    f_ref, g_ref, _ = O.step(P, f1, g1, n=10, check=False)
    with gpu_lattice(lb, rho * 0 + 0.2, T, O.THERMAL_EQ24, "fp64", tile_x=128, tile_y=0) as L:
        L.set_populations(f1, g1)
        L.step(10)
        f, g = L.populations()
    assert np.array_equal(f, f_ref, equal_nan=True) and np.array_equal(g, g_ref, equal_nan=True)


@pytest.mark.parametrize("shape,tile", [((64, 64), (32, 8)), ((64, 64), (128, 0)),
                                        ((17, 260), (256, 0)), ((45, 72), (256, 0)),
                                        ((3, 4), (256, 0)), ((40, 512), (128, 0)),
                                        ((13, 301), (256, 0)), ((11, 45), (128, 0))])
def test_fp32_kernels_agree_one_step(lb, shape, tile):
    """All FP32 kernels (strip widths, tiles) compute the same step: one step from a
    shared state within FP32 rounding (their FMA contractions may differ)."""
    ny, nx = shape
    rho, T = I.slab_fields(nx, ny, width=max(2, nx // 2), noise=1e-3)
    P = oracle_params(O.THERMAL_EQ24, nx=nx, ny=ny)
    f0, g0 = O.init_equilibrium(P, rho, T)
    f0, g0, _ = O.step(P, f0, g0, n=30)
    f32 = f0.astype(np.float32).astype(np.float64)
    g32 = g0.astype(np.float32).astype(np.float64)
    f_ref, g_ref, _ = O.step(P, f32, g32, n=1)
    with gpu_lattice(lb, rho, T, O.THERMAL_EQ24, "fp32", tile_x=tile[0], tile_y=tile[1]) as L:
        L.set_populations(f32, g32)
        L.step(1)
        f, g = L.populations()
    for i in range(9):
        assert emax(f[i], f_ref[i]) < 2e-6 and emax(g[i], g_ref[i]) < 2e-6


def test_fp32_strip_translation_invariance(lb):
    """Strip kernel: a periodic shift by a non-multiple of the strip width and the
    chunk height shifts the result bit for bit."""
    rho, T = I.slab_fields(512, 96)
    sh = (7, -132)
    with gpu_lattice(lb, rho, T, O.THERMAL_EQ24, "fp32", tile_x=256, tile_y=0) as A, \
            gpu_lattice(lb, np.roll(rho, sh, (0, 1)), np.roll(T, sh, (0, 1)), O.THERMAL_EQ24,
                        "fp32", tile_x=256, tile_y=0) as B:
        A.step(60)
        B.step(60)
        fa, ga = A.populations()
        fb, gb = B.populations()
    assert np.array_equal(np.roll(fa, sh, (1, 2)), fb)
    assert np.array_equal(np.roll(ga, sh, (1, 2)), gb)


def test_fp32_translation_invariance(lb):
    """Periodic shift of the input shifts the output bit for bit (tile-position independent)."""
    rho, T = I.slab_fields(96, 72)
    sh = (5, -13)
    with gpu_lattice(lb, rho, T, O.THERMAL_EQ24, "fp32") as A, \
            gpu_lattice(lb, np.roll(rho, sh, (0, 1)), np.roll(T, sh, (0, 1)), O.THERMAL_EQ24,
                        "fp32") as B:
        A.step(100)
        B.step(100)
        fa, ga = A.populations()
        fb, gb = B.populations()
    assert np.array_equal(np.roll(fa, sh, (1, 2)), fb)
    assert np.array_equal(np.roll(ga, sh, (1, 2)), gb)


def test_fp32_uniform_state_and_determinism(lb):
    rho, T = I.uniform_fields(40, 24, 0.2, 0.8 * I.CS_TC)
    with gpu_lattice(lb, rho, T, O.THERMAL_EQ7, "fp32") as L:
        L.step(50)
        f, g = L.populations()
    assert np.all(f == f[:, :1, :1]) and np.all(g == g[:, :1, :1])
    rho, T = I.slab_fields(64, 64)
    out = []
    for _ in range(2):
        with gpu_lattice(lb, rho, T, O.THERMAL_EQ24, "fp32") as L:
            L.step(300)
            out.append(L.populations())
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


def test_checkpoint_resume_bit_identical(lb):
    rho, T = I.slab_fields(64, 64)
    for prec in ("fp32", "fp16"):
        with gpu_lattice(lb, rho, T, O.THERMAL_EQ24, prec) as A:
            A.step(50)
            blob = lb.lb_save_state(A.ctx)
            A.step(50)
            fa, ga = A.populations()
        with gpu_lattice(lb, rho, T, O.THERMAL_EQ24, prec) as B:
            lb.lb_load_state(B.ctx, blob)
            assert B.time == 50
            B.step(50)
            fb, gb = B.populations()
        assert np.array_equal(fa, fb) and np.array_equal(ga, gb)


def test_zero_steps_is_identity(lb):
    rho, T = I.slab_fields(64, 64)
    P = oracle_params(O.THERMAL_EQ24)
    f0, g0 = O.init_equilibrium(P, rho, T)
    with gpu_lattice(lb, rho, T, O.THERMAL_EQ24, "fp64") as L:
        L.step(0)
        f, g = L.populations()
    assert np.array_equal(f, f0) and np.array_equal(g, g0)


# ------------------------------------------------------------------ 16-bit
@pytest.mark.parametrize("prec,u,shape,tile", [("fp16", 2.0 ** -11, (64, 64), (0, 0)),
                                              ("bf16", 2.0 ** -8, (64, 64), (0, 0)),
                                              ("fp16", 2.0 ** -11, (37, 261), (256, 0)),
                                              ("bf16", 2.0 ** -8, (29, 131), (128, 0)),
                                              ("bf16", 2.0 ** -8, (37, 45), (32, 8))])
def test_16bit_one_step_within_rounding_bound(lb, prec, u, shape, tile):
    """One step from a state the 16-bit mode represents exactly: every stored
    population within (half an ulp of its deviation) + (FP32 step error), on the
    strip kernel (any nx) and the tile kernel."""
    check_16bit_one_step(lb, prec, u, shape, tile)


# shapes of the 16-bit strip kernel's edge cases: strips narrower than one
# 16-byte unit and than a warp (the row's tensor copy clips at nx), odd and
# even job counts per row chunk (two rows per iteration), one- and
# many-chunk strips, a ragged second strip
@pytest.mark.parametrize("prec,u", [("fp16", 2.0 ** -11), ("bf16", 2.0 ** -8)])
@pytest.mark.parametrize("shape,tile", [((5, 3), (256, 0)), ((3, 6), (256, 0)), ((7, 40), (256, 0)), ((50, 300), (256, 0)),
                                        ((9, 257), (128, 0)), ((64, 136), (128, 0))])
def test_16bit_strip_shapes_within_rounding_bound(lb, prec, u, shape, tile):
    check_16bit_one_step(lb, prec, u, shape, tile)


def check_16bit_one_step(lb, prec, u, shape, tile):
    rho0, T0 = 0.12, 0.75 * I.CS_TC
    ny, nx = shape
    rho, T = I.spinodal_fields(nx, ny)
    P = oracle_params(O.THERMAL_EQ24, beta=SPIN_BETA, nx=nx, ny=ny)
    f, g = O.init_equilibrium(P, rho, T)
    f, g, _ = O.step(P, f, g, n=20)
    with gpu_lattice(lb, rho, T, O.THERMAL_EQ24, prec, rho0=rho0, T0=T0, beta=SPIN_BETA,
                     tile_x=tile[0], tile_y=tile[1]) as L:
        L.set_populations(f, g)
        fs, gs = L.populations()  # the exactly representable state
        f_ref, g_ref, _ = O.step(P, fs, gs, n=1)
        L.step(1)
        f1, g1 = L.populations()
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)[:, None, None]
    base_f = (w * rho0).astype(np.float32).astype(np.float64)
    base_g = (w * rho0 * T0).astype(np.float32).astype(np.float64)
    for got, ref, base in ((f1, f_ref, base_f), (g1, g_ref, base_g)):
        # moving populations: unit roundoff u of the 16-bit format on the
        # deviation, half the FP16 subnormal spacing (deviations below 6.1e-5
        # are subnormal), the FP32 step
        sub = 2.0 ** -25 if prec == "fp16" else 0.0
        bound = u * np.abs(ref - base) * 1.01 + sub + 2e-6 * np.abs(ref).max() + 1e-12
        assert np.all(np.abs(got[1:] - ref[1:]) <= bound[1:])
        # the rest population (an FP32 deviation) closes the site's mass or
        # energy: it carries with the opposite sign the errors of the eight
        # populations that left the site, which now sit at x + e_i, plus its
        # own FP32 step error
        ex = [0, 1, 0, -1, 0, 1, -1, -1, 1]
        ey = [0, 0, 1, 0, -1, 1, 1, -1, -1]
        bound0 = sum(np.roll(bound[i], (-ey[i], -ex[i]), (0, 1)) for i in range(1, 9))
        bound0 = bound0 + 2e-6 * np.abs(ref[0]).max()
        assert np.all(np.abs(got[0] - ref[0]) <= bound0)



# Mass and energy drift bounds: the paper's method conserves both exactly
# (Eq. (13); sum C_i = 0 after Eq. (25)).  FP32 storage closes them through the
# rest populations at FP32 precision; the 16-bit modes keep the rest
# populations as FP32 deviations and close each site's stored deviation sums
# (one FP32 rounding of a deviation of at most ~0.1 per site and step), so all
# three drift by FP32 roundings only: 1e-6 after 400 steps.
@pytest.mark.parametrize("prec,drift_max,frac_tol", [("fp32", 1e-6, 0.01), ("fp16", 1e-6, 0.03),
                                                    ("bf16", 1e-6, 0.10)])
def test_spinodal_statistics_against_fp64(lb, prec, drift_max, frac_tol):
    """Spinodal decomposition amplifies any perturbation exponentially, so after a few
    hundred steps reduced-precision runs differ from FP64 site by site by design.  They
    are compared by what must agree: mass and energy conservation, the fraction of the
    lattice in the liquid phase (rho > rho_c) and the density variance, against the
    FP64 path (which is bit-identical to the oracle)."""
    n, steps = 256, 400
    rho, T = I.spinodal_fields(n, n)
    stats = {}
    for p in ("fp64", prec):
        with gpu_lattice(lb, rho, T, O.THERMAL_EQ24, p, rho0=0.12, T0=0.75 * I.CS_TC,
                         beta=SPIN_BETA) as L:
            t0 = L.totals()
            L.step(steps)
            r = L.moments()[0]
            t1 = L.totals()
        stats[p] = (abs(t1[0] / t0[0] - 1), float((r > I.CS_RHOC).mean()), float(r.var()),
                    abs(t1[1] / t0[1] - 1))
    d, fr, var, de = stats[prec]
    d64, fr64, var64, de64 = stats["fp64"]
    print(f"{prec} spinodal {n}^2 {steps} steps: mass drift {d:.2e} (fp64 {d64:.1e}), energy drift "
          f"{de:.2e}, liquid fraction {fr:.4f} (fp64 {fr64:.4f}), var {var:.4e} (fp64 {var64:.4e})")
    assert d64 < 1e-13 and de64 < 1e-13
    assert d < drift_max and de < drift_max
    assert abs(fr - fr64) < frac_tol
    assert abs(var / var64 - 1) < 10 * frac_tol


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
def test_16bit_slab_error_report(lb, prec):
    """64x64 slab, 200 steps, deviations from w_i rho0 with rho0 the mean density:
    the per-field error against the oracle is reported (the 16-bit modes carry no
    parity claim beyond the one-step rounding bound); sanity bounds only."""
    rho, T, P, f_ref, g_ref, st, m_ref = oracle_run(O.THERMAL_EQ24, 200)
    with gpu_lattice(lb, rho, T, O.THERMAL_EQ24, prec, rho0=float(rho.mean()),
                     T0=0.85 * I.CS_TC) as L:
        L.step(200)
        m = L.moments()
    e = field_errors(m, m_ref)
    print(f"{prec} slab 64^2 200 steps: e_rho={e[0]:.3e} e_u={e[1]:.3e} e_T={e[2]:.3e}")
    bound = 0.05 if prec == "fp16" else 0.5
    assert np.all(np.isfinite(m[0])) and e[0] < bound and e[2] < bound
