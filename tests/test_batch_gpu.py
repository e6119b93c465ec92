"""Batched solver (lb_batch_*) against the FP64 oracle, domain by domain.

A batch advances many independent domains (different sizes, relaxation times,
G, EOS, temperatures) in one persistent kernel; each domain must evolve exactly
as it would alone.  FP64 storage is compared bit for bit, FP32 within 2e-5
(rho, T) after 40 steps."""
import ctypes

import numpy as np
import pytest

import oracle as O
from paper_1405_2232_gb300 import inputs as I


@pytest.fixture(scope="module")
def lb():
    from paper_1405_2232_gb300 import lb as _lb
    _lb.load()
    return _lb


# (nx, ny, tau_f, G, eos, T/Tc, kind)
DOMAINS = [
    (16, 12, 1.0, -1.0, "cs", 0.85, "slab"),
    (64, 64, 0.8, -1.1, "cs", 0.80, "droplet"),
    (36, 20, 1.2, -1.0, "cs", 0.90, "slab"),
    (260, 9, 1.0, -0.9, "cs", 0.85, "slab"),
    (132, 17, 0.9, -1.0, "vdw", 0.90, "droplet"),
    (516, 140, 1.0, -1.0, "cs", 0.85, "droplet"),
    # sides that are not a multiple of the 16-byte row unit (rounded-up row copies)
    (37, 21, 1.0, -1.0, "cs", 0.85, "droplet"),
    (131, 19, 0.9, -1.0, "cs", 0.85, "slab"),
    (257, 33, 1.1, -1.1, "cs", 0.80, "droplet"),
]
VDW = dict(a=9.0 / 49.0, b=2.0 / 21.0, R=1.0)


def domain_setup(spec, thermal, passive=False):
    nx, ny, tau_f, G, eos, tt, kind = spec
    if eos == "cs":
        Tc, kw = I.CS_TC, dict(eos=O.EOS_CS, a=1.0, b=4.0, R=1.0)
        rl, rg = 0.30, 0.04
    else:
        Tc, kw = 8 * VDW["a"] / (27 * VDW["b"]), dict(eos=O.EOS_VDW, **VDW)
        rl, rg = 5.0, 2.0
    if kind == "slab":
        rho, _ = I.slab_fields(nx, ny, width=max(2, nx // 2), rho_l=rl, rho_g=rg, noise=1e-3)
    else:
        rho, _ = I.droplet_fields(nx, ny, max(2, min(nx, ny) // 4), rho_l=rl, rho_g=rg, Tc=Tc)
    T = np.full((ny, nx), tt * Tc)
    P = O.params(nx, ny, tau_f=tau_f, tau_g=0.8, G=G, beta=1.0, thermal=thermal,
                 psi_uses_local_T=0 if passive else 1, T_psi=tt * Tc if passive else 0.0, **kw)
    return rho, T, P, kw


def lb_params_from(lb, P, precision):
    return lb.lb_params_default(nx=P.nx, ny=P.ny, tau_f=P.tau_f, tau_g=P.tau_g, G=P.G, beta=P.beta,
                                eos=P.eos, a=P.a, b=P.b, R=P.R, cv=P.cv, thermal=P.thermal,
                                precision=precision, psi_uses_local_T=P.psi_uses_local_T,
                                T_psi=P.T_psi)


@pytest.mark.gpu
def test_fp64_batch_bit_identical_per_domain(lb):
    setups = [domain_setup(s, O.THERMAL_EQ24) for s in DOMAINS]
    params = [lb_params_from(lb, P, "fp64") for _, _, P, _ in setups]
    with lb.Batch(params, [s[0] for s in setups], [s[1] for s in setups]) as B:
        B.step(40)
        for d, (rho0, T0, P, _) in enumerate(setups):
            f, g = O.init_equilibrium(P, rho0, T0)
            f, g, st = O.step(P, f, g, n=40, check=False)
            m = O.moments(P, f, g)
            rho, T = B.fields(d)
            assert np.array_equal(rho, m[0], equal_nan=True), d
            assert np.array_equal(T, m[3], equal_nan=True), d


@pytest.mark.gpu
def test_fp32_batch_per_domain(lb):
    setups = [domain_setup(s, O.THERMAL_EQ24) for s in DOMAINS]
    params = [lb_params_from(lb, P, "fp32") for _, _, P, _ in setups]
    with lb.Batch(params, [s[0] for s in setups], [s[1] for s in setups]) as B:
        B.step(40)
        for d, (rho0, T0, P, _) in enumerate(setups):
            f, g = O.init_equilibrium(P, rho0, T0)
            f, g, _ = O.step(P, f, g, n=40, check=False)
            m = O.moments(P, f, g)
            rho, T = B.fields(d)
            e_rho = np.abs(rho - m[0]).max() / np.abs(m[0]).max()
            e_T = np.abs(T - m[3]).max() / np.abs(m[3]).max()
            assert e_rho < 2e-5 and e_T < 2e-5, (d, e_rho, e_T)


@pytest.mark.gpu
def test_batch_check_residual_mass_energy(lb):
    setups = [domain_setup(s, O.THERMAL_EQ24) for s in DOMAINS[:4]]
    params = [lb_params_from(lb, P, "fp64") for _, _, P, _ in setups]
    with lb.Batch(params, [s[0] for s in setups], [s[1] for s in setups]) as B:
        B.step(20)
        r0, m0, e0, st0 = B.check()
        assert np.all(r0 == 0.0) and np.all(st0 == 0)
        B.step(30)
        r1, m1, e1, st1 = B.check()
    for d, (rho0, T0, P, _) in enumerate(setups):
        f, g = O.init_equilibrium(P, rho0, T0)
        fa, ga, _ = O.step(P, f, g, n=20)
        fb, gb, _ = O.step(P, fa, ga, n=30)
        ma, mb = O.moments(P, fa, ga), O.moments(P, fb, gb)
        assert r1[d] == pytest.approx(O.residual(ma[0], ma[3], mb[0], mb[3], 30), rel=1e-9)
        tot = O.totals(P, fb, gb)
        assert m1[d] == pytest.approx(tot[0], rel=1e-13)
        assert e1[d] == pytest.approx(tot[1], rel=1e-13)
        assert m1[d] == pytest.approx(m0[d], rel=1e-13)  # mass conserved


@pytest.mark.gpu
def test_batch_run_to_steady_state(lb):
    """Droplets and a slab relax to r < 1e-8 (psi from T0: with psi(rho, local T) a
    slab under Eq. (24) develops a slowly growing flow and never settles); every
    domain converges, its reported residual is below the tolerance, and its state
    equals a lone run of the same number of steps (FP64: bit for bit)."""
    specs = [(32, 32, 1.0, -1.0, "cs", 0.90, "droplet"), (40, 24, 0.9, -1.0, "cs", 0.92, "slab"),
             (24, 24, 1.1, -1.0, "cs", 0.88, "droplet")]
    setups = [domain_setup(s, O.THERMAL_EQ24, passive=True) for s in specs]
    params = [lb_params_from(lb, P, "fp64") for _, _, P, _ in setups]
    with lb.Batch(params, [s[0] for s in setups], [s[1] for s in setups]) as B:
        steps, resid, status = B.run(1e-8, K=100, max_steps=400000)
        assert np.all(status == lb.LB_OK), status
        assert np.all(resid < 1e-8) and np.all(steps > 0) and np.all(steps % 100 == 0)
        for d, (rho0, T0, P, _) in enumerate(setups):
            rho, T = B.fields(d)
            with lb.Lattice(rho0, T0, nx=P.nx, ny=P.ny, precision="fp64", tau_f=P.tau_f, G=P.G,
                            thermal=P.thermal, psi_uses_local_T=0, T_psi=P.T_psi) as L:
                L.step(int(steps[d]))
                m = L.moments()
            assert np.array_equal(rho, m[0]) and np.array_equal(T, m[3]), d


@pytest.mark.gpu
def test_batch_failed_domain_is_retired(lb):
    """Eq. (7) with psi(rho, T) leaves the psi domain on the 64x64 slab (step 33);
    in a batch that domain is retired with LB_ERR_PSI_DOMAIN and the other domain
    (passive T) runs on unharmed."""
    rho, T = I.slab_fields(64, 64)
    pa = lb.lb_params_default(nx=64, ny=64, thermal=lb.LB_THERMAL_EQ7, precision="fp32")
    pb = lb.lb_params_default(nx=64, ny=64, thermal=lb.LB_THERMAL_EQ7, precision="fp32",
                              psi_uses_local_T=0, T_psi=0.85 * I.CS_TC)
    with lb.Batch([pa, pb], [rho, rho], [T, T]) as B:
        steps, resid, status = B.run(1e-12, K=20, max_steps=400)
        assert status[0] == lb.LB_ERR_PSI_DOMAIN
        assert status[1] == lb.LB_ERR_NOT_CONVERGED and steps[1] == 400
        assert steps[0] <= 60
        r1, T1 = B.fields(1)
        assert np.all(np.isfinite(r1)) and np.all(np.isfinite(T1))


def test_batch_init_validates_on_host(lb):
    """Mismatched precision, a too-small domain and unsupported storage are rejected
    before any device work (runs without a GPU; any nx >= 3 is accepted)."""
    rho = np.ones((12, 16))
    dp = ctypes.POINTER(ctypes.c_double)
    for mutate, code in [
        (lambda p: setattr(p[1], "precision", lb.LB_PREC_FP64), lb.LB_ERR_ARG),
        (lambda p: setattr(p[1], "nx", 2), lb.LB_ERR_ARG),
        (lambda p: [setattr(q, "precision", lb.LB_PREC_FP16_DEV) for q in p], lb.LB_ERR_UNSUPPORTED),
        (lambda p: setattr(p[1], "thermal", lb.LB_THERMAL_EQ7), lb.LB_ERR_ARG),
        (lambda p: setattr(p[0], "tau_f", 0.4), lb.LB_ERR_ARG),
    ]:
        ps = [lb.lb_params_default(nx=16, ny=12, precision="fp32") for _ in range(2)]
        mutate(ps)
        arr = (lb.lb_params * 2)(*ps)
        fields = [np.ones((q.ny, q.nx)) for q in ps]
        ptrs = (dp * 2)(*[f.ctypes.data_as(dp) for f in fields])
        b = ctypes.c_void_p()
        st = lb.load().lb_batch_init(arr, 2, ptrs, ptrs, None, ctypes.byref(b))
        assert st == code and b.value is None


@pytest.mark.gpu
def test_batch_restart_domain(lb):
    """lb_batch_restart: a restarted domain evolves as a fresh start (FP64: bit for
    bit, from host or device fields, either initial state), the others are
    untouched, and a domain that had failed comes back onto the work list."""
    import torch
    setups = [domain_setup(s, O.THERMAL_EQ24) for s in DOMAINS[:3]]
    params = [lb_params_from(lb, P, "fp64") for _, _, P, _ in setups]
    with lb.Batch(params, [s[0] for s in setups], [s[1] for s in setups]) as B:
        B.step(30)
        B.restart(0, setups[0][0], setups[0][1], init_balanced=0)                # host fields
        d_rho = torch.from_numpy(setups[2][0]).cuda()
        d_T = torch.from_numpy(setups[2][1]).cuda()
        torch.cuda.synchronize()
        B.restart(2, d_rho, d_T, init_balanced=1)                                # device fields
        B.step(25)
        for d, n, bal in ((0, 25, 0), (1, 55, 0), (2, 25, 1)):
            rho0, T0, P, _ = setups[d]
            f, g = O.init_balanced(P, rho0, T0)[:2] if bal else O.init_equilibrium(P, rho0, T0)
            f, g, _ = O.step(P, f, g, n=n, check=False)
            m = O.moments(P, f, g)
            rho, T = B.fields(d)
            assert np.array_equal(rho, m[0]) and np.array_equal(T, m[3]), d
    # a failed domain is reactivated by a restart
    rho, T = I.slab_fields(64, 64)
    pa = lb.lb_params_default(nx=64, ny=64, thermal=lb.LB_THERMAL_EQ7, precision="fp32")
    with lb.Batch([pa], [rho], [T]) as B:
        steps, _, st = B.run(1e-12, K=20, max_steps=400)
        assert st[0] == lb.LB_ERR_PSI_DOMAIN
        B.restart(0, rho, T)
        steps2, _, st2 = B.run(1e-12, K=20, max_steps=20)
        assert steps2[0] == steps[0] + 20 and st2[0] in (lb.LB_ERR_NOT_CONVERGED, lb.LB_ERR_PSI_DOMAIN)
    with pytest.raises(lb.LbError):
        lb.lb_batch_restart(None, 0, rho, T)


@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_batch_many_items_per_cta_match_lone_runs(lb, precision):
    """More work items than persistent CTAs (each CTA takes several items from
    the global counter through its shared-memory queue, then the end mark),
    full and half items (strips at most half the kernel's width, rows split
    over the two halves of the CTA, odd and even row counts): every domain
    equals a lone single-lattice run of the same steps, FP64 bit for bit
    (both compiled without contraction, both bit-identical to the oracle);
    FP32 to a few FP32 roundings (the two kernels' units may contract
    products into fused multiply-adds differently)."""
    rng = np.random.default_rng(11)
    specs = []
    for k in range(48):
        nx = int(rng.choice([37, 64, 100, 131, 260, 300, 333]))
        ny = int(rng.integers(9, 70))
        kind = "droplet" if k % 2 else "slab"
        specs.append((nx, ny, float(rng.uniform(0.7, 1.2)), float(rng.uniform(-1.1, -0.9)), "cs",
                      float(rng.uniform(0.8, 0.92)), kind))
    setups = [domain_setup(s, O.THERMAL_EQ24) for s in specs]
    params = [lb_params_from(lb, P, precision) for _, _, P, _ in setups]
    with lb.Batch(params, [s[0] for s in setups], [s[1] for s in setups]) as B:
        lb.lb_batch_set_chunk_rows(B.b, 16)
        B.step(12)
        for d, (rho0, T0, P, _) in enumerate(setups):
            rho, T = B.fields(d)
            with lb.Lattice(rho0, T0, nx=P.nx, ny=P.ny, precision=precision, tau_f=P.tau_f, G=P.G,
                            thermal=P.thermal, beta=P.beta, psi_uses_local_T=P.psi_uses_local_T,
                            T_psi=P.T_psi, eos=P.eos, tile_x=32, tile_y=8) as L:
                L.step(12)
                m = L.moments()
            if precision == "fp64":
                assert np.array_equal(rho, m[0]) and np.array_equal(T, m[3]), (d, specs[d][:2])
            else:
                e_rho = np.abs(rho - m[0]).max() / np.abs(m[0]).max()
                e_T = np.abs(T - m[3]).max() / np.abs(m[3]).max()
                assert e_rho < 1e-6 and e_T < 1e-6, (d, specs[d][:2], e_rho, e_T)
