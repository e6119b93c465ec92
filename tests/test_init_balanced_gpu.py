"""The start at rest under the force (lb_params.init_balanced) against the FP64
oracle's init_balanced, through the C ABI.

FP64 populations are compared bit for bit (context tile and strip layouts,
ragged lattices, three force forms, batched domains), FP32 as the one
rounding of the FP64 value, the 16-bit modes within the rounding of the
stored deviation; the moments of the start have zero velocity; the state
after 200 steps from it matches the oracle bit for bit (FP64)."""
import numpy as np
import pytest

import oracle as O
from paper_1405_2232_gb300 import inputs as I


@pytest.fixture(scope="module")
def lb():
    import torch  # noqa: F401  (initialises CUDA in this process)
    from paper_1405_2232_gb300 import lb as _lb
    _lb.load()
    return _lb


def _fields(kind, nx, ny):
    if kind == "slab":
        rg, rl = I.coexistence_densities(0.8)
        rho, _ = I.slab_fields(nx, ny, width=2 * (nx // 5), rho_l=rl, rho_g=rg, noise=1e-3)
        return rho, np.full((ny, nx), 0.8 * I.CS_TC)
    return I.droplet_fields(nx, ny, min(nx, ny) / 4, rho_l=0.3, rho_g=0.05, T_lo=0.85, T_hi=0.9)


# (name, kind, nx, ny, beta, psi_local, tile)
CASES = [
    ("slab_mixed_passive_tile", "slab", 45, 37, 1.3, 0, (32, 8)),
    ("droplet_beta1_local_tile", "droplet", 41, 33, 1.0, 1, (0, 0)),
    ("droplet_beta0_local_tile", "droplet", 40, 36, 0.0, 1, (32, 8)),
    ("slab_mixed_passive_strip", "slab", 130, 37, 1.3, 0, (128, 0)),
]


def _oracle(kind, nx, ny, beta, psi_local):
    rho, T = _fields(kind, nx, ny)
    T_psi = 0.8 * I.CS_TC if not psi_local else 0.0
    P = O.params(nx, ny, tau_f=0.9, tau_g=0.8, G=-1.0, beta=beta, eos=O.EOS_CS, a=1.0, b=4.0, R=1.0,
                 thermal=O.THERMAL_EQ24, psi_uses_local_T=psi_local, T_psi=T_psi)
    return rho, T, P


def _lattice(lb, rho, T, P, precision, tile):
    return lb.Lattice(rho, T, nx=P.nx, ny=P.ny, tau_f=P.tau_f, tau_g=P.tau_g, G=P.G, beta=P.beta,
                      eos=P.eos, a=P.a, b=P.b, R=P.R, cv=P.cv, thermal=P.thermal,
                      precision=lb.PRECISIONS[precision], psi_uses_local_T=P.psi_uses_local_T,
                      T_psi=P.T_psi, tile_x=tile[0], tile_y=tile[1], init_balanced=1)


@pytest.mark.gpu
@pytest.mark.parametrize("name,kind,nx,ny,beta,psi_local,tile", CASES, ids=[c[0] for c in CASES])
def test_fp64_start_bit_identical(lb, name, kind, nx, ny, beta, psi_local, tile):
    rho, T, P = _oracle(kind, nx, ny, beta, psi_local)
    f_ref, g_ref, st = O.init_balanced(P, rho, T)
    assert st == O.OK
    L = _lattice(lb, rho, T, P, "fp64", tile)
    f, g = L.populations()
    assert np.array_equal(f, f_ref) and np.array_equal(g, g_ref)
    # at rest: the moments the step computes have u = 0 to rounding
    r, ux, uy, Tm = L.moments()
    Fx_ref = O.moments(P, f_ref, g_ref)[4]
    scale = max(np.abs(Fx_ref / rho).max(), 1e-30)
    assert max(np.abs(ux).max(), np.abs(uy).max()) <= 1e-12 * scale
    # and the step from it is the oracle's step
    L.step(200)
    L.synchronize()
    f_ref, g_ref, _ = O.step(P, f_ref, g_ref, n=200, check=False)
    f, g = L.populations()
    assert np.array_equal(f, f_ref) and np.array_equal(g, g_ref)
    m = O.moments(P, f_ref, g_ref)
    r, ux, uy, Tm = L.moments()
    assert np.abs(r - m[0]).max() <= 1e-12 * np.abs(m[0]).max()
    assert np.abs(Tm - m[3]).max() <= 1e-12 * np.abs(m[3]).max()
    umax = max(np.abs(m[1]).max(), np.abs(m[2]).max())
    assert max(np.abs(ux - m[1]).max(), np.abs(uy - m[2]).max()) <= 1e-12 * umax


@pytest.mark.gpu
@pytest.mark.parametrize("tile", [(0, 0), (32, 8)])
def test_fp32_start_one_rounding(lb, tile):
    rho, T, P = _oracle("slab", 64, 24, 1.3, 0)
    f_ref, g_ref, _ = O.init_balanced(P, rho, T)
    L = _lattice(lb, rho, T, P, "fp32", tile)
    f, g = L.populations()
    assert np.all(f == f_ref.astype(np.float32).astype(np.float64))
    assert np.all(g == g_ref.astype(np.float32).astype(np.float64))


@pytest.mark.gpu
@pytest.mark.parametrize("prec,tol", [("fp16", 2.0 ** -11), ("bf16", 2.0 ** -8)])
def test_16bit_start_within_deviation_rounding(lb, prec, tol):
    rho, T, P = _oracle("droplet", 48, 40, 1.0, 1)
    f_ref, g_ref, _ = O.init_balanced(P, rho, T)
    L = lb.Lattice(rho, T, nx=48, ny=40, tau_f=0.9, tau_g=0.8, G=-1.0, beta=1.0,
                   precision=lb.PRECISIONS[prec], rho0=0.15, T0=0.87 * I.CS_TC, init_balanced=1)
    f, g = L.populations()
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)[:, None, None]
    dev_f = np.abs(f_ref - w * 0.15)
    dev_g = np.abs(g_ref - w * 0.15 * 0.87 * I.CS_TC)
    # one 16-bit rounding of the deviation, plus the FP32 roundings of the value
    # and of the base (and fp16's subnormal spacing)
    assert np.all(np.abs(f - f_ref) <= tol * dev_f + 4e-8 * np.abs(f_ref) + 6e-8)
    assert np.all(np.abs(g - g_ref) <= tol * dev_g + 4e-8 * np.abs(g_ref) + 6e-8)


@pytest.mark.gpu
def test_start_reports_psi_domain(lb):
    rho = np.full((16, 32), 0.2)
    rho[5, 5] = 0.9
    T = np.full((16, 32), 0.09)
    L = lb.Lattice(rho, T, nx=32, ny=16, precision=lb.PRECISIONS["fp64"], beta=1.0, init_balanced=1)
    with pytest.raises(lb.LbError) as exc:
        L.synchronize()
    assert exc.value.status == lb.LB_ERR_PSI_DOMAIN


@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_batch_start_per_domain(lb, precision):
    """Batched domains with and without the start at rest evolve as the oracle
    does from the same start (FP64 bit for bit, FP32 within 2e-5 after 40 steps)."""
    specs = [("slab", 64, 20, 1), ("droplet", 48, 48, 0), ("slab", 132, 17, 1), ("droplet", 36, 28, 1)]
    setups = []
    for kind, nx, ny, bal in specs:
        rho, T, P = _oracle(kind, nx, ny, 1.3, 0)
        setups.append((rho, T, P, bal))
    params = [lb.lb_params_default(nx=P.nx, ny=P.ny, tau_f=P.tau_f, tau_g=P.tau_g, G=P.G, beta=P.beta,
                                   precision=lb.PRECISIONS[precision], psi_uses_local_T=0, T_psi=P.T_psi,
                                   init_balanced=bal) for _, _, P, bal in setups]
    with lb.Batch(params, [s[0] for s in setups], [s[1] for s in setups]) as B:
        B.step(40)
        for d, (rho0, T0, P, bal) in enumerate(setups):
            if bal:
                f, g, _ = O.init_balanced(P, rho0, T0)
            else:
                f, g = O.init_equilibrium(P, rho0, T0)
            f, g, _ = O.step(P, f, g, n=40, check=False)
            m = O.moments(P, f, g)
            rho, T = B.fields(d)
            if precision == "fp64":
                assert np.array_equal(rho, m[0]) and np.array_equal(T, m[3]), d
            else:
                e_rho = np.abs(rho - m[0]).max() / np.abs(m[0]).max()
                e_T = np.abs(T - m[3]).max() / np.abs(m[3]).max()
                assert e_rho < 2e-5 and e_T < 2e-5, (d, e_rho, e_T)
