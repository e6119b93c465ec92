"""Two fused time steps per launch (the FP32 two-step strip kernel) against
single steps: bit-identical populations for odd and even step counts, ragged
and narrow strips, both temperature treatments and every force form."""
import numpy as np
import pytest

from paper_1405_2232_gb300 import inputs as I


@pytest.fixture(scope="module")
def lb():
    from paper_1405_2232_gb300 import lb as _lb
    _lb.load()
    return _lb


def run(lb, rho, T, n, fusion, **kw):
    with lb.Lattice(rho, T, precision="fp32", step_fusion=fusion, **kw) as L:
        L.step(n)
        f, g = L.populations()
    return f, g


CASES = [
    dict(thermal=1, beta=1.0),
    dict(thermal=0, beta=1.0, psi_uses_local_T=0, T_psi=0.85 * I.CS_TC),
    dict(thermal=1, beta=1.3),
    dict(thermal=1, beta=0.0),
]


@pytest.mark.gpu
@pytest.mark.parametrize("nx,ny", [(64, 64), (8, 12), (132, 17), (260, 33), (244, 70), (4, 9)])
@pytest.mark.parametrize("case", range(len(CASES)))
def test_two_step_fusion_is_bit_identical(lb, nx, ny, case):
    kw = CASES[case]
    # beta = 0 (psi^2 form) gets a milder contrast: it diverges on the narrowest slabs
    rl, rg = (0.3, 0.04) if kw["beta"] != 0.0 else (0.2, 0.08)
    rho, T = I.slab_fields(nx, ny, width=max(2, nx // 2), rho_l=rl, rho_g=rg, noise=1e-3)
    for n in (2, 21):
        f1, g1 = run(lb, rho, T, n, 1, nx=nx, ny=ny, **kw)
        f2, g2 = run(lb, rho, T, n, 0, nx=nx, ny=ny, **kw)
        assert np.array_equal(f1, f2, equal_nan=True) and np.array_equal(g1, g2, equal_nan=True), (nx, ny, case, n)
        assert np.all(np.isfinite(f1)), (nx, ny, case, n)


@pytest.mark.gpu
def test_two_step_fusion_spinodal_1024(lb):
    rho, T = I.spinodal_fields(1024, 1024)
    kw = dict(nx=1024, ny=1024, beta=1.3, rho0=0.12, T0=0.75 * I.CS_TC)
    f1, g1 = run(lb, rho, T, 40, 1, **kw)
    f2, g2 = run(lb, rho, T, 40, 0, **kw)
    assert np.array_equal(f1, f2) and np.array_equal(g1, g2)


@pytest.mark.gpu
def test_invalid_fusion_value(lb):
    rho, T = I.slab_fields(16, 12)
    with pytest.raises(lb.LbError):
        lb.Lattice(rho, T, nx=16, ny=12, step_fusion=2)
