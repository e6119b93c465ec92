"""The throughput workload at full size, in the launch configuration the
benchmark times (4096 x 4096 spinodal quench, T = 0.75 T_c, rho = 0.12 +-
0.01, beta = 1.3, Eq. (24), the strip kernel with its production grid).

The oracle cannot step 16.8 M sites inside a test, so it steps 4096 sampled
sites one by one from the GPU's own state after 20 steps; the GPU's next step
must agree at those sites: bit for bit with FP64 storage, within the one-step
FP32 rounding bound (2e-6 of the largest population) with FP32 storage."""
import numpy as np
import pytest

import bench
import oracle as O
from paper_1405_2232_gb300 import inputs as I


@pytest.fixture(scope="module")
def lb():
    from paper_1405_2232_gb300 import lb as _lb
    _lb.load()
    return _lb


@pytest.mark.gpu
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_spinodal4096_sampled_step(lb, prec):
    p = bench.workload_params(lb, prec)
    assert (p.nx, p.ny) == (4096, 4096)
    rho, T = I.spinodal_fields(p.nx, p.ny)
    kw = {name: getattr(p, name) for name, _ in p._fields_}
    with lb.Lattice(rho, T, **kw) as L:
        used = lb.lb_get_params(L.ctx)
        assert used.tile_y == 0  # the strip kernel, as in the benchmark
        L.step(20)
        f, g = L.populations()
        L.step(1)
        f1, g1 = L.populations()
        L.synchronize()
    P = O.params(p.nx, p.ny, tau_f=p.tau_f, tau_g=p.tau_g, G=p.G, beta=p.beta, eos=O.EOS_CS,
                 a=p.a, b=p.b, R=p.R, cv=p.cv, thermal=O.THERMAL_EQ24,
                 psi_uses_local_T=p.psi_uses_local_T, T_psi=p.T_psi)
    sites = np.sort(np.random.default_rng(11).choice(p.nx * p.ny, 4096, replace=False))
    # include the lattice corners and strip / chunk seams
    extra = np.array([0, p.nx - 1, (p.ny - 1) * p.nx, p.nx * p.ny - 1, 255, 256, 256 * p.nx + 511])
    sites = np.unique(np.concatenate([sites, extra]))
    of, og = O.step_sites(P, f, g, sites)
    gf = f1.reshape(9, -1)[:, sites].T
    gg = g1.reshape(9, -1)[:, sites].T
    if prec == "fp64":
        assert np.array_equal(of, gf) and np.array_equal(og, gg)
    else:
        assert np.abs(gf - of).max() <= 2e-6 * np.abs(of).max()
        assert np.abs(gg - og).max() <= 2e-6 * np.abs(og).max()
