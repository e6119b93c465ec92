"""Autotuner on the GPU: the chosen shape is the fastest measured one, shapes
that do not apply are skipped, a tuned lattice gives the same results, and
tuning a batch leaves its state untouched."""
import math

import numpy as np
import pytest

import oracle as O
from paper_1405_2232_gb300 import autotune as A
from paper_1405_2232_gb300 import inputs as I


@pytest.fixture(scope="module")
def lb():
    from paper_1405_2232_gb300 import lb as _lb
    _lb.load()
    return _lb


@pytest.mark.gpu
@pytest.mark.parametrize("prec,nx,ny,invalid", [
    ("fp32", 512, 256, []),
    ("fp64", 256, 128, [0]),          # the FP64 strip kernel is 128 wide only
    ("fp32", 130, 64, []),            # any nx: the strip kernel's row copies are rounded up
    ("bf16", 1024, 512, []),
])
def test_autotune_picks_the_fastest_valid_shape(lb, prec, nx, ny, invalid):
    p = lb.lb_params_default(nx=nx, ny=ny, precision=prec, beta=1.3, psi_uses_local_T=0,
                             T_psi=0.075)
    best, ms = lb.lb_autotune(p, 6)
    for k in range(lb.LB_TUNE_N):
        assert math.isnan(ms[k]) == (k in invalid), (k, ms)
    k_best = int(np.nanargmin(ms))
    assert (best.tile_x, best.tile_y) == lb.lb_tune_candidate(k_best)
    assert best.nx == nx and best.precision == p.precision and best.beta == 1.3


@pytest.mark.gpu
def test_tuned_lattice_matches_default_bit_for_bit(lb, tmp_path):
    rho, T = I.slab_fields(96, 64)
    p = lb.lb_params_default(nx=96, ny=64, precision="fp64")
    q = A.tuned_params(p, A.TuneCache(str(tmp_path / "t.json")), steps=4)
    out = []
    for par in (p, q):
        with lb.Lattice(rho, T, **{n: getattr(par, n) for n, _ in par._fields_}) as L:
            L.step(50)
            out.append(L.populations())
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


@pytest.mark.gpu
def test_batch_autotune_restores_state(lb):
    specs = [(64, 48), (132, 36), (256, 200), (36, 260)]
    params, rhos, Ts = [], [], []
    for k, (nx, ny) in enumerate(specs):
        rho, T = I.droplet_fields(nx, ny, min(nx, ny) // 4, rho_l=0.3, rho_g=0.04)
        params.append(lb.lb_params_default(nx=nx, ny=ny, precision="fp64", tau_f=0.8 + 0.1 * k,
                                           psi_uses_local_T=0, T_psi=0.085))
        rhos.append(rho)
        Ts.append(np.full((ny, nx), 0.085))
    with lb.Batch(params, rhos, Ts) as A_, lb.Batch(params, rhos, Ts) as B_:
        A_.step(10)
        B_.step(10)
        before = [A_.fields(d) for d in range(len(specs))]
        rows, ms = A_.autotune(4)
        assert rows in (16, 32, 64, 128) and A_.chunk_rows == rows
        assert np.all(np.isfinite(ms)) and ms[[16, 32, 64, 128].index(rows)] == ms.min()
        assert A_.time == 10
        after = [A_.fields(d) for d in range(len(specs))]
        for (r0, t0), (r1, t1) in zip(before, after):
            assert np.array_equal(r0, r1) and np.array_equal(t0, t1)
        A_.step(30)
        B_.step(30)
        for d in range(len(specs)):
            (ra, ta), (rb, tb) = A_.fields(d), B_.fields(d)
            assert np.array_equal(ra, rb) and np.array_equal(ta, tb), d
        A_.chunk_rows = 16
        A_.step(2)
        B_.step(2)
        for d in range(len(specs)):
            assert np.array_equal(A_.fields(d)[0], B_.fields(d)[0]), d
