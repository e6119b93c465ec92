"""Failure detection on the GPU, without faulting it: the device error word
reports a non-finite state planted from the host, and a bounded wait of the
strip kernels that is made to run out returns LB_ERR_TIMEOUT with the context
still usable afterwards.

Nothing here traps, hangs or faults the device: the NaN is ordinary data, and
the timeout is the kernels' own bounded mbarrier wait given a limit of one
clock cycle (the copies already issued are still waited for, with the default
limit, before a CTA leaves)."""
import numpy as np
import pytest

from paper_1405_2232_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lb():
    import torch  # noqa: F401  (initialises CUDA in this process)
    from paper_1405_2232_gb300 import lb as _lb
    _lb.load()
    return _lb


def lattice(lb, nx, ny, precision, tile=(0, 0), thermal=None, beta=1.0):
    rho, T = I.slab_fields(nx, ny, width=nx // 2, noise=1e-3)
    return lb.Lattice(rho, T, nx=nx, ny=ny, precision=precision, tile_x=tile[0], tile_y=tile[1],
                      beta=beta, thermal=lb.LB_THERMAL_EQ24 if thermal is None else thermal)


@pytest.mark.parametrize("precision,tile", [("fp32", (256, 0)), ("fp32", (32, 8)), ("fp64", (128, 0)),
                                            ("fp16", (256, 0)), ("bf16", (32, 8))])
def test_nan_population_reports_nonfinite(lb, precision, tile):
    """A NaN written into one population through lb_set_populations: the next
    step's moments are non-finite at that site and the step reports
    LB_ERR_NONFINITE; after valid populations are set again the context steps on."""
    with lattice(lb, 512, 40, precision, tile) as L:
        L.step(5)
        L.synchronize()
        f, g = L.populations()
        good_f, good_g = f.copy(), g.copy()
        f[3, 17, 200] = np.nan
        L.set_populations(f, g)
        L.step(1)
        with pytest.raises(lb.LbError) as ei:
            L.synchronize()
        assert ei.value.status == lb.LB_ERR_NONFINITE
        L.synchronize()  # the error word was cleared by the report
        L.set_populations(good_f, good_g)
        L.step(3)
        L.synchronize()
        assert np.all(np.isfinite(L.moments()[0]))


@pytest.mark.parametrize("precision,thermal", [("fp32", None), ("fp64", None), ("fp16", None),
                                               ("fp32", "fd")])
def test_bounded_wait_times_out_and_context_recovers(lb, precision, thermal):
    """With a one-cycle limit the strip kernel's first mbarrier wait gives up:
    lb_synchronize reports LB_ERR_TIMEOUT.  With the default limit restored and
    the state put back, the context steps on bit for bit like an untouched one."""
    th = lb.LB_THERMAL_FD26 if thermal == "fd" else None
    nx, ny = 512, 64
    with lattice(lb, nx, ny, precision, thermal=th) as L, lattice(lb, nx, ny, precision, thermal=th) as R:
        assert lb.lb_get_params(L.ctx).tile_y == 0  # the strip kernel runs
        L.step(4)
        R.step(4)
        L.synchronize()
        if th is None:
            blob = lb.lb_save_state(L.ctx)
        lb.lb_set_wait_limit(L.ctx, 1)
        L.step(1)
        with pytest.raises(lb.LbError) as ei:
            L.synchronize()
        assert ei.value.status == lb.LB_ERR_TIMEOUT
        lb.lb_set_wait_limit(L.ctx, 0)
        if th is None:
            lb.lb_load_state(L.ctx, blob)
            L.step(10)
            R.step(10)
            fl, gl = L.populations()
            fr, gr = R.populations()
            assert np.array_equal(fl, fr) and np.array_equal(gl, gr)
        else:
            # the FD context has no population state calls: it just steps on
            L.step(10)
            L.synchronize()
            assert np.all(np.isfinite(L.moments()[0]))
    with pytest.raises(lb.LbError):
        lb.lb_set_wait_limit(None, 1)
