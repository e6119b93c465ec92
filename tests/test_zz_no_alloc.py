"""The allocation-free totals entry point (lb_field_totals_noalloc), called
through the C ABI, against the context-based lb_totals.

Callers that must not have device memory allocated for them (allocation-free
stream capture, their own memory pools, fixed memory budgets) use the variant
whose scratch is a static device array.  This file is collected last so that a
failure here leaves every other test already run; it must pass both alone in a
fresh process and after the other tests (the scratch keeps the previous call's
contents)."""
import numpy as np
import pytest

from paper_1405_2232_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def test_noalloc_totals_match_lb_totals_two_calls():
    import torch
    from paper_1405_2232_gb300 import lb
    torch.cuda.set_device(0)
    lb.load()
    nx, ny = 192, 96
    rho, T = I.slab_fields(nx, ny, width=64)
    stream = torch.cuda.Stream()
    L = lb.Lattice(rho, T, stream=stream, nx=nx, ny=ny, precision="fp64",
                   thermal=lb.LB_THERMAL_EQ24)
    try:
        f = lambda: torch.empty((ny, nx), dtype=torch.float64, device="cuda")
        ref = [f() for _ in range(4)]
        cur = [f() for _ in range(4)]
        L.step(100)
        lb.lb_moments_device(L.ctx, *ref)
        t_ref = L.totals()              # lb_totals keeps (rho, T) at t = 100
        L.step(50)
        lb.lb_moments_device(L.ctx, *cur)
        expect = L.totals()             # residual over K = 50 steps
        L.synchronize()
        for call in range(2):           # twice in a row: the shared scratch is reused
            out = torch.full((lb.LB_TOTALS_N,), float("nan"), dtype=torch.float64, device="cuda")
            torch.cuda.synchronize()    # the fill ran on torch's stream
            lb.lb_field_totals_noalloc(nx, ny, 1.0, cur[0], cur[1], cur[2], cur[3], out,
                                       d_ref_rho=ref[0], d_ref_T=ref[3], K=50, stream=stream)
            stream.synchronize()
            got = out.cpu().numpy()
            assert got[0] == pytest.approx(expect[0], rel=1e-12), call
            assert got[1] == pytest.approx(expect[1], rel=1e-12), call
            assert abs(got[2] - expect[2]) <= 1e-12 * expect[0], call
            assert abs(got[3] - expect[3]) <= 1e-12 * expect[0], call
            assert got[4] == pytest.approx(expect[4], rel=1e-9), call
        assert t_ref[0] == pytest.approx(expect[0], rel=1e-13)  # mass conserved meanwhile
        # no reference fields: residual is zero, the rest unchanged
        out = torch.zeros(lb.LB_TOTALS_N, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        lb.lb_field_totals_noalloc(nx, ny, 1.0, cur[0], cur[1], cur[2], cur[3], out, stream=stream)
        stream.synchronize()
        got = out.cpu().numpy()
        assert got[4] == 0.0 and got[0] == pytest.approx(expect[0], rel=1e-12)
        # beyond the stated maximum: a clear error from the library itself, nothing
        # launched (called through ctypes directly: the binding would already
        # refuse these tensors as too small for 4097 x 4096 sites)
        import ctypes
        so = lb.load()
        st = so.lb_field_totals_noalloc(4097, 4096, 1.0, *[ctypes.c_void_p(t.data_ptr()) for t in cur],
                                        None, None, 0, ctypes.c_void_p(out.data_ptr()),
                                        ctypes.c_void_p(stream.cuda_stream))
        assert st == lb.LB_ERR_ARG and "limit" in lb.lb_last_error()
    finally:
        L.close()


def test_noalloc_totals_full_scratch_no_device_memory_change():
    """A 4096 x 4096 lattice fills every slot of the static scratch (4096 CTAs of
    4096 sites).  Its totals match lb_totals of the same state on two calls in a
    row, the free device memory reported by the driver is the same before and
    after those calls (nothing is allocated), and the caller's current device is
    unchanged."""
    import torch
    from paper_1405_2232_gb300 import lb
    torch.cuda.set_device(0)
    lb.load()
    n = 4096
    rho, T = I.spinodal_fields(n, n)
    stream = torch.cuda.Stream()
    # FP64 storage: the moments lb_totals sums are then exactly the fields handed over
    L = lb.Lattice(rho, T, stream=stream, nx=n, ny=n, precision="fp64", beta=1.3,
                   thermal=lb.LB_THERMAL_EQ24)
    try:
        fields = [torch.empty((n, n), dtype=torch.float64, device="cuda") for _ in range(6)]
        torch.cuda.synchronize()
        L.step(10)
        lb.lb_moments_device(L.ctx, fields[4], None, None, fields[5])  # reference at t = 10
        L.totals()
        L.step(20)
        lb.lb_moments_device(L.ctx, *fields[:4])
        expect = L.totals()                # residual over K = 20 steps
        L.synchronize()
        outs = [torch.full((lb.LB_TOTALS_N,), float("nan"), dtype=torch.float64, device="cuda")
                for _ in range(2)]
        torch.cuda.synchronize()
        # set-up call (the first call on a device may load the library's device code)
        lb.lb_field_totals_noalloc(n, n, 1.0, *fields[:4], outs[0], d_ref_rho=fields[4],
                                   d_ref_T=fields[5], K=20, stream=stream)
        stream.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        for out in outs:                   # two calls in a row on the same scratch
            lb.lb_field_totals_noalloc(n, n, 1.0, *fields[:4], out, d_ref_rho=fields[4],
                                       d_ref_T=fields[5], K=20, stream=stream)
        stream.synchronize()
        free1 = torch.cuda.mem_get_info()[0]
        assert free1 == free0, (free0, free1)
        assert torch.cuda.current_device() == 0
        for out in outs:
            got = out.cpu().numpy()
            assert got[0] == pytest.approx(expect[0], rel=1e-12)
            assert got[1] == pytest.approx(expect[1], rel=1e-12)
            assert abs(got[2] - expect[2]) <= 1e-12 * expect[0]
            assert abs(got[3] - expect[3]) <= 1e-12 * expect[0]
            assert got[4] == pytest.approx(expect[4], rel=1e-9) and got[4] > 0
    finally:
        L.close()
