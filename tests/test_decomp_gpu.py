"""One lattice decomposed into y-slabs (ghost-row contexts, lb_halo_pack /
lb_halo_unpack) on the GPU, against the same lattice run whole.

The slabs of the decomposition are held by one process on one stream (one
GPU); their exchange is device copies between the contexts, issued in order
on that stream, so no kernel waits on another.  After every step the owned
rows of every slab must equal the same rows of the whole lattice BIT FOR BIT
in every storage mode (the per-site arithmetic of a slab is that of the
whole lattice's kernel)."""
import numpy as np
import pytest

from paper_1405_2232_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    import torch  # noqa: F401
    from paper_1405_2232_gb300 import decomp as D
    from paper_1405_2232_gb300 import lb
    lb.load()
    return lb, D


def case(nx, ny):
    rho, _ = I.droplet_fields(nx, ny, min(nx, ny) // 5, rho_l=0.3, rho_g=0.04)
    rho = rho + I.site_noise(7, nx, ny, 1e-3)
    T = np.full((ny, nx), 0.85 * I.CS_TC) + I.site_noise(8, nx, ny, 1e-4)
    return np.ascontiguousarray(rho), np.ascontiguousarray(T)


@pytest.mark.parametrize("prec,tile,shape,world", [
    ("fp64", (128, 0), (67, 260), 2),
    ("fp64", (128, 0), (67, 260), 3),
    ("fp64", (32, 8), (45, 70), 3),
    ("fp32", (256, 0), (96, 515), 2),
    ("fp32", (256, 0), (96, 515), 5),
    ("bf16", (256, 0), (64, 512), 3),
    ("fp16", (32, 8), (40, 72), 2),
])
def test_slabs_match_the_whole_lattice(mods, prec, tile, shape, world):
    import torch
    lb, D = mods
    ny, nx = shape
    rho, T = case(nx, ny)
    kw = dict(precision=prec, tile_x=tile[0], tile_y=tile[1], thermal=lb.LB_THERMAL_EQ24,
              rho0=0.12, T0=0.85 * I.CS_TC)
    stream = torch.cuda.Stream()
    slabs = [D.SlabLattice(rho, T, rank=r, world=world, stream=stream, **kw) for r in range(world)]
    try:
        with lb.Lattice(rho, T, nx=nx, ny=ny, **kw) as W:
            assert (lb.lb_get_params(W.ctx).tile_x, lb.lb_get_params(W.ctx).tile_y) == tile
            for n in (1, 39):
                W.step(n)
                D.step_local(slabs, n)
                fw, gw = W.populations()
                parts = [s.populations() for s in slabs]
                f = np.concatenate([p[0] for p in parts], axis=1)
                g = np.concatenate([p[1] for p in parts], axis=1)
                assert np.array_equal(f, fw) and np.array_equal(g, gw), n
            mw = W.moments()
            ms = [s.moments() for s in slabs]
            for k in range(4):
                assert np.array_equal(np.concatenate([m[k] for m in ms], axis=0), mw[k])
            for s in slabs:
                s.synchronize()
    finally:
        for s in slabs:
            s.close()


def test_single_slab_exchanges_with_itself(mods):
    """world = 1: the exchange is the periodic wrap; the slab steps as the lattice."""
    lb, D = mods
    rho, T = case(256, 40)
    kw = dict(precision="fp32", thermal=lb.LB_THERMAL_EQ24)
    with D.SlabLattice(rho, T, **kw) as S, lb.Lattice(rho, T, nx=256, ny=40, **kw) as W:
        S.step(25)
        W.step(25)
        fs, gs = S.populations()
        fw, gw = W.populations()
    assert np.array_equal(fs, fw) and np.array_equal(gs, gw)


def test_ghost_rows_are_needed(mods):
    """Without the exchange the slabs drift away from the whole lattice: the
    ghost rows carry information the owned rows need every step."""
    import torch
    lb, D = mods
    rho, T = case(128, 30)
    kw = dict(precision="fp64", thermal=lb.LB_THERMAL_EQ24)
    stream = torch.cuda.Stream()
    slabs = [D.SlabLattice(rho, T, rank=r, world=2, stream=stream, **kw) for r in range(2)]
    try:
        with lb.Lattice(rho, T, nx=128, ny=30, **kw) as W:
            W.step(5)
            for s in slabs:
                lb.lb_step(s.L.ctx, 5)  # no exchange
            fw, _ = W.populations()
            f = np.concatenate([s.populations()[0] for s in slabs], axis=1)
        assert not np.array_equal(f, fw)
    finally:
        for s in slabs:
            s.close()
