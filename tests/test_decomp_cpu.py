"""The y-slab decomposition of one lattice (paper_1405_2232_gb300/decomp.py) on
CPU ranks over gloo (127.0.0.1): the row split, the slab fields with their
ghost rows, and the ghost-row exchange schedule.

Each rank steps its slab (owned rows plus two ghost rows per side, periodic
in its own rows) with the FP64 oracle, then runs the product's exchange; after
K steps the owned rows of all ranks, put together, must equal the oracle's run
of the whole lattice BIT FOR BIT.  The oracle holds pre-collision populations
at their site and streams inside its step; the rows a slab needs from its
neighbours are the same two rows per face as on the GPU, so the exchange is
the same.  One, two (lower and upper neighbour the same rank) and three ranks,
with uneven slabs."""
import json
import os
import socket

import numpy as np
import pytest

import oracle as O
from paper_1405_2232_gb300 import decomp as D
from paper_1405_2232_gb300 import inputs as I

NX, NY, STEPS = 40, 23, 30


def global_case():
    rho, _ = I.droplet_fields(NX, NY, 6, rho_l=0.3, rho_g=0.04)
    rho = rho + I.site_noise(7, NX, NY, 1e-3)   # structure along y at every x
    T = np.full((NY, NX), 0.85 * I.CS_TC) + I.site_noise(8, NX, NY, 1e-4)
    return np.ascontiguousarray(rho), np.ascontiguousarray(T)


def params(ny):
    return O.params(NX, ny, tau_f=1.0, tau_g=0.8, G=-1.0, beta=1.0, eos=O.EOS_CS, a=1.0, b=4.0, R=1.0,
                    thermal=O.THERMAL_EQ24)


def run_slab(rank, world, dist):
    """Step this rank's slab with the oracle and the product exchange; returns
    its owned rows of (f, g)."""
    import torch
    rho, T = global_case()
    y0, y1 = D.split_rows(NY, world)[rank]
    ny_loc = (y1 - y0) + 2 * D.HALO
    P = params(ny_loc)
    f, g = O.init_equilibrium(P, D.slab_rows(rho, y0, y1), D.slab_rows(T, y0, y1))
    h = D.HALO
    state = {"f": f, "g": g}

    def pack(face):
        rows = slice(h, 2 * h) if face == 0 else slice(ny_loc - 2 * h, ny_loc - h)
        return torch.from_numpy(np.concatenate([state["f"][:, rows], state["g"][:, rows]]).copy())

    def unpack(face, t):
        rows = slice(0, h) if face == 0 else slice(ny_loc - h, ny_loc)
        a = t.numpy()
        state["f"][:, rows] = a[:9]
        state["g"][:, rows] = a[9:]

    for _ in range(STEPS):
        state["f"], state["g"], _ = O.step(P, state["f"], state["g"], n=1, check=False)
        D.exchange(pack, unpack, rank, world, dist)
    return state["f"][:, h:ny_loc - h], state["g"][:, h:ny_loc - h]


def _worker(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        f, g = run_slab(rank, world, dist)
        np.save(os.path.join(out_dir, f"f{rank}.npy"), f)
        np.save(os.path.join(out_dir, f"g{rank}.npy"), g)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.fixture(scope="module")
def whole_lattice():
    rho, T = global_case()
    P = params(NY)
    f, g = O.init_equilibrium(P, rho, T)
    f, g, st = O.step(P, f, g, n=STEPS)
    assert st == O.OK
    return f, g


def test_split_rows_covers_the_lattice():
    for ny, world in ((23, 1), (23, 2), (23, 3), (4096, 8), (9, 3)):
        parts = D.split_rows(ny, world)
        assert parts[0][0] == 0 and parts[-1][1] == ny
        assert all(a[1] == b[0] for a, b in zip(parts, parts[1:]))
        sizes = [b - a for a, b in parts]
        assert max(sizes) - min(sizes) <= 1 and min(sizes) >= D.HALO + 1
    with pytest.raises(ValueError):
        D.split_rows(8, 3)
    assert D.neighbours(0, 3) == (2, 1) and D.neighbours(2, 3) == (1, 0) and D.neighbours(0, 1) == (0, 0)


def test_slab_rows_wrap_periodically():
    a = np.arange(7 * 3).reshape(7, 3)
    s = D.slab_rows(a, 0, 3)
    assert np.array_equal(s[:2], a[5:7]) and np.array_equal(s[2:5], a[0:3]) and np.array_equal(s[5:], a[3:5])


def test_single_slab_exchange_is_the_periodic_lattice(whole_lattice):
    f, g = run_slab(0, 1, None)
    assert np.array_equal(f, whole_lattice[0]) and np.array_equal(g, whole_lattice[1])


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_ranks_step_a_decomposed_lattice_bit_for_bit(tmp_path, whole_lattice, world):
    pytest.importorskip("torch")
    import torch.multiprocessing as mp
    mp.start_processes(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    f = np.concatenate([np.load(tmp_path / f"f{r}.npy") for r in range(world)], axis=1)
    g = np.concatenate([np.load(tmp_path / f"g{r}.npy") for r in range(world)], axis=1)
    assert f.shape == whole_lattice[0].shape
    assert np.array_equal(f, whole_lattice[0]) and np.array_equal(g, whole_lattice[1])


def test_a_wrong_exchange_is_caught(whole_lattice):
    """The test is sensitive to the exchange: a schedule that swaps the faces
    (the first owned rows sent up instead of down) breaks the bit-for-bit match."""
    def swapped(pack, unpack, rank, world, dist=None):
        down, up = pack(0), pack(1)
        unpack(0, down)
        unpack(1, up)
    orig = D.exchange
    D.exchange = swapped
    try:
        f, g = run_slab(0, 1, None)
    finally:
        D.exchange = orig
    assert not np.array_equal(f, whole_lattice[0])
