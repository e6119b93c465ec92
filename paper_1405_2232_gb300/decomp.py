"""One periodic lattice decomposed into y-slabs, one slab per rank (GPU).

The fused step at row y reads the post-collision populations of rows y - 2 ..
y + 2: the pull reaches one row, and the psi of the force stencil (Eq. 2/4)
at the pulled rows one more.  So a slab that owns the global rows [y0, y1)
keeps LB_HALO_ROWS = 2 ghost rows on each side: it is a context of
(y1 - y0) + 4 rows holding the global rows [y0 - 2, y1 + 2) (periodic), whose
steps update only the owned rows.  After every step each rank sends its first
two owned rows to the rank below (they become that slab's upper ghost rows)
and its last two owned rows to the rank above (its lower ghost rows), and
receives the same from its neighbours; the owned rows then evolve bit for bit
as the same rows of the whole lattice.  Per face that is every population
plane x 2 rows x the padded row width: 0.6 MB at nx = 4096 in FP32.

The exchange is written against two callables, ``pack(face) -> tensor`` and
``unpack(face, tensor)``, so that the same schedule drives the GPU slabs
(lb_halo_pack / lb_halo_unpack of the C ABI, device tensors, NCCL) and any
other row store (CPU tensors over gloo).  With world == 1 the exchange is
the periodic wrap of a single slab.

Message order: every rank posts, in this order, send(face 0 -> lower),
send(face 1 -> upper), recv(upper ghost <- upper), recv(lower ghost <- lower),
with tag 0 for messages that move down and tag 1 for messages that move up.
With two ranks the lower and the upper neighbour are the same rank; the two
messages between them then pair up in posting order (face 0 with the upper
ghost rows, face 1 with the lower ghost rows), which is also how NCCL, which
ignores tags, matches them.
"""
from __future__ import annotations

import numpy as np

HALO = 2  # ghost rows per side (LB_HALO_ROWS of include/lb.h)


def split_rows(ny: int, world: int):
    """Owned global rows [y0, y1) of each rank: contiguous, sizes differing by at
    most one row, every slab at least HALO + 1 rows (the ghost rows of a slab
    come from its two neighbours' owned rows)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    if ny < world * (HALO + 1):
        raise ValueError(f"ny = {ny} too small for {world} slabs of at least {HALO + 1} rows")
    bounds = [(r * ny) // world for r in range(world + 1)]
    return [(bounds[r], bounds[r + 1]) for r in range(world)]


def neighbours(rank: int, world: int):
    """(lower, upper) neighbour ranks of a slab on the periodic lattice."""
    return (rank - 1) % world, (rank + 1) % world


def slab_rows(field, y0: int, y1: int, halo: int = HALO):
    """Rows [y0 - halo, y1 + halo) of a global [ny, nx] field, wrapped periodically."""
    ny = field.shape[0]
    idx = np.arange(y0 - halo, y1 + halo) % ny
    return np.ascontiguousarray(field[idx])


def exchange(pack, unpack, rank: int, world: int, dist=None):
    """One ghost-row exchange of this rank's slab (see the module docstring).

    pack(face) returns this slab's first (face 0) or last (face 1) HALO owned
    rows as a tensor; unpack(face, t) writes t into the lower (face 0) or upper
    (face 1) ghost rows.  dist: torch.distributed (world > 1)."""
    down, up = pack(0), pack(1)
    if world == 1:
        # the slab is the whole periodic lattice: its first rows sit above its last
        unpack(1, down)
        unpack(0, up)
        return
    lower, upper = neighbours(rank, world)
    from_upper = down.new_empty(down.shape)
    from_lower = up.new_empty(up.shape)
    ops = [dist.P2POp(dist.isend, down, lower, tag=0),
           dist.P2POp(dist.isend, up, upper, tag=1),
           dist.P2POp(dist.irecv, from_upper, upper, tag=0),
           dist.P2POp(dist.irecv, from_lower, lower, tag=1)]
    for req in dist.batch_isend_irecv(ops):
        req.wait()
    unpack(1, from_upper)
    unpack(0, from_lower)


class SlabLattice:
    """The slab of one rank as a lattice Boltzmann context with ghost rows.

    rho, T: the GLOBAL initial fields [ny, nx] (host arrays); params: lb_params
    fields as for lb.Lattice (periodic, Eq. (7) or (24)).  step(n) advances n
    time steps, each one fused kernel launch followed by the ghost-row
    exchange.  All of this slab's device work runs on ``stream`` (a
    torch.cuda.Stream); NCCL collectives are issued under it so they follow
    the packs and precede the unpacks.
    """

    def __init__(self, rho, T, rank=0, world=1, dist=None, stream=None, **params):
        import torch
        from . import lb
        self.lb, self.torch = lb, torch
        self.rank, self.world, self.dist = rank, world, dist
        ny, nx = rho.shape
        self.y0, self.y1 = split_rows(ny, world)[rank]
        self.stream = stream if stream is not None else torch.cuda.Stream()
        local = (self.y1 - self.y0) + 2 * HALO
        self.L = lb.Lattice(slab_rows(rho, self.y0, self.y1), slab_rows(T, self.y0, self.y1),
                            stream=self.stream, nx=nx, ny=local, halo_rows=HALO, **params)
        nb = lb.lb_halo_bytes(self.L.ctx)
        dev = torch.device("cuda", torch.cuda.current_device())
        self._send = [torch.empty(nb, dtype=torch.uint8, device=dev) for _ in range(2)]

    # row store callables of the exchange
    def pack(self, face):
        self.lb.lb_halo_pack(self.L.ctx, face, self._send[face])
        return self._send[face]

    def unpack(self, face, buf):
        self.lb.lb_halo_unpack(self.L.ctx, face, buf)

    def exchange(self):
        # the receive buffers are allocated on the slab's stream, and NCCL
        # orders its sends and receives after the packs on it
        with self.torch.cuda.stream(self.stream):
            exchange(self.pack, self.unpack, self.rank, self.world, self.dist)

    def step(self, n=1):
        for _ in range(int(n)):
            self.lb.lb_step(self.L.ctx, 1)
            self.exchange()
        return self

    def owned(self, a):
        """The owned rows of a local [..., ny_local, nx] array."""
        return a[..., HALO:a.shape[-2] - HALO, :]

    def populations(self):
        f, g = self.L.populations()
        return self.owned(f), self.owned(g)

    def moments(self):
        return tuple(self.owned(m) for m in self.L.moments())

    def synchronize(self):
        self.L.synchronize()

    def close(self):
        self.L.close()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
        return False


def exchange_local(slabs):
    """The ghost-row exchange of several slabs of one lattice held by one
    process (all on one stream): every slab packs both faces, then every slab
    unpacks its neighbours' faces.  No kernel waits on another; used to run a
    decomposed lattice on one GPU."""
    world = len(slabs)
    for s in slabs:
        s.pack(0)
        s.pack(1)
    for r, s in enumerate(slabs):
        lower, upper = neighbours(r, world)
        s.unpack(1, slabs[upper]._send[0])
        s.unpack(0, slabs[lower]._send[1])


def step_local(slabs, n=1):
    """n time steps of a lattice decomposed into slabs held by one process."""
    for _ in range(int(n)):
        for s in slabs:
            s.lb.lb_step(s.L.ctx, 1)
        exchange_local(slabs)
