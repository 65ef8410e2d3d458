"""Z-split of one slab over ranks (domain decomposition).

The EV-FDLB stage is an explicit stencil in z (Sec. III): a node reads F and
G over +-3 nodes (the WENO-5 face fluxes) and the density over +-M nodes
(the Eq. (F1) force integral, M = r_cut / dz for EV1).  A slab of nz nodes
therefore splits into contiguous parts, one per rank; each rank keeps its
part plus G ghost nodes per side (G = ``halo_width``) and, before every RK
stage, swaps one message per side with each neighbour: on a ring for a
periodic slab, on a line for an outflow slab, whose first and last parts
keep no ghost band at the slab's ends (those ends are its outflow
boundaries).  The interior nodes then evolve bit-identically to the unsplit
slab.

The pieces:

* ``partition`` / ``local_slice``: which nodes a rank owns and the periodic
  slice (interior plus ghosts) of a global field it starts from.
* ``HaloDriver``: the order of a step -- stage, exchange, three times -- over
  an *engine* (``stage(s)``, ``pack()``, ``unpack(from_left, from_right)``)
  and an *exchange* (``(to_left, to_right) -> (from_left, from_right)``).
* ``CudaSlabPart``: the engine on the CUDA library (a context with
  ``bc = BC_HALO``; pack / unpack / stage are its kernels).
* ``DistExchange``: the exchange over ``torch.distributed`` point-to-point
  (NCCL for CUDA tensors, gloo for CPU tensors), no collective.
* ``step_lockstep``: several parts advanced in one process (the exchange a
  plain routing of the packed messages), for a split that runs on one device.
"""
from __future__ import annotations

import dataclasses

import numpy as np


def partition(nz: int, world: int, G: int):
    """Contiguous parts (start, count) of nz nodes over world ranks, counts
    differing by at most one; every part must hold at least G nodes so that
    a neighbour's ghosts come from one rank."""
    if world < 1 or nz < world:
        raise ValueError("need 1 <= world <= nz")
    base, extra = divmod(nz, world)
    parts, start = [], 0
    for r in range(world):
        count = base + (1 if r < extra else 0)
        parts.append((start, count))
        start += count
    if min(c for _, c in parts) < G:
        raise ValueError(f"each part needs >= {G} nodes (the ghost width); got {base}")
    return parts


def bands(rank: int, world: int, G: int, periodic: bool = True):
    """Ghost nodes (below, above) the interior of a rank's part: G on every
    side with a neighbour; none at the ends of an outflow slab."""
    if periodic:
        return G, G
    return (0 if rank == 0 else G), (0 if rank == world - 1 else G)


def local_slice(field, start: int, count: int, G: int, periodic: bool = True, lo: int | None = None,
                hi: int | None = None):
    """Nodes start - lo .. start + count + hi - 1 of a field (last axis),
    wrapped for a periodic slab; lo, hi default to G."""
    nz = field.shape[-1]
    lo = G if lo is None else lo
    hi = G if hi is None else hi
    idx = np.arange(start - lo, start + count + hi)
    if periodic:
        idx %= nz
    elif idx[0] < 0 or idx[-1] >= nz:
        raise ValueError("an outflow part reaches past the slab")
    return field[..., idx]


class HaloDriver:
    """Advances one rank's part: every RK stage is followed by a halo
    exchange, so the ghosts always hold the neighbours' edge columns of the
    state the next stage reads."""

    def __init__(self, engine, exchange):
        self.engine = engine
        self.exchange = exchange

    def exchange_halos(self):
        to_left, to_right = self.engine.pack()
        from_left, from_right = self.exchange(to_left, to_right)
        self.engine.unpack(from_left, from_right)

    def step(self, nsteps: int = 1):
        if not getattr(self.engine, "ghosts_valid", True):   # after init
            self.exchange_halos()
        for _ in range(int(nsteps)):
            for s in range(3):
                self.engine.stage(s)
                self.exchange_halos()


def route_ring(messages, periodic: bool = True):
    """In-process exchange: messages[r] = (to_left, to_right) of part r;
    returns (from_left, from_right) per part -- around a ring, or along a
    line whose end parts receive None at the slab's ends."""
    W = len(messages)
    out = []
    for r in range(W):
        fl = messages[(r - 1) % W][1] if (periodic or r > 0) else None
        fr = messages[(r + 1) % W][0] if (periodic or r < W - 1) else None
        out.append((fl, fr))
    return out


def step_lockstep(engines, nsteps: int = 1, periodic: bool = True):
    """Advances the parts of one slab held in this process (in order): each
    stage runs on every part, then the packed messages are routed."""
    if not all(getattr(e, "ghosts_valid", True) for e in engines):   # after init
        exchange_lockstep(engines, periodic)
    for _ in range(int(nsteps)):
        for s in range(3):
            for e in engines:
                e.stage(s)
            exchange_lockstep(engines, periodic)


def exchange_lockstep(engines, periodic: bool = True):
    routed = route_ring([e.pack() for e in engines], periodic)
    for e, (fl, fr) in zip(engines, routed):
        e.unpack(fl, fr)


class DistExchange:
    """Halo exchange with the neighbours (ring for a periodic slab, line for
    an outflow slab) over torch.distributed point-to-point operations, one
    message each way per side.

    The operations are posted in one order on every rank -- send right, send
    left, receive from the left, receive from the right -- with tags 0 for
    right-going and 1 for left-going messages, so that they match whether the
    backend honours tags (gloo) or pairs grouped operations per peer in order
    (NCCL), also when both neighbours are the same rank (two ranks)."""

    def __init__(self, group=None, periodic: bool = True):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.periodic = periodic
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)
        glob = (lambda r: dist.get_global_rank(group, r)) if group is not None else (lambda r: r)
        W, r = self.world, self.rank
        self.left = glob((r - 1) % W) if (periodic or r > 0) else None
        self.right = glob((r + 1) % W) if (periodic or r < W - 1) else None

    def __call__(self, to_left, to_right):
        import torch
        if self.world == 1:
            if self.periodic:                     # the slab wraps onto itself
                return to_right.clone(), to_left.clone()
            return None, None
        dist = self.dist
        msg = to_left if to_left is not None else to_right
        fl = torch.empty_like(msg) if self.left is not None else None
        fr = torch.empty_like(msg) if self.right is not None else None
        ops = []
        if self.right is not None:
            ops.append(dist.P2POp(dist.isend, to_right, self.right, self.group, tag=0))
        if self.left is not None:
            ops.append(dist.P2POp(dist.isend, to_left, self.left, self.group, tag=1))
            ops.append(dist.P2POp(dist.irecv, fl, self.left, self.group, tag=0))
        if self.right is not None:
            ops.append(dist.P2POp(dist.irecv, fr, self.right, self.group, tag=1))
        for req in dist.batch_isend_irecv(ops):
            req.wait()
        return fl, fr


class CudaSlabPart:
    """Rank ``rank`` of ``world`` parts of a z-split slab on the CUDA library.

    ``params`` describes the whole slab (nx = nz; bc PERIODIC or OUTFLOW).
    The part is a context over its interior plus its ghost bands (nodes
    start - lo .. start + count + hi - 1, wrapped for a periodic slab) with
    bc HALO, or HALO_OUTFLOW_LO / _HI for the end parts of an outflow slab
    (a single outflow part is a plain OUTFLOW context).  dt is resolved from
    the whole slab's parameters, so every part steps with the same dt."""

    def __init__(self, params, rank: int, world: int, stream=None):
        from . import BC_HALO, BC_HALO_OUTFLOW_HI, BC_HALO_OUTFLOW_LO, BC_OUTFLOW, BC_PERIODIC, Sim, halo_width
        import torch
        if params.bc not in (BC_PERIODIC, BC_OUTFLOW) or params.dim != 1:
            raise ValueError("a split slab is a 1D periodic or outflow slab")
        self.periodic = params.bc == BC_PERIODIC
        self.G = halo_width(params)
        self.start, self.count = partition(params.nx, world, self.G)[rank]
        self.lo, self.hi = bands(rank, world, self.G, self.periodic)
        if self.lo and self.hi:
            bc = BC_HALO
        elif self.hi:
            bc = BC_HALO_OUTFLOW_LO
        elif self.lo:
            bc = BC_HALO_OUTFLOW_HI
        else:
            bc = BC_OUTFLOW
        local = dataclasses.replace(params, nx=self.count + self.lo + self.hi, bc=bc)
        self.sim = Sim(local, stream=stream)
        n = self.sim.halo_len()
        dev = torch.device("cuda", torch.cuda.current_device())
        f64 = torch.float64
        mk = lambda side: torch.empty(n, dtype=f64, device=dev) if (side and n) else None
        self._out = (mk(self.lo), mk(self.hi))
        self.ghosts_valid = not (self.lo or self.hi)

    def init(self, n0, u0, T0):
        """Projected Maxwellian of the whole slab's fields (numpy, length nz)
        on this part; its ghosts are filled by the first exchange."""
        sl = lambda f: np.ascontiguousarray(local_slice(np.asarray(f, dtype=np.float64), self.start, self.count,
                                                        self.G, self.periodic, self.lo, self.hi))
        self.sim.init(sl(n0), sl(u0), sl(T0))
        self.ghosts_valid = not (self.lo or self.hi)

    def stage(self, s):
        self.sim.stage(s)

    def pack(self):
        if self.lo or self.hi:
            self.sim.halo_pack(*self._out)
        return self._out

    def unpack(self, from_left, from_right):
        if self.lo or self.hi:
            c = lambda x: x.contiguous() if x is not None else None
            self.sim.halo_unpack(c(from_left) if self.lo else None, c(from_right) if self.hi else None)
        self.ghosts_valid = True

    def interior_state(self):
        """(F, G) of the owned nodes, shape (Q, count) each (synchronises)."""
        F, Gd = self.sim.get_state()
        Q = self.sim.Q[0]
        n = self.count + self.lo + self.hi
        i = slice(self.lo, self.lo + self.count)
        return F.reshape(Q, n)[:, i].copy(), Gd.reshape(Q, n)[:, i].copy()

    def close(self):
        self.sim.close()
