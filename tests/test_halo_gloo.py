"""Z-split of one slab over gloo ranks on CPU: the exchange logic of the
domain decomposition (paper_2503_15187_gb300.halo) with the oracle as the
per-rank engine.

Each rank owns a contiguous part of a slab plus ghost nodes on an outflow
slab of its own, runs every Shu-Osher stage (Sec. III) on it, and swaps
edge columns with its neighbours through DistExchange: on a ring for a
periodic slab, on a line for an outflow slab (whose end parts keep no ghost
band at the slab's ends).  The interior nodes must come out bit-identical
to the unsplit slab stepped with the same stage arithmetic: a wrong
neighbour, a swapped side, an off-by-one column or a missing exchange
changes them.
"""
import dataclasses
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
NZ, Q, DZ, STEPS = 96, 8, 0.25, 3


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def setup_and_state(bc=0):
    import oracle as O
    xi, _ = O.gauss_hermite(Q)
    S = O.Setup(nz=NZ, Q=Q, dz=DZ, dt=0.5 * DZ / abs(xi).max(), bc=bc)
    orc = O.Oracle(S)
    rng = np.random.default_rng(5)
    z = np.arange(NZ) * DZ
    n = 0.25 + 0.08 * np.sin(2 * np.pi * z / (NZ * DZ)) + 0.005 * rng.standard_normal(NZ)
    u = 0.05 * np.cos(4 * np.pi * z / (NZ * DZ))
    T = 0.9 + 0.02 * rng.standard_normal(NZ)
    F0, G0 = orc.equilibrium(n, u, T)
    return S, np.ascontiguousarray(F0), np.ascontiguousarray(G0)


def oracle_reach(S):
    """Ghost width of the oracle engine: the oracle recomputes every node
    field from F and G, so its ghosts cover the whole read of a stage --
    the force taps (r_cut / dz) plus the WENO-5 stencil."""
    return int(round(S.rcut / S.dz)) + 3


def stage_update(s, U, L, dt):
    """Shu-Osher stage s from the state list U = [u, u1, u2] and L = L(U[s])."""
    if s == 0:
        return U[0] + dt * L
    if s == 1:
        return 0.75 * U[0] + 0.25 * (U[1] + dt * L)
    return U[0] / 3.0 + 2.0 / 3.0 * (U[2] + dt * L)


class OracleSlabPart:
    """Engine of one part on the oracle: the part plus Go ghost nodes per
    side as an outflow slab; a stage updates the interior nodes only."""

    def __init__(self, S, start, count, Go, lo=None, hi=None):
        import oracle as O
        self.lo = Go if lo is None else lo
        self.hi = Go if hi is None else hi
        self.periodic = S.bc == 0
        self.orc = O.Oracle(dataclasses.replace(S, nz=count + self.lo + self.hi, bc=1))
        self.dt, self.Go, self.count, self.start = S.dt, Go, count, start
        self.ghosts_valid = False
        self.cur = 0

    def init(self, F0, G0):
        from paper_2503_15187_gb300.halo import local_slice
        sl = lambda f: local_slice(f, self.start, self.count, self.Go, self.periodic, self.lo, self.hi)
        u = np.concatenate([sl(F0), sl(G0)])
        u[:, :self.lo] = 0.0                      # ghosts come from the first exchange
        u[:, self.lo + self.count:] = 0.0
        self.U = [u, u.copy(), u.copy()]
        self.cur = 0

    def stage(self, s):
        src = self.U[s]
        RF, RG = self.orc.rhs(src[:Q], src[Q:])
        new = stage_update(s, self.U, np.concatenate([RF, RG]), self.dt)
        i = slice(self.lo, self.lo + self.count)
        dst = (s + 1) % 3
        self.U[dst][:, i] = new[:, i]
        self.cur = dst

    def pack(self):
        import torch
        u, Go, lo, c = self.U[self.cur], self.Go, self.lo, self.count
        msg = lambda cols: torch.from_numpy(np.ascontiguousarray(u[:, cols]).ravel())
        return (msg(slice(lo, lo + Go)) if self.lo else None,
                msg(slice(lo + c - Go, lo + c)) if self.hi else None)

    def unpack(self, from_left, from_right):
        u, lo, c = self.U[self.cur], self.lo, self.count
        if self.lo:
            u[:, :lo] = from_left.numpy().reshape(2 * Q, lo)
        if self.hi:
            u[:, lo + c:] = from_right.numpy().reshape(2 * Q, self.hi)
        self.ghosts_valid = True

    def interior(self):
        return self.U[0][:, self.lo:self.lo + self.count]


def unsplit(S, F0, G0, nsteps):
    """The whole slab, same stage arithmetic, no exchange."""
    import oracle as O
    orc = O.Oracle(S)
    U = [np.concatenate([F0, G0]), None, None]
    for _ in range(nsteps):
        for s in range(3):
            RF, RG = orc.rhs(U[s][:Q], U[s][Q:])
            U[(s + 1) % 3] = stage_update(s, U, np.concatenate([RF, RG]), S.dt)
    return U[0]


def _worker(rank, world, port, out_dir, bc):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2503_15187_gb300 import halo
    S, F0, G0 = setup_and_state(bc)
    Go = oracle_reach(S)
    start, count = halo.partition(NZ, world, Go)[rank]
    lo, hi = halo.bands(rank, world, Go, periodic=(bc == 0))
    part = OracleSlabPart(S, start, count, Go, lo, hi)
    part.init(F0, G0)
    drv = halo.HaloDriver(part, halo.DistExchange(periodic=(bc == 0)))
    drv.step(STEPS)
    np.save(os.path.join(out_dir, f"rank{rank}.npy"), part.interior())
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world,bc", [(2, 0), (3, 0), (2, 1), (3, 1)])
def test_split_slab_equals_unsplit_bit_for_bit(tmp_path, world, bc):
    import torch.multiprocessing as mp
    sys.path.insert(0, ROOT)
    mp.spawn(_worker, args=(world, free_port(), str(tmp_path), bc), nprocs=world, join=True)
    got = np.concatenate([np.load(tmp_path / f"rank{r}.npy") for r in range(world)], axis=1)
    S, F0, G0 = setup_and_state(bc)
    ref = unsplit(S, F0, G0, STEPS)
    assert got.shape == ref.shape
    assert np.array_equal(got, ref)


def test_unsplit_stage_arithmetic_matches_the_oracle_step():
    """The stage composition above is the oracle's own RK3 step (to
    rounding: the oracle may group the combination differently)."""
    import oracle as O
    S, F0, G0 = setup_and_state()
    ref = unsplit(S, F0, G0, 2)
    F, G = O.Oracle(S).step(F0, G0, 2)
    assert np.abs(ref - np.concatenate([F, G])).max() < 1e-13 * np.abs(ref).max()


def test_world_one_wraps_onto_itself():
    """A single rank in halo form (its exchange the periodic wrap) equals
    the unsplit slab."""
    import torch
    from paper_2503_15187_gb300 import halo
    S, F0, G0 = setup_and_state()
    Go = oracle_reach(S)
    part = OracleSlabPart(S, 0, NZ, Go)
    part.init(F0, G0)
    wrap = lambda tl, tr: (tr.clone(), tl.clone())
    halo.HaloDriver(part, wrap).step(STEPS)
    assert np.array_equal(part.interior(), unsplit(S, F0, G0, STEPS))


def test_partition_and_routing():
    from paper_2503_15187_gb300 import halo
    parts = halo.partition(100, 3, 24)
    assert parts == [(0, 34), (34, 33), (67, 33)]
    with pytest.raises(ValueError):
        halo.partition(60, 3, 24)              # a part smaller than the ghost width
    f = np.arange(10.0)
    assert list(halo.local_slice(f, 0, 4, 2)) == [8, 9, 0, 1, 2, 3, 4, 5]
    routed = halo.route_ring([("L0", "R0"), ("L1", "R1"), ("L2", "R2")])
    assert routed == [("R2", "L1"), ("R0", "L2"), ("R1", "L0")]
    line = halo.route_ring([(None, "R0"), ("L1", "R1"), ("L2", None)], periodic=False)
    assert line == [(None, "L1"), ("R0", "L2"), ("R1", None)]
    assert halo.bands(0, 3, 24, periodic=False) == (0, 24)
    assert halo.bands(2, 3, 24, periodic=False) == (24, 0)
    assert list(halo.local_slice(f, 0, 4, 2, periodic=False, lo=0)) == [0, 1, 2, 3, 4, 5]
