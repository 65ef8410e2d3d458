"""Z-split slab on the CUDA library: RK stages one call at a time, and the
halo exchange of a slab split into parts, run on one device with the parts
in lockstep (every part's stage, then the messages routed between them; no
kernel waits on another).

The split is the domain decomposition of the explicit z stencil (Sec. III):
the interior nodes of the parts must equal the unsplit slab bit for bit --
periodic slabs on a ring, outflow slabs on a line -- in FP64 and FP32, EV1
and EV2, and on the full 1D liquid-slab evaporation workload (Nz = 4096,
dz = 0.1, Q = 32, outflow ends) split four ways.  The split also matches the
oracle's step to 1e-12.
"""
import numpy as np
import pytest

import oracle as O
import paper_2503_15187_gb300 as ev
from paper_2503_15187_gb300 import halo
from paper_2503_15187_gb300 import workloads as W

pytestmark = pytest.mark.gpu
E_UNSUPPORTED, E_STATE = -8, -7


def fields(nz, seed=3):
    rng = np.random.default_rng(seed)
    z = np.arange(nz)
    n = 0.3 + 0.1 * np.sin(2 * np.pi * z / nz) + 0.01 * rng.standard_normal(nz)
    u = 0.03 * np.cos(6 * np.pi * z / nz)
    T = 0.95 + 0.02 * rng.standard_normal(nz)
    return n, u, T


def unsplit(p, n, u, T, steps):
    sim = ev.Sim(p)
    sim.init(n, u, T)
    sim.step(steps)
    F, G = sim.get_state()
    sim.close()
    return F.reshape(p.Q, p.nx), G.reshape(p.Q, p.nx)


def split(p, n, u, T, steps, world):
    parts = [halo.CudaSlabPart(p, r, world) for r in range(world)]
    for e in parts:
        e.init(n, u, T)
    halo.step_lockstep(parts, steps, periodic=(p.bc == ev.BC_PERIODIC))
    got = [e.interior_state() for e in parts]
    for e in parts:
        e.close()
    return np.concatenate([g[0] for g in got], axis=1), np.concatenate([g[1] for g in got], axis=1)


def test_three_stage_calls_equal_one_step():
    p = ev.Params(nx=200, dx=0.25, Q=16)
    n, u, T = fields(p.nx)
    ref = unsplit(p, n, u, T, 2)
    sim = ev.Sim(p)
    sim.init(n, u, T)
    for _ in range(2):
        for s in range(3):
            sim.stage(s)
    F, G = sim.get_state()
    assert np.array_equal(F.reshape(p.Q, p.nx), ref[0]) and np.array_equal(G.reshape(p.Q, p.nx), ref[1])
    with pytest.raises(ev.EvfdlbError) as e:           # stages in order only
        sim.stage(1)
    assert e.value.code == E_STATE
    sim.stage(0)
    with pytest.raises(ev.EvfdlbError) as e:           # no whole step in the middle of one
        sim.step(1)
    assert e.value.code == E_STATE
    sim.close()


@pytest.mark.parametrize("bc,world", [(ev.BC_PERIODIC, 1), (ev.BC_PERIODIC, 2), (ev.BC_PERIODIC, 3),
                                      (ev.BC_OUTFLOW, 2), (ev.BC_OUTFLOW, 3)])
@pytest.mark.parametrize("prec", [ev.FP64, ev.FP32])
def test_split_equals_unsplit_bit_for_bit(bc, world, prec):
    p = ev.Params(nx=157, dx=0.25, Q=16, bc=bc, precision=prec)      # ragged parts (53, 52, 52)
    n, u, T = fields(p.nx)
    F, G = split(p, n, u, T, 6, world)
    Fr, Gr = unsplit(p, n, u, T, 6)
    assert np.array_equal(F, Fr) and np.array_equal(G, Gr)


@pytest.mark.parametrize("bc", [ev.BC_PERIODIC, ev.BC_OUTFLOW])
def test_split_ev2_and_odd_q(bc):
    p = ev.Params(nx=90, dx=0.25, Q=15, bc=bc, force_model=ev.EV2, gamma=8.0)
    n, u, T = fields(p.nx, seed=8)
    F, G = split(p, n, u, T, 5, 3)
    Fr, Gr = unsplit(p, n, u, T, 5)
    assert np.array_equal(F, Fr) and np.array_equal(G, Gr)


def test_split_against_the_oracle():
    p = ev.Params(nx=120, dx=0.25, Q=12)
    n, u, T = fields(p.nx, seed=11)
    parts = [halo.CudaSlabPart(p, r, 2) for r in range(2)]
    for e in parts:
        e.init(n, u, T)
    sim0 = ev.Sim(p)
    sim0.init(n, u, T)
    F0, G0 = sim0.get_state()
    dt = sim0.dt()
    sim0.close()
    halo.step_lockstep(parts, 3)
    F = np.concatenate([e.interior_state()[0] for e in parts], axis=1)
    G = np.concatenate([e.interior_state()[1] for e in parts], axis=1)
    orc = O.Oracle(O.Setup(nz=p.nx, Q=p.Q, dz=p.dx, dt=dt))
    Fo, Go = orc.step(F0.reshape(p.Q, p.nx), G0.reshape(p.Q, p.nx), 3)
    rel = lambda a, b: np.abs(a - b).max() / np.abs(b).max()
    assert rel(F, Fo) < 1e-12 and rel(G, Go) < 1e-12
    for e in parts:
        e.close()


def test_halo_context_rules():
    p = ev.Params(nx=120, dx=0.25, Q=12)
    G = ev.halo_width(p)
    assert G == 24                                     # r_cut / dz = 6 / 0.25
    part = halo.CudaSlabPart(p, 0, 2)
    assert part.sim.halo_len() == 6 * p.Q + 6 * G
    n, u, T = fields(p.nx)
    part.init(n, u, T)
    for call in (lambda: part.sim.step(1), lambda: part.sim.rhs(), lambda: part.sim.set_persistent(True)):
        with pytest.raises(ev.EvfdlbError) as e:
            call()
        assert e.value.code == E_UNSUPPORTED
    import torch
    short = torch.zeros(5, dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        part.sim.halo_pack(short, short)
    with pytest.raises(ValueError):
        part.sim.halo_pack(np.zeros(part.sim.halo_len()), np.zeros(part.sim.halo_len()))
    part.close()
    with pytest.raises(ValueError):                    # 3 parts of 20 nodes < G
        halo.CudaSlabPart(ev.Params(nx=60, dx=0.25, Q=12), 0, 3)
    with pytest.raises(ev.EvfdlbError):                # too few interior nodes for a HALO context
        ev.Sim(ev.Params(nx=3 * G - 1, dx=0.25, Q=12, bc=ev.BC_HALO))


def test_split_full_liquid_slab_workload():
    """Nz = 4096, dz = 0.1, Q = 32, outflow ends (G = 60), four parts."""
    p = ev.Params(nx=4096, dx=0.1, Q=32, bc=ev.BC_OUTFLOW)
    T = 0.8 * ev.critical_T(p)
    nv, nl = ev.coexistence(p, T)
    n0 = W.liquid_slab(p.nx, p.dx, nl, nv, thickness=20.0, width=2.0)
    u0, T0 = np.zeros(p.nx), np.full(p.nx, T)
    F, G = split(p, n0, u0, T0, 4, 4)
    Fr, Gr = unsplit(p, n0, u0, T0, 4)
    assert np.array_equal(F, Fr) and np.array_equal(G, Gr)
