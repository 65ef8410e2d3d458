"""Batched slabs: many independent periodic slabs of different length, order
Q, temperature and density advanced together by one launch per RK stage.

Parity: every slab of a mixed batch against its own oracle run; the full
phase-separation batch (256 slabs, Nz log-uniform in [128, 8192],
Q in {16, 24, 32}, T/T_c in [0.6, 0.95], mean n in [0.15, 0.35], +-1% noise)
on sampled slabs one step at a time, and mass/momentum conservation of every
slab (a property that holds at any size).  The tile size is a speed knob
only: results are bit-identical across tiles, and the autotuner's choice is
one of its candidates.
"""
import numpy as np
import pytest

import oracle as O
import paper_2503_15187_gb300 as ev
from paper_2503_15187_gb300 import autotune as AT
from paper_2503_15187_gb300 import workloads as W

pytestmark = pytest.mark.gpu
DZ = 0.25


def rel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300))


def build(slabs):
    params = [ev.Params(nx=s["nz"], dx=DZ, Q=s["Q"]) for s in slabs]
    n0 = np.concatenate([s["n0"] for s in slabs])
    T0 = np.concatenate([np.full(s["nz"], s["T_ratio"] * ev.critical_T(p)) for s, p in zip(slabs, params)])
    return params, n0, np.zeros_like(n0), T0


def slab_view(arr, sim, s):
    off = sum(sim.nx[i] * sim.Q[i] for i in range(s))
    return arr[off:off + sim.nx[s] * sim.Q[s]].reshape(sim.Q[s], sim.nx[s])


def test_mixed_batch_against_oracle_per_slab():
    slabs = W.batch_slabs(nslab=6, seed=7, nz_min=24, nz_max=200)
    params, n0, u0, T0 = build(slabs)
    sim = ev.Sim(params)
    sim.tune(13)                                 # ragged tiles in every slab
    sim.init(n0, u0, T0)
    F0, G0 = sim.get_state()
    sim.step(3)
    F, G = sim.get_state()
    for s, p in enumerate(params):
        orc = O.Oracle(O.Setup(nz=p.nx, Q=p.Q, dz=DZ, dt=sim.dt(s)))
        Fo, Go = orc.step(slab_view(F0, sim, s), slab_view(G0, sim, s), 3)
        eF, eG = rel(slab_view(F, sim, s), Fo), rel(slab_view(G, sim, s), Go)
        print(f"slab {s}: nz {p.nx} Q {p.Q} err F {eF:.1e} G {eG:.1e}")
        assert eF < 1e-12 and eG < 1e-12


def test_tile_size_changes_nothing_but_speed():
    slabs = W.batch_slabs(nslab=5, seed=3, nz_min=40, nz_max=300)
    params, n0, u0, T0 = build(slabs)
    sim = ev.Sim(params)
    states = []
    for z in (1, 7, 27, 64):
        sim.tune(z)
        sim.init(n0, u0, T0)
        sim.step(4)
        states.append(np.concatenate(sim.get_state()))
    for st in states[1:]:
        assert np.array_equal(st, states[0])


def test_autotuner_picks_a_candidate_and_caches(tmp_path):
    slabs = W.batch_slabs(nslab=8, seed=11, nz_min=64, nz_max=1024)
    params, n0, u0, T0 = build(slabs)
    cache = str(tmp_path / "tune.json")
    best, times = AT.autotune(params, n0, u0, T0, cache=cache)
    assert best in times and times[best] == min(times.values())
    best2, times2 = AT.autotune(params, n0, u0, T0, cache=cache)    # served from the cache
    assert best2 == best and times2 == times
    sim = ev.Sim(params)
    sim.tune(best)
    assert sim.tile_nodes() == best


def test_phase_separation_batch_full_size():
    """256 slabs as one context: sampled slabs one step against the oracle,
    and mass / momentum of every slab conserved over 20 steps."""
    slabs = W.batch_slabs(nslab=256)
    params, n0, u0, T0 = build(slabs)
    sim = ev.Sim(params)
    sim.init(n0, u0, T0)
    t0 = sim.moments()[4]
    F0, G0 = sim.get_state()
    sim.step(1)
    F, G = sim.get_state()
    order = np.argsort([p.nx * p.Q for p in params])
    for s in list(order[:3]) + [int(order[len(order) // 2])]:
        p = params[s]
        orc = O.Oracle(O.Setup(nz=p.nx, Q=p.Q, dz=DZ, dt=sim.dt(s)))
        Fo, Go = orc.step(slab_view(F0, sim, s), slab_view(G0, sim, s), 1)
        eF, eG = rel(slab_view(F, sim, s), Fo), rel(slab_view(G, sim, s), Go)
        print(f"slab {s}: nz {p.nx} Q {p.Q} err F {eF:.1e} G {eG:.1e}")
        assert eF < 1e-12 and eG < 1e-12
    sim.step(19)
    t1 = sim.moments()[4]
    assert np.all(np.abs(t1[:, 0] - t0[:, 0]) < 1e-12 * t0[:, 0])
    assert np.all(np.abs(t1[:, 1] - t0[:, 1]) < 1e-12 * t0[:, 0])
