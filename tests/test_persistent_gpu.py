"""Persistent form of the batched step: one launch per graph of steps whose
resident CTAs take (RK stage, slab tile) items from a queue in stage order
and wait, on the device, only for the previous stage of their own slab.

It is the same Shu-Osher RK3 step (Sec. 3) as the launch-per-stage form,
so results must be bit-identical to it, and within 1e-12 of the oracle per
slab.  The waits are bounded: with the gate flag closed every wait runs to
its spin limit and the call reports EVFDLB_E_TIMEOUT, after which the
context refuses to step until a new init, and then steps correctly again.
"""
import numpy as np
import pytest

import oracle as O
import paper_2503_15187_gb300 as ev
from paper_2503_15187_gb300 import workloads as W

pytestmark = pytest.mark.gpu
DZ = 0.25
E_TIMEOUT, E_STATE, E_UNSUPPORTED = -6, -7, -8


def build(slabs):
    params = [ev.Params(nx=s["nz"], dx=DZ, Q=s["Q"]) for s in slabs]
    n0 = np.concatenate([s["n0"] for s in slabs])
    T0 = np.concatenate([np.full(s["nz"], s["T_ratio"] * ev.critical_T(p)) for s, p in zip(slabs, params)])
    return params, n0, np.zeros_like(n0), T0


def slab_view(arr, sim, s):
    off = sum(sim.nx[i] * sim.Q[i] for i in range(s))
    return arr[off:off + sim.nx[s] * sim.Q[s]].reshape(sim.Q[s], sim.nx[s])


def rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def run(params, n0, u0, T0, steps, persistent, tile=None):
    sim = ev.Sim(params)
    if tile is not None:
        sim.tune(tile)
    if persistent:
        sim.set_persistent(True)
    sim.init(n0, u0, T0)
    sim.step(steps)
    out = np.concatenate(sim.get_state())
    mom = sim.moments()
    sim.close()
    return out, mom


@pytest.mark.parametrize("steps", [1, 5, 37])    # one-step graph, chunk graphs + tail
def test_persistent_bit_identical_to_per_stage(steps):
    slabs = W.batch_slabs(nslab=6, seed=7, nz_min=24, nz_max=200)
    params, n0, u0, T0 = build(slabs)
    a, ma = run(params, n0, u0, T0, steps, False, tile=13)
    b, mb = run(params, n0, u0, T0, steps, True, tile=13)
    assert np.array_equal(a, b)
    for x, y in zip(ma, mb):
        assert np.array_equal(np.asarray(x), np.asarray(y))


def test_persistent_mixed_batch_against_oracle_per_slab():
    slabs = W.batch_slabs(nslab=5, seed=21, nz_min=17, nz_max=150)
    params, n0, u0, T0 = build(slabs)
    sim = ev.Sim(params)
    sim.tune(11)
    sim.set_persistent(True)
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
    sim.close()


def test_persistent_single_slab_and_retile():
    """One slab (every item waits on the same counter) and a tile change
    while the persistent form is on (the per-slab item counts are rebuilt)."""
    slabs = W.batch_slabs(nslab=1, seed=5, nz_min=300, nz_max=300)
    params, n0, u0, T0 = build(slabs)
    ref, _ = run(params, n0, u0, T0, 20, False)
    sim = ev.Sim(params)
    sim.set_persistent(True)
    for z in (7, 27):
        sim.tune(z)
        sim.init(n0, u0, T0)
        sim.step(20)
        assert np.array_equal(np.concatenate(sim.get_state()), ref)
    sim.set_persistent(False)
    sim.init(n0, u0, T0)
    sim.step(20)
    assert np.array_equal(np.concatenate(sim.get_state()), ref)
    sim.close()


def test_bounded_wait_times_out_and_context_recovers():
    slabs = W.batch_slabs(nslab=3, seed=9, nz_min=40, nz_max=120)
    params, n0, u0, T0 = build(slabs)
    ref, _ = run(params, n0, u0, T0, 4, False)
    sim = ev.Sim(params)
    sim.set_persistent(True, spin_limit=2000)     # ~0.2 ms of polling per wait
    sim.init(n0, u0, T0)
    sim.debug_gate(False)                         # every wait now waits on a flag nothing sets
    with pytest.raises(ev.EvfdlbError) as e:
        sim.step(4)
    assert e.value.code == E_TIMEOUT
    with pytest.raises(ev.EvfdlbError) as e:      # poisoned until a new init
        sim.step(1)
    assert e.value.code == E_STATE
    sim.debug_gate(True)
    sim.init(n0, u0, T0)
    sim.step(4)
    assert np.array_equal(np.concatenate(sim.get_state()), ref)
    sim.close()


def test_persistent_refuses_unsupported_modes():
    p = ev.Params(nx=64, dx=DZ, Q=16)
    for q in (ev.Params(nx=64, dx=DZ, Q=16, precision=ev.FP32),
              ev.Params(nx=64, dx=DZ, Q=16, T_iso=0.9)):
        sim = ev.Sim([q])
        with pytest.raises(ev.EvfdlbError) as e:
            sim.set_persistent(True)
        assert e.value.code == E_UNSUPPORTED
        sim.close()
    sim = ev.Sim([p])
    with pytest.raises(ev.EvfdlbError) as e:      # the gate exists only once enabled
        sim.debug_gate(True)
    assert e.value.code == E_STATE
    sim.close()


def test_persistent_full_phase_separation_batch():
    """The 256-slab phase-separation batch (Nz log-uniform in [128, 8192]):
    persistent and per-stage forms bit-identical over 20 steps."""
    slabs = W.batch_slabs(nslab=256)
    params, n0, u0, T0 = build(slabs)
    a, _ = run(params, n0, u0, T0, 20, False)
    b, _ = run(params, n0, u0, T0, 20, True)
    assert np.array_equal(a, b)
