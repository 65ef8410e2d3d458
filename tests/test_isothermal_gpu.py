"""GPU parity of the isothermal mode (T_iso > 0: after every step each
node's temperature is set back to T_iso, density, velocity and
non-equilibrium part kept) against the oracle's isothermal path (pinned in
test_oracle_isothermal_pins.py) on the same seeded inputs.

Bars are those of the thermal parity tests: 1e-12 per step, 1e-11 after 20
steps; FP32 at 1e-5 per step.  A uniform Maxwellian at another temperature
becomes the projected Maxwellian at T_iso after one step.
"""
import numpy as np
import pytest

import oracle as O
import paper_2503_15187_gb300 as ev
from paper_2503_15187_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300))


CASES = {
    # name: (nz, Q, dz, bc, force_model, tile)
    "periodic_q16_ev1_tile7": (64, 16, 0.25, 0, 0, 7),
    "outflow_q24_ev1": (97, 24, 0.25, 1, 0, 13),
    "periodic_q16_ev2_dz01": (150, 16, 0.1, 0, 1, 27),
}


def make(name, T_ratio=0.7, prec=ev.FP64):
    nz, Q, dz, bc, fm, tile = CASES[name]
    p = ev.Params(nx=nz, dx=dz, Q=Q, bc=bc, force_model=fm, precision=prec)
    T_iso = T_ratio * ev.critical_T(p)
    p.T_iso = T_iso
    sim = ev.Sim(p)
    sim.tune(tile)
    orc = O.Oracle(O.Setup(nz=nz, Q=Q, dz=dz, dt=sim.dt(), bc=bc, force_model=fm, T_iso=T_iso))
    nv, nl = O.coexistence(T_iso, orc.discrete_a())
    n0 = W.liquid_slab(nz, dz, nl, nv, thickness=0.35 * nz * dz, width=2.0)
    u0 = 0.02 * np.sin(2 * np.pi * np.arange(nz) / nz)
    T0 = T_iso * (1 + 0.05 * np.cos(2 * np.pi * np.arange(nz) / nz))    # kinetic T off T_iso
    return sim, orc, n0, u0, T0


@pytest.mark.parametrize("name", list(CASES))
def test_isothermal_rhs_and_step(name):
    sim, orc, n0, u0, T0 = make(name)
    F, G = orc.step(*orc.equilibrium(n0, u0, T0), 2)
    sim.set_state(F.ravel(), G.ravel())
    RF, RG = sim.rhs()                             # the thermal right-hand side
    RFo, RGo = orc.rhs(F, G)
    Q, nz = F.shape
    assert rel(RF.reshape(Q, nz), RFo) < 1e-11 and rel(RG.reshape(Q, nz), RGo) < 1e-11
    sim.step(1)
    Fo, Go = orc.step(F, G, 1)
    Fg, Gg = sim.state_2d()
    assert rel(Fg, Fo) < 1e-12 and rel(Gg, Go) < 1e-12


@pytest.mark.parametrize("name", ["periodic_q16_ev1_tile7", "outflow_q24_ev1"])
def test_isothermal_twenty_steps(name):
    sim, orc, n0, u0, T0 = make(name)
    sim.init(n0, u0, T0)
    Fo, Go = orc.step(*orc.equilibrium(n0, u0, T0), 20)
    sim.step(20)
    Fg, Gg = sim.state_2d()
    assert rel(Fg, Fo) < 1e-11 and rel(Gg, Go) < 1e-11
    n, u, T, q, tot = sim.moments()
    assert np.abs(T - orc.s.T_iso).max() < 1e-13 * orc.s.T_iso


def test_isothermal_fp32_step():
    sim, orc, n0, u0, T0 = make("periodic_q16_ev1_tile7", prec=ev.FP32)
    F, G = orc.step(*orc.equilibrium(n0, u0, T0), 2)
    sim.set_state(F.ravel(), G.ravel())
    sim.step(1)
    Fo, Go = orc.step(F, G, 1)
    Fg, Gg = sim.state_2d()
    assert rel(Fg, Fo) < 1e-5 and rel(Gg, Go) < 1e-5


def test_uniform_maxwellian_reset_on_gpu():
    nz, Q = 40, 16
    p = ev.Params(nx=nz, dx=0.25, Q=Q, T_iso=0.55)
    sim = ev.Sim(p)
    th = O.Oracle(O.Setup(nz=nz, Q=Q, dz=0.25, dt=sim.dt()))
    n0 = np.full(nz, 0.3)
    Fe, Ge = th.equilibrium(n0, np.zeros(nz), np.full(nz, 0.55))
    sim.init(n0, np.zeros(nz), np.full(nz, 0.72))
    sim.step(1)
    Fg, Gg = sim.state_2d()
    assert np.abs(Fg - Fe).max() < 1e-14 * Fe.max() and np.abs(Gg - Ge).max() < 1e-14 * Ge.max()
    assert sim.launches_per_step() == 4


def test_isothermal_adjoint_unsupported():
    sim, orc, n0, u0, T0 = make("periodic_q16_ev1_tile7")
    sim.init(n0, u0, T0)
    N = sim.NF
    with pytest.raises(ev.EvfdlbError) as e:
        sim.rhs_vjp(np.ones(N), np.ones(N))
    assert e.value.code == -8
