"""GPU parity of the FP64_DF variant (FP64 state and arithmetic, Hermite
analysis and synthesis as double-float pairs with the Dot2 compensated dot
product) against the FP64 oracle, at the FP64 bars: 1e-11 for one
right-hand side, 1e-12 per step, 1e-11 after 20 steps, on ragged tiles,
both boundary rules, Q = 8..32, EV1 and EV2, and the full-size liquid slab.
Double-float sums carry ~2^-48 relative error per term against the FP64
oracle's 2^-53, well inside the bars.
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
    "periodic_q16_tile7": (64, 16, 0.25, 0, 0, 7),
    "outflow_q24_slab": (97, 24, 0.25, 1, 0, 13),
    "outflow_q32_dz01": (150, 32, 0.1, 1, 0, 27),
    "periodic_q8_ev2": (50, 8, 0.25, 0, 1, 64),
}


def make(name):
    nz, Q, dz, bc, fm, tile = CASES[name]
    sim = ev.Sim(ev.Params(nx=nz, dx=dz, Q=Q, bc=bc, force_model=fm, precision=ev.FP64_DF))
    sim.tune(tile)
    orc = O.Oracle(O.Setup(nz=nz, Q=Q, dz=dz, dt=sim.dt(), bc=bc, force_model=fm))
    T = 0.8 * orc.critical_T()
    nv, nl = O.coexistence(T, orc.discrete_a())
    n0 = W.liquid_slab(nz, dz, nl, nv, thickness=0.35 * nz * dz, width=2.0)
    u0 = 0.02 * np.sin(2 * np.pi * np.arange(nz) / nz)
    T0 = T * (1 + 0.01 * np.cos(2 * np.pi * np.arange(nz) / nz))
    return sim, orc, n0, u0, T0


@pytest.mark.parametrize("name", list(CASES))
def test_df_rhs_and_one_step(name):
    sim, orc, n0, u0, T0 = make(name)
    F, G = orc.step(*orc.equilibrium(n0, u0, T0), 2)
    sim.set_state(F.ravel(), G.ravel())
    RF, RG = sim.rhs()
    RFo, RGo = orc.rhs(F, G)
    Q, nz = F.shape
    eF, eG = rel(RF.reshape(Q, nz), RFo), rel(RG.reshape(Q, nz), RGo)
    sim.step(1)
    Fg, Gg = sim.state_2d()
    Fo, Go = orc.step(F, G, 1)
    sF, sG = rel(Fg, Fo), rel(Gg, Go)
    print(f"FP64_DF {name}: rhs {eF:.1e} {eG:.1e} step {sF:.1e} {sG:.1e}")
    assert eF < 1e-11 and eG < 1e-11 and sF < 1e-12 and sG < 1e-12


@pytest.mark.parametrize("name", ["periodic_q16_tile7", "outflow_q24_slab"])
def test_df_twenty_steps(name):
    sim, orc, n0, u0, T0 = make(name)
    sim.init(n0, u0, T0)
    Fo, Go = orc.step(*orc.equilibrium(n0, u0, T0), 20)
    sim.step(20)
    Fg, Gg = sim.state_2d()
    assert rel(Fg, Fo) < 1e-11 and rel(Gg, Go) < 1e-11
    tot = sim.moments()[4]
    to = orc.totals(Fo, Go)
    assert abs(tot[0, 0] - to[0]) < 1e-12 * abs(to[0])


def test_df_adjoint_unsupported():
    sim, orc, n0, u0, T0 = make("periodic_q16_tile7")
    sim.init(n0, u0, T0)
    with pytest.raises(ev.EvfdlbError) as e:
        sim.rhs_vjp(np.ones(sim.NF), np.ones(sim.NF))
    assert e.value.code == -8


def test_df_liquid_slab_full_size_one_step():
    """Nz = 4096, dz = 0.1, Q = 32, outflow, 20-sigma slab at T = 0.8 T_c, the
    default launch configuration: one step against the oracle."""
    nz, Q, dz = 4096, 32, 0.1
    sim = ev.Sim(ev.Params(nx=nz, dx=dz, Q=Q, bc=ev.BC_OUTFLOW, precision=ev.FP64_DF))
    orc = O.Oracle(O.Setup(nz=nz, Q=Q, dz=dz, dt=sim.dt(), bc=1))
    T = 0.8 * orc.critical_T()
    nv, nl = O.coexistence(T, orc.discrete_a())
    n0 = W.liquid_slab(nz, dz, nl, nv, thickness=20.0, width=2.0)
    F, G = orc.equilibrium(n0, np.zeros(nz), np.full(nz, T))
    sim.set_state(F.ravel(), G.ravel())
    sim.step(1)
    Fg, Gg = sim.state_2d()
    Fo, Go = orc.step(F, G, 1)
    assert rel(Fg, Fo) < 1e-12 and rel(Gg, Go) < 1e-12
