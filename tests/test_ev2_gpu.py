"""GPU parity of the EV2 force model (Eq. (F2)) against the oracle's EV2 path
(pinned in test_oracle_ev2_pins.py) on the same seeded inputs.

The library applies EV2 as one merged antisymmetric 5-point force stencil and
a 5-point energy stencil inside the tap blocks the EV1 path uses, so every
kernel (forward FP64 and FP32, batched, adjoint, allocation-free step) runs
the same code with EV2 taps; the oracle forms 2a D4 n + kappa D3 n from the
two stencils separately.  Bars are those of the EV1 parity tests: 1e-12 for
node fields and one step, 1e-11 for one right-hand side and after 20 steps,
FP32 at 1e-5 per step, adjoint dot products at 1e-11 of the Cauchy-Schwarz
scale.  Tiles are ragged; both boundary rules; batches mix EV1 and EV2 slabs.
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
    # name: (nz, Q, dz, bc, profile, tile)
    "periodic_q16_tile7": (64, 16, 0.25, 0, "noise", 7),
    "outflow_q24_slab": (97, 24, 0.25, 1, "slab", 13),
    "outflow_q32_dz01": (150, 32, 0.1, 1, "slab", 27),
    "periodic_q8_short": (16, 8, 0.25, 0, "noise", 5),
}


def inputs(orc, nz, dz, prof):
    Tc = orc.critical_T()
    if prof == "noise":
        T = 0.7 * Tc
        n0 = W.noisy_uniform(nz, 0.25, 0.05)
    else:
        T = 0.8 * Tc
        nv, nl = O.coexistence(T, orc.discrete_a())
        n0 = W.liquid_slab(nz, dz, nl, nv, thickness=0.35 * nz * dz, width=2.0)
    u0 = 0.02 * np.sin(2 * np.pi * np.arange(nz) / nz)
    T0 = T * (1 + 0.01 * np.cos(2 * np.pi * np.arange(nz) / nz))
    return n0, u0, T0


def make(name, prec=ev.FP64):
    nz, Q, dz, bc, prof, tile = CASES[name]
    sim = ev.Sim(ev.Params(nx=nz, dx=dz, Q=Q, bc=bc, force_model=ev.EV2, precision=prec))
    if tile:
        sim.tune(tile)
    orc = O.Oracle(O.Setup(nz=nz, Q=Q, dz=dz, dt=sim.dt(), bc=bc, force_model=1))
    return sim, orc, *inputs(orc, nz, dz, prof)


def nonequilibrium_state(orc, n0, u0, T0, steps=2):
    F, G = orc.equilibrium(n0, u0, T0)
    return orc.step(F, G, steps)


@pytest.mark.parametrize("name", list(CASES))
def test_ev2_force_and_fields(name):
    sim, orc, n0, u0, T0 = make(name)
    F, G = nonequilibrium_state(orc, n0, u0, T0)
    sim.set_state(F.ravel(), G.ravel())
    fg = sim.fields()
    fo = orc.node_fields(F, G)
    # the stencil sums cancel O(kappa/dz^3 n) terms: measure on that scale
    dz = CASES[name][2]
    scale = max(np.abs(fo["force"]).max(), 2.5 / dz ** 3 * fo["n"].max() * 1e-3)
    assert np.abs(fg["force"] - fo["force"]).max() / scale < 1e-12
    for k, ko in (("n", "n"), ("T", "T"), ("chi", "chi"), ("nu", "rate"), ("nbar", "nbar")):
        assert rel(fg[k], fo[ko]) < 1e-12, k


@pytest.mark.parametrize("name", list(CASES))
def test_ev2_rhs_and_one_step(name):
    sim, orc, n0, u0, T0 = make(name)
    F, G = nonequilibrium_state(orc, n0, u0, T0)
    sim.set_state(F.ravel(), G.ravel())
    RF, RG = sim.rhs()
    RFo, RGo = orc.rhs(F, G)
    Q, nz = F.shape
    assert rel(RF.reshape(Q, nz), RFo) < 1e-11 and rel(RG.reshape(Q, nz), RGo) < 1e-11
    sim.step(1)
    Fg, Gg = sim.state_2d()
    Fo, Go = orc.step(F, G, 1)
    assert rel(Fg, Fo) < 1e-12 and rel(Gg, Go) < 1e-12


@pytest.mark.parametrize("name", ["periodic_q16_tile7", "outflow_q24_slab"])
def test_ev2_twenty_steps_and_totals(name):
    sim, orc, n0, u0, T0 = make(name)
    sim.init(n0, u0, T0)
    F, G = orc.equilibrium(n0, u0, T0)
    sim.step(20)
    Fo, Go = orc.step(F, G, 20)
    Fg, Gg = sim.state_2d()
    assert rel(Fg, Fo) < 1e-11 and rel(Gg, Go) < 1e-11
    tot = sim.moments()[4]
    to = orc.totals(Fo, Go)
    assert abs(tot[0, 0] - to[0]) < 1e-12 * abs(to[0])
    assert abs(tot[0, 1] - to[1]) < 1e-12 * abs(to[0])
    assert abs(tot[0, 2] - to[2]) < 1e-11 * abs(to[2])
    assert abs(tot[0, 3] - to[3]) < 1e-11 * abs(to[3])


@pytest.mark.parametrize("name", ["periodic_q16_tile7", "outflow_q24_slab"])
def test_ev2_fp32_step(name):
    sim, orc, n0, u0, T0 = make(name, prec=ev.FP32)
    F, G = nonequilibrium_state(orc, n0, u0, T0)
    sim.set_state(F.ravel(), G.ravel())
    sim.step(1)
    Fg, Gg = sim.state_2d()
    Fo, Go = orc.step(F, G, 1)
    eF, eG = rel(Fg, Fo), rel(Gg, Go)
    print(f"EV2 FP32 {name}: step F {eF:.1e} G {eG:.1e}")
    assert eF < 1e-5 and eG < 1e-5


def test_ev2_periodic_conservation_200_steps():
    sim, orc, n0, u0, T0 = make("periodic_q16_tile7")
    sim.init(n0, u0, T0)
    t0 = sim.moments()[4][0]
    sim.step(200)
    t1 = sim.moments()[4][0]
    assert abs(t1[0] - t0[0]) < 1e-12 * t0[0]
    assert abs(t1[1] - t0[1]) < 1e-13 * t0[0]


def test_batch_mixing_ev1_and_ev2_slabs():
    """Four slabs in one context, EV1 and EV2 alternating, different sizes and
    boundary rules: each slab against the oracle of its own force model."""
    specs = [(64, 16, 0.25, 0, 0), (97, 16, 0.25, 1, 1), (40, 16, 0.25, 1, 0), (33, 16, 0.25, 0, 1)]
    ps = [ev.Params(nx=nz, dx=dz, Q=Q, bc=bc, force_model=fm) for nz, Q, dz, bc, fm in specs]
    sim = ev.Sim(ps)
    states, orcs = [], []
    for (nz, Q, dz, bc, fm) in specs:
        orc = O.Oracle(O.Setup(nz=nz, Q=Q, dz=dz, dt=sim.dt(), bc=bc, force_model=fm))
        n0, u0, T0 = inputs(orc, nz, dz, "slab" if bc else "noise")
        states.append(nonequilibrium_state(orc, n0, u0, T0))
        orcs.append(orc)
    sim.set_state(np.concatenate([F.ravel() for F, _ in states]), np.concatenate([G.ravel() for _, G in states]))
    sim.step(2)
    Fg, Gg = sim.get_state()
    off = 0
    for (F, G), orc in zip(states, orcs):
        Fo, Go = orc.step(F, G, 2)
        n = Fo.size
        assert rel(Fg[off:off + n], Fo.ravel()) < 1e-12 and rel(Gg[off:off + n], Go.ravel()) < 1e-12
        off += n


@pytest.mark.parametrize("case", [(64, 16, 0.25, 0, 7), (97, 24, 0.25, 0, 13)])   # the adjoint is periodic-only
def test_ev2_adjoint_dot_product_identity(case):
    nz, Q, dz, bc, tile = case
    sim = ev.Sim(ev.Params(nx=nz, dx=dz, Q=Q, bc=bc, force_model=ev.EV2))
    sim.tune(tile)
    orc = O.Oracle(O.Setup(nz=nz, Q=Q, dz=dz, dt=sim.dt(), bc=bc, force_model=1))
    rng = np.random.default_rng(nz + 1)
    z = np.arange(nz)
    n0 = 0.25 * (1 + 0.3 * np.sin(2 * np.pi * z / nz) + 0.02 * rng.uniform(-1, 1, nz))
    F, G = nonequilibrium_state(orc, n0, 0.04 * np.cos(2 * np.pi * z / nz), np.full(nz, 0.6))
    sim.set_state(F.ravel(), G.ravel())
    for trial in range(3):
        vF, vG = F * rng.uniform(-1, 1, F.shape), G * rng.uniform(-1, 1, G.shape)
        wF, wG = rng.uniform(-1, 1, F.shape), rng.uniform(-1, 1, G.shape)
        dphi_dir = rng.uniform(-1, 1)
        _, _, jF, jG = orc.rhs_tl(F, G, vF, vG, dphi=dphi_dir)
        lhs = (wF * jF).sum() + (wG * jG).sum()
        oF, oG, dphi = sim.rhs_vjp(wF.ravel(), wG.ravel())
        rhs = (oF.reshape(Q, nz) * vF).sum() + (oG.reshape(Q, nz) * vG).sum() + dphi[0] * dphi_dir
        scale = np.sqrt((wF ** 2).sum() + (wG ** 2).sum()) * np.sqrt((jF ** 2).sum() + (jG ** 2).sum())
        print(f"EV2 {case}: rel {abs(lhs - rhs) / scale:.2e}")
        assert abs(lhs - rhs) < 1e-11 * scale


def test_ev2_liquid_slab_full_size_one_step():
    """The liquid-slab workload (Nz = 4096, dz = 0.1, Q = 32, outflow, 20-sigma
    slab at the EV2 coexistence densities of T = 0.8 T_c) under EV2, default
    launch configuration: one step against the oracle."""
    nz, Q, dz = 4096, 32, 0.1
    sim = ev.Sim(ev.Params(nx=nz, dx=dz, Q=Q, bc=ev.BC_OUTFLOW, force_model=ev.EV2))
    orc = O.Oracle(O.Setup(nz=nz, Q=Q, dz=dz, dt=sim.dt(), bc=1, force_model=1))
    T = 0.8 * orc.critical_T()
    nv, nl = O.coexistence(T, orc.discrete_a())
    n0 = W.liquid_slab(nz, dz, nl, nv, thickness=20.0, width=2.0)
    F, G = orc.equilibrium(n0, np.zeros(nz), np.full(nz, T))
    sim.set_state(F.ravel(), G.ravel())
    sim.step(1)
    Fg, Gg = sim.state_2d()
    Fo, Go = orc.step(F, G, 1)
    assert rel(Fg, Fo) < 1e-12 and rel(Gg, Go) < 1e-12
