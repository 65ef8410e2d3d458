"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the
same seeded inputs.

Error measure (per distribution F, G): ||GPU - oracle||_inf / ||oracle||_inf.
Bars: 1e-12 per step (state), 1e-11 for a single right-hand side (which can
be small against its terms), 1e-8 on end-of-run moments.  Cases span tiles
of several sizes with a ragged last tile, both boundary rules, both
relaxation readings and Q = 8..32, odd orders included.
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
    # name: (nz, Q, dz, bc, relax, profile, tile)
    "periodic_q16": (64, 16, 0.25, 0, 0, "noise", None),
    "periodic_q16_tile7": (64, 16, 0.25, 0, 0, "noise", 7),
    "outflow_q24_slab": (97, 24, 0.25, 1, 0, "slab", 13),
    "outflow_q32_dz01": (150, 32, 0.1, 1, 0, "slab", 27),
    "periodic_q8_chi_over_tau": (50, 8, 0.25, 0, 1, "noise", 64),
    "periodic_q12_short": (16, 12, 0.25, 0, 0, "noise", 5),
    # odd orders: a zero velocity node, the middle of the parity split
    "periodic_q9_odd": (40, 9, 0.25, 0, 0, "noise", 6),
    "outflow_q31_odd": (77, 31, 0.25, 1, 0, "slab", 11),
}


def make(name):
    nz, Q, dz, bc, relax, prof, tile = CASES[name]
    p = ev.Params(nx=nz, dx=dz, Q=Q, bc=bc, relax_mode=relax)
    sim = ev.Sim(p)
    if tile:
        sim.tune(tile)
    orc = O.Oracle(O.Setup(nz=nz, Q=Q, dz=dz, dt=sim.dt(), bc=bc, relax=relax))
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
    return sim, orc, n0, u0, T0


def nonequilibrium_state(orc, n0, u0, T0, steps=2):
    F, G = orc.equilibrium(n0, u0, T0)
    return orc.step(F, G, steps)


@pytest.mark.parametrize("name", list(CASES))
def test_init_is_projected_maxwellian(name):
    sim, orc, n0, u0, T0 = make(name)
    sim.init(n0, u0, T0)
    Fg, Gg = sim.state_2d()
    Fo, Go = orc.equilibrium(n0, u0, T0)
    assert rel(Fg, Fo) < 1e-13 and rel(Gg, Go) < 1e-13


@pytest.mark.parametrize("name", list(CASES))
def test_node_fields(name):
    sim, orc, n0, u0, T0 = make(name)
    F, G = nonequilibrium_state(orc, n0, u0, T0)
    sim.set_state(F.ravel(), G.ravel())
    fg = sim.fields()
    fo = orc.node_fields(F, G)
    names = {"n": "n", "u": "u", "T": "T", "q": "q", "nbar": "nbar", "chi": "chi", "force": "force",
             "mu": "mu", "tau": "tau", "Pr": "Pr", "nu": "rate", "A": "A", "B": "B", "D": "D", "X": "X",
             "bnchi": "bnchi"}
    dz = CASES[name][2]
    for k, ko in names.items():
        if k in ("A", "B", "D"):
            # fourth-order differences of nearly uniform fields: rounding in
            # the inputs is amplified by ~1/dz, the natural scale of the result
            scale = max(np.abs(fo[ko]).max(), (np.sqrt(fo["T"].max()) if k == "D" else 1.0) / dz)
            err = np.abs(fg[k] - fo[ko]).max() / scale
        elif k == "q":
            # the heat flux is a small difference of O(n T^1.5) moments: measure
            # it on that scale (the GPU forms it from raw sums, the oracle from
            # centred sums)
            scale = np.max(fo["n"] * fo["T"] ** 1.5)
            err = np.abs(fg[k] - fo[ko]).max() / scale
        else:
            err = rel(fg[k], fo[ko])
        assert err < 1e-12, (k, err)


@pytest.mark.parametrize("name", list(CASES))
def test_rhs(name):
    sim, orc, n0, u0, T0 = make(name)
    F, G = nonequilibrium_state(orc, n0, u0, T0)
    sim.set_state(F.ravel(), G.ravel())
    RF, RG = sim.rhs()
    RFo, RGo = orc.rhs(F, G)
    Q, nz = F.shape
    assert rel(RF.reshape(Q, nz), RFo) < 1e-11
    assert rel(RG.reshape(Q, nz), RGo) < 1e-11


@pytest.mark.parametrize("name", list(CASES))
def test_one_step(name):
    sim, orc, n0, u0, T0 = make(name)
    F, G = nonequilibrium_state(orc, n0, u0, T0)
    sim.set_state(F.ravel(), G.ravel())
    sim.step(1)
    Fg, Gg = sim.state_2d()
    Fo, Go = orc.step(F, G, 1)
    assert rel(Fg, Fo) < 1e-12 and rel(Gg, Go) < 1e-12


@pytest.mark.parametrize("name", ["periodic_q16_tile7", "outflow_q24_slab"])
def test_twenty_steps_and_totals(name):
    sim, orc, n0, u0, T0 = make(name)
    sim.init(n0, u0, T0)
    F, G = orc.equilibrium(n0, u0, T0)
    sim.step(20)
    Fo, Go = orc.step(F, G, 20)
    Fg, Gg = sim.state_2d()
    assert rel(Fg, Fo) < 1e-11 and rel(Gg, Go) < 1e-11
    n, u, T, q, tot = sim.moments()
    no, uo, To, qo = orc.moments(Fo, Go)
    assert rel(n, no) < 1e-11 and rel(T, To) < 1e-11 and rel(u, uo) < 1e-9
    to = orc.totals(Fo, Go)
    assert abs(tot[0, 0] - to[0]) < 1e-12 * abs(to[0])
    assert abs(tot[0, 1] - to[1]) < 1e-12 * abs(to[0])
    assert abs(tot[0, 2] - to[2]) < 1e-11 * abs(to[2])
    assert abs(tot[0, 3] - to[3]) < 1e-11 * abs(to[3])


def test_moments_with_and_without_totals_agree():
    """The node moments come from the totals' first pass when totals are asked
    for and from a kernel of their own otherwise: the same values, and the
    oracle's."""
    sim, orc, n0, u0, T0 = make("outflow_q24_slab")
    F, G = nonequilibrium_state(orc, n0, u0, T0)
    sim.set_state(F.ravel(), G.ravel())
    a = sim.moments()
    b = sim.moments(with_totals=False)
    for x, y in zip(a[:4], b[:4]):
        assert rel(x, y) < 1e-15
    no, uo, To, qo = orc.moments(F, G)
    assert rel(b[0], no) < 1e-13 and rel(b[2], To) < 1e-12 and rel(b[3], qo) < 1e-9


def test_bad_state_is_reported_by_the_next_synchronising_call():
    """set_state returns once its copies have run; a state whose moment sums
    are not finite is reported by the next call that synchronises, after which
    the context refuses to step until a new state is set."""
    sim, orc, n0, u0, T0 = make("periodic_q16")
    F, G = nonequilibrium_state(orc, n0, u0, T0)
    bad = F.copy()
    bad[3, 5] = np.nan
    sim.set_state(bad.ravel(), G.ravel())
    with pytest.raises(ev.EvfdlbError) as e:
        sim.step(1)
    assert e.value.code == -4
    with pytest.raises(ev.EvfdlbError) as e:
        sim.step(1)
    assert e.value.code == -7
    sim.set_state(F.ravel(), G.ravel())            # recovers
    sim.step(1)
    Fg, Gg = sim.state_2d()
    Fo, Go = orc.step(F, G, 1)
    assert rel(Fg, Fo) < 1e-12 and rel(Gg, Go) < 1e-12


def test_set_state_from_page_locked_memory_releases_the_arrays():
    """From page-locked host arrays the copies are asynchronous; set_state
    returns only once they have run, so the caller may overwrite its arrays at
    once."""
    import torch
    sim, orc, n0, u0, T0 = make("outflow_q32_dz01")
    F, G = nonequilibrium_state(orc, n0, u0, T0)
    Fp = torch.empty(F.size, dtype=torch.float64, pin_memory=True).numpy()
    Gp = torch.empty(G.size, dtype=torch.float64, pin_memory=True).numpy()
    for _ in range(3):
        Fp[:] = F.ravel()
        Gp[:] = G.ravel()
        sim.set_state(Fp, Gp)
        Fp[:] = -1.0
        Gp[:] = np.nan
        sim.step(1)
        Fg, Gg = sim.state_2d()
    Fo, Go = orc.step(F, G, 1)
    assert rel(Fg, Fo) < 1e-12 and rel(Gg, Go) < 1e-12


def test_mass_momentum_conserved_on_gpu():
    sim, orc, n0, u0, T0 = make("periodic_q16")
    sim.init(n0, u0, T0)
    t0 = sim.moments()[4][0]
    sim.step(200)
    t1 = sim.moments()[4][0]
    assert abs(t1[0] - t0[0]) < 1e-12 * t0[0]
    assert abs(t1[1] - t0[1]) < 1e-13 * t0[0]


def test_errors_are_reported_not_faulted():
    """Invalid states are caught by the kernels' checks and returned as status
    codes; the context stays usable after init."""
    sim, orc, n0, u0, T0 = make("periodic_q16")
    with pytest.raises(ev.EvfdlbError) as e:
        sim.step(1)
    assert e.value.code == -7                      # step before init
    bad = n0.copy()
    bad[5] = -0.1
    with pytest.raises(ev.EvfdlbError) as e:
        sim.init(bad, u0, T0)
    assert e.value.code == -5
    bad[5] = np.nan
    with pytest.raises(ev.EvfdlbError) as e:
        sim.init(bad, u0, T0)
    assert e.value.code == -4
    sim.init(n0, u0, T0)                           # recovers
    sim.step(2)


# ---------------------------------------------------------------------------
# full-size workloads
# ---------------------------------------------------------------------------
def test_liquid_slab_evaporation_full_size_one_step():
    """Nz = 4096, dz = 0.1, Q = 32, outflow ends, centred 20-sigma liquid slab at
    the coexistence density of T = 0.8 T_c, in the default launch configuration
    the benchmark times; one step against the oracle on every output."""
    nz, Q, dz = 4096, 32, 0.1
    p = ev.Params(nx=nz, dx=dz, Q=Q, bc=ev.BC_OUTFLOW)
    sim = ev.Sim(p)
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


def test_phase_separation_full_run_moments():
    """Nz = 256, dz = 0.25, Q = 16, periodic, T = 0.7 T_c, mean n = 0.25 with
    +-1% seeded noise, 2000 steps at CFL 0.5: end-of-run n, T against the oracle."""
    nz, Q, dz = 256, 16, 0.25
    p = ev.Params(nx=nz, dx=dz, Q=Q)
    sim = ev.Sim(p)
    orc = O.Oracle(O.Setup(nz=nz, Q=Q, dz=dz, dt=sim.dt()))
    T = 0.7 * orc.critical_T()
    n0 = W.noisy_uniform(nz, 0.25, 0.01)
    sim.init(n0, np.zeros(nz), np.full(nz, T))
    sim.step(2000)
    F, G = orc.equilibrium(n0, np.zeros(nz), np.full(nz, T))
    Fo, Go = orc.step(F, G, 2000)
    n, u, Tg, q, _ = sim.moments()
    no, uo, To, qo = orc.moments(Fo, Go)
    assert rel(n, no) < 1e-8 and rel(Tg, To) < 1e-8
