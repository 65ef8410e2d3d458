"""GPU parity of the two-dimensional model (evfdlb_2d.cu) against the 2D
oracle (evfdlb_oracle2d.c) on the same seeded inputs.

FP64 build: projected initial state 1e-13, one right-hand side 1e-11, one
RK step 1e-12 (the 1D bars).  FP32 build (the phase-separation variant:
FP32 bulk, FP64 conserved sums): 2e-7 for the projected state (one FP32
rounding), 1e-5 per step (Q^2-term Hermite transforms and WENO in FP32,
u = 2^-24).  Grids are not multiples of the 16x16 field tiles, the 8-node
collision groups or the 32x16 advection tiles.  At the full 1024 x 1024,
16 x 16-velocity size the checks are properties that hold at any size: a
uniform state is stationary, mass and momentum are conserved.
"""
import numpy as np
import pytest

import oracle as O
import paper_2503_15187_gb300 as ev

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300))


def fields(nx, ny, seed=3):
    rng = np.random.default_rng(seed)
    X, Y = np.meshgrid(np.arange(nx), np.arange(ny))
    n = 0.25 * (1 + 0.25 * np.sin(2 * np.pi * X / nx) * np.cos(2 * np.pi * Y / ny) + 0.02 * rng.uniform(-1, 1, (ny, nx)))
    ux = 0.03 * np.cos(2 * np.pi * Y / ny)
    uy = 0.02 * np.sin(2 * np.pi * X / nx)
    T = 0.6 * (1 + 0.04 * np.cos(2 * np.pi * (X / nx + Y / ny)))
    return n, ux, uy, T


def make(nx, ny, Q, prec, dx=0.25):
    p = ev.Params(nx=nx, dx=dx, Q=Q, dim=2, ny=ny, precision=prec)
    sim = ev.Sim(p)
    orc = O.Oracle2D(O.Setup2(nx=nx, ny=ny, Q=Q, dx=dx, dt=sim.dt()))
    return sim, orc


# (19, 17, 16): the velocity count of the 2D workload; 323 nodes leave a
# ragged last collision group of 3 nodes
CASES = [(24, 20, 6), (19, 33, 8), (19, 17, 16)]


@pytest.mark.parametrize("nx,ny,Q", CASES)
def test_2d_fp64_init_rhs_step(nx, ny, Q):
    sim, orc = make(nx, ny, Q, ev.FP64)
    n, ux, uy, T = fields(nx, ny)
    sim.init(n.ravel(), np.concatenate([ux.ravel(), uy.ravel()]), T.ravel())
    Fg, Gg = sim.state_2d()
    Fo, Go = orc.equilibrium(n, ux, uy, T)
    assert rel(Fg, Fo) < 1e-13 and rel(Gg, Go) < 1e-13
    F, G = orc.step(Fo, Go, 1)                     # a non-equilibrium state
    sim.set_state(F.ravel(), G.ravel())
    RF, RG = sim.rhs()
    RFo, RGo = orc.rhs(F, G)
    eF, eG = rel(RF.reshape(RFo.shape), RFo), rel(RG.reshape(RGo.shape), RGo)
    print(f"2D FP64 {nx}x{ny} Q={Q}: rhs F {eF:.1e} G {eG:.1e}")
    assert eF < 1e-11 and eG < 1e-11
    sim.step(1)
    Fg, Gg = sim.state_2d()
    Fo2, Go2 = orc.step(F, G, 1)
    eF, eG = rel(Fg, Fo2), rel(Gg, Go2)
    print(f"2D FP64 {nx}x{ny} Q={Q}: step F {eF:.1e} G {eG:.1e}")
    assert eF < 1e-12 and eG < 1e-12
    n_g, u_g, T_g, q_g, tot = sim.moments()
    n_o, ux_o, uy_o, T_o, qx_o, qy_o = orc.moments(Fo2, Go2)
    assert rel(n_g, n_o.ravel()) < 1e-12 and rel(T_g, T_o.ravel()) < 1e-12
    assert rel(q_g[0], qx_o.ravel()) < 1e-9 and rel(q_g[1], qy_o.ravel()) < 1e-9
    to = orc.totals(Fo2, Go2)
    assert np.allclose(tot[0], to, rtol=1e-12, atol=1e-12 * to[0])


@pytest.mark.parametrize("nx,ny,Q", CASES)
def test_2d_fp32_against_fp64_oracle(nx, ny, Q):
    sim, orc = make(nx, ny, Q, ev.FP32)
    n, ux, uy, T = fields(nx, ny, seed=5)
    sim.init(n.ravel(), np.concatenate([ux.ravel(), uy.ravel()]), T.ravel())
    Fg, Gg = sim.state_2d()
    Fo, Go = orc.equilibrium(n, ux, uy, T)
    assert rel(Fg, Fo) < 2e-7 and rel(Gg, Go) < 2e-7
    F, G = orc.step(Fo, Go, 1)
    sim.set_state(F.ravel(), G.ravel())
    sim.step(1)
    Fg, Gg = sim.state_2d()
    Fo2, Go2 = orc.step(F, G, 1)
    eF, eG = rel(Fg, Fo2), rel(Gg, Go2)
    print(f"2D FP32 {nx}x{ny} Q={Q}: step F {eF:.1e} G {eG:.1e}")
    assert eF < 1e-5 and eG < 1e-5


def test_2d_conservation_fp32():
    nx, ny, Q = 48, 40, 8
    sim, _ = make(nx, ny, Q, ev.FP32)
    n, ux, uy, T = fields(nx, ny, seed=9)
    sim.init(n.ravel(), np.concatenate([ux.ravel(), uy.ravel()]), T.ravel())
    t0 = sim.moments()[4][0]
    steps = 50
    sim.step(steps)
    t1 = sim.moments()[4][0]
    dm = abs(t1[0] - t0[0]) / t0[0]
    dpx, dpy = abs(t1[1] - t0[1]) / t0[0], abs(t1[2] - t0[2]) / t0[0]
    print(f"2D FP32 drift over {steps} steps: mass {dm:.1e} momentum {dpx:.1e} {dpy:.1e}")
    # FP64 sums of an FP32 state: each step stores the state once in FP32
    assert dm < steps * 2.0 ** -24 and dpx < steps * 2.0 ** -24 and dpy < steps * 2.0 ** -24


def test_2d_phase_separation_full_size_properties():
    """1024 x 1024 periodic grid, dx = 0.25, 16 x 16 velocities, FP32 bulk
    with FP64 conserved sums, T = 0.75 T_c, mean n = 0.25 with +-1% seeded
    noise: 10 steps conserve mass and momentum; a uniform state of the same
    size stays uniform."""
    nx = ny = 1024
    Q = 16
    p = ev.Params(nx=nx, dx=0.25, Q=Q, dim=2, ny=ny, precision=ev.FP32)
    T = 0.75 * ev.critical_T(p)
    sim = ev.Sim(p)
    rng = np.random.default_rng(15187)
    n0 = 0.25 * (1 + 0.01 * rng.uniform(-1, 1, nx * ny))
    sim.init(n0, np.zeros(2 * nx * ny), np.full(nx * ny, T))
    t0 = sim.moments()[4][0]
    sim.step(10)
    n, u, Tg, q, t1 = sim.moments()
    t1 = t1[0]
    assert abs(t1[0] - t0[0]) < 10 * 2.0 ** -24 * t0[0]
    assert abs(t1[1]) < 10 * 2.0 ** -24 * t0[0] and abs(t1[2]) < 10 * 2.0 ** -24 * t0[0]
    assert np.all(n > 0) and np.all(np.isfinite(Tg))
    sim.init(np.full(nx * ny, 0.25), np.zeros(2 * nx * ny), np.full(nx * ny, T))
    sim.step(3)
    n, u, Tg, q, _ = sim.moments()
    assert np.abs(n - 0.25).max() < 1e-6 and np.abs(u).max() < 1e-6 and np.abs(Tg - T).max() < 1e-6 * T
    sim.close()


@pytest.mark.parametrize("prec,bar", [(ev.FP64, 1e-12), (ev.FP32, 1e-5)])
@pytest.mark.parametrize("dx,rcut", [(0.5, 4.5), (0.5, 6.0)])
def test_2d_other_disc_shapes(prec, bar, dx, rcut):
    """The force disc as column plans other than the workload's: dx = 0.5
    with r_cut = 4.5 (9 offset columns each side) and 6 (12), odd and
    ragged grids; one step against the oracle in each precision."""
    nx, ny, Q = 23, 17, 8
    p = ev.Params(nx=nx, dx=dx, Q=Q, dim=2, ny=ny, precision=prec, r_cut=rcut)
    sim = ev.Sim(p)
    orc = O.Oracle2D(O.Setup2(nx=nx, ny=ny, Q=Q, dx=dx, dt=sim.dt(), rcut=rcut))
    n, ux, uy, T = fields(nx, ny, seed=11)
    F, G = orc.equilibrium(n, ux, uy, T)
    F, G = orc.step(F, G, 1)
    sim.set_state(F.ravel(), G.ravel())
    sim.step(1)
    Fg, Gg = sim.state_2d()
    Fo, Go = orc.step(F, G, 1)
    eF, eG = rel(Fg, Fo), rel(Gg, Go)
    print(f"2D dx={dx} r_cut={rcut} prec={prec}: step F {eF:.1e} G {eG:.1e}")
    assert eF < bar and eG < bar


# A grid wider than the force disc on both axes (r_cut = 6 at dx = 0.25: 49
# nodes across), and a multiple of no tile edge: the 16 x 16 field tiles,
# the 32 x 16 advection tiles and the 8-node collision groups all have
# interior instances and ragged edges, and every force tap wraps the
# periodic domain at most once -- the configuration of the 1024 x 1024 run.
BIG = (72, 61, 16)


@pytest.fixture(scope="module")
def big_case():
    import oracle as Om
    nx, ny, Q = BIG
    xi, _ = Om.gauss_hermite(Q)
    dx = 0.25
    dt = 0.5 * dx / (2 * np.abs(xi).max())          # the library's default CFL step
    orc = Om.Oracle2D(Om.Setup2(nx=nx, ny=ny, Q=Q, dx=dx, dt=dt))
    n, ux, uy, T = fields(nx, ny, seed=21)
    F0, G0 = orc.equilibrium(n, ux, uy, T)
    F, G = orc.step(F0, G0, 1)                       # a non-equilibrium state
    RF, RG = orc.rhs(F, G)
    F1, G1 = orc.step(F, G, 1)
    return dict(dt=dt, F=F, G=G, RF=RF, RG=RG, F1=F1, G1=G1)


@pytest.mark.parametrize("prec,bar_step", [(ev.FP64, 1e-12), (ev.FP32, 1e-5)])
def test_2d_parity_beyond_the_force_disc(big_case, prec, bar_step):
    """72 x 61 grid, dx 0.25, r_cut 6, 16 x 16 velocities: one right-hand
    side (FP64, 1e-11) and one RK3 step (FP64 1e-12, FP32 1e-5) against the
    2D oracle, reaching the interior k2_fields / k2_adv tiles and the full
    1809-tap force column plan."""
    nx, ny, Q = BIG
    p = ev.Params(nx=nx, dx=0.25, Q=Q, dim=2, ny=ny, precision=prec)
    sim = ev.Sim(p)
    assert abs(sim.dt() - big_case["dt"]) < 1e-15 * big_case["dt"]
    sim.set_state(big_case["F"].ravel(), big_case["G"].ravel())
    if prec == ev.FP64:
        RF, RG = sim.rhs()
        eF = rel(RF.reshape(big_case["RF"].shape), big_case["RF"])
        eG = rel(RG.reshape(big_case["RG"].shape), big_case["RG"])
        print(f"2D FP64 {nx}x{ny}: rhs F {eF:.1e} G {eG:.1e}")
        assert eF < 1e-11 and eG < 1e-11
    sim.step(1)
    Fg, Gg = sim.state_2d()
    eF, eG = rel(Fg, big_case["F1"]), rel(Gg, big_case["G1"])
    print(f"2D prec={prec} {nx}x{ny}: step F {eF:.1e} G {eG:.1e}")
    assert eF < bar_step and eG < bar_step
    sim.close()
