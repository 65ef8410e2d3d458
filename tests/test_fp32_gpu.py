"""GPU parity of the FP32 variant against the FP64 oracle.

The FP32 variant stores F, G and does the per-velocity work (WENO faces,
Hermite analysis and synthesis, force convolution, coefficient recurrences,
RK combine) and the transport coefficients and coefficient constants in
FP32, and keeps FP64 for the Fischer-Methfessel average and chi, the
gradients' differences, the heat flux and the per-node sums of the
conserved moments.  Its error against
the FP64 oracle is therefore set by FP32 rounding, u = 2^-24 = 6.0e-8 per
operation.  The bars below are derived from that: a right-hand side sums
O(Q) = 32 terms of the size of the state (Hermite synthesis), so its error is
bounded by about Q u |F| = 2e-6 of the state; one RK step adds three such
right-hand sides times dt plus the rounding of the stored state, so 1e-5
normwise per step (measured values are printed by -s); node fields formed
from FP32 sums (and, for the transport, in FP32 arithmetic over a few
operations) are good to ~1e-6.  Over a run the error grows at most
linearly in the number of steps on these non-chaotic cases.
Error measure: ||GPU - oracle||_inf / ||oracle||_inf per distribution.
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
    "outflow_q32_slab": (150, 32, 0.1, 1, "slab", None),
    "periodic_q16_noise": (64, 16, 0.25, 0, "noise", 7),
    "outflow_q24_slab_ragged": (97, 24, 0.25, 1, "slab", 13),
    "periodic_q15_odd": (55, 15, 0.25, 0, "noise", 9),
}


def make(name):
    nz, Q, dz, bc, prof, tile = CASES[name]
    p = ev.Params(nx=nz, dx=dz, Q=Q, bc=bc, precision=ev.FP32)
    sim = ev.Sim(p)
    if tile:
        sim.tune(tile)
    orc = O.Oracle(O.Setup(nz=nz, Q=Q, dz=dz, dt=sim.dt(), bc=bc))
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


def force_scale(orc, nmax):
    """sum_j |s_j g(j dz)| * max n: the size of the terms of the Eq. (F1) sum."""
    dz, M = orc.s.dz, int(round(orc.s.rcut / orc.s.dz))
    j = np.arange(-M, M + 1)
    s = np.where((j == -M) | (j == M), 1.0, np.where((j + M) % 2 == 1, 4.0, 2.0)) * dz / 3.0
    g = np.array([orc.force_kernel(x * dz) for x in j])
    return float(np.abs(s * g).sum() * nmax)


@pytest.mark.parametrize("name", list(CASES))
def test_fp32_init_and_fields(name):
    sim, orc, n0, u0, T0 = make(name)
    sim.init(n0, u0, T0)
    Fg, Gg = sim.state_2d()
    Fo, Go = orc.equilibrium(n0, u0, T0)
    eF, eG = rel(Fg, Fo), rel(Gg, Go)
    print(f"{name}: init F {eF:.2e} G {eG:.2e}")
    assert eF < 2e-7 and eG < 2e-7                  # one FP32 rounding of the state
    fg = sim.fields()
    fo = orc.node_fields(Fo, Go)
    for k in ("n", "T", "chi", "force", "nu"):
        if k == "force":
            # the force is a difference of tap terms of size sum_j |s_j g_j| n:
            # FP32 products and sums err on that scale, not on |F1|
            e = np.abs(fg[k] - fo[k]).max() / force_scale(orc, n0.max())
        else:
            e = rel(fg[k], fo[k if k != "nu" else "rate"])
        print(f"  field {k}: {e:.2e}")
        assert e < 2e-6, (k, e)


@pytest.mark.parametrize("name", list(CASES))
def test_fp32_one_step(name):
    sim, orc, n0, u0, T0 = make(name)
    F, G = orc.equilibrium(n0, u0, T0)
    F, G = orc.step(F, G, 2)
    sim.set_state(F.ravel(), G.ravel())
    sim.step(1)
    Fg, Gg = sim.state_2d()
    Fo, Go = orc.step(F, G, 1)
    eF, eG = rel(Fg, Fo), rel(Gg, Go)
    print(f"{name}: one step F {eF:.2e} G {eG:.2e}")
    assert eF < 1e-5 and eG < 1e-5


def test_fp32_hundred_steps_moments():
    sim, orc, n0, u0, T0 = make("outflow_q32_slab")
    sim.init(n0, u0, T0)
    F, G = orc.equilibrium(n0, u0, T0)
    sim.step(100)
    Fo, Go = orc.step(F, G, 100)
    n, u, T, q, tot = sim.moments()
    no, uo, To, qo = orc.moments(Fo, Go)
    en, eT = rel(n, no), rel(T, To)
    print(f"100 steps: n {en:.2e} T {eT:.2e}")
    assert en < 1e-4 and eT < 1e-4                 # 100 x the per-step bar


@pytest.mark.parametrize("name", ["outflow_q32_slab", "periodic_q15_odd"])
@pytest.mark.parametrize("after", ["stage", "set_state"])
def test_fp32_conserved_sums_are_fp64_sums_of_the_state(name, after):
    """The per-node sums of the conserved moments of an FP32 state are FP64
    sums of its stored float values: n = sum_k F_k, n u = sum_k xi_k F_k,
    n (3/2 T + u^2/2) = sum_k (xi_k^2 F_k / 2 + G_k), to FP64 rounding of a
    Q-term sum (Q 2^-53 of the sum of magnitudes), where FP32 accumulation
    would err by ~1e-7.  Formed by the stage kernel (the pair terms of its
    synthesis) and, after set_state, by the sums kernel."""
    sim, orc, n0, u0, T0 = make(name)
    if after == "stage":
        sim.init(n0, u0, T0)
        sim.step(3)
    else:
        F, G = orc.equilibrium(n0, u0, T0)
        F, G = orc.step(F, G, 2)
        sim.set_state(F.ravel(), G.ravel())
    F, G = sim.state_2d()                          # the stored floats, widened exactly
    assert np.array_equal(F, F.astype(np.float32).astype(np.float64))
    xi, _ = ev.velocity_set(F.shape[0])
    n, u, T, _, _ = sim.moments()
    Q = F.shape[0]
    bound = 4 * Q * 2.0 ** -53
    S0 = F.sum(axis=0)
    S1 = (xi[:, None] * F).sum(axis=0)
    E = (0.5 * xi[:, None] ** 2 * F + G).sum(axis=0)
    mag1 = (np.abs(xi)[:, None] * F).sum(axis=0)
    e0 = np.abs(n - S0).max() / S0.max()
    e1 = (np.abs(n * u - S1) / mag1).max()
    e2 = (np.abs(n * (1.5 * T + 0.5 * u * u) - E) / E).max()
    print(f"{name} after {after}: mass {e0:.1e} momentum {e1:.1e} energy {e2:.1e} (bound {bound:.1e})")
    assert e0 < bound and e1 < 4 * bound and e2 < 4 * bound


def test_fp32_mass_conserved_to_fp32_rounding():
    sim, orc, n0, u0, T0 = make("periodic_q16_noise")
    sim.init(n0, u0, T0)
    t0 = sim.moments()[4][0]
    sim.step(200)
    t1 = sim.moments()[4][0]
    drift = abs(t1[0] - t0[0]) / t0[0]
    print(f"mass drift over 200 FP32 steps: {drift:.2e}")
    # the FP64 sums see an FP32 state, and the flux-form update telescopes
    # only up to the rounding of each stored element: the mass can move by at
    # most about one FP32 rounding (u = 2^-24) of the state per step
    assert drift < 200 * 2.0 ** -24


def plateaus(n, dz):
    """Mean density of the liquid core (|z| < 3) and of the vapour band
    (15 < |z| < 18) of a centred slab, z measured from the domain centre."""
    z = (np.arange(n.size) - n.size / 2) * dz
    return n[np.abs(z) < 3.0].mean(), n[(np.abs(z) > 15.0) & (np.abs(z) < 18.0)].mean()


def test_fp32_coexistence_densities_against_oracle():
    """Liquid-slab evaporation family at a size the oracle runs in seconds:
    Nz = 400, dz = 0.1, Q = 32, outflow ends, 20-sigma slab at the coexistence
    densities of T = 0.8 T_c; after 600 steps the FP32 liquid and vapour
    densities agree with the FP64 oracle's to 1e-3 relative (the bar set for
    FP32 coexistence densities), and the whole profile to 1e-4."""
    nz, Q, dz = 400, 32, 0.1
    sim = ev.Sim(ev.Params(nx=nz, dx=dz, Q=Q, bc=ev.BC_OUTFLOW, precision=ev.FP32))
    orc = O.Oracle(O.Setup(nz=nz, Q=Q, dz=dz, dt=sim.dt(), bc=1))
    T = 0.8 * orc.critical_T()
    nv, nl = O.coexistence(T, orc.discrete_a())
    n0 = W.liquid_slab(nz, dz, nl, nv, thickness=20.0, width=2.0)
    sim.init(n0, np.zeros(nz), np.full(nz, T))
    sim.step(600)
    n32 = sim.moments()[0]
    F, G = orc.equilibrium(n0, np.zeros(nz), np.full(nz, T))
    Fo, Go = orc.step(F, G, 600)
    no = orc.moments(Fo, Go)[0]
    (l32, v32), (lo, vo) = plateaus(n32, dz), plateaus(no, dz)
    print(f"liquid {l32:.7f} (oracle {lo:.7f}); vapour {v32:.7f} (oracle {vo:.7f}); profile {rel(n32, no):.2e}")
    assert abs(l32 - lo) < 1e-3 * lo and abs(v32 - vo) < 1e-3 * vo
    assert rel(n32, no) < 1e-4


def test_fp32_liquid_slab_full_size_long_run():
    """Nz = 4096, dz = 0.1, Q = 32, outflow ends, 20-sigma liquid slab at the
    coexistence densities of T = 0.8 T_c, 20000 steps (t = 99): the FP32 and
    FP64 runs agree on the liquid and vapour plateau densities to 1e-3
    relative.  (The oracle takes hours at this size; the FP64 path it is
    checked against is pinned to the oracle step by step.)  The plateaus
    themselves move by about 1 % from the initial Maxwell densities as the
    non-equilibrium tanh interfaces relax and release heat; printed by -s."""
    nz, Q, dz = 4096, 32, 0.1
    orc = O.Oracle(O.Setup(nz=nz, Q=Q, dz=dz, dt=0.01, bc=1))
    T = 0.8 * orc.critical_T()
    nv, nl = O.coexistence(T, orc.discrete_a())
    n0 = W.liquid_slab(nz, dz, nl, nv, thickness=20.0, width=2.0)
    res = {}
    for prec in (ev.FP32, ev.FP64):
        sim = ev.Sim(ev.Params(nx=nz, dx=dz, Q=Q, bc=ev.BC_OUTFLOW, precision=prec))
        sim.init(n0, np.zeros(nz), np.full(nz, T))
        sim.step(20000)
        n, u, Tg = sim.moments()[:3]
        z = (np.arange(nz) - nz / 2) * dz
        liq = n[np.abs(z) < 3.0].mean()
        vap = n[(np.abs(z) > 60.0) & (np.abs(z) < 150.0)].mean()
        res[prec] = (liq, vap, Tg[np.abs(z) < 3.0].mean())
        sim.close()
    (l32, v32, T32), (l64, v64, T64) = res[ev.FP32], res[ev.FP64]
    print(f"liquid {l32:.6f} (fp64 {l64:.6f}, initial {nl:.6f}); vapour {v32:.6f} (fp64 {v64:.6f}, "
          f"initial {nv:.6f}); liquid T {T32:.6f} (fp64 {T64:.6f}, initial {T:.6f})")
    assert abs(l32 - l64) < 1e-3 * l64 and abs(v32 - v64) < 1e-3 * v64
