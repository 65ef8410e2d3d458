"""Pins of the oracle's isothermal mode (Sec. III.A holds T constant; the
reading: every node field is formed at T = T_iso, so the collisions hold the
fluid at T_iso).

* A uniform fluid at rest with a Maxwellian at T1 != T_iso obeys the linear
  ODE dF/dt = -nu (F - F_eq(T_iso)) node by node (no streaming, no force, no
  J1 for a uniform state), with nu = 1/tau at (n, T_iso).  Shu-Osher RK3 on a
  linear ODE multiplies the deviation by the stability polynomial
  R(z) = 1 + z + z^2/2 + z^3/6 per step, z = -nu dt.  The oracle's state
  after k steps must be F_eq + R^k (F0 - F_eq), elementwise, for F and G.
* On a state whose kinetic temperature is already uniform and equal to
  T_iso, the isothermal right-hand side is the thermal one.
* Mass and momentum stay conserved on a periodic grid; B = 0 exactly.
"""
import numpy as np
import pytest

import oracle as O


def mk(nz=48, Q=16, dz=0.25, bc=0, T_iso=0.0, fm=0, dt=None):
    if dt is None:
        xi, _ = O.gauss_hermite(Q)
        dt = 0.5 * dz / np.abs(xi).max()
    return O.Oracle(O.Setup(nz=nz, Q=Q, dz=dz, dt=dt, bc=bc, T_iso=T_iso, force_model=fm))


@pytest.mark.parametrize("T1,T_iso,fm", [(0.7, 0.55, 0), (0.45, 0.6, 1), (0.6, 0.6, 0)])
def test_uniform_fluid_relaxes_by_the_rk3_stability_polynomial(T1, T_iso, fm):
    nz, n0, k = 24, 0.3, 7
    o = mk(nz=nz, T_iso=T_iso, fm=fm)
    F0, G0 = o.equilibrium(np.full(nz, n0), np.zeros(nz), np.full(nz, T1))
    Fe, Ge = o.equilibrium(np.full(nz, n0), np.zeros(nz), np.full(nz, T_iso))
    thermal = mk(nz=nz, fm=fm)
    nu = thermal.node_fields(Fe, Ge)["rate"][0]        # 1/tau at (n0, T_iso), Eq. (tau)
    z = -nu * o.s.dt
    R = 1 + z + z * z / 2 + z ** 3 / 6
    F, G = o.step(F0, G0, k)
    assert np.abs(F - (Fe + R ** k * (F0 - Fe))).max() < 1e-14 * F0.max()
    assert np.abs(G - (Ge + R ** k * (G0 - Ge))).max() < 1e-14 * G0.max()
    T = o.moments(F, G)[2]
    assert np.allclose(T, T_iso + R ** k * (T1 - T_iso), rtol=1e-13, atol=0)


def test_isothermal_rhs_equals_thermal_rhs_at_uniform_T_iso():
    nz = 40
    rng = np.random.default_rng(3)
    n = 0.25 * (1 + 0.2 * np.sin(2 * np.pi * np.arange(nz) / nz) + 0.02 * rng.uniform(-1, 1, nz))
    u = 0.03 * np.cos(2 * np.pi * np.arange(nz) / nz)
    for fm in (0, 1):
        iso, th = mk(nz=nz, T_iso=0.6, fm=fm), mk(nz=nz, fm=fm)
        F, G = th.equilibrium(n, u, np.full(nz, 0.6))
        RFi, RGi = iso.rhs(F, G)
        RFt, RGt = th.rhs(F, G)
        # the kinetic T of the projected state is 0.6 to rounding
        assert np.abs(RFi - RFt).max() < 1e-12 * np.abs(RFt).max()
        assert np.abs(RGi - RGt).max() < 1e-12 * np.abs(RGt).max()


def test_isothermal_fields_and_conservation():
    nz = 64
    o = mk(nz=nz, T_iso=0.55)
    rng = np.random.Generator(np.random.PCG64(31))
    n = 0.25 * (1 + 0.05 * rng.uniform(-1, 1, nz))
    u = 0.02 * rng.uniform(-1, 1, nz)
    T = 0.55 * (1 + 0.1 * rng.uniform(-1, 1, nz))
    F, G = o.equilibrium(n, u, T)
    f = o.node_fields(F, G)
    assert np.all(f["T"] == 0.55) and np.abs(f["B"]).max() < 1e-15     # stencil rounding only
    X = f["n"] ** 2 * f["chi"] * 0.55
    assert np.allclose(f["X"], X, rtol=1e-15)
    t0 = o.totals(F, G)
    t1 = o.totals(*o.step(F, G, 5))
    assert abs(t1[0] - t0[0]) < 1e-13 * t0[0]
    assert abs(t1[1] - t0[1]) < 1e-14 * t0[0]
    # the kinetic temperature moves towards T_iso
    T1 = o.moments(*o.step(F, G, 20))[2]
    assert np.abs(T1 - 0.55).max() < np.abs(T - 0.55).max()
