"""Pins of the oracle's isothermal mode.  Sec. III.A keeps the temperature
constant without saying how; the reading: after every step each node's
temperature is set back to T_iso, keeping its density, velocity and
non-equilibrium part (F += F_MB(n, u, T_iso) - F_MB(n, u, T), likewise G).

The pins check what that operation must do, against the thermal step and the
moment definitions, not by restating it:
* a uniform Maxwellian at T1 becomes the projected Maxwellian at T_iso after
  one step (the thermal step leaves a uniform equilibrium unchanged);
* after a step every node's kinetic temperature is T_iso, and the density,
  velocity, heat flux q and the anisotropy T_x - T (T_x the temperature of
  the p_x motion alone) equal those of the thermal step;
* mass and momentum are conserved on a periodic grid; the right-hand side
  itself is the thermal one.
"""
import numpy as np
import pytest

import oracle as O


def mk(nz=48, Q=16, dz=0.25, bc=0, T_iso=0.0, fm=0, dt=None):
    if dt is None:
        xi, _ = O.gauss_hermite(Q)
        dt = 0.5 * dz / np.abs(xi).max()
    return O.Oracle(O.Setup(nz=nz, Q=Q, dz=dz, dt=dt, bc=bc, T_iso=T_iso, force_model=fm))


def kinetic_moments(o, F, G):
    """n, u, T, q from the definitions, and T_x = sum (xi - u)^2 F / n."""
    xi = o.xi[:, None]
    n = F.sum(0)
    u = (xi * F).sum(0) / n
    c = xi - u
    Tx = (c * c * F).sum(0) / n
    T = (2.0 / 3.0) * ((0.5 * c * c * F + G).sum(0)) / n
    q = (c * (0.5 * c * c * F + G)).sum(0)
    return n, u, T, q, Tx


@pytest.mark.parametrize("T1,T_iso,fm", [(0.7, 0.55, 0), (0.45, 0.6, 1)])
def test_uniform_maxwellian_is_reset_to_T_iso(T1, T_iso, fm):
    nz = 24
    o = mk(nz=nz, T_iso=T_iso, fm=fm)
    F0, G0 = o.equilibrium(np.full(nz, 0.3), np.zeros(nz), np.full(nz, T1))
    Fe, Ge = o.equilibrium(np.full(nz, 0.3), np.zeros(nz), np.full(nz, T_iso))
    F, G = o.step(F0, G0, 1)
    assert np.abs(F - Fe).max() < 1e-14 * Fe.max()
    assert np.abs(G - Ge).max() < 1e-14 * Ge.max()


@pytest.mark.parametrize("fm,bc", [(0, 0), (1, 1)])
def test_step_sets_T_and_keeps_the_other_moments_of_the_thermal_step(fm, bc):
    nz = 40
    rng = np.random.default_rng(5)
    z = np.arange(nz)
    n = 0.25 * (1 + 0.3 * np.sin(2 * np.pi * z / nz) + 0.02 * rng.uniform(-1, 1, nz))
    u = 0.04 * np.cos(2 * np.pi * z / nz)
    T = 0.6 * (1 + 0.05 * np.sin(4 * np.pi * z / nz))
    th = mk(nz=nz, fm=fm, bc=bc)
    iso = mk(nz=nz, fm=fm, bc=bc, T_iso=0.58)
    F, G = th.step(*th.equilibrium(n, u, T), 2)          # a non-equilibrium state
    Ft, Gt = th.step(F, G, 1)
    Fi, Gi = iso.step(F, G, 1)
    nt, ut, Tt, qt, Txt = kinetic_moments(th, Ft, Gt)
    ni, ui, Ti, qi, Txi = kinetic_moments(th, Fi, Gi)
    assert np.abs(Ti - 0.58).max() < 1e-14
    assert np.abs(ni - nt).max() < 1e-15 and np.abs(ui - ut).max() < 1e-15
    assert np.abs(qi - qt).max() < 1e-14 * (nt * Tt ** 1.5).max()     # q cancels O(n T^1.5) terms
    assert np.abs((Txi - Ti) - (Txt - Tt)).max() < 1e-14
    # the right-hand side is the thermal one
    RFi, RGi = iso.rhs(F, G)
    RFt, RGt = th.rhs(F, G)
    assert np.array_equal(RFi, RFt) and np.array_equal(RGi, RGt)


def test_isothermal_conserves_mass_and_momentum():
    nz = 64
    o = mk(nz=nz, T_iso=0.55)
    rng = np.random.Generator(np.random.PCG64(31))
    n = 0.25 * (1 + 0.05 * rng.uniform(-1, 1, nz))
    u = 0.02 * rng.uniform(-1, 1, nz)
    T = 0.55 * (1 + 0.1 * rng.uniform(-1, 1, nz))
    F, G = o.equilibrium(n, u, T)
    t0 = o.totals(F, G)
    F1, G1 = o.step(F, G, 5)
    t1 = o.totals(F1, G1)
    assert abs(t1[0] - t0[0]) < 1e-13 * t0[0]
    assert abs(t1[1] - t0[1]) < 1e-14 * t0[0]
    assert np.abs(o.moments(F1, G1)[2] - 0.55).max() < 1e-14
