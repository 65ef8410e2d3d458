"""The paper's three numerical experiments (Sec. III) at its discretisation
(dx = sigma/10, dt = 5e-3, Q = 16) on the GPU path, with shortened runs and
checks of what must hold at any length:

* planar interfaces at constant T (Sec. III.A): after 1e5 steps at T = 0.7
  the bulk densities sit within 0.3% of the Maxwell construction of the force
  model's own attraction constant, the flow has decayed, T = T_iso at every
  node, the profile is mirror-symmetric and mass is conserved; at T = 0.55
  EV2 stays finite (the paper's lowest temperature);
* phase separation from a sinusoid (Sec. III.B): mass, momentum and energy
  conserved, mirror symmetry kept, density contrast growing;
* evaporation into metastable vapour (Sec. III.C): outward flow on each side,
  evaporative cooling below T_i and compression heating above it, n even and
  u odd in x, mass conserved.
"""
import numpy as np
import pytest

import paper_2503_15187_gb300 as ev
from paper_2503_15187_gb300 import experiments as E

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("fm", [ev.EV1, ev.EV2])
def test_interface_at_constant_temperature(fm):
    T = 0.7
    r = E.run_interface(T, fm, steps=(100000,))
    n, u, Tk = r["n"][-1], r["u"][-1], r["T"][-1]
    nz = len(n)
    assert abs(n[nz // 2] / r["n_l"] - 1) < 3e-3       # liquid at x = 0
    assert abs(n[0] / r["n_v"] - 1) < 3e-3             # vapour at x = +-100 sigma
    assert np.abs(u).max() < 1e-3
    assert np.abs(Tk - T).max() < 1e-13
    assert np.abs(n - n[::-1]).max() < 1e-12
    m0 = r["n0"].sum() * E.DX
    assert abs(r["totals"][-1][0] - m0) < 1e5 * 2e-16 * m0      # FP64 rounding per step


def test_interface_ev2_lowest_temperature_stays_finite():
    r = E.run_interface(0.55, ev.EV2, steps=(20000,))
    n, u = r["n"][-1], r["u"][-1]
    assert np.all(np.isfinite(n)) and n.min() > 0.5 * r["n_v"] and np.abs(u).max() < 0.05


@pytest.mark.parametrize("fm", [ev.EV1, ev.EV2])
def test_phase_separation_from_sinusoid(fm):
    r = E.run_phase_separation(0.7, 0.4, fm, steps=(1, 20000))
    n0 = r["n0"]
    t0, t1 = r["totals"][0], r["totals"][-1]
    assert abs(t1[0] / t0[0] - 1) < 1e-11
    assert abs(t1[1]) < 1e-13 * t0[0]
    assert abs(t1[2] / t0[2] - 1) < 5e-5                 # energy, to truncation error
    n = r["n"][-1]
    assert np.abs(n - n[::-1]).max() < 1e-12
    assert n.max() > n0.max() and n.min() < n0.min()


@pytest.mark.parametrize("fm", [ev.EV1, ev.EV2])
def test_evaporation_into_metastable_vapour(fm):
    T_i = 0.7
    r = E.run_evaporation(T_i, fm, times=(25.0,))
    x, n, u, T = r["x"], r["n"][-1], r["u"][-1], r["T"][-1]
    right = x > 0
    assert u[right].max() > 0.03 and u[right].max() > 10 * abs(min(u[right].min(), 0.0))
    assert T.min() < T_i - 0.03 and T.max() > T_i + 0.005
    assert np.abs(n - n[::-1]).max() < 1e-12 and np.abs(u + u[::-1]).max() < 1e-12
    m0 = r["n0"].sum() * E.DX
    assert abs(r["totals"][-1][0] - m0) < 1e-12 * m0
