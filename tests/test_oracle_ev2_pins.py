"""Pins of the oracle's EV2 force (Eq. (F2), Sec. III) against facts that do
not come from the oracle's own EV2 code.

* The printed a and kappa of Eq. (F2) are the first and third moments of the
  EV1 plane kernel g of Eq. (F1): 2a = int s g(s) ds, 6 kappa = int s^3 g(s) ds
  (the gradient expansion of the convolution).  g is pinned in
  test_oracle_pins.py to the plane integral of the Sutherland force.
* On a periodic sinusoid the EV2 force equals the Fourier symbols of the two
  stencils, worked out by hand: the fourth-order first difference gives
  (8 sin kh - sin 2kh)/(6h) and the five-point third difference gives
  (sin 2kh - 2 sin kh)/h^3.  A wrong coefficient, sign or offset in either
  stencil fails it.
* The symbol converges to the continuum 2ak - kappa k^3 at second order.
* The oracle's Simpson EV1 force, at long wavelength, is 2 a_d k - kappa_R k^3
  with kappa_R = kappa - 2 pi phi sigma^6/(3R) the third moment of the kernel
  cut at R: EV2 is the gradient expansion of EV1.
* Antisymmetric stencils conserve momentum to rounding on a periodic grid; a
  uniform state is stationary under both boundary conditions.
"""
import math

import numpy as np
import pytest
from scipy import integrate

import oracle as O


def mk(nz=64, Q=8, dz=0.25, bc=0, fm=1, rcut=6.0, dt=None):
    if dt is None:
        xi, _ = O.gauss_hermite(Q)
        dt = 0.5 * dz / np.abs(xi).max()
    return O.Oracle(O.Setup(nz=nz, Q=Q, dz=dz, dt=dt, bc=bc, rcut=rcut, force_model=fm))


def kernel_moment(o, p, R=np.inf):
    f = lambda s: s ** p * o.force_kernel(s)
    return 2 * (integrate.quad(f, 0, 1, epsabs=1e-14)[0] + integrate.quad(f, 1, R, epsabs=1e-14)[0])


def symbol(o, nz, dz, kidx):
    """Force per unit amplitude of n = 0.3 + 0.01 sin(kz): the force is
    S(k) 0.01 cos(kz) for a linear, translation-invariant force."""
    L = nz * dz
    k = 2 * math.pi * kidx / L
    z = dz * np.arange(nz)
    n = 0.3 + 0.01 * np.sin(k * z)
    F, G = o.equilibrium(n, np.zeros(nz), np.full(nz, 0.7))
    f = o.node_fields(F, G)["force"]
    c = np.cos(k * z)
    big = np.abs(c) > 0.5
    S = f[big] / (0.01 * c[big])
    assert np.ptp(S) < 1e-9 * abs(S).max()          # the force is a pure cosine
    return float(S.mean()), k


def test_printed_a_and_kappa_are_moments_of_the_F1_kernel():
    o = mk()
    a_printed = 2 * math.pi / 3 * 6 / 3                 # sigma = phi = 1, gamma = 6
    kappa_printed = 2 * math.pi / 15 * 6 / 1
    assert abs(kernel_moment(o, 1) - 2 * a_printed) < 1e-10
    assert abs(kernel_moment(o, 3) - 6 * kappa_printed) < 1e-9
    assert abs(o.discrete_a() - a_printed) < 1e-14       # EV2 reports the printed a


@pytest.mark.parametrize("dz", [0.25, 0.125])
def test_ev2_force_fourier_symbol(dz):
    nz = int(round(64 / dz))
    o = mk(nz=nz, dz=dz)
    a, kappa = kernel_moment(o, 1) / 2, kernel_moment(o, 3) / 6
    h = dz
    for kidx in (1, 3, 7, 20):
        S, k = symbol(o, nz, dz, kidx)
        ref = 2 * a * (8 * math.sin(k * h) - math.sin(2 * k * h)) / (6 * h) \
            + kappa * (math.sin(2 * k * h) - 2 * math.sin(k * h)) / h ** 3
        assert abs(S - ref) < 1e-9 * abs(ref), (kidx, S, ref)


def test_ev2_symbol_converges_to_continuum_at_second_order():
    o0 = mk()
    a, kappa = kernel_moment(o0, 1) / 2, kernel_moment(o0, 3) / 6
    err = []
    for dz in (0.25, 0.125, 0.0625):
        nz = int(round(128 / dz))
        S, k = symbol(mk(nz=nz, dz=dz), nz, dz, 4)
        cont = 2 * a * k - kappa * k ** 3
        err.append(abs(S - cont) / abs(cont))
    assert err[0] < 1e-5 and 3.6 < err[0] / err[1] < 4.4 and 3.6 < err[1] / err[2] < 4.4, err


@pytest.mark.parametrize("R", [6.0, 12.0])
def test_ev2_is_the_gradient_expansion_of_ev1(R):
    nz, dz = 1024, 0.125
    o1 = mk(nz=nz, dz=dz, fm=0, rcut=R)
    kappa_R = kernel_moment(o1, 3, R) / 6
    assert abs(kappa_R - (2 * math.pi / 15 * 6 - 2 * math.pi / (3 * R))) < 1e-10
    a_d = o1.discrete_a()
    ratios = []
    for kidx in (1, 2, 4):
        S1, k = symbol(o1, nz, dz, kidx)
        ratios.append((S1 - 2 * a_d * k) / (-kappa_R * k ** 3))
    # the k^3 term of the Simpson EV1 force is the cut kernel's kappa; the next
    # term (k^5 log k for gamma = 6) shrinks with k
    assert abs(ratios[0] - 1) < 2e-3 and abs(ratios[1] - 1) < 6e-3 and abs(ratios[2] - 1) < 2.5e-2, ratios
    assert abs(ratios[0] - 1) < abs(ratios[1] - 1) < abs(ratios[2] - 1)
    # and EV1 (uncut in the limit) and EV2 agree to the cut and Simpson error
    o2 = mk(nz=nz, dz=dz)
    S2, k = symbol(o2, nz, dz, 1)
    S1, _ = symbol(o1, nz, dz, 1)
    assert abs(S1 / S2 - 1) < 2 * math.pi / (3 * R ** 3) / (4 * math.pi / 3) + 1e-4


@pytest.mark.parametrize("Q,bc", [(16, 0), (24, 1)])
def test_ev2_uniform_state_is_stationary(Q, bc):
    nz = 48
    o = mk(nz=nz, Q=Q, bc=bc)
    F, G = o.equilibrium(np.full(nz, 0.25), np.zeros(nz), np.full(nz, 0.55))
    RF, RG, f = o.rhs(F, G, with_fields=True)
    assert np.abs(f["force"]).max() < 1e-15           # rounding of the stencil sums
    assert np.abs(RF).max() < 1e-14 * F.max() / o.s.dt
    assert np.abs(RG).max() < 1e-14 * G.max() / o.s.dt


def test_ev2_conserves_mass_and_momentum_periodic():
    """n . D n = 0 for an antisymmetric stencil D, so the EV2 force does no net
    momentum work on a periodic grid."""
    nz = 64
    o = mk(nz=nz, Q=16)
    rng = np.random.Generator(np.random.PCG64(21))
    n = 0.25 * (1 + 0.05 * rng.uniform(-1, 1, nz))
    u = 0.02 * rng.uniform(-1, 1, nz)
    T = 0.55 * (1 + 0.02 * rng.uniform(-1, 1, nz))
    F, G = o.equilibrium(n, u, T)
    f = o.node_fields(F, G)
    assert abs(np.sum(f["n"] * f["force"])) < 1e-15 * nz
    t0 = o.totals(F, G)
    t1 = o.totals(*o.step(F, G, 5))
    assert abs(t1[0] - t0[0]) < 1e-13 * t0[0]
    assert abs(t1[1] - t0[1]) < 1e-14 * t0[0]


def test_ev2_energy_drift_falls_under_refinement():
    """E_kin + E_int + (1/2) sum n psi with psi = -2a n - kappa n'' is
    conserved to truncation order: the drift over a fixed time falls by more
    than 3.5x per halving of dz."""
    L, drift = 16.0, []
    for nz in (64, 128, 256):
        dz = L / nz
        xi, _ = O.gauss_hermite(16)
        nsteps = int(round(0.2 / (0.5 * dz / np.abs(xi).max())))
        o = mk(nz=nz, Q=16, dz=dz, dt=0.2 / nsteps)
        z = dz * np.arange(nz)
        n = 0.25 * (1 + 0.05 * np.cos(2 * np.pi * z / L))
        u = 0.02 * np.sin(2 * np.pi * z / L)
        T = 0.55 * (1 + 0.02 * np.cos(4 * np.pi * z / L))
        F, G = o.equilibrium(n, u, T)
        t0 = o.totals(F, G)
        t1 = o.totals(*o.step(F, G, nsteps))
        drift.append(abs(t1[2] - t0[2]))
    assert drift[0] / drift[1] > 3.5 and drift[1] / drift[2] > 3.5, drift


def test_ev2_uniform_mean_field_energy():
    """Uniform n: psi = -2a n, E_mf = -a n^2 L with the printed a."""
    nz, dz, n0 = 64, 0.25, 0.3
    o = mk(nz=nz, dz=dz)
    F, G = o.equilibrium(np.full(nz, n0), np.zeros(nz), np.full(nz, 0.6))
    tot = o.totals(F, G)
    assert abs(tot[3] + 4 * math.pi / 3 * n0 ** 2 * nz * dz) < 1e-12
