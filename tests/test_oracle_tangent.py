"""Pins of the oracle's tangent-linear maps (complex-step build).

The adjoint of the time step is checked against these maps, so they are
pinned here against things other than themselves:
  * the complex build evaluates exactly the FP64 oracle (zero tangent);
  * the tangent agrees with central finite differences of the FP64 oracle
    (a check of the differentiation itself, to the FD truncation error);
  * the tangent of a mass- and momentum-conserving right-hand side conserves
    mass and momentum too (Sec. II.B: the collision terms keep n and n u; the
    WENO flux form telescopes; the force term moves no mass and its odd kernel
    gives no net momentum), to rounding;
  * tangents are linear in the direction (superposition).
"""
import numpy as np
import pytest

import oracle as O


def mk(nz=48, Q=12, dz=0.25, bc=0, relax=0, phi=1.0):
    xi, _ = O.gauss_hermite(Q)
    dt = 0.5 * dz / np.abs(xi).max()
    return O.Oracle(O.Setup(nz=nz, Q=Q, dz=dz, dt=dt, bc=bc, relax=relax, phi=phi))


def state(orc, seed=3, steps=2):
    rng = np.random.default_rng(seed)
    nz = orc.s.nz
    z = np.arange(nz)
    n0 = 0.25 * (1 + 0.3 * np.sin(2 * np.pi * z / nz) + 0.02 * rng.uniform(-1, 1, nz))
    u0 = 0.05 * np.cos(2 * np.pi * z / nz)
    T0 = 0.6 * (1 + 0.05 * np.sin(4 * np.pi * z / nz))
    F, G = orc.equilibrium(n0, u0, T0)
    return orc.step(F, G, steps)


def direction(orc, F, G, seed=11):
    rng = np.random.default_rng(seed)
    return F * rng.uniform(-1, 1, F.shape), G * rng.uniform(-1, 1, G.shape)


def rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


@pytest.mark.parametrize("bc", [0, 1])
def test_complex_build_is_the_fp64_oracle(bc):
    orc = mk(bc=bc)
    F, G = state(orc)
    RF, RG = orc.rhs(F, G)
    rf, rg, dF, dG = orc.rhs_tl(F, G, np.zeros_like(F), np.zeros_like(G))
    assert rel(rf, RF) < 1e-14 and rel(rg, RG) < 1e-14
    assert np.abs(dF).max() == 0.0 and np.abs(dG).max() == 0.0
    F2, G2 = orc.step(F, G, 3)
    f2, g2, _, _ = orc.step_tl(F, G, np.zeros_like(F), np.zeros_like(G), 3)
    assert rel(f2, F2) < 1e-14 and rel(g2, G2) < 1e-14


@pytest.mark.parametrize("bc,relax", [(0, 0), (1, 0), (0, 1)])
def test_rhs_tangent_matches_central_differences(bc, relax):
    orc = mk(bc=bc, relax=relax)
    F, G = state(orc)
    vF, vG = direction(orc, F, G)
    _, _, dF, dG = orc.rhs_tl(F, G, vF, vG)

    def fd_err(h):
        pF, pG = orc.rhs(F + h * vF, G + h * vG)
        mF, mG = orc.rhs(F - h * vF, G - h * vG)
        return rel(dF, (pF - mF) / (2 * h)), rel(dG, (pG - mG) / (2 * h))

    # central differences converge to the tangent as h^2 (x100 per decade)
    # until rounding takes over near h = 1e-7
    e4, e5, e6 = fd_err(1e-4), fd_err(1e-5), fd_err(1e-6)
    for a, b, c in zip(e4, e5, e6):
        assert 50 < a / b < 200 and c < 1e-7, (a, b, c)


def test_phi_tangent_matches_central_differences():
    """d/dphi of the right-hand side and of three steps: phi scales the
    Eq. (F1) kernel, so the oracle re-run at phi +- h is the reference."""
    orc = mk()
    F, G = state(orc)
    z = np.zeros_like(F)
    _, _, dF, dG = orc.rhs_tl(F, G, z, z, dphi=1.0)
    _, _, sF, sG = orc.step_tl(F, G, z, z, 3, dphi=1.0)
    h = 1e-5
    op, om = mk(phi=1.0 + h), mk(phi=1.0 - h)
    pF, pG = op.rhs(F, G)
    mF, mG = om.rhs(F, G)
    assert rel(dF, (pF - mF) / (2 * h)) < 1e-7 and rel(dG, (pG - mG) / (2 * h)) < 1e-7
    pF, pG = op.step(F, G, 3)
    mF, mG = om.step(F, G, 3)
    assert rel(sF, (pF - mF) / (2 * h)) < 1e-7 and rel(sG, (pG - mG) / (2 * h)) < 1e-7


def test_trajectory_tangent_matches_central_differences():
    """Projection of (n0, u0, T0) followed by five steps, along a seeded
    direction in n0 and a uniform change of T0."""
    orc = mk(nz=40, Q=10)
    nz = orc.s.nz
    rng = np.random.default_rng(5)
    n0 = 0.25 * (1 + 0.05 * rng.uniform(-1, 1, nz))
    u0 = np.zeros(nz)
    T0 = np.full(nz, 0.6)
    dn = 0.25 * rng.uniform(-1, 1, nz)
    dT = np.full(nz, 1.0)
    _, _, tF, tG = orc.trajectory_tl(n0, u0, T0, dn, np.zeros(nz), dT, 5)
    h = 1e-6

    def run(s):
        F, G = orc.equilibrium(n0 + s * dn, u0, T0 + s * dT)
        return orc.step(F, G, 5)

    pF, pG = run(h)
    mF, mG = run(-h)
    assert rel(tF, (pF - mF) / (2 * h)) < 1e-7 and rel(tG, (pG - mG) / (2 * h)) < 1e-7


def test_rhs_tangent_conserves_mass_and_momentum():
    """Periodic slab: sum_{k,i} dR_F = 0 and sum_{k,i} xi_k dR_F = 0 for any
    direction, because the nonlinear right-hand side conserves n and n u."""
    orc = mk(nz=48, Q=12)
    F, G = state(orc)
    vF, vG = direction(orc, F, G)
    _, _, dF, dG = orc.rhs_tl(F, G, vF, vG)
    scale = np.abs(dF).sum()
    assert abs(dF.sum()) < 1e-13 * scale
    assert abs((orc.xi[:, None] * dF).sum()) < 1e-13 * np.abs(orc.xi[:, None] * dF).sum()


def test_tangent_is_linear_in_the_direction():
    orc = mk()
    F, G = state(orc)
    aF, aG = direction(orc, F, G, seed=1)
    bF, bG = direction(orc, F, G, seed=2)
    _, _, ta, ua = orc.rhs_tl(F, G, aF, aG)
    _, _, tb, ub = orc.rhs_tl(F, G, bF, bG)
    _, _, tc, uc = orc.rhs_tl(F, G, 2.0 * aF - 3.0 * bF, 2.0 * aG - 3.0 * bG)
    assert rel(tc, 2.0 * ta - 3.0 * tb) < 1e-13 and rel(uc, 2.0 * ua - 3.0 * ub) < 1e-13
