"""Pins of the two-dimensional oracle (evfdlb_oracle2d.c) against things other
than itself: direct quadrature of the Sutherland force of Eq. (force), the
1D kernel of Eq. (F1) and the paper's constant a (Eq. F2), an independent
numpy reduction of the 3D Shakhov and J1 expressions of Sec. II.B over the
transverse velocity, Gaussian moment identities of the tensor-product
projection, conservation, and convergence of a y-uniform 2D slab to the 1D
model under refinement.
"""
import math

import numpy as np
import pytest
from numpy.polynomial.hermite_e import hermegauss
from scipy import integrate

import oracle as O


def mk2(nx=8, ny=8, Q=6, dx=0.25, rcut=6.0, dt=None):
    if dt is None:
        xi, _ = O.gauss_hermite(Q)
        dt = 0.5 * dx / (2 * np.abs(xi).max())
    return O.Oracle2D(O.Setup2(nx=nx, ny=ny, Q=Q, dx=dx, dt=dt, rcut=rcut))


def sutherland_force_line(rx, ry, sigma=1.0, phi=1.0, gamma=6.0):
    """x, y components of int dz phi'(r) r_vec / r over r = |(rx, ry, z)| > sigma,
    phi(r) = -phi (r/sigma)^-gamma (Eq. (sutherland)), by adaptive quadrature."""
    rho2 = rx * rx + ry * ry
    f = lambda z: gamma * phi * sigma ** gamma * (rho2 + z * z) ** (-(gamma + 2) / 2)
    if rho2 >= sigma * sigma:
        J = 2 * integrate.quad(f, 0, np.inf, epsabs=0, epsrel=1e-13, limit=200)[0]
    else:
        z0 = math.sqrt(sigma * sigma - rho2)
        J = 2 * integrate.quad(f, z0, np.inf, epsabs=0, epsrel=1e-13, limit=200)[0]
    return J * rx, J * ry


@pytest.mark.parametrize("r", [(0.25, 0.0), (0.5, 0.25), (0.7, 0.7), (1.0, 0.0), (1.5, -0.5), (3.0, 4.0)])
def test_in_plane_kernel_is_z_integral_of_eq_force(r):
    o = mk2()
    got = o.force_kernel(*r)
    ref = sutherland_force_line(*r)
    assert np.allclose(got, ref, rtol=1e-11, atol=1e-14)


@pytest.mark.parametrize("x", [0.3, 0.8, 1.0, 1.7, 3.0])
def test_in_plane_kernel_integrates_to_eq_F1_kernel(x):
    """int g2_x(x, y) dy over y is the plane-integrated kernel g(x) of Eq. (F1)."""
    o = mk2()
    pts = [math.sqrt(1 - x * x)] if x < 1 else None
    val = 2 * integrate.quad(lambda y: o.force_kernel(x, y)[0], 0, np.inf, points=None, epsabs=0,
                             epsrel=1e-11, limit=400)[0] if pts is None else \
        2 * (integrate.quad(lambda y: o.force_kernel(x, y)[0], 0, pts[0], epsabs=0, epsrel=1e-11)[0]
             + integrate.quad(lambda y: o.force_kernel(x, y)[0], pts[0], np.inf, epsabs=0, epsrel=1e-11,
                              limit=400)[0])
    g = 2 * math.pi * x if x < 1 else 2 * math.pi * x / x ** 6
    assert abs(val - g) < 1e-9 * abs(g)


def test_continuous_a_of_in_plane_kernel_is_eq_F2():
    """(1/2) int rho_x g2_x d^2 rho = (pi/2) int rho^2 |g2|(rho) d rho = a of
    Eq. (F2): 2 pi sigma^3 phi gamma / (3 (gamma - 3)) = 4 pi / 3 for gamma = 6."""
    o = mk2()
    f = lambda r: r * r * o.force_kernel(r, 0.0)[0]
    val = 0.5 * math.pi * (integrate.quad(f, 0, 1, epsabs=0, epsrel=1e-12)[0]
                           + integrate.quad(f, 1, np.inf, epsabs=0, epsrel=1e-12, limit=200)[0])
    assert abs(val - 4 * math.pi / 3) < 1e-10


@pytest.mark.parametrize("Q,ux,uy,T", [(6, 0.0, 0.0, 1.0), (8, 0.3, -0.2, 0.6), (10, -0.5, 0.1, 0.8)])
def test_projected_2d_maxwellian_moments(Q, ux, uy, T):
    o = mk2(nx=1, ny=1, Q=Q)
    n = 0.37
    F, G = o.equilibrium(n, ux, uy, T)
    F, G = F[:, :, 0, 0], G[:, :, 0, 0]
    z, wz = hermegauss(40)
    wz = wz / math.sqrt(2 * math.pi)
    ex = lambda u, a: float((wz * (u + math.sqrt(T) * z) ** a).sum())
    for a in range(Q):
        for b in range(Q):
            mom = (F * np.outer(o.xi ** a, o.xi ** b)).sum()
            ref = n * ex(ux, a) * ex(uy, b)
            assert abs(mom - ref) < 1e-12 * max(1.0, abs(ref)) * 10 ** (0.3 * (a + b))
            momG = (G * np.outer(o.xi ** a, o.xi ** b)).sum()
            assert abs(momG - 0.5 * T * ref) < 1e-12 * max(1.0, abs(ref)) * 10 ** (0.3 * (a + b))


def reduced_by_quadrature(n, ux, uy, T, qx, qy, Pr, chi, A, B, D, Q, xi, w, nq=24):
    """Independent reduction: the 3D reduced Shakhov f^S and J1 of Sec. II.B
    (with 3D peculiar velocity c, zeta = c / sqrt(2T), q = (qx, qy, 0),
    gradients in-plane) integrated over c_z by Gauss-Hermite quadrature,
    then projected onto the tensor Hermite basis; returns FS, GS, JF, JG."""
    b = 2 * math.pi / 3
    z, wz = hermegauss(nq)
    wz = wz / math.sqrt(2 * math.pi)
    s = (1 - Pr) / (n * T * T)
    Dm = np.array([[D[0], D[1], 0.0], [D[2], D[3], 0.0], [0.0, 0.0, 0.0]])   # D_ij = d_i u_j
    divu = D[0] + D[3]
    coef = {k: np.zeros((Q, Q)) for k in ("FS", "GS", "JF", "JG")}
    he = lambda x: np.array([np.polynomial.hermite_e.hermeval(x, [0] * l + [1]) for l in range(Q)])
    for i in range(nq):
        cx = math.sqrt(T) * z[i]
        hx = he(ux + cx)
        for j in range(nq):
            cy = math.sqrt(T) * z[j]
            hy = he(uy + cy)
            W = wz[i] * wz[j] * n
            pS = pG = pJF = pJG = 0.0
            for k in range(nq):
                cz = math.sqrt(T) * z[k]
                c = np.array([cx, cy, cz])
                c2 = c @ c
                zeta2 = c2 / (2 * T)
                shak = 1 + s * (c2 / (5 * T) - 1) * (cx * qx + cy * qy)
                j1 = -b * n * chi * (c[0] * A[0] + c[1] * A[1] + 0.6 * (zeta2 - 2.5) * (c[0] * B[0] + c[1] * B[1])
                                     + 0.4 * (2 * (c @ Dm @ c) / (2 * T) + (zeta2 - 2.5) * divu))
                pS += wz[k] * shak
                pG += wz[k] * 0.5 * cz * cz * shak
                pJF += wz[k] * j1
                pJG += wz[k] * 0.5 * cz * cz * j1
            hh = W * np.outer(hx, hy)
            coef["FS"] += pS * hh
            coef["GS"] += pG * hh
            coef["JF"] += pJF * hh
            coef["JG"] += pJG * hh
    fact = np.array([math.factorial(l) for l in range(Q)], dtype=float)
    H = np.array([[np.polynomial.hermite_e.hermeval(x, [0] * l + [1]) for l in range(Q)] for x in xi]) / fact
    out = []
    for k in ("FS", "GS", "JF", "JG"):
        out.append(np.outer(w, w) * (H @ coef[k] @ H.T))
    return out


def test_reduced_shakhov_and_J1_match_3d_reduction():
    Q = 6
    o = mk2(nx=1, ny=1, Q=Q)
    fields = dict(n=0.3, ux=0.2, uy=-0.1, T=0.7, qx=0.05, qy=-0.03, Pr=0.8, chi=1.6, Ax=0.4, Ay=-0.2,
                  Bx=0.1, By=0.3, Dxx=0.05, Dxy=-0.02, Dyx=0.03, Dyy=-0.04)
    got = o.equilibria_node(fields)
    ref = reduced_by_quadrature(0.3, 0.2, -0.1, 0.7, 0.05, -0.03, 0.8, 1.6, (0.4, -0.2), (0.1, 0.3),
                                (0.05, -0.02, 0.03, -0.04), Q, o.xi, o.w)
    for g, r in zip(got, ref):
        assert np.abs(g - r).max() < 1e-13 * max(np.abs(r).max(), 1e-3)


def test_shakhov_heat_flux_and_J1_moments_2d():
    Q = 8
    o = mk2(nx=1, ny=1, Q=Q)
    n, ux, uy, T, qx, qy, Pr, chi = 0.3, 0.1, -0.2, 0.7, 0.04, -0.02, 0.75, 1.4
    Ax, Ay, Bx, By = 0.3, -0.1, 0.2, 0.05
    FS, GS, JF, JG = o.equilibria_node(dict(n=n, ux=ux, uy=uy, T=T, qx=qx, qy=qy, Pr=Pr, chi=chi, Ax=Ax, Ay=Ay,
                                            Bx=Bx, By=By, Dxx=0.02, Dxy=0.01, Dyx=-0.03, Dyy=0.04))
    X, Y = np.meshgrid(o.xi, o.xi, indexing="ij")
    cx, cy = X - ux, Y - uy
    e = 0.5 * (cx * cx + cy * cy) * FS + GS
    assert abs((cx * e).sum() - (1 - Pr) * qx) < 1e-13
    assert abs((cy * e).sum() - (1 - Pr) * qy) < 1e-13
    assert abs(FS.sum() - n) < 1e-14
    b = 2 * math.pi / 3
    assert abs(JF.sum()) < 1e-14
    # momentum source of J1: -b n chi n T A (Sec. II.B; the viscous and B terms carry none)
    assert abs((X * JF).sum() + b * n * chi * n * T * Ax) < 1e-13
    assert abs((Y * JF).sum() + b * n * chi * n * T * Ay) < 1e-13


def test_uniform_state_is_stationary_2d():
    o = mk2(nx=6, ny=5, Q=6)
    F, G = o.equilibrium(0.3, 0.15, -0.1, 0.65)
    RF, RG = o.rhs(F, G)
    assert np.abs(RF).max() < 1e-13 * np.abs(F).max() and np.abs(RG).max() < 1e-13 * np.abs(G).max()


def test_mass_and_momentum_conserved_2d():
    nx, ny = 10, 9
    o = mk2(nx=nx, ny=ny, Q=6)
    X, Y = np.meshgrid(np.arange(nx), np.arange(ny))
    n = 0.25 * (1 + 0.2 * np.sin(2 * np.pi * X / nx) * np.cos(2 * np.pi * Y / ny))
    F, G = o.equilibrium(n, 0.02 * np.cos(2 * np.pi * Y / ny), 0.01 * np.sin(2 * np.pi * X / nx), 0.6)
    t0 = o.totals(F, G)
    F, G = o.step(F, G, 3)
    t1 = o.totals(F, G)
    assert abs(t1[0] - t0[0]) < 1e-13 * t0[0]
    assert abs(t1[1] - t0[1]) < 1e-14 * t0[0] and abs(t1[2] - t0[2]) < 1e-14 * t0[0]


def test_y_uniform_slab_converges_to_the_1d_model():
    """For fields that vary along x only, the 2D right-hand side reduced over
    xi_y (F1 = sum_ky F, G1 = sum_ky (xi_y^2/2 F + G)) is the 1D right-hand
    side up to the discretisation differences of the two quadratures (the 2D
    rectangle rule over the force disc and the chord-weighted FM disc, whose
    kernel kinks at rho = sigma, against the 1D Simpson rules) and the
    nonlinearity of WENO weights.  The difference must fall under refinement
    (measured x3.0 per halving of dx: 12.5 % -> 4.2 % of the right-hand side);
    a wrong factor or term in the 2D model would not converge.  Cut radius
    12 sigma, so that the disc and line cuts agree to 1e-7."""
    Q, L, rc = 8, 16.0, 12.0
    errs = []
    for dx in (0.25, 0.125):
        nx = int(round(L / dx))
        x = dx * np.arange(nx)
        n = 0.25 * (1 + 0.2 * np.sin(2 * np.pi * x / L))
        u = 0.03 * np.sin(4 * np.pi * x / L)
        T = 0.6 * (1 + 0.05 * np.cos(2 * np.pi * x / L))
        xi, _ = O.gauss_hermite(Q)
        o1 = O.Oracle(O.Setup(nz=nx, Q=Q, dz=dx, dt=0.01, rcut=rc))
        o2 = O.Oracle2D(O.Setup2(nx=nx, ny=1, Q=Q, dx=dx, dt=0.01, rcut=rc))
        F1, G1 = o1.equilibrium(n, u, T)
        F2, G2 = o2.equilibrium(n[None, :], u[None, :], 0.0, T[None, :])
        R1F, R1G = o1.rhs(F1, G1)
        R2F, R2G = o2.rhs(F2, G2)
        rF = R2F[:, :, 0, :].sum(axis=1)
        rG = (0.5 * (o2.xi ** 2)[None, :, None] * R2F[:, :, 0, :] + R2G[:, :, 0, :]).sum(axis=1)
        errs.append((np.abs(rF - R1F).max() / np.abs(R1F).max(), np.abs(rG - R1G).max() / np.abs(R1G).max()))
    print("y-uniform 2D vs 1D:", errs)
    for a, b in zip(errs[0], errs[1]):
        assert b < a / 2.5 and b < 0.06
