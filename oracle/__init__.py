"""Plain FP64 CPU reference ("the oracle") for the EV-FDLB time step of
Busuioc & Sofonea, arXiv:2503.15187.

TEST INFRASTRUCTURE ONLY: only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA library in ``paper_2503_15187_gb300``; neither imports the other.

Contents
--------
* ``build()`` compiles ``evfdlb_oracle.c`` (plain C, FP64) with gcc.
* ``gauss_hermite(Q)``: the full-range Gauss-Hermite velocity set (Sec. III),
  taken from numpy's ``hermegauss`` and normalised to unit total weight.
* Equation of state, Eq. (EOSS), with its critical point, spinodal and Maxwell
  construction (Sec. III.A), in numpy/scipy.
* ``Oracle``: a ctypes wrapper around the C routines (moments, node fields,
  right-hand side, Shu-Osher RK3 steps, projected equilibria, totals).
* Tangent-linear maps (``rhs_tl``, ``step_tl``, ``equilibrium_tl``,
  ``trajectory_tl``): the same C source compiled over double complex
  (``evfdlb_oracle_cs.c``) and evaluated by complex step, the reference for
  the adjoint of the time step.

Parity status: every function here is pinned by ``tests/test_oracle_pins.py``
(closed forms, identities, brute-force quadrature, textbook routines and the
paper's printed critical temperature) and, for the tangent-linear maps, by
``tests/test_oracle_tangent.py`` (finite differences of the FP64 oracle with
their h^2 convergence, linearised mass and momentum conservation).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np
from numpy.polynomial import Polynomial
from numpy.polynomial.hermite_e import hermegauss

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "evfdlb_oracle.c")
_SRC_CS = os.path.join(_HERE, "evfdlb_oracle_cs.c")
_SRC_2D = os.path.join(_HERE, "evfdlb_oracle2d.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liborc.so")
NFIELDS = 16
FIELD_NAMES = ("n", "u", "T", "q", "nbar", "chi", "force", "mu", "tau", "Pr",
               "rate", "A", "B", "D", "X", "bnchi")

PI = np.pi


def build(force: bool = False) -> str:
    """Compile the C oracle into oracle/_build/liborc.so (gcc, -O2, IEEE FP):
    the FP64 routines and their complex-step twins from the same source, with
    OpenMP over the independent node loops where the compiler offers it (the
    thread count changes no result; ``set_threads``)."""
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(f) for f in (_SRC, _SRC_CS, _SRC_2D, os.path.abspath(__file__)))
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        tmp = _LIB + f".tmp{os.getpid()}"
        base = ["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-ffp-contract=off"]
        try:
            subprocess.check_call(base + ["-fopenmp", "-o", tmp, _SRC, _SRC_CS, _SRC_2D, "-lm"],
                                  stderr=subprocess.DEVNULL)
        except subprocess.CalledProcessError:      # no OpenMP runtime: serial build
            subprocess.check_call(base + ["-o", tmp, _SRC, _SRC_CS, _SRC_2D, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def set_threads(n: int | None = None) -> int:
    """Threads of the oracle's node loops (n > 0 sets them; None only reads);
    returns the count in effect (1 for a build without OpenMP).  The default is
    one thread, or ORACLE_THREADS from the environment."""
    return int(_load().orc_set_threads(0 if n is None else int(n)))


def available_cores() -> int:
    """Host cores this process may run on (its CPU affinity)."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:                          # pragma: no cover
        return os.cpu_count() or 1


_lib = None


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        d, i, vp = ctypes.c_double, ctypes.c_int, ctypes.c_void_p
        P = ctypes.POINTER(_Params)
        _lib.orc_force_kernel.restype = d
        _lib.orc_force_kernel.argtypes = [P, d]
        _lib.orc_force_potential.restype = d
        _lib.orc_force_potential.argtypes = [P, d]
        _lib.orc_plane_potential.restype = d
        _lib.orc_plane_potential.argtypes = [P, d]
        _lib.orc_chi.restype = d
        _lib.orc_chi.argtypes = [P, d]
        _lib.orc_discrete_a.restype = d
        _lib.orc_discrete_a.argtypes = [P]
        _lib.orc_weno5.restype = d
        _lib.orc_weno5.argtypes = [d, d, d, d, d, d]
        _lib.orc_moments.argtypes = [P, vp, vp, vp, vp, vp, vp]
        _lib.orc_node_fields.argtypes = [P, vp, vp, vp, vp, vp]
        _lib.orc_equilibria_node.argtypes = [P, d, d, d, d, d, d, d, d, d, vp, vp, vp, vp]
        _lib.orc_equilibrium.argtypes = [P, vp, vp, vp, vp, vp]
        _lib.orc_dxi.argtypes = [P, vp, vp]
        _lib.orc_rhs.argtypes = [P, vp, vp, vp, vp, vp]
        _lib.orc_advect_row.argtypes = [P, d, vp, vp]
        _lib.orc_step.argtypes = [P, vp, vp, i]
        _lib.orc_totals.argtypes = [P, vp, vp, vp]
        _lib.orc_cs_moments.argtypes = [P, vp, vp, vp, vp, vp, vp]
        _lib.orc_cs_equilibrium.argtypes = [P, vp, vp, vp, vp, vp]
        _lib.orc_cs_rhs.argtypes = [P, vp, vp, vp, vp, vp]
        _lib.orc_cs_step.argtypes = [P, vp, vp, i]
        P2 = ctypes.POINTER(_Params2)
        _lib.orc2_force_kernel.argtypes = [P2, d, d, vp]
        _lib.orc2_discrete_a.restype = d
        _lib.orc2_discrete_a.argtypes = [P2]
        _lib.orc2_moments.argtypes = [P2, vp, vp, vp, vp, vp, vp, vp, vp]
        _lib.orc2_node_fields.argtypes = [P2, vp, vp, vp, vp, vp, vp, vp]
        _lib.orc2_equilibria_node.argtypes = [P2, vp, vp, vp, vp, vp]
        _lib.orc2_equilibrium.argtypes = [P2, vp, vp, vp, vp, vp, vp]
        _lib.orc2_dxi.argtypes = [P2, vp, vp, vp]
        _lib.orc2_rhs.argtypes = [P2, vp, vp, vp, vp, vp]
        _lib.orc2_step.argtypes = [P2, vp, vp, i]
        _lib.orc2_totals.argtypes = [P2, vp, vp, vp]
        _lib.orc_set_threads.restype = i
        _lib.orc_set_threads.argtypes = [i]
        _lib.orc_set_threads(max(1, int(os.environ.get("ORACLE_THREADS", "1"))))
    return _lib


class _Params(ctypes.Structure):
    _fields_ = [("nz", ctypes.c_int), ("Q", ctypes.c_int), ("dz", ctypes.c_double),
                ("dt", ctypes.c_double), ("sigma", ctypes.c_double),
                ("phi", ctypes.c_double), ("gamma", ctypes.c_double),
                ("rcut", ctypes.c_double), ("bc", ctypes.c_int), ("relax", ctypes.c_int),
                ("weno_eps", ctypes.c_double), ("xi", ctypes.c_void_p),
                ("w", ctypes.c_void_p), ("nq", ctypes.c_int), ("zq", ctypes.c_void_p),
                ("wq", ctypes.c_void_p), ("phi_tl", ctypes.c_double), ("force_model", ctypes.c_int),
                ("T_iso", ctypes.c_double)]


class _Params2(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("Q", ctypes.c_int),
                ("dx", ctypes.c_double), ("dt", ctypes.c_double), ("sigma", ctypes.c_double),
                ("phi", ctypes.c_double), ("gamma", ctypes.c_double), ("rcut", ctypes.c_double),
                ("weno_eps", ctypes.c_double), ("relax", ctypes.c_int), ("xi", ctypes.c_void_p),
                ("w", ctypes.c_void_p), ("nq", ctypes.c_int), ("zq", ctypes.c_void_p),
                ("wq", ctypes.c_void_p)]


# --------------------------------------------------------------------------
# Velocity set (Sec. III: full-range Gauss-Hermite quadrature)
# --------------------------------------------------------------------------
def gauss_hermite(Q: int):
    """Nodes xi_k (roots of the probabilists' He_Q) and weights w_k normalised
    to sum 1, i.e. the rule for the standard normal density."""
    x, w = hermegauss(Q)
    return np.ascontiguousarray(x, dtype=np.float64), np.ascontiguousarray(w / np.sqrt(2 * PI))


# --------------------------------------------------------------------------
# Equation of state, Eq. (EOSS), and the Maxwell construction (Sec. III.A)
# --------------------------------------------------------------------------
def _y_poly():
    """y(eta) = eta * Z_CS(eta) = N(eta) / (1-eta)^3, with
    Z_CS = (1 + eta + eta^2 - eta^3)/(1-eta)^3 (the repulsive part of Eq. (EOSS))."""
    N = Polynomial([0.0, 1.0, 1.0, 1.0, -1.0])
    D = Polynomial([1.0, -1.0]) ** 3
    return N, D


def _y_derivs(eta):
    N, D = _y_poly()
    N1, D1 = N.deriv(), D.deriv()
    num1 = N1 * D - N * D1                      # y' = num1 / D^2
    num2 = num1.deriv() * D - 2.0 * num1 * D1   # y'' = num2 / D^3
    d = D(eta)
    return N(eta) / d, num1(eta) / d ** 2, num2(eta) / d ** 3


def pressure(n, T, a, sigma=1.0):
    """P = n T (1+eta+eta^2-eta^3)/(1-eta)^3 - a n^2, eta = pi sigma^3 n / 6 (Eq. (EOSS))."""
    eta = PI * sigma ** 3 * np.asarray(n) / 6.0
    return n * T * (1 + eta + eta ** 2 - eta ** 3) / (1 - eta) ** 3 - a * n * n


def chem_potential(n, T, a, sigma=1.0):
    """Chemical potential of Eq. (EOSS) up to a function of T:
    mu = T [ln n + (8 eta - 9 eta^2 + 3 eta^3)/(1-eta)^3] - 2 a n
    (from the Carnahan-Starling free energy T[(4 eta - 3 eta^2)/(1-eta)^2] - a n
    per particle, so that n dmu/dn = dP/dn)."""
    eta = PI * sigma ** 3 * np.asarray(n) / 6.0
    return T * (np.log(n) + (8 * eta - 9 * eta ** 2 + 3 * eta ** 3) / (1 - eta) ** 3) - 2 * a * n


def dP_dn(n, T, a, sigma=1.0):
    k = 6.0 / (PI * sigma ** 3)
    _, y1, _ = _y_derivs(np.asarray(n) / k)
    return T * y1 - 2.0 * a * n


def critical_point(a, sigma=1.0):
    """(n_c, T_c) of Eq. (EOSS): dP/dn = d2P/dn2 = 0.  With y = eta Z_CS and
    n = k eta, the two conditions give y'(eta) = eta y''(eta) (independent of
    a and T) and T_c = 2 a k / y''(eta_c)."""
    from scipy.optimize import brentq
    k = 6.0 / (PI * sigma ** 3)

    def f(eta):
        _, y1, y2 = _y_derivs(eta)
        return y1 - eta * y2

    eta_c = brentq(f, 0.01, 0.4, xtol=1e-16, rtol=1e-15, maxiter=500)
    _, _, y2 = _y_derivs(eta_c)
    return k * eta_c, 2.0 * a * k / y2


def spinodal(T, a, sigma=1.0):
    """Densities where dP/dn = 0 at fixed T (T < T_c)."""
    from scipy.optimize import brentq
    n_c, T_c = critical_point(a, sigma)
    if T >= T_c:
        raise ValueError("T must be below T_c")
    n_max = 0.99 * 6.0 / (PI * sigma ** 3)
    lo = brentq(lambda n: dP_dn(n, T, a, sigma), 1e-12, n_c, xtol=1e-16, rtol=1e-15, maxiter=500)
    hi = brentq(lambda n: dP_dn(n, T, a, sigma), n_c, n_max, xtol=1e-16, rtol=1e-15, maxiter=500)
    return lo, hi


def coexistence(T, a, sigma=1.0):
    """Maxwell construction (Sec. III.A): (n_v, n_l) with equal pressure and
    equal chemical potential at temperature T."""
    from scipy.optimize import brentq
    s_lo, s_hi = spinodal(T, a, sigma)
    n_max = 0.99 * 6.0 / (PI * sigma ** 3)
    p_lo = max(pressure(s_hi, T, a, sigma), 1e-300)
    p_hi = pressure(s_lo, T, a, sigma)

    def dens_at(P_s):
        nv = brentq(lambda n: pressure(n, T, a, sigma) - P_s, 1e-300, s_lo,
                    xtol=1e-300, rtol=1e-15, maxiter=1000)
        nl = brentq(lambda n: pressure(n, T, a, sigma) - P_s, s_hi, n_max,
                    xtol=1e-16, rtol=1e-15, maxiter=1000)
        return nv, nl

    def dmu(P_s):
        nv, nl = dens_at(P_s)
        return chem_potential(nl, T, a, sigma) - chem_potential(nv, T, a, sigma)

    P_s = brentq(dmu, p_lo * (1 + 1e-12), p_hi * (1 - 1e-12), xtol=1e-300, rtol=1e-15, maxiter=1000)
    return dens_at(P_s)


# --------------------------------------------------------------------------
# ctypes wrapper
# --------------------------------------------------------------------------
@dataclass
class Setup:
    nz: int
    Q: int
    dz: float
    dt: float
    sigma: float = 1.0
    phi: float = 1.0
    gamma: float = 6.0
    rcut: float = 6.0
    bc: int = 0            # 0 periodic, 1 outflow
    relax: int = 0         # 0: rate 1/tau, 1: rate chi/tau
    weno_eps: float = 1e-6
    nq: int = 64           # points of the projection rule
    force_model: int = 0   # 0: EV1, Eq. (F1); 1: EV2, Eq. (F2)
    T_iso: float = 0.0     # > 0: isothermal mode at this temperature


class Oracle:
    """FP64 CPU reference of one EV1 right-hand side and of RK3 time steps.
    Distributions are numpy arrays of shape (Q, nz), float64, C order."""

    def __init__(self, setup: Setup):
        self.s = setup
        self.lib = _load()
        self.xi, self.w = gauss_hermite(setup.Q)
        self.zq, self.wq = gauss_hermite(setup.nq)
        self._p = _Params(setup.nz, setup.Q, setup.dz, setup.dt, setup.sigma, setup.phi,
                          setup.gamma, setup.rcut, setup.bc, setup.relax, setup.weno_eps,
                          self.xi.ctypes.data, self.w.ctypes.data, setup.nq,
                          self.zq.ctypes.data, self.wq.ctypes.data, 0.0, setup.force_model,
                          setup.T_iso)
        self.p = ctypes.byref(self._p)

    # scalar kernels -------------------------------------------------------
    def force_kernel(self, z):
        return self.lib.orc_force_kernel(self.p, float(z))

    def force_potential(self, z):
        return self.lib.orc_force_potential(self.p, float(z))

    def plane_potential(self, z):
        return self.lib.orc_plane_potential(self.p, float(z))

    def chi(self, n):
        return self.lib.orc_chi(self.p, float(n))

    def discrete_a(self):
        return self.lib.orc_discrete_a(self.p)

    def critical_T(self):
        """T_c of Eq. (EOSS) with the model's own force constant a_d."""
        return critical_point(self.discrete_a(), self.s.sigma)[1]

    @staticmethod
    def weno5(v, eps=1e-6):
        return _load().orc_weno5(*[float(x) for x in v], float(eps))

    # array routines -------------------------------------------------------
    def _arr(self, x, shape=None):
        a = np.ascontiguousarray(x, dtype=np.float64)
        if shape is not None:
            assert a.shape == shape, (a.shape, shape)
        return a

    def moments(self, F, G):
        F = self._arr(F, (self.s.Q, self.s.nz))
        G = self._arr(G, (self.s.Q, self.s.nz))
        out = [np.empty(self.s.nz) for _ in range(4)]
        self.lib.orc_moments(self.p, F.ctypes.data, G.ctypes.data, *[o.ctypes.data for o in out])
        return tuple(out)

    def node_fields(self, F, G):
        n, u, T, q = self.moments(F, G)
        out = np.empty((NFIELDS, self.s.nz))
        self.lib.orc_node_fields(self.p, n.ctypes.data, u.ctypes.data, T.ctypes.data,
                                 q.ctypes.data, out.ctypes.data)
        return {k: out[i] for i, k in enumerate(FIELD_NAMES)}

    def equilibria_node(self, n, u, T, q=0.0, Pr=1.0, bnchi=0.0, A=0.0, B=0.0, D=0.0):
        Q = self.s.Q
        outs = [np.empty(Q) for _ in range(4)]
        self.lib.orc_equilibria_node(self.p, n, u, T, q, Pr, bnchi, A, B, D,
                                     *[o.ctypes.data for o in outs])
        return tuple(outs)

    def equilibrium(self, n, u, T):
        nz, Q = self.s.nz, self.s.Q
        n, u, T = self._arr(n, (nz,)), self._arr(u, (nz,)), self._arr(T, (nz,))
        F = np.empty((Q, nz))
        G = np.empty((Q, nz))
        self.lib.orc_equilibrium(self.p, n.ctypes.data, u.ctypes.data, T.ctypes.data,
                                 F.ctypes.data, G.ctypes.data)
        return F, G

    def dxi(self, h):
        h = self._arr(h, (self.s.Q,))
        out = np.empty(self.s.Q)
        self.lib.orc_dxi(self.p, h.ctypes.data, out.ctypes.data)
        return out

    def advect_row(self, xi, h):
        """-xi dh/dz by WENO-5 with the boundary rule, for one velocity row."""
        h = self._arr(h, (self.s.nz,))
        out = np.empty(self.s.nz)
        self.lib.orc_advect_row(self.p, float(xi), h.ctypes.data, out.ctypes.data)
        return out

    def rhs(self, F, G, with_fields=False):
        nz, Q = self.s.nz, self.s.Q
        F = self._arr(F, (Q, nz))
        G = self._arr(G, (Q, nz))
        RF = np.empty((Q, nz))
        RG = np.empty((Q, nz))
        fl = np.empty((NFIELDS, nz))
        self.lib.orc_rhs(self.p, F.ctypes.data, G.ctypes.data, RF.ctypes.data,
                         RG.ctypes.data, fl.ctypes.data)
        if with_fields:
            return RF, RG, {k: fl[i] for i, k in enumerate(FIELD_NAMES)}
        return RF, RG

    def step(self, F, G, nsteps=1):
        """Returns new arrays after nsteps Shu-Osher RK3 steps."""
        nz, Q = self.s.nz, self.s.Q
        F = self._arr(F, (Q, nz)).copy()
        G = self._arr(G, (Q, nz)).copy()
        self.lib.orc_step(self.p, F.ctypes.data, G.ctypes.data, int(nsteps))
        return F, G

    # tangent-linear maps by complex step ---------------------------------
    # Each routine evaluates the oracle's own arithmetic at x + i h v
    # (double complex build) and returns (f(x), J v) = (Re, Im / h); h is
    # tiny, so J v is exact to rounding (Squire & Trapp 1998).
    CS_H = 1e-30

    def _c(self, x, dx, shape):
        z = np.empty(shape, dtype=np.complex128)
        z.real = np.asarray(x, dtype=np.float64).reshape(shape)
        z.imag = (self.CS_H * np.asarray(dx, dtype=np.float64)).reshape(shape) if dx is not None else 0.0
        return z

    def _with_phi_tangent(self, dphi):
        self._p.phi_tl = self.CS_H * float(dphi)

    def rhs_tl(self, F, G, dF, dG, dphi=0.0):
        """(RF, RG) and the tangent (dRF, dRG) of the right-hand side along
        (dF, dG) and a change dphi of the well depth phi."""
        nz, Q = self.s.nz, self.s.Q
        Fc, Gc = self._c(F, dF, (Q, nz)), self._c(G, dG, (Q, nz))
        RF = np.empty((Q, nz), dtype=np.complex128)
        RG = np.empty((Q, nz), dtype=np.complex128)
        fl = np.empty((NFIELDS, nz), dtype=np.complex128)
        self._with_phi_tangent(dphi)
        try:
            self.lib.orc_cs_rhs(self.p, Fc.ctypes.data, Gc.ctypes.data, RF.ctypes.data,
                                RG.ctypes.data, fl.ctypes.data)
        finally:
            self._with_phi_tangent(0.0)
        return RF.real.copy(), RG.real.copy(), RF.imag / self.CS_H, RG.imag / self.CS_H

    def step_tl(self, F, G, dF, dG, nsteps=1, dphi=0.0):
        """nsteps RK3 steps and their tangent along (dF, dG, dphi)."""
        nz, Q = self.s.nz, self.s.Q
        Fc, Gc = self._c(F, dF, (Q, nz)), self._c(G, dG, (Q, nz))
        self._with_phi_tangent(dphi)
        try:
            self.lib.orc_cs_step(self.p, Fc.ctypes.data, Gc.ctypes.data, int(nsteps))
        finally:
            self._with_phi_tangent(0.0)
        return Fc.real.copy(), Gc.real.copy(), Fc.imag / self.CS_H, Gc.imag / self.CS_H

    def equilibrium_tl(self, n, u, T, dn, du, dT):
        """Projected Maxwellian pair and its tangent along (dn, du, dT)."""
        nz, Q = self.s.nz, self.s.Q
        nc, uc, Tc = self._c(n, dn, (nz,)), self._c(u, du, (nz,)), self._c(T, dT, (nz,))
        F = np.empty((Q, nz), dtype=np.complex128)
        G = np.empty((Q, nz), dtype=np.complex128)
        self.lib.orc_cs_equilibrium(self.p, nc.ctypes.data, uc.ctypes.data, Tc.ctypes.data,
                                    F.ctypes.data, G.ctypes.data)
        return F.real.copy(), G.real.copy(), F.imag / self.CS_H, G.imag / self.CS_H

    def trajectory_tl(self, n0, u0, T0, dn0, du0, dT0, nsteps, dphi=0.0):
        """State after projecting (n0, u0, T0) and nsteps RK3 steps, and the
        tangent of that state along (dn0, du0, dT0, dphi)."""
        F, G, dF, dG = self.equilibrium_tl(n0, u0, T0, dn0, du0, dT0)
        return self.step_tl(F, G, dF, dG, nsteps, dphi)

    def totals(self, F, G):
        """[mass, momentum, energy (incl. E_mf), E_mf]"""
        nz, Q = self.s.nz, self.s.Q
        F = self._arr(F, (Q, nz))
        G = self._arr(G, (Q, nz))
        out = np.empty(4)
        self.lib.orc_totals(self.p, F.ctypes.data, G.ctypes.data, out.ctypes.data)
        return out


# --------------------------------------------------------------------------
# Two-dimensional extension (evfdlb_oracle2d.c)
# --------------------------------------------------------------------------
NFIELDS2 = 22
FIELD_NAMES2 = ("n", "ux", "uy", "T", "qx", "qy", "nbar", "chi", "Fx", "Fy", "mu", "tau", "Pr", "nu",
                "Ax", "Ay", "Bx", "By", "Dxx", "Dxy", "Dyx", "Dyy")


@dataclass
class Setup2:
    nx: int
    ny: int
    Q: int
    dx: float
    dt: float
    sigma: float = 1.0
    phi: float = 1.0
    gamma: float = 6.0
    rcut: float = 6.0
    weno_eps: float = 1e-6
    relax: int = 0
    nq: int = 32


class Oracle2D:
    """FP64 CPU reference of the 2D tensor-product model.  Distributions are
    arrays of shape (Q, Q, ny, nx) (index [kx, ky, y, x]), float64."""

    def __init__(self, setup: Setup2):
        self.s = setup
        self.lib = _load()
        self.xi, self.w = gauss_hermite(setup.Q)
        self.zq, self.wq = gauss_hermite(setup.nq)
        self._p = _Params2(setup.nx, setup.ny, setup.Q, setup.dx, setup.dt, setup.sigma, setup.phi,
                           setup.gamma, setup.rcut, setup.weno_eps, setup.relax, self.xi.ctypes.data,
                           self.w.ctypes.data, setup.nq, self.zq.ctypes.data, self.wq.ctypes.data)
        self.p = ctypes.byref(self._p)
        self.shape = (setup.Q, setup.Q, setup.ny, setup.nx)

    def _a(self, x, shape):
        a = np.ascontiguousarray(x, dtype=np.float64)
        assert a.shape == shape, (a.shape, shape)
        return a

    def force_kernel(self, rx, ry):
        out = np.empty(2)
        self.lib.orc2_force_kernel(self.p, float(rx), float(ry), out.ctypes.data)
        return out

    def discrete_a(self):
        return self.lib.orc2_discrete_a(self.p)

    def critical_T(self):
        return critical_point(self.discrete_a(), self.s.sigma)[1]

    def moments(self, F, G):
        F, G = self._a(F, self.shape), self._a(G, self.shape)
        grid = (self.s.ny, self.s.nx)
        out = [np.empty(grid) for _ in range(6)]
        self.lib.orc2_moments(self.p, F.ctypes.data, G.ctypes.data, *[o.ctypes.data for o in out])
        return tuple(out)

    def node_fields(self, F, G):
        mom = self.moments(F, G)
        out = np.empty((NFIELDS2, self.s.ny, self.s.nx))
        self.lib.orc2_node_fields(self.p, *[m.ctypes.data for m in mom], out.ctypes.data)
        return {k: out[i] for i, k in enumerate(FIELD_NAMES2)}

    def equilibria_node(self, fields: dict):
        """(F^S, G^S, J1_F, J1_G), each (Q, Q), for one node's fields (missing
        entries 0; chi and Pr default to 1)."""
        fl = np.zeros(NFIELDS2)
        fl[FIELD_NAMES2.index("chi")] = 1.0
        fl[FIELD_NAMES2.index("Pr")] = 1.0
        for k, v in fields.items():
            fl[FIELD_NAMES2.index(k)] = v
        Q = self.s.Q
        outs = [np.empty((Q, Q)) for _ in range(4)]
        self.lib.orc2_equilibria_node(self.p, fl.ctypes.data, *[o.ctypes.data for o in outs])
        return tuple(outs)

    def equilibrium(self, n, ux, uy, T):
        grid = (self.s.ny, self.s.nx)
        args = [self._a(np.broadcast_to(a, grid), grid) for a in (n, ux, uy, T)]
        F, G = np.empty(self.shape), np.empty(self.shape)
        self.lib.orc2_equilibrium(self.p, *[a.ctypes.data for a in args], F.ctypes.data, G.ctypes.data)
        return F, G

    def dxi(self, h):
        Q = self.s.Q
        h = self._a(h, (Q, Q))
        ox, oy = np.empty((Q, Q)), np.empty((Q, Q))
        self.lib.orc2_dxi(self.p, h.ctypes.data, ox.ctypes.data, oy.ctypes.data)
        return ox, oy

    def rhs(self, F, G, with_fields=False):
        F, G = self._a(F, self.shape), self._a(G, self.shape)
        RF, RG = np.empty(self.shape), np.empty(self.shape)
        fl = np.empty((NFIELDS2, self.s.ny, self.s.nx))
        self.lib.orc2_rhs(self.p, F.ctypes.data, G.ctypes.data, RF.ctypes.data, RG.ctypes.data, fl.ctypes.data)
        if with_fields:
            return RF, RG, {k: fl[i] for i, k in enumerate(FIELD_NAMES2)}
        return RF, RG

    def step(self, F, G, nsteps=1):
        F, G = self._a(F, self.shape).copy(), self._a(G, self.shape).copy()
        self.lib.orc2_step(self.p, F.ctypes.data, G.ctypes.data, int(nsteps))
        return F, G

    def totals(self, F, G):
        """[mass, momentum x, momentum y, kinetic + internal energy]"""
        F, G = self._a(F, self.shape), self._a(G, self.shape)
        out = np.empty(4)
        self.lib.orc2_totals(self.p, F.ctypes.data, G.ctypes.data, out.ctypes.data)
        return out
