"""GB300 (sm_103a) EV-FDLB time step: thin Python binding of libevfdlb.

Every step of the model runs in the CUDA library (``csrc/``, C ABI in
``include/evfdlb.h``); this module only marshals arguments.  There is no CPU
fallback: if the library is not built, or no CUDA device is present, the
calls raise.

Paper: Busuioc & Sofonea, "Thermal Enskog-Vlasov Lattice Boltzmann model
with phase separation", arXiv:2503.15187.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass, fields as dc_fields

import numpy as np

from .buildlib import LIB as LIB_PATH, build  # noqa: F401

EVFDLB_NFIELDS = 16
FIELD_NAMES = ("n", "u", "T", "q", "nbar", "chi", "force", "mu", "tau", "Pr",
               "nu", "A", "B", "D", "X", "bnchi")

BC_PERIODIC, BC_OUTFLOW, BC_HALO, BC_HALO_OUTFLOW_LO, BC_HALO_OUTFLOW_HI = 0, 1, 2, 3, 4
FP64, FP32, FP64_DF = 0, 1, 2
EV1, EV2 = 0, 1
RELAX_INV_TAU, RELAX_CHI_OVER_TAU = 0, 1

STATUS = {0: "ok", -1: "invalid argument", -2: "CUDA runtime error", -3: "out of device memory",
          -4: "non-finite value in the state", -5: "non-positive density or temperature",
          -6: "bounded device wait timed out", -7: "call out of order", -8: "not supported"}


class EvfdlbError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        super().__init__(f"{where}: {STATUS.get(code, code)} ({code})")


class CParams(ctypes.Structure):
    """Mirror of evfdlb_params (include/evfdlb.h)."""
    _fields_ = [("dim", ctypes.c_int32), ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
                ("dx", ctypes.c_double), ("sigma", ctypes.c_double), ("phi_a", ctypes.c_double),
                ("gamma", ctypes.c_double), ("r_cut", ctypes.c_double), ("Q", ctypes.c_int32),
                ("bc", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("force_model", ctypes.c_int32), ("relax_mode", ctypes.c_int32),
                ("dt", ctypes.c_double), ("cfl", ctypes.c_double), ("ckpt_every", ctypes.c_int32),
                ("weno_eps", ctypes.c_double), ("T_iso", ctypes.c_double)]


@dataclass
class Params:
    """Python view of evfdlb_params with the defaults of the paper's Sec. III."""
    nx: int
    dx: float
    Q: int = 16
    bc: int = BC_PERIODIC
    sigma: float = 1.0
    phi_a: float = 1.0
    gamma: float = 6.0
    r_cut: float = 6.0
    precision: int = FP64
    force_model: int = EV1
    relax_mode: int = RELAX_INV_TAU
    dt: float = 0.0
    cfl: float = 0.5
    ckpt_every: int = 0
    weno_eps: float = 1e-6
    dim: int = 1
    ny: int = 1
    T_iso: float = 0.0     # > 0: isothermal mode at this temperature

    def c(self) -> CParams:
        return CParams(**{f.name: getattr(self, f.name) for f in dc_fields(self)})


_lib = None


def lib():
    """The loaded libevfdlb (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libevfdlb is not built ({LIB_PATH}); call "
                               "paper_2503_15187_gb300.build() first")
        L = ctypes.CDLL(LIB_PATH)
        P = ctypes.POINTER(CParams)
        vp, i32, i64, d = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
        sig = {
            "evfdlb_default_params": (None, [P]),
            "evfdlb_create": (i32, [P, i32, P, vp, ctypes.POINTER(vp)]),
            "evfdlb_init": (i32, [vp, vp, vp, vp, i32]),
            "evfdlb_step": (i32, [vp, i64]),
            "evfdlb_step_async": (i32, [vp, i64]),
            "evfdlb_moments": (i32, [vp, vp, vp, vp, vp, vp, i32]),
            "evfdlb_get_state": (i32, [vp, vp, vp, i32]),
            "evfdlb_set_state": (i32, [vp, vp, vp, i32]),
            "evfdlb_rhs": (i32, [vp, vp, vp, i32]),
            "evfdlb_fields": (i32, [vp, vp, i32]),
            "evfdlb_slab_info": (i32, [vp, i32, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(d)]),
            "evfdlb_launches_per_step": (i32, [vp]),
            "evfdlb_tune": (i32, [vp, i32]),
            "evfdlb_tile_nodes": (i32, [vp]),
            "evfdlb_destroy": (None, [vp]),
            "evfdlb_status_string": (ctypes.c_char_p, [i32]),
            "evfdlb_discrete_a": (d, [P]),
            "evfdlb_critical_T": (d, [P]),
            "evfdlb_coexistence": (i32, [P, d, ctypes.POINTER(d), ctypes.POINTER(d)]),
            "evfdlb_velocity_set": (i32, [i32, vp, vp]),
            "evfdlb_step_static": (i32, [P, vp, i64, vp]),
            "evfdlb_rhs_vjp": (i32, [vp, vp, vp, i32, vp, vp, vp]),
            "evfdlb_adjoint_state": (i32, [vp, vp, vp, i32, vp, vp, vp, vp, vp, vp]),
            "evfdlb_adjoint": (i32, [vp, vp, i32, vp, vp, vp]),
            "evfdlb_probe_fp64_fma": (i32, [i32, vp, ctypes.POINTER(d)]),
            "evfdlb_divide_fp64": (i32, [vp, vp, vp, vp, i64, vp]),
            "evfdlb_profile_stage": (i32, [vp, i32]),
            "evfdlb_set_persistent": (i32, [vp, i32, i64]),
            "evfdlb_debug_gate": (i32, [vp, i32]),
            "evfdlb_halo_width": (i32, [P]),
            "evfdlb_halo_len": (i64, [vp]),
            "evfdlb_stage": (i32, [vp, i32]),
            "evfdlb_halo_pack": (i32, [vp, vp, vp]),
            "evfdlb_halo_unpack": (i32, [vp, vp, vp]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(code, where):
    if code != 0:
        raise EvfdlbError(code, where)


def _host(a, n=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if n is not None and a.size != n:
        raise ValueError(f"expected {n} values, got {a.size}")
    return a


def _ptr(x):
    """(pointer, on_device) for a numpy array or a CUDA torch tensor."""
    if isinstance(x, np.ndarray):
        return x.ctypes.data, 0
    if hasattr(x, "data_ptr") and getattr(x, "is_cuda", False):
        if not x.is_contiguous() or str(x.dtype) != "torch.float64":
            raise ValueError("device arrays must be contiguous float64 tensors")
        return x.data_ptr(), 1
    raise TypeError("expected a numpy array or a CUDA float64 tensor")


# ---------------------------------------------------------------------------
# host-side model constants
# ---------------------------------------------------------------------------
def velocity_set(Q: int):
    xi, w = np.empty(Q), np.empty(Q)
    _check(lib().evfdlb_velocity_set(Q, xi.ctypes.data, w.ctypes.data), "evfdlb_velocity_set")
    return xi, w


def discrete_a(p: Params) -> float:
    return lib().evfdlb_discrete_a(ctypes.byref(p.c()))


def critical_T(p: Params) -> float:
    return lib().evfdlb_critical_T(ctypes.byref(p.c()))


def coexistence(p: Params, T: float):
    nv, nl = ctypes.c_double(), ctypes.c_double()
    _check(lib().evfdlb_coexistence(ctypes.byref(p.c()), T, ctypes.byref(nv), ctypes.byref(nl)),
           "evfdlb_coexistence")
    return nv.value, nl.value


def step_static(p: Params, state, nsteps: int = 1, stream=None):
    """Advances a caller-owned device state (contiguous float64 CUDA tensor of
    2 * Q * nx values, F then G) by nsteps steps in place, without any device
    allocation: for callers that cannot allocate device memory (a host
    application's own pool, a fixed memory budget).  Calls that overlap on
    the GPU share the library's static working memory and must be serialised.
    ``stream`` is a torch.cuda.Stream (None: torch's current stream)."""
    import torch
    ptr, dev = _ptr(state)
    if not dev or state.numel() != 2 * p.Q * p.nx:
        raise ValueError("state must be a CUDA float64 tensor of 2 * Q * nx values")
    s = stream if stream is not None else torch.cuda.current_stream()
    _check(lib().evfdlb_step_static(ctypes.byref(p.c()), ptr, int(nsteps), ctypes.c_void_p(s.cuda_stream)),
           "evfdlb_step_static")


def halo_width(p: Params) -> int:
    """Ghost nodes per side of a z-split (BC_HALO) slab with parameters p:
    the widest read of one RK stage about a node (host computation)."""
    g = lib().evfdlb_halo_width(ctypes.byref(p.c()))
    if g < 0:
        raise ValueError("invalid parameters")
    return g


def probe_fp64_fma(reps: int = 5, stream=None) -> float:
    """Measured FP64 FMA throughput of the current device, GFLOP/s (the peak
    of the FP64 step's roofline); ``stream``: torch.cuda.Stream or None."""
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    g = ctypes.c_double()
    _check(lib().evfdlb_probe_fp64_fma(int(reps), ctypes.c_void_p(s.cuda_stream), ctypes.byref(g)),
           "evfdlb_probe_fp64_fma")
    return g.value


def divide_fp64(a, b, with_ieee=True, stream=None):
    """(q, q_ieee): the library's FP64 quotient a / b of two CUDA float64
    tensors, and the IEEE quotient beside it (None unless with_ieee)."""
    import torch
    if a.shape != b.shape:
        raise ValueError("a and b must have the same shape")
    (pa, da), (pb, db) = _ptr(a), _ptr(b)
    if not (da and db):
        raise ValueError("a and b must be CUDA float64 tensors")
    q = torch.empty_like(a)
    qi = torch.empty_like(a) if with_ieee else None
    s = stream if stream is not None else torch.cuda.current_stream()
    _check(lib().evfdlb_divide_fp64(pa, pb, q.data_ptr(), qi.data_ptr() if qi is not None else None,
                                    a.numel(), ctypes.c_void_p(s.cuda_stream)), "evfdlb_divide_fp64")
    return q, qi


# ---------------------------------------------------------------------------
# simulation context
# ---------------------------------------------------------------------------
class Sim:
    """One evfdlb context: nbatch independent slabs advanced together.

    ``stream`` is a torch.cuda.Stream (or None for torch's current stream)."""

    def __init__(self, params, stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("no CUDA device: the EV-FDLB library runs on the GPU only")
        plist = list(params) if isinstance(params, (list, tuple)) else [params]
        self.params = plist
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        arr = (CParams * len(plist))(*[p.c() for p in plist])
        self._arr = arr
        h = ctypes.c_void_p()
        _check(lib().evfdlb_create(None, len(plist), arr, ctypes.c_void_p(self.stream.cuda_stream),
                                   ctypes.byref(h)), "evfdlb_create")
        self.h = h
        self.dim = plist[0].dim
        self.nx = [p.nx for p in plist]
        self.Q = [p.Q for p in plist]
        if self.dim == 2:        # one plane periodic domain: nodes nx * ny, velocities Q * Q
            p0 = plist[0]
            self.NN = p0.nx * p0.ny
            self.NF = p0.Q * p0.Q * self.NN
        else:
            self.NN = sum(self.nx)
            self.NF = sum(p.nx * p.Q for p in plist)

    def close(self):
        if getattr(self, "h", None):
            lib().evfdlb_destroy(self.h)
            self.h = None

    __del__ = close

    def dt(self, s=0):
        nx, Q, dt = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_double()
        _check(lib().evfdlb_slab_info(self.h, s, ctypes.byref(nx), ctypes.byref(Q), ctypes.byref(dt)),
               "evfdlb_slab_info")
        return dt.value

    def launches_per_step(self):
        return lib().evfdlb_launches_per_step(self.h)

    def tune(self, tile_nodes):
        _check(lib().evfdlb_tune(self.h, int(tile_nodes)), "evfdlb_tune")

    def tile_nodes(self):
        return lib().evfdlb_tile_nodes(self.h)

    def set_persistent(self, enable=True, spin_limit=0):
        """The persistent form of the step (one launch per graph of steps,
        per-slab stage dependencies waited on the device with bounded polls),
        or back to one launch per RK stage."""
        _check(lib().evfdlb_set_persistent(self.h, int(bool(enable)), int(spin_limit)), "evfdlb_set_persistent")

    def debug_gate(self, open_):
        """Testing hook: with open_ False every dependency wait of the
        persistent form waits on a flag nothing sets (bounded-wait path)."""
        _check(lib().evfdlb_debug_gate(self.h, int(bool(open_))), "evfdlb_debug_gate")

    def stage(self, s):
        """Queues RK stage s (0, 1, 2 in order) of one step."""
        _check(lib().evfdlb_stage(self.h, int(s)), "evfdlb_stage")

    def halo_len(self):
        return int(lib().evfdlb_halo_len(self.h))

    def _halo_ptrs(self, a, b):
        """Device pointers of two halo messages (None: the side of an outflow
        end, which the library skips)."""
        n = self.halo_len()
        out = []
        for x in (a, b):
            if x is None:
                out.append(None)
                continue
            p, dev = _ptr(x)
            if not dev or x.numel() != n:
                raise ValueError(f"halo messages are CUDA float64 tensors of {n} values")
            out.append(p)
        return out

    def halo_pack(self, to_left, to_right):
        """Edge columns of the state the next stage reads into two CUDA
        float64 tensors of halo_len() values (queued on the stream)."""
        _check(lib().evfdlb_halo_pack(self.h, *self._halo_ptrs(to_left, to_right)), "evfdlb_halo_pack")

    def halo_unpack(self, from_left, from_right):
        """The neighbours' messages into the ghost nodes (queued on the stream)."""
        _check(lib().evfdlb_halo_unpack(self.h, *self._halo_ptrs(from_left, from_right)), "evfdlb_halo_unpack")

    def profile_stage(self, stage):
        """Queues stage 0, 1 or 2 of one step (as evfdlb_step runs it) on the
        context's stream without changing the state, for timing."""
        _check(lib().evfdlb_profile_stage(self.h, int(stage)), "evfdlb_profile_stage")

    def init(self, n0, u0, T0):
        """Projected Maxwellian state of (n0, u0, T0); in 2D u0 holds ux then
        uy ([2, nx * ny])."""
        nu = self.NN * (2 if self.dim == 2 else 1)
        if isinstance(n0, np.ndarray) or not hasattr(n0, "data_ptr"):
            n0, u0, T0 = _host(n0, self.NN), _host(u0, nu), _host(T0, self.NN)
        (pn, dev), (pu, _), (pT, _) = _ptr(n0), _ptr(u0), _ptr(T0)
        _check(lib().evfdlb_init(self.h, pn, pu, pT, dev), "evfdlb_init")

    def step(self, nsteps=1):
        _check(lib().evfdlb_step(self.h, int(nsteps)), "evfdlb_step")

    def step_async(self, nsteps=1):
        _check(lib().evfdlb_step_async(self.h, int(nsteps)), "evfdlb_step_async")

    def get_state(self, F=None, G=None):
        if F is None:
            F, G = np.empty(self.NF), np.empty(self.NF)
        (pF, dev), (pG, _) = _ptr(F), _ptr(G)
        _check(lib().evfdlb_get_state(self.h, pF, pG, dev), "evfdlb_get_state")
        return F, G

    def set_state(self, F, G):
        if isinstance(F, np.ndarray) or not hasattr(F, "data_ptr"):
            F, G = _host(F, self.NF), _host(G, self.NF)
        (pF, dev), (pG, _) = _ptr(F), _ptr(G)
        _check(lib().evfdlb_set_state(self.h, pF, pG, dev), "evfdlb_set_state")

    def rhs(self):
        """One right-hand side at the current state (state layout)."""
        RF, RG = np.empty(self.NF), np.empty(self.NF)
        _check(lib().evfdlb_rhs(self.h, RF.ctypes.data, RG.ctypes.data, 0), "evfdlb_rhs")
        return RF, RG

    def fields(self):
        out = np.empty((EVFDLB_NFIELDS, self.NN))
        _check(lib().evfdlb_fields(self.h, out.ctypes.data, 0), "evfdlb_fields")
        return {k: out[i] for i, k in enumerate(FIELD_NAMES)}

    def moments(self, with_totals=True):
        """(n, u, T, q, totals): per node; in 2D u and q are [2, nx * ny] and
        totals are {mass, momentum x, momentum y, kinetic + internal energy}."""
        vec = 2 if self.dim == 2 else 1
        n, T = np.empty(self.NN), np.empty(self.NN)
        u, q = np.empty(vec * self.NN), np.empty(vec * self.NN)
        tot = np.empty(4 * len(self.params)) if with_totals else None
        _check(lib().evfdlb_moments(self.h, n.ctypes.data, u.ctypes.data, T.ctypes.data, q.ctypes.data,
                                    tot.ctypes.data if tot is not None else None, 0), "evfdlb_moments")
        if vec == 2:
            u, q = u.reshape(2, self.NN), q.reshape(2, self.NN)
        return n, u, T, q, (tot.reshape(-1, 4) if tot is not None else None)

    # adjoint ----------------------------------------------------------------
    def rhs_vjp(self, WF, WG):
        """(J^T W_F, J^T W_G, dphi): the transpose of the Jacobian of one
        right-hand side at the current state applied to (W_F, W_G), and
        sum W . dR/dphi_a per slab."""
        WF, WG = _host(WF, self.NF), _host(WG, self.NF)
        oF, oG = np.empty(self.NF), np.empty(self.NF)
        dphi = np.empty(len(self.params))
        _check(lib().evfdlb_rhs_vjp(self.h, WF.ctypes.data, WG.ctypes.data, 0, oF.ctypes.data, oG.ctypes.data,
                                    dphi.ctypes.data), "evfdlb_rhs_vjp")
        return oF, oG, dphi

    def adjoint_state(self, barF, barG, fields=True):
        """Reverse sweep over every step since the last init / set_state for
        the cotangent (barF, barG) of the current state.  Returns a dict with
        dphi [nbatch], dF0, dG0 [NF] and, if fields and the trajectory began
        at init, dn0, du0, dT0 [NN] (gradients per node)."""
        barF, barG = _host(barF, self.NF), _host(barG, self.NF)
        out = {"dphi": np.empty(len(self.params)), "dF0": np.empty(self.NF), "dG0": np.empty(self.NF)}
        ptr = {k: None for k in ("dn0", "du0", "dT0")}
        if fields:
            for k in ptr:
                out[k] = np.empty(self.NN)
                ptr[k] = out[k].ctypes.data
        _check(lib().evfdlb_adjoint_state(self.h, barF.ctypes.data, barG.ctypes.data, 0, out["dphi"].ctypes.data,
                                          out["dF0"].ctypes.data, out["dG0"].ctypes.data, ptr["dn0"], ptr["du0"],
                                          ptr["dT0"]), "evfdlb_adjoint_state")
        return out

    def adjoint(self, dL_dn):
        """Gradient of a loss L(n_end) given dL/dn_end [NN]: (dphi [nbatch],
        dT0 [NN], dn0 [NN]) with respect to phi_a and the initial T0, n0."""
        g = _host(dL_dn, self.NN)
        dphi, dT0, dn0 = np.empty(len(self.params)), np.empty(self.NN), np.empty(self.NN)
        _check(lib().evfdlb_adjoint(self.h, g.ctypes.data, 0, dphi.ctypes.data, dT0.ctypes.data, dn0.ctypes.data),
               "evfdlb_adjoint")
        return dphi, dT0, dn0

    # helpers for one slab --------------------------------------------------
    def state_2d(self, s=0):
        """(F, G) of slab s as (Q, nx) arrays; for a 2D context as
        (Q, Q, ny, nx) arrays (index [kx, ky, y, x])."""
        F, G = self.get_state()
        if self.dim == 2:
            p = self.params[0]
            shp = (p.Q, p.Q, p.ny, p.nx)
            return F.reshape(shp), G.reshape(shp)
        off = sum(self.nx[i] * self.Q[i] for i in range(s))
        n = self.nx[s] * self.Q[s]
        return (F[off:off + n].reshape(self.Q[s], self.nx[s]),
                G[off:off + n].reshape(self.Q[s], self.nx[s]))
