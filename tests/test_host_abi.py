"""CPU-side checks of libevfdlb: the library builds and loads, exports every
entry point include/evfdlb.h declares, and its host-side model constants
(velocity set, force constant, critical point, Maxwell construction) agree
with the oracle's independent implementations.  No CUDA call is made."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

import oracle as O
import paper_2503_15187_gb300 as ev
from paper_2503_15187_gb300.buildlib import build as build_lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    build_lib()
    return ev.lib()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "evfdlb.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(evfdlb_[A-Za-z0-9_]+)\s*\(", src)))


def exported_functions():
    """Names of the evfdlb_* functions the built library exports (the
    dynamic symbol table as `nm -D --defined-only` lists it)."""
    import shutil
    import subprocess
    nm = shutil.which("nm")
    if nm is None:
        pytest.skip("nm is not available")
    out = subprocess.run([nm, "-D", "--defined-only", ev.LIB_PATH], capture_output=True, text=True, check=True)
    names = set()
    for line in out.stdout.splitlines():
        parts = line.split()
        if len(parts) == 3 and parts[1] == "T" and parts[2].startswith("evfdlb_"):
            names.add(parts[2])
    return sorted(names)


def test_exports_every_declared_symbol(L):
    names = declared_functions()
    assert len(names) >= 18
    for n in names:
        assert hasattr(L, n), n


def test_declares_every_exported_symbol(L):
    """The header and the library agree in both directions: every evfdlb_*
    function the library exports is declared in include/evfdlb.h."""
    declared = set(declared_functions())
    exported = exported_functions()
    assert len(exported) >= 18
    missing = [n for n in exported if n not in declared]
    assert not missing, f"exported but not declared in include/evfdlb.h: {missing}"


def test_status_strings(L):
    for code in range(-8, 1):
        assert L.evfdlb_status_string(code)
    assert L.evfdlb_status_string(-4) == b"non-finite value in the state"


@pytest.mark.parametrize("Q", [4, 8, 16, 24, 32, 48])
def test_velocity_set_matches_oracle(L, Q):
    xi, w = ev.velocity_set(Q)
    xo, wo = O.gauss_hermite(Q)
    o = np.argsort(xo)
    assert np.all(np.diff(xi) > 0)
    assert np.allclose(xi, xo[o], rtol=0, atol=2e-14 * max(1, np.abs(xo).max()))
    assert np.allclose(w, wo[o], rtol=1e-12, atol=0)
    assert abs(w.sum() - 1) < 1e-14


def test_default_params_are_the_papers(L):
    cp = ev.CParams()
    L.evfdlb_default_params(ctypes.byref(cp))
    assert (cp.sigma, cp.phi_a, cp.gamma, cp.r_cut, cp.Q) == (1.0, 1.0, 6.0, 6.0, 16)
    assert cp.weno_eps == 1e-6 and cp.cfl == 0.5 and cp.dim == 1


@pytest.mark.parametrize("dx", [0.25, 0.1, 0.125])
def test_force_constant_and_critical_point(L, dx):
    p = ev.Params(nx=64, dx=dx)
    orc = O.Oracle(O.Setup(nz=64, Q=8, dz=dx, dt=0.01))
    assert abs(ev.discrete_a(p) - orc.discrete_a()) < 1e-13 * orc.discrete_a()
    assert abs(ev.critical_T(p) - orc.critical_T()) < 1e-12


@pytest.mark.parametrize("r", [0.6, 0.7, 0.8, 0.95])
def test_coexistence_matches_oracle(L, r):
    p = ev.Params(nx=64, dx=0.25)
    a = ev.discrete_a(p)
    T = r * ev.critical_T(p)
    nv, nl = ev.coexistence(p, T)
    nvo, nlo = O.coexistence(T, a)
    assert abs(nv - nvo) < 1e-9 * nvo and abs(nl - nlo) < 1e-9 * nlo


def test_invalid_params_rejected(L):
    for bad in (dict(dx=0.3), dict(dx=0.25, Q=40), dict(dx=0.25, r_cut=5.75),
                dict(dx=0.25, gamma=3.0), dict(dx=0.25, bc=7)):
        kw = dict(nx=64)
        kw.update(bad)
        p = ev.Params(**kw)
        assert math.isnan(ev.critical_T(p)), bad


@pytest.mark.parametrize("dx", [0.25, 0.1])
def test_ev2_constants_match_oracle(L, dx):
    """EV2 reports the printed a of Eq. (F2); the critical point and the
    coexistence densities follow from it."""
    p = ev.Params(nx=64, dx=dx, force_model=ev.EV2, r_cut=5.3)   # r_cut is not used by EV2
    orc = O.Oracle(O.Setup(nz=64, Q=8, dz=dx, dt=0.01, force_model=1))
    assert abs(ev.discrete_a(p) - orc.discrete_a()) < 1e-15 * orc.discrete_a()
    assert abs(ev.critical_T(p) - orc.critical_T()) < 1e-12
    T = 0.8 * ev.critical_T(p)
    nv, nl = ev.coexistence(p, T)
    nvo, nlo = O.coexistence(T, orc.discrete_a())
    assert abs(nv - nvo) < 1e-9 * nvo and abs(nl - nlo) < 1e-9 * nlo


def test_ev2_invalid_params_rejected(L):
    for bad in (dict(gamma=5.0), dict(gamma=4.5), dict(dx=0.3), dict(force_model=2)):
        kw = dict(nx=64, dx=0.25, force_model=ev.EV2)
        kw.update(bad)
        assert math.isnan(ev.critical_T(ev.Params(**kw))), bad


def _create(L, plist, nbatch=None, with_out=True):
    """evfdlb_create on a batch of Params; (status, handle or None)."""
    arr = (ev.CParams * len(plist))(*[p.c() for p in plist]) if plist else None
    h = ctypes.c_void_p(0x1234)                    # create must clear it on failure
    rc = L.evfdlb_create(None, len(plist) if nbatch is None else nbatch, arr, None,
                         ctypes.byref(h) if with_out else None)
    return rc, h.value


def test_create_rejects_invalid_arguments_before_any_device_call(L):
    """Argument validation of evfdlb_create runs on the host before its first
    CUDA call: empty or tiny grids, Q outside the supported orders, unknown
    enums, an empty batch, mixed precisions in one batch and a missing output
    pointer return E_INVALID_ARG and leave no handle; 2D requests this model
    does not cover return E_UNSUPPORTED."""
    INVALID, UNSUPPORTED = -1, -8
    base = dict(nx=64, dx=0.25)
    for bad in (dict(nx=0), dict(nx=7), dict(Q=3), dict(Q=33), dict(dx=0.0), dict(bc=5),
                dict(precision=9), dict(relax_mode=4), dict(force_model=3), dict(weno_eps=0.0),
                dict(dt=0.0, cfl=0.0), dict(T_iso=-1.0), dict(dim=1, ny=2)):
        kw = dict(base)
        kw.update(bad)
        rc, h = _create(L, [ev.Params(**kw)])
        assert rc == INVALID and h is None, bad
    assert _create(L, [ev.Params(**base)], nbatch=0) == (INVALID, None)
    mixed = [ev.Params(**base), ev.Params(precision=ev.FP32, **base)]
    assert _create(L, mixed) == (INVALID, None)
    assert _create(L, [ev.Params(**base)], with_out=False)[0] == INVALID
    # 2D: more nodes than 32-bit node offsets address, odd Q, outflow ends
    for bad in (dict(nx=50000, ny=50000), dict(Q=7), dict(bc=ev.BC_OUTFLOW)):
        kw = dict(dim=2, nx=64, ny=64, dx=0.25, Q=8)
        kw.update(bad)
        assert _create(L, [ev.Params(**kw)]) == (INVALID, None), bad
    two_d = dict(dim=2, nx=64, ny=64, dx=0.25, Q=8)
    assert _create(L, [ev.Params(**two_d)] * 2)[0] == UNSUPPORTED
    assert _create(L, [ev.Params(force_model=ev.EV2, **two_d)]) == (UNSUPPORTED, None)
