"""The allocation-free time step, evfdlb_step_static.

Some callers of this library cannot allocate device memory: a plugin whose
host application owns all device memory through its own pool and only hands
out pointers, or a process held to a device-memory budget fixed at start-up.
evfdlb_step_static serves them: the caller passes the state, and every
intermediate buffer lives in one fixed-size static device array inside the
library.  These tests call it through the C ABI and check it, on two calls
in a row (the second call starts from what the first left behind in the
shared array), against the context path (evfdlb_create / evfdlb_set_state /
evfdlb_step) and against the FP64 oracle, on the same input, including cases
at the documented limits (nx = 8192, so 54-node tiles, and a force tap
half-width of 300).  The file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

import oracle as O
import paper_2503_15187_gb300 as ev
from paper_2503_15187_gb300 import workloads as W


def rel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300))


def test_oversize_requests_rejected_before_any_cuda_call():
    """Sizes beyond the static array's limits come back as E_INVALID_ARG; the
    checks run on the host before any CUDA call, so this needs no GPU."""
    L = ev.lib()
    dummy = ctypes.c_void_p(16)          # never dereferenced: the call returns first
    for kw in (dict(nx=8193, dx=0.25, Q=4),              # nx > EVFDLB_STATIC_MAX_NODES
               dict(nx=4096, dx=0.25, Q=17),             # Q * nx > EVFDLB_STATIC_MAX_ELEMENTS
               dict(nx=4096, dx=0.01, Q=8, r_cut=6.0),   # r_cut / dx > EVFDLB_STATIC_MAX_HALFWIDTH
               dict(nx=4096, dx=0.001, Q=8, force_model=ev.EV2)):  # sigma / dx + 2 > the same limit
        p = ev.Params(**kw)
        assert L.evfdlb_step_static(ctypes.byref(p.c()), dummy, 1, None) == -1, kw
    p = ev.Params(nx=64, dx=0.25)
    assert L.evfdlb_step_static(ctypes.byref(p.c()), None, 1, None) == -1
    assert L.evfdlb_step_static(ctypes.byref(p.c()), dummy, -1, None) == -1


@pytest.mark.gpu
@pytest.mark.parametrize("case", [(97, 24, 0.25, ev.BC_OUTFLOW, ev.EV1, False),
                                  (150, 32, 0.1, ev.BC_PERIODIC, ev.EV1, False),
                                  (97, 24, 0.25, ev.BC_OUTFLOW, ev.EV2, False),
                                  (64, 16, 0.25, ev.BC_PERIODIC, ev.EV1, True),     # isothermal mode
                                  (8192, 8, 0.25, ev.BC_PERIODIC, ev.EV1, False),   # nx at its limit: 54-node tiles
                                  (1200, 8, 0.02, ev.BC_OUTFLOW, ev.EV1, False)])   # 300-tap force half-width
def test_static_step_matches_context_step_and_oracle_twice(case):
    import torch
    nz, Q, dz, bc, fm, iso = case
    torch.cuda.set_device(0)
    p = ev.Params(nx=nz, dx=dz, Q=Q, bc=bc, force_model=fm)
    if iso:
        p.T_iso = 0.75 * ev.critical_T(p)
    sim = ev.Sim(p)
    orc = O.Oracle(O.Setup(nz=nz, Q=Q, dz=dz, dt=sim.dt(), bc=bc, force_model=fm, T_iso=p.T_iso))
    T = 0.8 * orc.critical_T()
    nv, nl = O.coexistence(T, orc.discrete_a())
    n0 = W.liquid_slab(nz, dz, nl, nv, thickness=0.35 * nz * dz, width=2.0)
    u0 = 0.02 * np.sin(2 * np.pi * np.arange(nz) / nz)
    sim.init(n0, u0, np.full(nz, T))
    F0, G0 = sim.get_state()
    state = torch.from_numpy(np.concatenate([F0, G0])).cuda()
    stream = torch.cuda.current_stream()
    L = ev.lib()
    for nsteps in (3, 2):                 # two calls in a row on the shared array
        start = state.cpu().numpy()
        code = L.evfdlb_step_static(ctypes.byref(p.c()), ctypes.c_void_p(state.data_ptr()), nsteps,
                                    ctypes.c_void_p(stream.cuda_stream))
        assert code == 0, ev.STATUS.get(code, code)
        sim.step(nsteps)
        Fc, Gc = sim.get_state()
        got = state.cpu().numpy()
        assert rel(got[:Q * nz], Fc) < 1e-12 and rel(got[Q * nz:], Gc) < 1e-12, nsteps
        Fo, Go = orc.step(start[:Q * nz].reshape(Q, nz), start[Q * nz:].reshape(Q, nz), nsteps)
        eF, eG = rel(got[:Q * nz], Fo.ravel()), rel(got[Q * nz:], Go.ravel())
        print(f"static nx={nz} Q={Q} dx={dz}: {nsteps} steps vs oracle F {eF:.1e} G {eG:.1e}")
        assert eF < 1e-12 and eG < 1e-12, nsteps
    sim.close()
