"""The benchmark picks the node tile of the stage kernels with the autotuner,
so the full-size liquid-slab workload (Nz = 4096, dz = 0.1, Q = 32, outflow
ends, 20-sigma slab at the coexistence densities of T = 0.8 T_c) is checked
against the oracle at EVERY tile the autotuner may choose, in each precision
the benchmark times: one step, FP64 and FP64_DF at 1e-12, FP32 at 1e-5
(normwise per distribution).  The tile changes which CTA owns which nodes,
never the arithmetic, so every tile must pass.
"""
import numpy as np
import pytest

import oracle as O
import paper_2503_15187_gb300 as ev
from paper_2503_15187_gb300 import autotune as AT
from paper_2503_15187_gb300 import workloads as W

pytestmark = pytest.mark.gpu

NZ, Q, DZ = 4096, 32, 0.1


def rel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300))


@pytest.fixture(scope="module")
def reference():
    p = ev.Params(nx=NZ, dx=DZ, Q=Q, bc=ev.BC_OUTFLOW)
    sim = ev.Sim(p)
    orc = O.Oracle(O.Setup(nz=NZ, Q=Q, dz=DZ, dt=sim.dt(), bc=1))
    sim.close()
    T = 0.8 * orc.critical_T()
    nv, nl = O.coexistence(T, orc.discrete_a())
    n0 = W.liquid_slab(NZ, DZ, nl, nv, thickness=20.0, width=2.0)
    F, G = orc.equilibrium(n0, np.zeros(NZ), np.full(NZ, T))
    Fo, Go = orc.step(F, G, 1)
    return F, G, Fo, Go


@pytest.mark.parametrize("prec,bar", [(ev.FP64, 1e-12), (ev.FP64_DF, 1e-12), (ev.FP32, 1e-5)])
def test_full_size_step_at_every_candidate_tile(reference, prec, bar):
    import torch
    F, G, Fo, Go = reference
    sim = ev.Sim(ev.Params(nx=NZ, dx=DZ, Q=Q, bc=ev.BC_OUTFLOW, precision=prec))
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    worst = 0.0
    for z in AT.candidates(NZ, sms):
        sim.tune(z)
        sim.set_state(F.ravel(), G.ravel())
        sim.step(1)
        Fg, Gg = sim.state_2d()
        e = max(rel(Fg, Fo), rel(Gg, Go))
        worst = max(worst, e)
        assert e < bar, (z, e)
    print(f"precision {prec}: worst over {len(AT.candidates(NZ, sms))} tiles {worst:.1e}")
    sim.close()
