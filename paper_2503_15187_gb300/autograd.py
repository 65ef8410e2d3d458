"""torch.autograd binding of the EV-FDLB time step and its adjoint.

``EVRun.apply(phi_a, T0, n0, params, nsteps)`` projects the initial fields
(n0 [nx], u0 = 0, uniform T0) onto the Gauss-Hermite velocity set, advances
``nsteps`` Shu-Osher RK3 steps in the CUDA library and returns the final
density n(z, t_end) as a float64 tensor on n0's device.  Its backward pass
is the library's hand-written discrete adjoint (evfdlb_adjoint): the forward
keeps the state every ``params.ckpt_every`` steps (100 if unset) and the
reverse sweep recomputes each segment from its checkpoint.  Gradients flow
to phi_a (the Sutherland well depth, through the Eq. (F1) force), to the
uniform initial temperature T0 and to every node of n0.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import torch

from . import Params, Sim


class EVRun(torch.autograd.Function):
    @staticmethod
    def forward(ctx, phi_a, T0, n0, params: Params, nsteps: int):
        p = dataclasses.replace(params, phi_a=float(phi_a), ckpt_every=params.ckpt_every or 100)
        if n0.numel() != p.nx:
            raise ValueError("n0 must hold nx values")
        sim = Sim(p)
        nh = n0.detach().to("cpu", torch.float64).numpy()
        sim.init(nh, np.zeros(p.nx), np.full(p.nx, float(T0)))
        sim.step(int(nsteps))
        n_end = sim.moments(with_totals=False)[0]
        ctx.sim = sim
        ctx.dev = n0.device
        ctx.sdev = (getattr(phi_a, "device", "cpu"), getattr(T0, "device", "cpu"))
        return torch.from_numpy(n_end).to(n0.device)

    @staticmethod
    def backward(ctx, grad_n):
        sim = ctx.sim
        dphi, dT, dn = sim.adjoint(grad_n.detach().to("cpu", torch.float64).numpy())
        sim.close()
        ctx.sim = None
        f64 = torch.float64
        return (torch.tensor(dphi[0], dtype=f64, device=ctx.sdev[0]),
                torch.tensor(dT.sum(), dtype=f64, device=ctx.sdev[1]),
                torch.from_numpy(dn).to(ctx.dev), None, None)
