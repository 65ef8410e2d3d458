"""torch.autograd binding of the EV-FDLB time step and its adjoint.

``EVRun.apply(phi_a, T0, n0, params, nsteps)`` projects the initial fields
(n0 [nx], u0 = 0, uniform T0) onto the Gauss-Hermite velocity set, advances
``nsteps`` Shu-Osher RK3 steps in the CUDA library and returns the final
density n(z, t_end) as a float64 CUDA tensor.  Its backward pass is the
library's hand-written discrete adjoint (evfdlb_adjoint): the forward keeps
the state every ``params.ckpt_every`` steps (100 if unset) and the reverse
sweep recomputes each segment from its checkpoint.  Gradients flow to phi_a
(the Sutherland well depth, through the Eq. (F1) force), to the uniform
initial temperature T0 and to every node of n0.

Every array crosses the C ABI as a device pointer (on_device = 1) on torch's
current stream of the device holding n0 (a CPU n0 is moved to the current
CUDA device); only the per-slab phi_a gradient comes back through host
memory, as the ABI defines it.
"""
from __future__ import annotations

import ctypes
import dataclasses

import torch

from . import Params, Sim, _check, lib


class EVRun(torch.autograd.Function):
    @staticmethod
    def forward(ctx, phi_a, T0, n0, params: Params, nsteps: int):
        p = dataclasses.replace(params, phi_a=float(phi_a), ckpt_every=params.ckpt_every or 100)
        if n0.numel() != p.nx:
            raise ValueError("n0 must hold nx values")
        dev = n0.device if n0.is_cuda else torch.device("cuda", torch.cuda.current_device())
        f64 = torch.float64
        with torch.cuda.device(dev):
            stream = torch.cuda.current_stream(dev)
            sim = Sim(p, stream=stream)
            nd = n0.detach().to(dev, f64).contiguous()
            ud = torch.zeros(p.nx, dtype=f64, device=dev)
            Td = torch.full((p.nx,), float(T0), dtype=f64, device=dev)
            sim.init(nd, ud, Td)
            sim.step(int(nsteps))
            n_end = torch.empty(p.nx, dtype=f64, device=dev)
            _check(lib().evfdlb_moments(sim.h, n_end.data_ptr(), None, None, None, None, 1), "evfdlb_moments")
        ctx.sim = sim
        ctx.dev = dev
        ctx.n0_dev = n0.device
        ctx.sdev = (getattr(phi_a, "device", "cpu"), getattr(T0, "device", "cpu"))
        return n_end

    @staticmethod
    def backward(ctx, grad_n):
        sim = ctx.sim
        f64 = torch.float64
        with torch.cuda.device(ctx.dev):
            g = grad_n.detach().to(ctx.dev, f64).contiguous()
            nx = g.numel()
            dn = torch.empty(nx, dtype=f64, device=ctx.dev)
            dT = torch.empty(nx, dtype=f64, device=ctx.dev)
            dphi = (ctypes.c_double * 1)()
            _check(lib().evfdlb_adjoint(sim.h, g.data_ptr(), 1, ctypes.addressof(dphi), dT.data_ptr(),
                                        dn.data_ptr()), "evfdlb_adjoint")
        sim.close()
        ctx.sim = None
        return (torch.tensor(dphi[0], dtype=f64, device=ctx.sdev[0]),
                dT.sum().to(ctx.sdev[1]),
                dn.to(ctx.n0_dev), None, None)
