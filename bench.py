"""Benchmark of the EV-FDLB time step on GB300.

Workload (one "step" = one Shu-Osher RK3 time step, i.e. all of the hot path
over the whole slab): 1D liquid-slab evaporation, Nz = 4096 nodes,
dz = 0.1 sigma, Q = 32 Gauss-Hermite velocities, outflow ends, a centred
liquid slab 20 sigma thick at the coexistence densities of T = 0.8 T_c with
tanh interfaces of width 2 sigma, FP64.  Metric: GNVUPS = nodes x velocities
x steps / s / 1e9 (F and G together count as one velocity).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun (N > 1) every rank advances its own copy of the slab (replicas;
weak scaling) and rank 0 prints the aggregate.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

NZ, Q, DZ, T_RATIO, SLAB, WIDTH = 4096, 32, 0.1, 0.8, 20.0, 2.0
WORKLOAD = (f"1D liquid-slab evaporation: Nz={NZ}, dz={DZ} sigma, Q={Q}, outflow ends, "
            f"{SLAB:g}-sigma liquid slab at coexistence, T={T_RATIO} T_c, tanh width {WIDTH:g} sigma, FP64")
METRIC = "GNVUPS (node x velocity updates/s)"
UNIT = "GNVUPS"
L2_FLUSH_BYTES = 512 << 20


def stage_flops_method(Q: int) -> float:
    """Algorithmic FP64 flops of one stage-kernel launch per node, on the
    method's own operation count per node-velocity and distribution: one
    WENO-5 face (about 60 flops with its divisions), the force term's Hermite
    analysis (2Q), the synthesis of the collision and force terms (2Q) and
    the collision / RK combine (8); two distributions:
    2 (68 + 4Q) per node-velocity, 392 at Q = 32."""
    return Q * 2.0 * (68 + 4 * Q)


def stage_flops(Q: int, M: int, m: int) -> float:
    """Detailed FP64 flop count of one stage-kernel launch per node (FMA = 2,
    division = 1), from the operation counts of this kernel's arithmetic:
      per node and distribution, per velocity: Hermite analysis 2(Q-1),
      synthesis 2Q, one WENO-5 face 65, advective difference, relaxation and
      RK combine 10, moment sums 6;
      per node: two coefficient recurrences 2 * 14 Q, force taps 2(2M+1),
      Fischer-Methfessel taps 2(2m+1), gradients, transport and heat flux 100."""
    per_vel = 2 * (Q - 1) + 2 * Q + 65 + 10 + 6
    per_node = 2 * 14 * Q + 2 * (2 * M + 1) + 2 * (2 * m + 1) + 100
    return 2 * Q * per_vel + per_node


def fp64_peak_gflops(sm_mhz: float, sms: int = 152) -> float:
    """Nominal FP64 FMA rate of GB300: 2 FP64 FMA per clock per SM (4 flops)."""
    return sms * 4 * sm_mhz * 1e6 / 1e9


def fp64_peak_measured(ev, stream):
    """FP64 FMA throughput measured on this device in this run (the library's
    probe: independent FMA chains on every SM, best of 5 timed launches)."""
    return ev.probe_fp64_fma(5, stream=stream)


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons in the background."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == 7:
                self.rows.append(parts)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[j] for r in self.rows for j in range(4) if r[3 + j].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


TILE = 0   # --tile: fixed node tile for every leg (0: the autotuner's choice per leg)
# 2D step: bytes of state the kernels move per node-velocity-step (FP32)
IMPL_BYTES_2D = 168
# DRAM bytes (read + write) of one stage_kernel<double> launch (its one-wave
# 12-warp form) of this workload at the one-wave 27-node tile, from
# `ncu --set full` of the current kernel (4.51 MB read, 0 written: the outputs
# stay in the 129 MB L2); to be re-measured whenever the stage kernel changes.
STAGE_TRAFFIC_BYTES = 4516352   # dram read + write of one stage_kernel<double> launch, tile 27 (ncu)


def tuned_tile(p, n0, T, stream):
    """Node tile of the stage kernels: --tile if given, else the one the
    project's autotuner picks (autotune.py: every candidate timed with CUDA
    events on a scratch context of the same slab).  Results do not depend on
    the tile; a fixed --tile makes profiling runs reproduce the timed
    configuration (the autotuner's timings shift under a profiler)."""
    import numpy as np
    from paper_2503_15187_gb300 import autotune as AT
    if TILE > 0:
        return TILE
    best, _ = AT.autotune(p, n0, np.zeros(NZ), np.full(NZ, T), cache=None, stream=stream)
    return best


def build_workload(ev, W):
    p = ev.Params(nx=NZ, dx=DZ, Q=Q, bc=ev.BC_OUTFLOW)
    T = T_RATIO * ev.critical_T(p)
    nv, nl = ev.coexistence(p, T)
    n0 = W.liquid_slab(NZ, DZ, nl, nv, thickness=SLAB, width=WIDTH)
    return p, T, n0


def run_ours(args, rank, world):
    import numpy as np
    import torch
    import paper_2503_15187_gb300 as ev
    from paper_2503_15187_gb300 import workloads as W

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    p, T, n0 = build_workload(ev, W)
    stream = torch.cuda.current_stream()
    sim = ev.Sim(p, stream=stream)
    sim.tune(tuned_tile(p, n0, T, stream))
    sim.init(n0, np.zeros(NZ), np.full(NZ, T))
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    # warm-up
    sim.step(args.warmup)
    barrier()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    with ClockSampler(dev.index) as clk:
        barrier()
        t_wall = time.perf_counter()
        for i in range(args.steps):
            flush.fill_(float(i))             # evict the slab from L2 (untimed)
            starts[i].record(stream)
            sim.step_async(1)
            ends[i].record(stream)
        barrier()
        t_wall = time.perf_counter() - t_wall
    sim.step(0)                               # reads the device error word
    ms_steps = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    ms_total = sum(ms_steps)

    # the stage kernel by itself: each of the three stage launches of a step
    # bracketed by events on the context's stream (the state is not changed),
    # L2 flushed before each step as in the timed loop
    nprof = min(args.steps, 200)
    sev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(nprof)]
    for i in range(nprof):
        flush.fill_(float(i))
        for j in range(3):
            sev[i][j].record(stream)
            sim.profile_stage(j)
        sev[i][3].record(stream)
    torch.cuda.synchronize()
    stage_ms = [statistics.mean(sev[i][j].elapsed_time(sev[i][j + 1]) for i in range(nprof)) for j in range(3)]
    peak_meas = fp64_peak_measured(ev, stream)

    # end-to-end through the public API with pinned host buffers: per step the
    # state goes host -> device, one step runs, the moments come back (the
    # step is queued with evfdlb_step_async; evfdlb_moments synchronises and
    # reports any device error of the step).
    Fh = torch.empty(sim.NF, dtype=torch.float64, pin_memory=True).numpy()
    Gh = torch.empty(sim.NF, dtype=torch.float64, pin_memory=True).numpy()
    sim.get_state(Fh, Gh)
    outs = [torch.empty(NZ, dtype=torch.float64, pin_memory=True).numpy() for _ in range(4)]
    tot = torch.empty(4, dtype=torch.float64, pin_memory=True).numpy()
    import ctypes
    L = ev.lib()
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(args.steps):
        ev._check(L.evfdlb_set_state(sim.h, Fh.ctypes.data, Gh.ctypes.data, 0), "set_state")
        ev._check(L.evfdlb_step_async(sim.h, 1), "step_async")
        ev._check(L.evfdlb_moments(sim.h, *[o.ctypes.data for o in outs], tot.ctypes.data, 0), "moments")
    e1.record(stream)
    barrier()
    e2e_ms = e0.elapsed_time(e1)
    h2d = 2 * sim.NF * 8
    d2h = 4 * NZ * 8 + 4 * 8

    # reduce: max time over ranks
    def maxred(x):
        if world == 1:
            return x
        t = torch.tensor([x], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        return float(t.item())

    ms_total = maxred(ms_total)
    e2e_ms = maxred(e2e_ms)
    nvu = NZ * Q * args.steps * world
    value = nvu / (ms_total * 1e-3) / 1e9
    e2e = nvu / (e2e_ms * 1e-3) / 1e9
    clocks = clk.summary()
    sd = [ev.lib()]  # keep the library loaded until here
    del sd
    M, m = int(round(6.0 / DZ)), int(round(1.0 / DZ))
    launch_ms = statistics.mean(stage_ms)          # measured per stage launch (above)
    flops = stage_flops_method(Q) * NZ
    flops_detail = stage_flops(Q, M, m) * NZ
    achieved = flops / (launch_ms * 1e-3) / 1e9
    peak = peak_meas
    peak_nom = fp64_peak_gflops(2070.0)
    hbm_bytes = 128 * NZ * Q                       # 8 array passes x 2 distributions x 8 B per NVU-step
    hbm = hbm_bytes / (ms_total / args.steps * 1e-3) / 1e9
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "nodes": NZ, "velocities": Q, "steps_timed": args.steps,
                   "l2": f"flushed between timed steps ({L2_FLUSH_BYTES >> 20} MiB write, untimed)",
                   "parallelism": f"replicas x{world}", "tile_nodes": sim.tile_nodes()},
        "roofline": {"bound": "alu", "kernel": "stage_kernel", "achieved": achieved, "peak": peak,
                     "unit": "GFLOP/s", "frac": achieved / peak,
                     "peak_note": "FP64 FMA throughput measured in this run (evfdlb_probe_fp64_fma, of measured)",
                     "peak_nominal": peak_nom, "frac_of_nominal": achieved / peak_nom,
                     "peak_nominal_note": "152 SMs x 2 FP64 FMA/clk x 2070 MHz",
                     "flops_per_launch": flops,
                     "flops_note": "2 (68 + 4Q) per node-velocity (WENO-5 face ~60, analysis 2Q, synthesis 2Q, "
                                   "collision and RK 8; two distributions)",
                     "flops_per_launch_detailed": flops_detail,
                     "frac_detailed": flops_detail / (launch_ms * 1e-3) / 1e9 / peak,
                     "launch_ms": launch_ms, "stage_ms": stage_ms,
                     "launch_note": "CUDA events around each stage launch alone (evfdlb_profile_stage), "
                                    f"mean over {nprof} steps",
                     "traffic": STAGE_TRAFFIC_BYTES,
                     "traffic_note": "dram__bytes_read.sum + dram__bytes_write.sum of one stage_kernel<double> "
                                     "launch at the 27-node tile (ncu, profiles/stage_kernel_liquid_slab_"
                                     "4096x32_fp64_full.md)"},
        "hbm": {"algorithmic_GBps": hbm, "frac_of_measured": hbm / hbm_peak},
        "clocks": clocks,
        "gpu_launches": sim.launches_per_step() * args.steps,
        "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "ms_per_step": e2e_ms / args.steps},
        "wall_s_timed_region": t_wall,
    }
    n64 = sim.moments(with_totals=False)[0]
    sim.close()
    if not args.no_variants:
        legs = {"fp32": lambda: fp32_variant(args, ev, p, T, n0, stream, flush, barrier, maxred, world, n64),
                "ev2": lambda: ev2_variant(args, ev, p, T, n0, stream, flush, barrier, maxred, world, n64),
                "fp64_df": lambda: df_variant(args, ev, p, T, n0, stream, flush, barrier, maxred, world, n64),
                "adjoint": lambda: adjoint_leg(ev, W, stream),
                "batched": lambda: batched_leg(ev, W, stream, rank, world, maxred),
                "two_d": lambda: two_d_leg(ev, stream, flush, maxred, world, size=args.two_d_size)}
        want = args.variants.split(",") if args.variants else list(legs)
        line["variants"] = {k: legs[k]() for k in want}
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.cpu_seconds, T, n0)
    return line


def fp32_variant(args, ev, p, T, n0, stream, flush, barrier, maxred, world, n64):
    """The FP32 variant on the same workload and timing protocol: FP32 state and
    per-velocity work, FP64 chi / transport / gradients / conserved sums.  Its
    density after the same number of steps is compared with the FP64 run."""
    import dataclasses
    import numpy as np
    import torch
    p32 = dataclasses.replace(p, precision=ev.FP32)
    sim = ev.Sim(p32, stream=stream)
    sim.tune(tuned_tile(p32, n0, T, stream))
    sim.init(n0, np.zeros(NZ), np.full(NZ, T))
    sim.step(args.warmup)
    barrier()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    for i in range(args.steps):
        flush.fill_(float(i))
        starts[i].record(stream)
        sim.step_async(1)
        ends[i].record(stream)
    barrier()
    sim.step(1)          # the FP64 state compared against has W + K + 1 steps (its end-to-end leg adds one)
    ms = maxred(sum(s.elapsed_time(e) for s, e in zip(starts, ends)))
    n32 = sim.moments(with_totals=False)[0]
    tile = sim.tile_nodes()
    sim.close()
    return {"value": NZ * Q * args.steps * world / (ms * 1e-3) / 1e9, "unit": UNIT, "dtype": "f32 (f64 FM average and chi, "
            "gradient differences, heat flux, conserved sums)", "ms_per_step": ms / args.steps,
            "max_rel_diff_n_vs_fp64": float(np.abs(n32 - n64).max() / np.abs(n64).max()),
            "gpu_launches": 3 * args.steps, "tile_nodes": tile}


def ev2_variant(args, ev, p, T, n0, stream, flush, barrier, maxred, world, n64):
    """The EV2 force model (Eq. (F2)) on the same slab and timing protocol, FP64:
    the 5-point force stencil replaces the 2 r_cut/dx + 1 Simpson taps.  The
    slab starts at the same profile and temperature and its density after the
    same number of steps is compared with the EV1 run."""
    import dataclasses
    import numpy as np
    import torch
    p2 = dataclasses.replace(p, force_model=ev.EV2)
    sim = ev.Sim(p2, stream=stream)
    sim.tune(tuned_tile(p2, n0, T, stream))
    sim.init(n0, np.zeros(NZ), np.full(NZ, T))
    sim.step(args.warmup)
    barrier()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    for i in range(args.steps):
        flush.fill_(float(i))
        starts[i].record(stream)
        sim.step_async(1)
        ends[i].record(stream)
    barrier()
    sim.step(1)
    ms = maxred(sum(s.elapsed_time(e) for s, e in zip(starts, ends)))
    n2 = sim.moments(with_totals=False)[0]
    tile = sim.tile_nodes()
    sim.close()
    return {"value": NZ * Q * args.steps * world / (ms * 1e-3) / 1e9, "unit": UNIT, "dtype": "f64",
            "ms_per_step": ms / args.steps, "force": "Eq. (F2), 5-point stencils",
            "max_rel_diff_n_vs_ev1": float(np.abs(n2 - n64).max() / np.abs(n64).max()),
            "gpu_launches": 3 * args.steps, "tile_nodes": tile}


def df_variant(args, ev, p, T, n0, stream, flush, barrier, maxred, world, n64):
    """The FP64_DF variant on the same slab and timing protocol: FP64 state and
    arithmetic except the stage's Hermite analysis and synthesis, which run as
    double-float (Dot2) sums on the FP32 pipe.  Its density after the same
    number of steps is compared with the FP64 run."""
    import dataclasses
    import numpy as np
    import torch
    pdf = dataclasses.replace(p, precision=ev.FP64_DF)
    sim = ev.Sim(pdf, stream=stream)
    sim.tune(tuned_tile(pdf, n0, T, stream))
    sim.init(n0, np.zeros(NZ), np.full(NZ, T))
    sim.step(args.warmup)
    barrier()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    for i in range(args.steps):
        flush.fill_(float(i))
        starts[i].record(stream)
        sim.step_async(1)
        ends[i].record(stream)
    barrier()
    sim.step(1)
    ms = maxred(sum(s.elapsed_time(e) for s, e in zip(starts, ends)))
    nd = sim.moments(with_totals=False)[0]
    tile = sim.tile_nodes()
    sim.close()
    return {"value": NZ * Q * args.steps * world / (ms * 1e-3) / 1e9, "unit": UNIT,
            "dtype": "f64 (Hermite transforms and WENO-5 faces as double-float pairs on the FP32 pipe)",
            "ms_per_step": ms / args.steps,
            "max_rel_diff_n_vs_fp64": float(np.abs(nd - n64).max() / np.abs(n64).max()),
            "gpu_launches": 3 * args.steps, "tile_nodes": tile}


def adjoint_leg(ev, W, stream, steps=2000):
    """Cost of the discrete adjoint against the forward run on the adjoint
    calibration workload (periodic slab Nz = 1024, dz = 0.25, Q = 24,
    T = 0.7 T_c, mean n = 0.25 with +-1% noise, checkpoint every 100 steps),
    over `steps` steps: backward (segment recompute + reverse sweep + initial
    projection) / forward (steps with checkpoint copies)."""
    import numpy as np
    import torch
    nz, Q, dz = 1024, 24, 0.25
    p = ev.Params(nx=nz, dx=dz, Q=Q, ckpt_every=100)
    T = 0.7 * ev.critical_T(p)
    n0 = W.noisy_uniform(nz, 0.25, 0.01)
    sim = ev.Sim(p, stream=stream)
    times = []
    for rep in range(2):                  # the first pass allocates the work buffers
        sim.init(n0, np.zeros(nz), np.full(nz, T))
        torch.cuda.synchronize()
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        e[0].record(stream)
        sim.step(steps)
        e[1].record(stream)
        n = sim.moments(with_totals=False)[0]
        sim.adjoint(2.0 * (n - 0.25))
        e[2].record(stream)
        torch.cuda.synchronize()
        times.append((e[0].elapsed_time(e[1]), e[1].elapsed_time(e[2])))
    sim.close()
    fwd, bwd = times[-1]
    return {"workload": f"periodic Nz={nz}, dz={dz}, Q={Q}, {steps} steps, checkpoint every 100", "forward_ms": fwd,
            "backward_ms": bwd, "backward_over_forward": bwd / fwd}


def batched_leg(ev, W, stream, rank=0, world=1, maxred=lambda x: x, steps=100):
    """Batched against per-instance launches on the phase-separation batch:
    256 independent periodic slabs, Nz log-uniform in [128, 8192],
    Q in {16, 24, 32}, T/T_c in [0.6, 0.95], mean n in [0.15, 0.35], +-1%
    noise, dz = 0.25, FP64.  Batched: one context, one launch per RK stage for
    all slabs, node tile from the autotuner.  Persistent: the same context
    and tile with one resident launch per graph of steps, each slab's stages
    ordered by device-side counters.  Per-instance: one context per
    slab, each with its own (one-wave) tile, launched back to back on the
    same stream.  Both are timed over `steps` steps from the same state.
    Under N ranks each rank advances its longest-processing-time share of the
    slabs (no exchange while stepping; weak in slab count), the rates are
    whole-job (all slabs / slowest rank), and the per-slab masses are gathered
    at the end."""
    import numpy as np
    import torch
    from paper_2503_15187_gb300 import autotune as AT
    from paper_2503_15187_gb300 import shard
    all_slabs = W.batch_slabs(nslab=256)
    mine = shard.my_share(all_slabs, rank, world) if world > 1 else list(range(len(all_slabs)))
    slabs = [all_slabs[i] for i in mine]
    DZb = 0.25
    params = [ev.Params(nx=s["nz"], dx=DZb, Q=s["Q"]) for s in slabs]
    n0 = np.concatenate([s["n0"] for s in slabs])
    T0 = np.concatenate([np.full(s["nz"], s["T_ratio"] * ev.critical_T(p)) for s, p in zip(slabs, params)])
    u0 = np.zeros_like(n0)
    nvu = sum(s["nz"] * s["Q"] for s in all_slabs) * steps
    best, tune_ms = AT.autotune(params, n0, u0, T0, stream=stream)
    sim = ev.Sim(params, stream=stream)
    sim.tune(best)
    sim.init(n0, u0, T0)
    sim.step(2)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sim.step_async(steps)
    e1.record(stream)
    sim.step(0)
    ms_b = maxred(e0.elapsed_time(e1))
    mass = sim.moments()[4][:, 0]
    state_b = np.concatenate(sim.get_state())
    # persistent form: one launch per graph of steps, stage dependencies per
    # slab waited on the device; same tile, same initial state
    sim.set_persistent(True)
    sim.init(n0, u0, T0)
    sim.step(2)
    e0.record(stream)
    sim.step_async(steps)
    e1.record(stream)
    sim.step(0)
    ms_q = maxred(e0.elapsed_time(e1))
    same = bool(np.array_equal(np.concatenate(sim.get_state()), state_b))
    sim.close()
    if world > 1:
        masses = shard.gather_by_slab({i: float(m) for i, m in zip(mine, mass)}, len(all_slabs))
        assert len(masses) == len(all_slabs)
    sims, off = [], 0
    for p, s in zip(params, slabs):
        one = ev.Sim(p, stream=stream)
        one.init(s["n0"], np.zeros(p.nx), T0[off:off + p.nx])
        off += p.nx
        one.step(2)
        sims.append(one)
    torch.cuda.synchronize()
    e0.record(stream)
    for one in sims:
        one.step_async(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_p = maxred(e0.elapsed_time(e1))
    for one in sims:
        one.step(0)
        one.close()
    vb, vp = nvu / (ms_b * 1e-3) / 1e9, nvu / (ms_p * 1e-3) / 1e9
    vq = nvu / (ms_q * 1e-3) / 1e9
    return {"workload": "256 periodic slabs, Nz log-uniform [128, 8192], Q in {16,24,32}, dz 0.25, FP64",
            "sharding": f"LPT over {world} rank(s), {len(mine)} slabs on rank {rank}",
            "nvu_per_step": nvu // steps, "steps": steps, "batched_GNVUPS": vb, "per_instance_GNVUPS": vp,
            "batched_over_per_instance": vb / vp, "tile_nodes": best,
            "persistent_GNVUPS": vq, "persistent_over_per_stage": vq / vb,
            "persistent_bit_identical": same,
            # the time the launch-per-stage form loses at its three grid-wide
            # stage boundaries per step (tails of the last wave, launch gaps)
            "stage_boundary_ms_per_step": (ms_b - ms_q) / steps,
            "ms_per_step": {"per_stage": ms_b / steps, "persistent": ms_q / steps,
                            "per_instance": ms_p / steps},
            "autotune_ms_per_step": {str(k): round(v, 3) for k, v in tune_ms.items()}}


def two_d_leg(ev, stream, flush, maxred, world, steps=3, size=1024):
    """2D phase separation: 1024 x 1024 periodic grid, dx = 0.25 sigma,
    tensor-product Gauss-Hermite 16 x 16 velocities, FP32 bulk with FP64
    conserved sums, T = 0.75 T_c, mean n = 0.25 with +-1% seeded noise.
    State 2 GiB per copy (larger than L2); timed over `steps` steps with CUDA
    events.  Algorithmic HBM bytes per node-velocity-step: the Shu-Osher RK3
    streams 8 array passes per step (stage 1 reads u and writes u1, stages 2
    and 3 read u and their input and write), 2 distributions x 4 B: 64 B.
    The implementation's own state traffic per node-velocity-step is
    reported beside it (IMPL_BYTES_2D)."""
    import numpy as np
    import torch
    nx = ny = size           # --two-d-size: a smaller grid for ncu captures only
    Q = 16
    p = ev.Params(nx=nx, dx=0.25, Q=Q, dim=2, ny=ny, precision=ev.FP32)
    T = 0.75 * ev.critical_T(p)
    sim = ev.Sim(p, stream=stream)
    rng = np.random.default_rng(15187)
    n0 = 0.25 * (1 + 0.01 * rng.uniform(-1, 1, nx * ny))
    sim.init(n0, np.zeros(2 * nx * ny), np.full(nx * ny, T))
    sim.step(2)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sim.step_async(steps)
    e1.record(stream)
    sim.step(0)
    ms = maxred(e0.elapsed_time(e1)) / steps
    mass = sim.moments()[4][0][0]
    launches = sim.launches_per_step()
    sim.close()
    nvu = nx * ny * Q * Q
    gbs = 64.0 * nvu / (ms * 1e-3) / 1e9
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    return {"workload": f"2D phase separation {nx}x{ny}, dx 0.25, 16x16 velocities, FP32 (FP64 conserved sums)",
            "value": nvu * world / (ms * 1e-3) / 1e9, "unit": UNIT, "ms_per_step": ms,
            "algorithmic_GBps": gbs, "algorithmic_bytes_per_nvu_step": 64,
            "hbm_frac_of_measured": gbs / hbm_peak, "hbm_peak_GBps": hbm_peak,
            "impl_state_bytes_per_nvu_step": IMPL_BYTES_2D,
            "impl_state_GBps": IMPL_BYTES_2D * nvu / (ms * 1e-3) / 1e9,
            "mass": mass, "gpu_launches_per_step": launches}


def _oracle_rate(O, threads, budget_s, T, n0, max_steps=10**9):
    """(GNVUPS, steps, seconds, threads used) of the FP64 oracle as it stands
    on the bench slab, whole slab per step, as many steps as fit in budget_s."""
    import numpy as np
    used = O.set_threads(threads)
    xi, _ = O.gauss_hermite(Q)
    dt = 0.5 * DZ / np.abs(xi).max()
    orc = O.Oracle(O.Setup(nz=NZ, Q=Q, dz=DZ, dt=dt, bc=1))
    F, G = orc.equilibrium(n0, np.zeros(NZ), np.full(NZ, T))
    steps, t0 = 0, time.perf_counter()
    while steps < max_steps:
        F, G = orc.step(F, G, 1)
        steps += 1
        if time.perf_counter() - t0 > budget_s:
            break
    el = time.perf_counter() - t0
    return NZ * Q * steps / el / 1e9, steps, el, used


def cpu_baseline(budget_s, T, n0):
    """Times the FP64 oracle as it stands on the host's cores on a bounded
    sample of the same workload: OpenMP over the nodes on every core this
    process may use (the primary figure), and on one core (`single_core`)."""
    import oracle as O
    cores = O.available_cores()
    v1, s1, e1, _ = _oracle_rate(O, 1, budget_s, T, n0)
    vn, sn, en, used = _oracle_rate(O, cores, budget_s, T, n0)
    O.set_threads(1)
    return {"value": vn, "unit": UNIT, "cores": used, "kind": "oracle",
            "sample": f"{sn} full time steps of the {NZ}x{Q} slab ({en:.1f} s, OpenMP over nodes, {used} threads)",
            "single_core": {"value": v1, "unit": UNIT, "cores": 1,
                            "sample": f"{s1} full time steps of the {NZ}x{Q} slab ({e1:.1f} s, one thread)"}}


def run_reference(args):
    """The oracle as the reference arm, on every host core this process may
    use (OpenMP over nodes): each step one full oracle time step, at most 100
    steps timed so that the run stays within a minute or two; the line
    reports the steps actually timed and the threads used."""
    import numpy as np
    import oracle as O
    used = O.set_threads(O.available_cores())
    xi, _ = O.gauss_hermite(Q)
    dt = 0.5 * DZ / np.abs(xi).max()
    orc = O.Oracle(O.Setup(nz=NZ, Q=Q, dz=DZ, dt=dt, bc=1))
    T = T_RATIO * orc.critical_T()
    nv, nl = O.coexistence(T, orc.discrete_a())
    from paper_2503_15187_gb300 import workloads as W
    n0 = W.liquid_slab(NZ, DZ, nl, nv, thickness=SLAB, width=WIDTH)
    F, G = orc.equilibrium(n0, np.zeros(NZ), np.full(NZ, T))
    F, G = orc.step(F, G, args.warmup)
    steps = min(args.steps, 100)
    t0 = time.perf_counter()
    F, G = orc.step(F, G, steps)
    el = time.perf_counter() - t0
    v = NZ * Q * steps / el / 1e9
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": 1,
            "steps": steps, "warmup": args.warmup, "ms_per_step": el * 1e3 / steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "nodes": NZ, "velocities": Q},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": used, "kind": "oracle",
                             "sample": f"{steps} full time steps of the {NZ}x{Q} slab, OpenMP over nodes, "
                                       f"{used} threads"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=10.0,
                    help="seconds of oracle time per CPU-baseline leg (one core, then all cores)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-variants", action="store_true",
                    help="report the headline FP64 leg only (no FP32 / adjoint / batched / 2D legs), e.g. for ncu")
    ap.add_argument("--variants", default="", help="comma-separated subset of fp32,ev2,fp64_df,adjoint,batched,two_d")
    ap.add_argument("--two-d-size", type=int, default=1024,
                    help="grid edge of the two_d leg (default 1024, the workload; smaller only for ncu captures)")
    ap.add_argument("--tile", type=int, default=0,
                    help="node tile for the 1D legs (default 0: each leg's autotuned tile), e.g. for ncu")
    args = ap.parse_args()
    global TILE
    TILE = args.tile
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args)), flush=True)
        return
    if world > 1:
        import torch
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        torch.distributed.init_process_group("nccl")
    from paper_2503_15187_gb300.buildlib import build
    if rank == 0 or world == 1:
        build()
    if world > 1:
        import torch
        torch.distributed.barrier()
    line = run_ours(args, rank, world)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
