"""Autotuner of the node tile of the stage kernels.

Each CTA of a stage kernel advances all velocities of ``tile_nodes``
consecutive nodes of one slab.  Small tiles give more CTAs per SM (latency
hiding across CTAs, less shared memory each) but repeat the per-tile work
(table staging, the density halo of the Eq. (F1) force); large tiles amortise
it over more nodes.  The best tile depends on the slab mix, Q and the
precision, so it is measured: every candidate is timed with CUDA events over
a few steps on a scratch context of the same slabs, and the fastest is
returned and kept in a JSON cache keyed by the device and the slab set.
Per-node arithmetic does not depend on the tile, so the choice changes
speed only, never results.
"""
from __future__ import annotations

import hashlib
import json
import os

import numpy as np

from . import Sim
from .buildlib import BUILD

CACHE = os.path.join(BUILD, "autotune.json")


def candidates(total_nodes: int, sms: int):
    """Tile sizes to try: one to six waves of CTAs over the SMs, and a fixed
    ladder, clipped to the kernels' limit of 64 nodes."""
    c = {max(1, min(64, -(-total_nodes // (sms * w)))) for w in (1, 2, 3, 4, 6)}
    c |= {z for z in (4, 8, 12, 16, 24, 32, 48, 64) if z <= max(1, total_nodes)}
    return sorted(c)


def _key(params, device_name):
    sig = [(p.nx, p.Q, p.dx, p.bc, p.precision, p.r_cut, p.sigma) for p in params]
    h = hashlib.sha1(json.dumps(sig).encode()).hexdigest()[:16]
    return f"{device_name}|{h}"


def _load_cache(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def autotune(params, n0, u0, T0, steps: int = 8, warmup: int = 2, cache: str | None = CACHE,
             cands=None, stream=None, repeats: int = 2):
    """Returns (best tile_nodes, {tile: ms per step}) for the slabs `params`
    (one Params or a list), timing `steps` steps per candidate from the
    projected state of (n0, u0, T0) on a scratch context; each candidate's
    figure is the best of `repeats` timed runs."""
    import torch
    plist = list(params) if isinstance(params, (list, tuple)) else [params]
    dev = torch.cuda.current_device()
    name = torch.cuda.get_device_name(dev)
    key = _key(plist, name)
    store = _load_cache(cache) if cache else {}
    if key in store and cands is None:
        ent = store[key]
        return int(ent["best"]), {int(k): v for k, v in ent["ms"].items()}
    sims = Sim(plist, stream=stream)
    st = sims.stream
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    cands = candidates(sims.NN, sms) if cands is None else cands
    times = {}
    try:
        for z in cands:
            sims.tune(z)
            sims.init(n0, u0, T0)
            sims.step(warmup)
            best_ms = float("inf")
            for _ in range(max(1, repeats)):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(st)
                sims.step_async(steps)
                e1.record(st)
                sims.step(0)
                best_ms = min(best_ms, e0.elapsed_time(e1) / steps)
            times[z] = best_ms
    finally:
        sims.close()
    best = min(times, key=times.get)
    if cache:
        store[key] = {"best": best, "ms": {str(k): v for k, v in times.items()}}
        os.makedirs(os.path.dirname(cache), exist_ok=True)
        tmp = cache + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(store, f, indent=1)
        os.replace(tmp, cache)
    return best, times


def tune_sim(sim: Sim, n0, u0, T0, **kw):
    """Autotunes `sim`'s slabs and applies the best tile to it (its state is
    untouched: the timing runs on a scratch context)."""
    best, times = autotune(sim.params, n0, u0, T0, stream=sim.stream, **kw)
    sim.tune(best)
    return best, times


def uniform_fields(params, n=0.25, T=0.6):
    """Seed fields for tuning: uniform n, u = 0, T for every node of `params`."""
    plist = list(params) if isinstance(params, (list, tuple)) else [params]
    NN = sum(p.nx for p in plist)
    return np.full(NN, n), np.zeros(NN), np.full(NN, T)
