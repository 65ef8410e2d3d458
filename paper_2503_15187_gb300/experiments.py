"""The paper's three numerical experiments (Sec. III) on the GPU path.

* Planar interfaces at constant temperature (Sec. III.A): periodic domain
  [-100 sigma, 100 sigma], liquid for |x| < 50 sigma, Eq. (tanh) profile at
  the Maxwell-construction densities, isothermal mode at T.  The paper runs
  1e6 iterations to the quasi-stationary profile.
* Phase separation from a sinusoid (Sec. III.B): periodic [-L/2, L/2],
  L = 100 sigma, Eq. (rho_init_takata) with A = (n_l + n_v)/2, uniform
  initial temperature T_i, thermal.
* Evaporation of a liquid slab into metastable vapour (Sec. III.C):
  periodic [-200 sigma, 200 sigma], interfaces at +-25 sigma, Eq. (tan)
  profile (vapour at n_v / 2), uniform T_i, thermal, profiles at t = 25, 50,
  75.
All at the paper's discretisation: dx = sigma/10, dt = 5e-3, Q = 16.  The
coexistence densities and T_c are those of the chosen force model's own
attraction constant (evfdlb_coexistence / evfdlb_critical_T); the
temperatures are the paper's absolute values.

Run from the command line, e.g.
    python -m paper_2503_15187_gb300.experiments interface --T 0.7 --force ev2 --steps 1000000 --out e1.json
"""
from __future__ import annotations

import argparse
import json
import math

import numpy as np

from . import BC_PERIODIC, EV1, EV2, FP64, Params, Sim, coexistence, critical_T
from . import workloads as W

DX, DT, QX = 0.1, 5e-3, 16


def _params(nz, force_model, precision, T_iso=0.0):
    return Params(nx=nz, dx=DX, Q=QX, bc=BC_PERIODIC, force_model=force_model, precision=precision, dt=DT,
                  T_iso=T_iso)


def _run(sim, nz, n0, T0, snapshot_steps):
    sim.init(n0, np.zeros(nz), np.full(nz, T0))
    out = {"step": [], "t": [], "n": [], "u": [], "T": [], "totals": []}
    done = 0
    for s in sorted(snapshot_steps):
        sim.step(s - done)
        done = s
        n, u, T, q, tot = sim.moments()
        out["step"].append(s)
        out["t"].append(s * DT)
        out["n"].append(n)
        out["u"].append(u)
        out["T"].append(T)
        out["totals"].append(tot[0])
    return out


def run_interface(T: float, force_model: int = EV1, steps=(20000,), precision: int = FP64,
                  half_length: float = 100.0, x0: float = 50.0) -> dict:
    """Sec. III.A: two planar interfaces held at temperature T; profiles after
    each entry of `steps`."""
    nz = int(round(2 * half_length / DX))
    p = _params(nz, force_model, precision, T_iso=T)
    Tc = critical_T(p)
    nv, nl = coexistence(p, T)
    n0 = W.interface_pair(nz, DX, nl, nv, x0, W.tanh_width(Tc, T))
    sim = Sim(p)
    try:
        out = _run(sim, nz, n0, T, steps)
    finally:
        sim.close()
    out.update(x=W.centred_nodes(nz, DX), n_l=nl, n_v=nv, T_c=Tc, n0=n0)
    return out


def run_phase_separation(T_i: float, omega: float, force_model: int = EV1, steps=(20000,),
                         precision: int = FP64, length: float = 100.0) -> dict:
    """Sec. III.B: a sinusoidal density of amplitude omega about
    A = (n_l + n_v)/2 at uniform T_i, thermal."""
    nz = int(round(length / DX))
    p = _params(nz, force_model, precision)
    nv, nl = coexistence(p, T_i)
    n0 = W.sinusoid(nz, DX, 0.5 * (nl + nv), omega)
    sim = Sim(p)
    try:
        out = _run(sim, nz, n0, T_i, steps)
    finally:
        sim.close()
    out.update(x=W.centred_nodes(nz, DX), n_l=nl, n_v=nv, T_c=critical_T(p), n0=n0)
    return out


def run_evaporation(T_i: float, force_model: int = EV1, times=(25.0, 50.0, 75.0), precision: int = FP64,
                    half_length: float = 200.0, x0: float = 25.0) -> dict:
    """Sec. III.C: liquid slab |x| < x0 in vapour at half the coexistence
    density, uniform T_i, thermal; profiles at the given times."""
    nz = int(round(2 * half_length / DX))
    p = _params(nz, force_model, precision)
    Tc = critical_T(p)
    nv, nl = coexistence(p, T_i)
    n0 = W.slab_in_metastable_vapour(nz, DX, nl, nv, x0, W.tanh_width(Tc, T_i))
    sim = Sim(p)
    try:
        out = _run(sim, nz, n0, T_i, [int(round(t / DT)) for t in times])
    finally:
        sim.close()
    out.update(x=W.centred_nodes(nz, DX), n_l=nl, n_v=nv, T_c=Tc, n0=n0)
    return out


def _jsonable(d):
    o = {}
    for k, v in d.items():
        if isinstance(v, np.ndarray):
            o[k] = v.tolist()
        elif isinstance(v, list):
            o[k] = [x.tolist() if isinstance(x, np.ndarray) else x for x in v]
        else:
            o[k] = v
    return o


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("experiment", choices=["interface", "phase_separation", "evaporation"])
    ap.add_argument("--T", type=float, required=True, help="T (interface) or initial T_i")
    ap.add_argument("--omega", type=float, default=0.4, help="sinusoid amplitude (phase_separation)")
    ap.add_argument("--force", choices=["ev1", "ev2"], default="ev1")
    ap.add_argument("--steps", type=int, nargs="+", default=[20000], help="snapshot steps (not evaporation)")
    ap.add_argument("--times", type=float, nargs="+", default=[25.0, 50.0, 75.0], help="evaporation snapshots")
    ap.add_argument("--out", default="")
    a = ap.parse_args(argv)
    fm = EV1 if a.force == "ev1" else EV2
    if a.experiment == "interface":
        r = run_interface(a.T, fm, a.steps)
    elif a.experiment == "phase_separation":
        r = run_phase_separation(a.T, a.omega, fm, a.steps)
    else:
        r = run_evaporation(a.T, fm, a.times)
    r = _jsonable(r)
    r.update(experiment=a.experiment, force=a.force, T=a.T)
    if a.out:
        with open(a.out, "w") as f:
            json.dump(r, f)
    last = np.asarray(r["n"][-1])
    print(json.dumps({"experiment": a.experiment, "force": a.force, "T": a.T, "t": r["t"][-1],
                      "n_min": float(last.min()), "n_max": float(last.max()), "n_l": r["n_l"], "n_v": r["n_v"],
                      "mass_drift": float(abs(r["totals"][-1][0] - r["totals"][0][0]) / r["totals"][0][0])
                      if len(r["totals"]) > 1 else 0.0}))


if __name__ == "__main__":
    main()
