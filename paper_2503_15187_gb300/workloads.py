"""Seeded synthetic inputs for the EV-FDLB slabs.

This module holds only input recipes (random numbers and initial profiles);
it contains none of the model's arithmetic.  Temperatures and coexistence
densities are passed in by the caller, who computes them with its own
equation-of-state code.  Both the CUDA path and the oracle-based tests draw
their inputs from here, so both see identical bits.

Recipes (paper: Busuioc & Sofonea, arXiv:2503.15187):
* noisy uniform slab: n = nbar (1 + a U(-1, 1)), numpy PCG64 with the given
  seed; a seeded analogue of the phase-separation runs of Sec. III.B;
* liquid slab: n = n_v + (n_l - n_v)/2 [1 - tanh((|z - z_c| - h/2)/w)], the
  tanh interface shape of Eq. (tanh) (Sec. III.A) around a centred slab of
  thickness h; a variant of the evaporation runs of Sec. III.C;
* batch of slabs: per-slab sizes, orders, temperature ratios and mean
  densities drawn from one seed, noise from SeedSequence.spawn.

Initial profiles of the paper's three numerical experiments (Sec. III), on
the periodic domain [-L/2, L/2) with nodes at cell centres
x_i = (i + 1/2) dx - L/2:
* planar interface pair (Eq. (tanh), Sec. III.A): liquid for |x| < x0;
* sinusoid (Eq. (rho_init_takata), Sec. III.B): A [1 + omega cos(2 pi x/L)];
* slab in metastable vapour (Eq. (tan), Sec. III.C): liquid for |x| < x0,
  vapour at half the coexistence vapour density;
with the interface width xi = sqrt(3 / (4 pi sqrt(3) (T_c - T))) of both
tanh recipes.
"""
from __future__ import annotations

import numpy as np

SEED = 15187


def noisy_uniform(nz: int, nbar: float, amp: float = 0.01, seed: int = SEED) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    return nbar * (1.0 + amp * rng.uniform(-1.0, 1.0, nz))


def liquid_slab(nz: int, dz: float, n_l: float, n_v: float, thickness: float, width: float) -> np.ndarray:
    z = dz * (np.arange(nz) + 0.5) - 0.5 * nz * dz
    return n_v + 0.5 * (n_l - n_v) * (1.0 - np.tanh((np.abs(z) - 0.5 * thickness) / width))


def batch_slabs(nslab: int = 256, seed: int = SEED, nz_min: int = 128, nz_max: int = 8192,
                tr_range=(0.6, 0.95), orders=(16, 24, 32), nbar_range=(0.15, 0.35), amp: float = 0.01):
    """List of dicts {nz, Q, T_ratio, nbar, n0} for independent periodic slabs:
    nz log-uniform in [nz_min, nz_max], Q uniform over `orders`, T/T_c and the
    mean density uniform in their ranges, n0 with seeded +-amp noise."""
    ss = np.random.SeedSequence(seed)
    rng = np.random.Generator(np.random.PCG64(ss))
    children = ss.spawn(nslab)
    out = []
    for s in range(nslab):
        nz = int(round(np.exp(rng.uniform(np.log(nz_min), np.log(nz_max)))))
        Q = int(orders[rng.integers(len(orders))])
        tr = float(rng.uniform(*tr_range))
        nbar = float(rng.uniform(*nbar_range))
        r = np.random.Generator(np.random.PCG64(children[s]))
        n0 = nbar * (1.0 + amp * r.uniform(-1.0, 1.0, nz))
        out.append(dict(nz=nz, Q=Q, T_ratio=tr, nbar=nbar, n0=n0))
    return out


def centred_nodes(nz: int, dz: float) -> np.ndarray:
    return dz * (np.arange(nz) + 0.5) - 0.5 * nz * dz


def tanh_width(T_c: float, T: float) -> float:
    """Interface width of Eqs. (tanh) and (tan)."""
    return float(np.sqrt(3.0 / (4.0 * np.pi * np.sqrt(3.0) * (T_c - T))))


def interface_pair(nz: int, dz: float, n_l: float, n_v: float, x0: float, xi: float) -> np.ndarray:
    """Eq. (tanh): n_l + (n_v - n_l)/2 [1 + tanh((|x| - x0)/xi)]."""
    x = centred_nodes(nz, dz)
    return n_l + 0.5 * (n_v - n_l) * (1.0 + np.tanh((np.abs(x) - x0) / xi))


def sinusoid(nz: int, dz: float, A: float, omega: float) -> np.ndarray:
    """Eq. (rho_init_takata) with wavelength L = nz dz: A [1 + omega cos(2 pi x / L)]."""
    x = centred_nodes(nz, dz)
    return A * (1.0 + omega * np.cos(2.0 * np.pi * x / (nz * dz)))


def slab_in_metastable_vapour(nz: int, dz: float, n_l: float, n_v: float, x0: float, xi: float) -> np.ndarray:
    """Eq. (tan): n_l + (n_v - 2 n_l)/4 [1 + tanh((|x| - x0)/xi)], vapour n_v/2."""
    x = centred_nodes(nz, dz)
    return n_l + 0.25 * (n_v - 2.0 * n_l) * (1.0 + np.tanh((np.abs(x) - x0) / xi))
