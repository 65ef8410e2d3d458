"""The oracle's OpenMP build shares its independent node loops among
threads; every node's arithmetic is the same in any thread, so the results
must be bit-identical for any thread count (1D and 2D, a full RK3 step)."""
import numpy as np
import pytest

import oracle as O


@pytest.fixture
def restore_threads():
    before = O.set_threads()
    yield
    O.set_threads(before)


def test_1d_step_bit_identical_across_thread_counts(restore_threads):
    nz, Q, dz = 211, 16, 0.25
    xi, _ = O.gauss_hermite(Q)
    o = O.Oracle(O.Setup(nz=nz, Q=Q, dz=dz, dt=0.5 * dz / np.abs(xi).max(), bc=1))
    rng = np.random.default_rng(7)
    F, G = o.equilibrium(0.3 * (1 + 0.1 * rng.uniform(-1, 1, nz)), 0.02 * rng.uniform(-1, 1, nz), np.full(nz, 0.6))
    out = []
    for th in (1, 3, max(2, O.available_cores())):
        O.set_threads(th)
        out.append(o.step(F.copy(), G.copy(), 1))
    for F2, G2 in out[1:]:
        assert np.array_equal(F2, out[0][0]) and np.array_equal(G2, out[0][1])


def test_2d_step_bit_identical_across_thread_counts(restore_threads):
    nx, ny, Q, dx = 13, 11, 6, 0.5
    xi, _ = O.gauss_hermite(Q)
    o = O.Oracle2D(O.Setup2(nx=nx, ny=ny, Q=Q, dx=dx, dt=0.5 * dx / (2 * np.abs(xi).max())))
    rng = np.random.default_rng(8)
    n = 0.25 * (1 + 0.05 * rng.uniform(-1, 1, (ny, nx)))
    F, G = o.equilibrium(n, np.zeros((ny, nx)), np.zeros((ny, nx)), np.full((ny, nx), 0.6))
    out = []
    for th in (1, 4):
        O.set_threads(th)
        out.append(o.step(F.copy(), G.copy(), 1))
    assert np.array_equal(out[1][0], out[0][0]) and np.array_equal(out[1][1], out[0][1])
