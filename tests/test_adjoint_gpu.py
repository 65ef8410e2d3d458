"""GPU parity of the discrete adjoint against the oracle's tangent-linear maps.

The adjoint of the time step (evfdlb_rhs_vjp, evfdlb_adjoint_state,
evfdlb_adjoint) is checked against the complex-step tangent of the FP64
oracle (pinned in test_oracle_tangent.py):
  * the full transposed Jacobian of one right-hand side on a tiny slab, built
    column by column from the oracle tangent, element by element;
  * dot-product identities <w, J v> = <J^T w, v> on larger slabs with ragged
    node tiles, both relaxation readings, Q = 8..32;
  * the gradient of a loss of the final density after many steps with
    checkpoints (ragged last segment) against oracle directional derivatives
    along seeded directions in n0, a uniform change of T0, phi_a and F0.
Bars: elementwise 1e-12 of the largest entry for the explicit transpose;
dot products to 1e-11 of the Cauchy-Schwarz scale |w| |J v| (FP64 rounding
of O(Q^2) sums); whole-trajectory directional derivatives to 1e-9 relative.
"""
import numpy as np
import pytest

import oracle as O
import paper_2503_15187_gb300 as ev
from paper_2503_15187_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def nonequilibrium(orc, seed=4, steps=2):
    rng = np.random.default_rng(seed)
    nz = orc.s.nz
    z = np.arange(nz)
    n0 = 0.25 * (1 + 0.3 * np.sin(2 * np.pi * z / nz) + 0.02 * rng.uniform(-1, 1, nz))
    u0 = 0.04 * np.cos(2 * np.pi * z / nz)
    T0 = 0.6 * (1 + 0.05 * np.sin(4 * np.pi * z / nz))
    F, G = orc.equilibrium(n0, u0, T0)
    return orc.step(F, G, steps)


def make(nz, Q, dz, relax=0, tile=None, ckpt=0):
    sim = ev.Sim(ev.Params(nx=nz, dx=dz, Q=Q, relax_mode=relax, ckpt_every=ckpt))
    if tile:
        sim.tune(tile)
    orc = O.Oracle(O.Setup(nz=nz, Q=Q, dz=dz, dt=sim.dt(), relax=relax))
    return sim, orc


def test_rhs_transpose_jacobian_elementwise():
    nz, Q = 16, 8
    sim, orc = make(nz, Q, 0.25, tile=5)
    F, G = nonequilibrium(orc)
    sim.set_state(F.ravel(), G.ravel())
    N = Q * nz
    J = np.empty((2 * N, 2 * N))           # J[:, c] = d R / d x_c
    for c in range(2 * N):
        e = np.zeros(2 * N)
        e[c] = 1.0
        _, _, dF, dG = orc.rhs_tl(F, G, e[:N].reshape(Q, nz), e[N:].reshape(Q, nz))
        J[:, c] = np.concatenate([dF.ravel(), dG.ravel()])
    rng = np.random.default_rng(7)
    for trial in range(2):
        w = rng.uniform(-1, 1, 2 * N)
        oF, oG, dphi = sim.rhs_vjp(w[:N], w[N:])
        ref = J.T @ w
        got = np.concatenate([oF, oG])
        err = np.abs(got - ref).max() / np.abs(ref).max()
        print(f"J^T w elementwise: {err:.2e}")
        assert err < 1e-12
        _, _, pF, pG = orc.rhs_tl(F, G, np.zeros((Q, nz)), np.zeros((Q, nz)), dphi=1.0)
        ref_phi = w @ np.concatenate([pF.ravel(), pG.ravel()])
        assert abs(dphi[0] - ref_phi) < 1e-12 * np.abs(w).sum() * np.abs(np.concatenate([pF.ravel(), pG.ravel()])).max()


# (nz, Q, dz, relax, tile): ragged last tiles (64 = 9 x 7 + 1), tiles of
# one to three nodes (every WENO-5 stencil leaves its tile on both sides),
# the sweep's tile cap (tile 64 -> 32), one tile for the whole periodic slab
# (stencils wrap onto the same tile), odd Q (a zero velocity, whose row has
# no faces, and the middle node of the parity split)
@pytest.mark.parametrize("case", [(64, 16, 0.25, 0, 7), (97, 24, 0.25, 0, 13), (50, 8, 0.25, 1, 64),
                                  (150, 32, 0.1, 0, 27), (40, 9, 0.25, 0, 2), (33, 15, 0.25, 1, 3),
                                  (36, 11, 0.25, 0, 1), (20, 12, 0.25, 0, 64), (29, 7, 0.25, 0, 29)])
def test_rhs_dot_product_identity(case):
    nz, Q, dz, relax, tile = case
    sim, orc = make(nz, Q, dz, relax=relax, tile=tile)
    F, G = nonequilibrium(orc)
    sim.set_state(F.ravel(), G.ravel())
    rng = np.random.default_rng(nz)
    for trial in range(3):
        vF, vG = F * rng.uniform(-1, 1, F.shape), G * rng.uniform(-1, 1, G.shape)
        wF, wG = rng.uniform(-1, 1, F.shape), rng.uniform(-1, 1, G.shape)
        dphi_dir = rng.uniform(-1, 1)
        _, _, jF, jG = orc.rhs_tl(F, G, vF, vG, dphi=dphi_dir)
        lhs = (wF * jF).sum() + (wG * jG).sum()
        oF, oG, dphi = sim.rhs_vjp(wF.ravel(), wG.ravel())
        rhs = (oF.reshape(Q, nz) * vF).sum() + (oG.reshape(Q, nz) * vG).sum() + dphi[0] * dphi_dir
        scale = np.sqrt((wF ** 2).sum() + (wG ** 2).sum()) * np.sqrt((jF ** 2).sum() + (jG ** 2).sum())
        print(f"{case}: <w,Jv> {lhs:.6e} <J^T w,v> {rhs:.6e} rel {abs(lhs - rhs) / scale:.2e}")
        assert abs(lhs - rhs) < 1e-11 * scale


@pytest.mark.parametrize("case", [(32, 12, 0.25, 20, 6, 5), (40, 16, 0.25, 9, 9, 64), (26, 9, 0.25, 8, 3, 2)])
def test_trajectory_gradient_against_oracle_tangent(case):
    """Loss L = sum_z (n_end - n_target)^2 after `steps` steps from the
    projected (n0, u0 = 0, T0), checkpoints every `ckpt` steps."""
    nz, Q, dz, steps, ckpt, tile = case
    sim, orc = make(nz, Q, dz, tile=tile, ckpt=ckpt)
    rng = np.random.default_rng(2025)
    z = np.arange(nz)
    n0 = 0.25 * (1 + 0.05 * rng.uniform(-1, 1, nz))
    u0 = np.zeros(nz)
    T0 = np.full(nz, 0.55)
    target = 0.25 * (1 + 0.02 * np.cos(2 * np.pi * z / nz + 0.3))
    sim.init(n0, u0, T0)
    sim.step(steps)
    n_end = sim.moments(with_totals=False)[0]
    dL_dn = 2.0 * (n_end - target)
    g = sim.adjoint_state(np.repeat(dL_dn[None, :], Q, axis=0).ravel(), np.zeros(Q * nz))
    dphi, dT, dn = sim.adjoint(dL_dn)
    assert np.allclose(dphi, g["dphi"], rtol=1e-14, atol=0) and np.allclose(dn, g["dn0"], rtol=1e-14, atol=0)

    def dL(dn0=None, dT0=None, dphi_dir=0.0):
        dn0 = np.zeros(nz) if dn0 is None else dn0
        dT0 = np.zeros(nz) if dT0 is None else dT0
        F, G, tF, tG = orc.trajectory_tl(n0, u0, T0, dn0, np.zeros(nz), dT0, steps, dphi=dphi_dir)
        n = F.sum(axis=0)
        return (2.0 * (n - target) * tF.sum(axis=0)).sum()

    d = rng.uniform(-1, 1, nz)
    checks = [("n0 direction", dL(dn0=d), (g["dn0"] * d).sum()),
              ("uniform T0", dL(dT0=np.ones(nz)), g["dT0"].sum()),
              ("phi_a", dL(dphi_dir=1.0), g["dphi"][0])]
    for name, ref, got in checks:
        print(f"{case} {name}: oracle {ref:.10e} gpu {got:.10e}")
        assert abs(got - ref) < 1e-9 * abs(ref), name
    # the cotangent of the initial distributions
    F0, G0 = orc.equilibrium(n0, u0, T0)
    vF, vG = F0 * rng.uniform(-1, 1, F0.shape), G0 * rng.uniform(-1, 1, G0.shape)
    F, G, tF, tG = orc.step_tl(F0, G0, vF, vG, steps)
    ref = (2.0 * (F.sum(axis=0) - target) * tF.sum(axis=0)).sum()
    got = (g["dF0"].reshape(Q, nz) * vF).sum() + (g["dG0"].reshape(Q, nz) * vG).sum()
    print(f"{case} F0 direction: oracle {ref:.10e} gpu {got:.10e}")
    assert abs(got - ref) < 1e-9 * abs(ref)


def test_rhs_vjp_of_a_batch_equals_its_slabs_alone():
    """Slabs of different length and Q in one context give, slab by slab,
    the same transposed right-hand side (bit for bit) as each slab in a
    context of its own with the same node tile."""
    cases = [(40, 9, 0.25), (33, 16, 0.25), (27, 12, 0.25)]
    tile = 5
    rng = np.random.default_rng(11)
    singles, states, ws = [], [], []
    for nz, Q, dz in cases:
        sim, orc = make(nz, Q, dz, tile=tile)
        F, G = nonequilibrium(orc, seed=nz)
        w = rng.uniform(-1, 1, 2 * Q * nz)
        sim.set_state(F.ravel(), G.ravel())
        singles.append(sim.rhs_vjp(w[:Q * nz], w[Q * nz:]))
        states.append((F.ravel(), G.ravel()))
        ws.append(w)
    batch = ev.Sim([ev.Params(nx=nz, dx=dz, Q=Q) for nz, Q, dz in cases])
    batch.tune(tile)
    batch.set_state(np.concatenate([f for f, _ in states]), np.concatenate([g for _, g in states]))
    oF, oG, dphi = batch.rhs_vjp(np.concatenate([w[:len(w) // 2] for w in ws]),
                                 np.concatenate([w[len(w) // 2:] for w in ws]))
    off = 0
    for i, (nz, Q, dz) in enumerate(cases):
        sF, sG, sphi = singles[i]
        assert np.array_equal(oF[off:off + Q * nz], sF), i
        assert np.array_equal(oG[off:off + Q * nz], sG), i
        assert dphi[i] == sphi[0], i
        off += Q * nz


def test_adjoint_requires_tracking_and_periodic():
    sim = ev.Sim(ev.Params(nx=32, dx=0.25, Q=8))                 # ckpt_every = 0
    sim.init(np.full(32, 0.25), np.zeros(32), np.full(32, 0.6))
    sim.step(2)
    with pytest.raises(ev.EvfdlbError) as e:
        sim.adjoint(np.ones(32))
    assert e.value.code == -7
    sim = ev.Sim(ev.Params(nx=32, dx=0.25, Q=8, bc=ev.BC_OUTFLOW, ckpt_every=4))
    sim.init(np.full(32, 0.25), np.zeros(32), np.full(32, 0.6))
    sim.step(2)
    with pytest.raises(ev.EvfdlbError) as e:
        sim.adjoint(np.ones(32))
    assert e.value.code == -8


def test_autograd_function_small_against_oracle():
    """EVRun (torch.autograd.Function) on a small periodic slab: phi_a.grad,
    T0.grad and n0.grad of L = sum (n_end - target)^2 against the oracle's
    complex-step directional derivatives."""
    import torch
    from paper_2503_15187_gb300.autograd import EVRun
    nz, Q, dz, steps = 32, 12, 0.25, 15
    p = ev.Params(nx=nz, dx=dz, Q=Q, ckpt_every=4)
    rng = np.random.default_rng(99)
    n0h = 0.25 * (1 + 0.05 * rng.uniform(-1, 1, nz))
    target = torch.full((nz,), 0.25, dtype=torch.float64, device="cuda")
    phi = torch.tensor(1.0, dtype=torch.float64, requires_grad=True)
    T0 = torch.tensor(0.55, dtype=torch.float64, requires_grad=True)
    n0 = torch.tensor(n0h, dtype=torch.float64, device="cuda", requires_grad=True)
    n_end = EVRun.apply(phi, T0, n0, p, steps)
    loss = ((n_end - target) ** 2).sum()
    loss.backward()
    xi, _ = O.gauss_hermite(Q)
    orc = O.Oracle(O.Setup(nz=nz, Q=Q, dz=dz, dt=0.5 * dz / np.abs(xi).max()))
    tgt = target.cpu().numpy()

    def dL(dn0, dT0, dphi):
        F, G, tF, tG = orc.trajectory_tl(n0h, np.zeros(nz), np.full(nz, 0.55), dn0, np.zeros(nz), dT0, steps,
                                         dphi=dphi)
        return (2.0 * (F.sum(axis=0) - tgt) * tF.sum(axis=0)).sum()

    d = rng.uniform(-1, 1, nz)
    for name, ref, got in [("phi_a", dL(np.zeros(nz), np.zeros(nz), 1.0), float(phi.grad)),
                           ("T0", dL(np.zeros(nz), np.ones(nz), 0.0), float(T0.grad)),
                           ("n0", dL(d, np.zeros(nz), 0.0), float((n0.grad.cpu().numpy() * d).sum()))]:
        print(f"autograd {name}: oracle {ref:.10e} gpu {got:.10e}")
        assert abs(got - ref) < 1e-9 * abs(ref), name


def test_adjoint_calibration_full_size_against_central_differences():
    """Adjoint calibration workload: periodic slab Nz = 1024, dz = 0.25, Q = 24,
    2000 steps at CFL 0.5, T = 0.7 T_c, mean n = 0.25 with +-1% seeded noise,
    checkpoint every 100 steps; loss = sum_z (n(z, t_end) - n_target(z))^2
    with n_target from a seeded forward run at perturbed phi_a and T.
    Gradients through the autograd function against central differences
    (h = 1e-6) of forward runs, for phi_a, T and four seeded directions in n0:
    agreement to 1e-6 relative."""
    import torch
    from paper_2503_15187_gb300.autograd import EVRun
    nz, Q, dz, steps = 1024, 24, 0.25, 2000
    p = ev.Params(nx=nz, dx=dz, Q=Q, ckpt_every=100)
    T = 0.7 * ev.critical_T(p)
    n0h = W.noisy_uniform(nz, 0.25, 0.01)
    rng = np.random.default_rng(15187)
    phi_t, T_t = 1.0 + 0.05 * rng.uniform(-1, 1), T * (1 + 0.02 * rng.uniform(-1, 1))

    def forward(phi, Tv, n0):
        sim = ev.Sim(ev.Params(nx=nz, dx=dz, Q=Q, phi_a=phi))
        sim.init(n0, np.zeros(nz), np.full(nz, Tv))
        sim.step(steps)
        n = sim.moments(with_totals=False)[0]
        sim.close()
        return n

    target = forward(phi_t, T_t, n0h)
    loss_of = lambda n: float(((n - target) ** 2).sum())
    phi = torch.tensor(1.0, dtype=torch.float64, requires_grad=True)
    Tt = torch.tensor(T, dtype=torch.float64, requires_grad=True)
    n0 = torch.tensor(n0h, dtype=torch.float64, device="cuda", requires_grad=True)
    n_end = EVRun.apply(phi, Tt, n0, p, steps)
    loss = ((n_end - torch.from_numpy(target).cuda()) ** 2).sum()
    loss.backward()
    h = 1e-6
    checks = [("phi_a", (loss_of(forward(1 + h, T, n0h)) - loss_of(forward(1 - h, T, n0h))) / (2 * h),
               float(phi.grad)),
              ("T", (loss_of(forward(1.0, T + h, n0h)) - loss_of(forward(1.0, T - h, n0h))) / (2 * h),
               float(Tt.grad))]
    g = n0.grad.cpu().numpy()
    for j in range(4):
        d = np.random.default_rng(100 + j).uniform(-1, 1, nz)
        fd = (loss_of(forward(1.0, T, n0h + h * d)) - loss_of(forward(1.0, T, n0h - h * d))) / (2 * h)
        checks.append((f"n0 direction {j}", fd, float((g * d).sum())))
    for name, fd, got in checks:
        print(f"calibration {name}: central difference {fd:.9e} adjoint {got:.9e} rel {abs(got - fd) / abs(fd):.2e}")
        assert abs(got - fd) < 1e-6 * abs(fd), name


def test_autograd_function_on_a_side_stream_matches_default_stream():
    """EVRun passes device pointers on torch's current stream: run inside a
    side stream, it gives bit-identical values and gradients to a run on the
    default stream (same kernels, same order)."""
    import torch
    from paper_2503_15187_gb300.autograd import EVRun
    nz, Q, dz, steps = 48, 8, 0.25, 9
    p = ev.Params(nx=nz, dx=dz, Q=Q, ckpt_every=4)
    n0h = 0.25 * (1 + 0.05 * np.random.default_rng(5).uniform(-1, 1, nz))

    def run():
        phi = torch.tensor(1.0, dtype=torch.float64, requires_grad=True)
        T0 = torch.tensor(0.6, dtype=torch.float64, requires_grad=True)
        n0 = torch.tensor(n0h, dtype=torch.float64, device="cuda", requires_grad=True)
        n_end = EVRun.apply(phi, T0, n0, p, steps)
        (n_end ** 2).sum().backward()
        torch.cuda.current_stream().synchronize()
        return n_end.detach().cpu().numpy(), float(phi.grad), float(T0.grad), n0.grad.cpu().numpy()

    ref = run()
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        got = run()
    for a, b in zip(ref, got):
        assert np.array_equal(np.asarray(a), np.asarray(b))
