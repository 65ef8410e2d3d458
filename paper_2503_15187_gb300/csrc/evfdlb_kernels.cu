// evfdlb_kernels.cu -- sm_103a kernels of libevfdlb (forward path, FP64 and
// FP32 variants).
//
// One launch of `stage_kernel` evaluates the right-hand side of the EV1
// equations (Busuioc & Sofonea, arXiv:2503.15187, Eqs. (ev1) and
// (enskog_approx)) on a tile of nodes of one slab and applies one stage of the
// Shu-Osher third-order TVD Runge-Kutta scheme (Sec. III):
//   out = alpha * base + beta * (src + dt * L(src)).
// Each CTA owns all Q velocities of both reduced distributions F, G on its
// node tile, so it can
//   (1) rebuild the node fields of its tile from the raw moment sums that the
//       previous stage wrote (n over a +-M halo for the Eq. (F1) force and the
//       Fischer-Methfessel average, u and T over +-2 nodes for the
//       fourth-order gradients of Eq. (J1));
//   (2) express the force, the Shakhov relaxation and J1 as ONE vector of
//       Hermite coefficients per node and distribution (orthonormal basis
//       psi_l = He_l / sqrt(l!)):
//         c_l = nu a^S_l + a^J_l + F1 sqrt(l) a_{l-1},
//       where a_l = sum_j F_j psi_l(xi_j) is the analysis of the state and
//       a^S, a^J are the projections of the reduced Shakhov equilibrium and of
//       J1, obtained from the Hermite moments of N(u, T) by recurrence;
//   (3) synthesise R_k = -xi_k dF/dz - nu F_k + w_k sum_l c_l psi_l(xi_k),
//       with dF/dz from WENO-5 (Jiang-Shu) faces computed once per face;
//   (4) write the new stage and its raw moment sums for the next stage.
// FP64 is the GB300's scarcest pipe (about 1/60 of FP32), so the design
// minimises FP64 instructions: one division per WENO face, per-node work
// shared by all velocities, no re-reads of the state.
//
// Precision variants.  The kernels are templated on R, the type of the stored
// distributions and of the per-velocity work (WENO faces, Hermite analysis and
// synthesis, the force convolution, the coefficient recurrences and the RK
// combine).  R = double is the plain FP64 form.  R = float is the FP32
// variant; it keeps FP64 for the Fischer-Methfessel average, chi and the
// transport coefficients (the equation-of-state part, which is sensitive near
// liquid packing), the gradients, and the per-node sums of the conserved
// moments (mass, momentum, energy); the heat-flux sums are FP32.
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <type_traits>
#include <utility>

#include "evfdlb_device.cuh"

namespace evfdlb {

// ---------------------------------------------------------------------------
// Kernels
// ---------------------------------------------------------------------------

// mode 0: out = alpha base + beta (src + dt R);  mode 1: rhs_out = R (FP64).
// DF (R = double only): the FP64_DF variant -- rtab holds the analysis and
// synthesis tables as double-float pairs, every other table value comes from
// the FP64 `tables`; the Hermite analysis and synthesis run as Dot2 sums of
// pairs on the FP32 pipe (state tile split into pairs once per stage in a
// block after the Hermite moments), everything else as in the FP64 kernel.
//
// The body runs one work item (slab tile) with the CTA's threads; CG: the
// stage input, base and moment sums are read with L2-coherent loads (the
// persistent form, where other CTAs of the same launch wrote them); FO: the
// node fields of the stage input are also written to fields_out (a
// compile-time choice, so that the other forms carry none of its registers).
template <typename R, bool DF, bool CG, bool FO = false>
__device__ __forceinline__ void stage_body(const SlabDesc& sd, const WorkItem& it, double* smem,
                                           const double* __restrict__ tables, const R* __restrict__ rtab,
                                           const double* __restrict__ taps, const R* __restrict__ rtaps,
                                           const R* src, const R* base, R* out, double* rhs_out,
                                           const double* mom_in, double* mom_out, double* fields_out,
                                           long long NF, long long NN, double alpha, double beta, int mode, int Z,
                                           unsigned* err) {
    const int Q = sd.Q, W = Z + 6, nz = it.nz;
    Smem<R> s = carve<R>(smem, Q, Z, sd.M);
    double* const fo = FO ? fields_out : nullptr;

    // FP64 / FP32: parity-split tables and state tile (half the transform
    // products); FP64_DF: the full tables as float pairs and the state tile
    // split into float pairs in the EO block.
    // The inputs that no stage writes come first (velocity tables, force and
    // Fischer-Methfessel taps, velocity powers): in a programmatic launch
    // they are staged while the previous stage still runs, and
    // griddepcontrol.wait then holds back the reads of its state and moment
    // sums until that stage has completed (a no-op in a plain launch).
    float2* Fd = DF ? reinterpret_cast<float2*>(s.EO) : nullptr;
    load_velocity_tables<R, !DF>(sd, s, rtab);
    for (int j = threadIdx.x; j < 2 * sd.M + 1; j += blockDim.x) s.Ftap[j] = rtaps[sd.tap_off + j];
    for (int j = threadIdx.x; j < 2 * sd.m + 1; j += blockDim.x) s.Mtap[j] = taps[sd.tap_off + 2 * sd.M + 1 + j];
    // velocity powers of the closing moment sums, formed once per CTA
    {
        const R* vt = DF ? reinterpret_cast<const R*>(tables) : rtab;
        const int xo = sd.tab_off + TableLayout(Q).xi;
        velocity_powers<R>(Q, tables + xo, vt + xo, s.Vp, s.Vr, threadIdx.x, blockDim.x);
    }
    if constexpr (!CG) asm volatile("griddepcontrol.wait;" ::: "memory");
    // the state tile by asynchronous copies, issued first, so that they are
    // in flight with the node inputs' loads and arithmetic
    if constexpr (!DF) issue_state_tile<R, CG>(sd, it, s, Z, src, NF);
    load_node_inputs<R, !DF, CG, false>(sd, it, s, Z, rtab, mom_in, NN);
    if constexpr (DF) load_state_tile<R>(sd, it, s, Z, src, NF, Fd);
    if constexpr (!DF && !CG) cp_async_wait_all();
    __syncthreads();
    // The node warps form the node-level quantities of the tile (node fields,
    // coefficient constants, Hermite moments of the local Gaussian) while the
    // other warps do the velocity-space work that needs only the state tile
    // (Hermite analysis, WENO-5 faces), so the serial node work overlaps it.
    // the tables of everything but the DF transforms
    const R* vtab = DF ? reinterpret_cast<const R*>(tables) : rtab;
    const R* rt = vtab + sd.tab_off;
    TableLayout L(Q);
    // Node warps: one, or two when pass 1 (nz + 4 nodes) would take a
    // second round on one warp; the passes are separated by a barrier of the
    // node warps only (named barrier 1).
    const int NW = (nz + 4 > 32) ? 2 : 1;
    auto node_sync = [&]() {
        if (NW == 1) __syncwarp();
        else asm volatile("bar.sync 1, 64;" ::: "memory");
    };
    // FP32: the Eq. (F1) force sums need only the staged densities, so the
    // worker warps (whose FP32 work finishes well before the node chain)
    // form them first, a half-warp per node, and signal on named barrier 3
    // without waiting; the node warps take them up before pass 2.  The last
    // worker warp forms the Hermite moments of the local Gaussian meanwhile.
    // FP64 keeps both in the node chain: there the worker warps are the
    // longer side of the phase and the FP64 pipe the bound.
    constexpr bool WF = std::is_same<R, float>::value && !DF;
    if (threadIdx.x < 32 * NW) {
        node_fields_pass1<R>(sd, it, s, s.Mtap, NN, fo, threadIdx.x, 32 * NW);
        node_sync();
        if constexpr (WF) asm volatile("bar.sync 3, %0;" ::"r"((int)blockDim.x) : "memory");
        node_fields_pass2<R, WF>(sd, it, s, Z, s.Ftap, mom_in, NN, err, fo, threadIdx.x, 32 * NW);
        node_sync();
        node_coefficients<R, !WF>(sd, it, s, Z, rt, threadIdx.x, 32 * NW);
    } else {
        const int tid = threadIdx.x - 32 * NW, nth = blockDim.x - 32 * NW;
        if constexpr (WF) {
            // the Hermite moments of the local Gaussian (a serial recurrence
            // per node) need only u and T of the node inputs: the last worker
            // warp, whose share of the force sums (a half-warp per node from
            // the first worker) is empty on tiles of up to nth/16 - 2 nodes,
            // forms them first, beside the other workers' force sums
            if (tid >= nth - 32) node_hermite_moments<R>(sd, it, s, Z, rt, tid - (nth - 32), 32);
            tile_force_sums<R>(sd, it, s, Z, s.Ftap, tid, nth);
            __threadfence_block();
            asm volatile("bar.arrive 3, %0;" ::"r"((int)blockDim.x) : "memory");
        }
        if constexpr (DF) {
            analysis_df(sd, it, s, Fd, reinterpret_cast<const float2*>(s.P), Z, tid, nth);
        } else {
            // the worker warps split the tile into parity parts, then join on
            // named barrier 2 (the node warps go on meanwhile)
            split_state_tile<R>(sd, it, s, Z, tid, nth);
            asm volatile("bar.sync 2, %0;" ::"r"(nth) : "memory");
            analysis_eo<R>(sd, it, s, Z, tid, nth);
        }
        if constexpr (DF) faces_df(sd, it, s, Z, tables, tid, nth);
        else faces<R>(sd, it, s, Z, vtab, tid, nth);
    }
    __syncthreads();
    coefficients<R, DF>(sd, it, s, Z, rt, threadIdx.x, blockDim.x);
    __syncthreads();
    // the next stage (a programmatic launch) may now be scheduled beside
    // this CTA and stage its constant inputs
    if constexpr (!CG) asm volatile("griddepcontrol.launch_dependents;" ::: "memory");

    // Phase 5: synthesis, advection, relaxation and the RK stage.
    const R* xi = rt + L.xi;
    const R dt = (R)sd.dt, inv_dx = (R)sd.inv_dx, ralpha = (R)alpha, rbeta = (R)beta;
    const bool rhs_form = (mode == 1), with_base = (alpha != 0.0);
    // The stage out = alpha base + beta (h + dt R) with
    // R = -xi_k/dx (f_{t+1/2} - f_{t-1/2}) - nu h + syn is formed as
    // fma(cx_k, df, fma(cs, syn, fma(ch, h, alpha base))): cs = beta dt,
    // ch = beta (1 - dt nu) per node, cx_k = -beta dt xi_k / dx.
    const R cs = rbeta * dt, csx = -cs * inv_dx;
    // output of velocity k of node t of distribution d; the two output forms
    // under one uniform branch, so that the RK form issues no FP64
    // conversion of the right-hand-side form
    // bv: the base value at (d, k, t), loaded by the caller ahead of its
    // synthesis loop so that the global load's latency is hidden
    auto gidx_of = [&](int d, int t, int k) { return d * NF + sd.f_off + (long long)k * sd.nx + it.i0 + t; };
    // The FP32 state's moment sums take their pair terms from the values
    // written here (PT); the other forms sum the new tile after the
    // synthesis, so emit stores it back into s.F.
    constexpr bool PT = std::is_same<R, float>::value && !DF;
    auto emit = [&](int d, int t, int k, R syn, R ch, R cx, R bv) -> R {
        R* hp = s.F + (size_t)(d * Q + k) * W + t + 3;
        const R h = *hp;
        const R* fc = s.Face + (size_t)(d * Q + k) * (Z + 1);
        const R df = fc[t + 1] - fc[t];
        const long long g = gidx_of(d, t, k);
        if (rhs_form) {
            rhs_out[g] = (double)fma(-xi[k] * inv_dx, df, fma(-s.Scr[t], h, syn));
            return R(0);
        }
        R o = with_base ? ralpha * bv : R(0);
        o = fma(ch, h, o);
        o = fma(cs, syn, o);
        o = fma(cx, df, o);
        out[g] = o;
        if constexpr (!PT) *hp = o;
        return o;
    };
    if constexpr (DF) {
        // four velocities per thread (four independent Dot2 chains hide the
        // FP32 latency)
        constexpr int VK = 4;
        const int nkg = (Q + VK - 1) / VK;
        for (int e = threadIdx.x; e < 2 * nkg * nz; e += blockDim.x) {
            int t = e % nz, r = e / nz;
            int k0 = VK * (r % nkg), d = r / nkg;
            const int nk = min(VK, Q - k0);
            const float2* Sd = reinterpret_cast<const float2*>(s.S);
            const float2* c = reinterpret_cast<const float2*>(s.C) + (size_t)d * Q * Z + t;
            float a[VK], b[VK];
#pragma unroll
            for (int q = 0; q < VK; ++q) a[q] = b[q] = 0.f;
            for (int l = 0; l < Q; ++l) {
                const float2 cl = c[l * Z];
#pragma unroll
                for (int q = 0; q < VK; ++q) dot2_acc(a[q], b[q], Sd[min(k0 + q, Q - 1) * Q + l], cl);
            }
            const R ch = fma(-cs, s.Scr[t], rbeta);
#pragma unroll
            for (int q = 0; q < VK; ++q)
                if (q < nk)
                    emit(d, t, k0 + q, df_join(a[q], b[q]), ch, csx * xi[k0 + q],
                         (with_base && !rhs_form) ? gload<CG>(base + gidx_of(d, t, k0 + q)) : R(0));
        }
    } else if constexpr (PT) {
        // FP32, parity split: the velocity pairs (k, Q-1-k) of group g
        // (k = 2g, 2g+1) for one node per task, so that each coefficient
        // load serves both pairs (four independent chains); even orders
        // build E, odd orders O, the synthesis is E + O at k and E - O at
        // Q-1-k.  The task also forms the group's terms of the moment sums.
        const ParitySplit ps(Q);
        const int H = ps.H, QE2 = ps.QE / 2, G = pair_groups(Q);
        const float2* Sp = reinterpret_cast<const float2*>(s.S);
        const bool lb = with_base && !rhs_form;
        for (int e = threadIdx.x; e < 2 * G * nz; e += blockDim.x) {
            const int t = e % nz, r = e / nz;
            const int g = r % G, d = r / G;
            const int k0 = 2 * g;
            const bool two = k0 + 1 < H;
            const int k1 = two ? k0 + 1 : k0;
            const bool pair0 = (Q - 1 - k0 != k0), pair1 = two && (Q - 1 - k1 != k1);
            const R b00 = lb ? gload<CG>(base + gidx_of(d, t, k0)) : R(0);
            const R b01 = (lb && pair0) ? gload<CG>(base + gidx_of(d, t, Q - 1 - k0)) : R(0);
            const R b10 = (lb && two) ? gload<CG>(base + gidx_of(d, t, k1)) : R(0);
            const R b11 = (lb && pair1) ? gload<CG>(base + gidx_of(d, t, Q - 1 - k1)) : R(0);
            const R* c = s.C + (size_t)d * Q * Z + t;
            const float2* sp0 = Sp + (size_t)k0 * QE2;
            const float2* sp1 = Sp + (size_t)k1 * QE2;
            R e0 = 0, o0 = 0, e1 = 0, o1 = 0;
            int l = 0;
            for (; l + 1 < Q; l += 2) {
                const R c0 = c[l * Z], c1 = c[(l + 1) * Z];
                const float2 u = sp0[l >> 1], w = sp1[l >> 1];
                e0 = fma(u.x, c0, e0);
                o0 = fma(u.y, c1, o0);
                e1 = fma(w.x, c0, e1);
                o1 = fma(w.y, c1, o1);
            }
            if (l < Q) {   // odd Q: the last (even) order
                const R c0 = c[l * Z];
                e0 = fma(sp0[l >> 1].x, c0, e0);
                e1 = fma(sp1[l >> 1].x, c0, e1);
            }
            const R ch = fma(-cs, s.Scr[t], rbeta), cx0 = csx * xi[k0], cx1 = csx * xi[k1];
            const R a0 = emit(d, t, k0, e0 + o0, ch, cx0, b00);
            const R m0 = pair0 ? emit(d, t, Q - 1 - k0, e0 - o0, ch, -cx0, b01) : R(0);
            R a1 = 0, m1 = 0;
            if (two) {
                a1 = emit(d, t, k1, e1 + o1, ch, cx1, b10);
                m1 = pair1 ? emit(d, t, Q - 1 - k1, e1 - o1, ch, -cx1, b11) : R(0);
            }
            if (!rhs_form) pair_terms_f32(d, g, two, t, Q, Z, a0, m0, a1, m1, s.Vp, s.Vr, s.Mp64, s.Mp32);
        }
    } else {
        // parity split: one velocity pair (k, Q-1-k) per task; even orders
        // build E, odd orders O (one two-wide table load per two orders); the
        // synthesis is E + O at k and E - O at Q-1-k
        using R2 = typename std::conditional<std::is_same<R, float>::value, float2, double2>::type;
        const ParitySplit ps(Q);
        const int H = ps.H, QE2 = ps.QE / 2;
        const R2* Sp = reinterpret_cast<const R2*>(s.S);
        // NODES nodes per task, t0 and t1 = t0 + ceil(nz/2) for two (four
        // independent chains per thread, each table load serving both
        // nodes); two where that saves a round of tasks or still fills
        // every thread, else one (small tiles: more warps in the phase)
        const bool lb = with_base && !rhs_form;
        auto synth = [&](auto nodes) {
            constexpr int NODES = decltype(nodes)::value;
            const int nzh = (nz + NODES - 1) / NODES;
            for (int e = threadIdx.x; e < 2 * H * nzh; e += blockDim.x) {
                const int t0 = e % nzh, r = e / nzh;
                const int t1 = t0 + nzh;
                const bool two = NODES == 2 && t1 < nz;
                const int k = r % H, d = r / H;
                const R* c = s.C + (size_t)d * Q * Z + t0;
                const R2* sp = Sp + (size_t)k * QE2;
                const bool pair = (Q - 1 - k != k);
                const R b0 = lb ? gload<CG>(base + gidx_of(d, t0, k)) : R(0);
                const R b1 = (lb && pair) ? gload<CG>(base + gidx_of(d, t0, Q - 1 - k)) : R(0);
                const R b2 = (lb && two) ? gload<CG>(base + gidx_of(d, t1, k)) : R(0);
                const R b3 = (lb && pair && two) ? gload<CG>(base + gidx_of(d, t1, Q - 1 - k)) : R(0);
                R ev = 0, od = 0, ev1 = 0, od1 = 0;
                const int dt1 = two ? nzh : 0;      // a lone last node repeats t0 (results unused)
                int l = 0;
                for (; l + 1 < Q; l += 2) {
                    const R2 sv = sp[l >> 1];
                    ev = fma(sv.x, c[l * Z], ev);
                    od = fma(sv.y, c[(l + 1) * Z], od);
                    if constexpr (NODES == 2) {
                        ev1 = fma(sv.x, c[l * Z + dt1], ev1);
                        od1 = fma(sv.y, c[(l + 1) * Z + dt1], od1);
                    }
                }
                if (l < Q) {   // odd Q: the last (even) order
                    ev = fma(sp[l >> 1].x, c[l * Z], ev);
                    if constexpr (NODES == 2) ev1 = fma(sp[l >> 1].x, c[l * Z + dt1], ev1);
                }
                const R cx = csx * xi[k];
                const R ch0 = fma(-cs, s.Scr[t0], rbeta);
                emit(d, t0, k, ev + od, ch0, cx, b0);
                if (pair) emit(d, t0, Q - 1 - k, ev - od, ch0, -cx, b1);
                if (two) {
                    const R ch1 = fma(-cs, s.Scr[t1], rbeta);
                    emit(d, t1, k, ev1 + od1, ch1, cx, b2);
                    if (pair) emit(d, t1, Q - 1 - k, ev1 - od1, ch1, -cx, b3);
                }
            }
        };
        const int nth = blockDim.x, T1 = 2 * H * nz, T2 = 2 * H * ((nz + 1) / 2);
        if ((T2 + nth - 1) / nth < (T1 + nth - 1) / nth || T2 >= nth) synth(std::integral_constant<int, 2>{});
        else synth(std::integral_constant<int, 1>{});
    }
    if (mode == 1) return;
    __syncthreads();

    // Phase 6: raw moment sums of the new stage for the next stage's node fields.
    if constexpr (PT) {
        // the group terms formed with the synthesis, summed per (moment, node)
        const int G = pair_groups(Q);
        const size_t blk = (size_t)G * Z;
        for (int e = threadIdx.x; e < kNumMoments * nz; e += blockDim.x) {
            const int which = e / nz, t = e - which * nz;
            double v;
            if (which == MOM_S3 || which == MOM_G1)
                v = (double)sum_pair_terms<float>(s.Mp32 + (which == MOM_S3 ? 0 : blk) + t, G, Z);
            else
                v = sum_pair_terms<double>(s.Mp64 + (which == MOM_G0 ? 3 : which) * blk + t, G, Z);
            mom_out[which * NN + sd.node_off + it.i0 + t] = v;
        }
    } else {
        tile_moment_sums_staged<R>(sd, it, s, Z, s.Vp, s.Vr, mom_out, NN);
    }
}

template <typename R, bool DF = false, int T = StageThreads<R, DF>::value>
__global__ void __launch_bounds__(T, DF ? 3 : ((std::is_same<R, double>::value || T <= 256) ? 2 : 1))
stage_kernel(const SlabDesc* __restrict__ slabs, const WorkItem* __restrict__ items,
             const double* __restrict__ tables, const R* __restrict__ rtab,
             const double* __restrict__ taps, const R* __restrict__ rtaps,
             const R* __restrict__ src, const R* base, R* out, double* rhs_out,
             const double* __restrict__ mom_in, double* __restrict__ mom_out,
             long long NF, long long NN, double alpha, double beta, int mode, int Z, unsigned* err) {
    extern __shared__ __align__(16) double smem[];
    const WorkItem it = items[blockIdx.x];
    const SlabDesc sd = slabs[it.slab];
    stage_body<R, DF, false>(sd, it, smem, tables, rtab, taps, rtaps, src, base, out, rhs_out, mom_in, mom_out,
                             nullptr, NF, NN, alpha, beta, mode, Z, err);
}

// The FP64 stage that also writes the node fields of its input state,
// [EVFDLB_NFIELDS][NN] (the adjoint's segment recompute; the reverse sweep
// reads them instead of forming them again).
__global__ void __launch_bounds__(StageThreads<double>::value, 2)
stage_fields_kernel(const SlabDesc* __restrict__ slabs, const WorkItem* __restrict__ items,
                    const double* __restrict__ tables, const double* __restrict__ taps,
                    const double* __restrict__ src, const double* base, double* out,
                    const double* __restrict__ mom_in, double* __restrict__ mom_out, double* __restrict__ fields_out,
                    long long NF, long long NN, double alpha, double beta, int Z, unsigned* err) {
    extern __shared__ __align__(16) double smem[];
    const WorkItem it = items[blockIdx.x];
    const SlabDesc sd = slabs[it.slab];
    stage_body<double, false, false, true>(sd, it, smem, tables, tables, taps, taps, src, base, out, nullptr, mom_in,
                                           mom_out, fields_out, NF, NN, alpha, beta, 0, Z, err);
}

// ---------------------------------------------------------------------------
// Persistent form of the step for a batch of independent slabs (FP64): one
// launch advances every slab by nsteps Shu-Osher steps.  The CTAs stay
// resident and pull work items (stage, slab tile) from a queue in stage
// order; an item of global stage g of slab b starts once every item of stage
// g-1 of that slab has completed (a per-slab counter of completed items,
// released after the item's writes and acquired before its reads), so slabs
// proceed independently and a short slab does not wait at the stage
// boundaries of a long one.  An item only ever waits for items dequeued
// before it, by CTAs that are running: the queue cannot deadlock, whatever
// the number of resident CTAs.  Every wait is bounded: after spin_limit polls
// the CTA sets ERR_TIMEOUT, and every CTA leaves at its next dequeue; nothing
// traps.  Data written in the same launch are read with L2-coherent loads.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__global__ void __launch_bounds__(StageThreads<double>::value, 2) persist_kernel(PersistArgs a) {
    extern __shared__ __align__(16) double smem[];
    __shared__ int s_q, s_stop;
    const int total = a.nstages * a.nitems;
    for (;;) {
        if (threadIdx.x == 0) {
            int stop = (ld_acquire_u32(a.err) & ERR_TIMEOUT) ? 1 : 0;
            const int q = stop ? total : (int)atomicAdd(a.queue, 1u);
            if (q < total) {
                const int g = q / a.nitems, b = a.items[q % a.nitems].slab;
                const unsigned need = (unsigned)g * (unsigned)a.tiles[b];
                long long polls = 0;
                while (ld_acquire_u32(a.gate) == 0u || ld_acquire_u32(a.done + b) < need) {
                    if (++polls > a.spin_limit) {
                        atomicOr(a.err, ERR_TIMEOUT);
                        stop = 1;
                        break;
                    }
                    if (ld_acquire_u32(a.err) & ERR_TIMEOUT) {   // another CTA gave up
                        stop = 1;
                        break;
                    }
                    __nanosleep(100);
                }
            }
            s_q = q;
            s_stop = stop || q >= total;
        }
        __syncthreads();
        if (s_stop) return;
        const int q = s_q, g = q / a.nitems, stage = g % 3;
        const WorkItem it = a.items[q % a.nitems];
        const SlabDesc sd = a.slabs[it.slab];
        // stage 0: u1 = u + dt L(u); 1: u2 = 3/4 u + 1/4 (u1 + dt L(u1));
        // 2: u = 1/3 u + 2/3 (u2 + dt L(u2)), over u
        const double* src = a.st[stage];
        const double* base = stage == 0 ? nullptr : a.st[0];
        double* out = a.st[(stage + 1) % 3];
        const double alpha = stage == 0 ? 0.0 : (stage == 1 ? 0.75 : 1.0 / 3.0);
        const double beta = stage == 0 ? 1.0 : (stage == 1 ? 0.25 : 2.0 / 3.0);
        stage_body<double, false, true>(sd, it, smem, a.tables, a.tables, a.taps, a.taps, src, base, out, nullptr,
                                        a.mom[stage], a.mom[(stage + 1) % 3], nullptr, a.NF, a.NN, alpha, beta, 0,
                                        a.Z, a.err);
        __threadfence();                               // this thread's writes, before the release
        __syncthreads();
        if (threadIdx.x == 0) atomicAdd(a.done + it.slab, 1u);
    }
}

cudaError_t configure_persist(size_t smem_bytes) {
    return cudaFuncSetAttribute(persist_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
}

// Resident CTAs of the persistent kernel on the current device (at least one).
int persist_grid(size_t smem_bytes) {
    int dev = 0, sms = 1, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, persist_kernel, StageThreads<double>::value, smem_bytes);
    return (sms > 0 ? sms : 1) * (per_sm > 0 ? per_sm : 1);
}

void launch_persist(int grid, size_t smem, cudaStream_t st, const PersistArgs& a) {
    persist_kernel<<<grid, StageThreads<double>::value, smem, st>>>(a);
}

// Projected Maxwellian pair (F_MB, T F_MB) from node fields, formed in FP64 and
// stored as R: F_k = sum_l S_kl n m_l(u, T), G_k = T F_k; also writes the raw
// moment sums of the stored state.
template <typename R>
__global__ void __launch_bounds__(kThreads)
init_kernel(const SlabDesc* __restrict__ slabs, const WorkItem* __restrict__ items,
            const double* __restrict__ tables, const R* __restrict__ rtab, const double* __restrict__ n0,
            const double* __restrict__ u0, const double* __restrict__ T0, R* state,
            double* mom, long long NF, long long NN, int Z, unsigned* err) {
    extern __shared__ __align__(16) double smem[];
    const WorkItem it = items[blockIdx.x];
    const SlabDesc sd = slabs[it.slab];
    const int Q = sd.Q, W = Z + 6, nz = it.nz;
    Smem<R> s = carve<R>(smem, Q, Z, sd.M);
    TableLayout L(Q);
    const double* tab = tables + sd.tab_off;
    // FP64 coefficients [Q][Z] in the R blocks C and A (2 Q Z + 2 Q Z R values
    // hold at least Q Z doubles for either R)
    double* coef = reinterpret_cast<double*>(s.C);
    for (int t = threadIdx.x; t < nz; t += blockDim.x) {
        long long o = sd.node_off + it.i0 + t;
        double n = n0[o], u = u0[o], T = T0[o];
        if (!(n > 0.0) || !(T > 0.0) || !finite(u))
            atomicOr(err, (finite(n) && finite(T) && finite(u)) ? ERR_NEGATIVE : ERR_NONFINITE);
        s.Sc[SC_T * Z + t] = T;
        double m0 = 1.0, m1 = 0.0, Tm1 = T - 1.0;
        for (int l = 0; l < Q; ++l) {
            coef[l * Z + t] = n * m0;
            double mn = fma(u * tab[L.rinv + l], m0, Tm1 * tab[L.rr + l] * m1);
            m1 = m0;
            m0 = mn;
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < Q * nz; e += blockDim.x) {
        int t = e % nz, k = e / nz;
        double acc = 0.0;
        for (int l = 0; l < Q; ++l) acc = fma(tab[L.S + k * Q + l], coef[l * Z + t], acc);
        double gval = s.Sc[SC_T * Z + t] * acc;
        long long g = sd.f_off + (long long)k * sd.nx + it.i0 + t;
        R fa = (R)acc, ga = (R)gval;
        state[g] = fa;
        state[NF + g] = ga;
        s.F[(size_t)k * W + t + 3] = fa;
        s.F[(size_t)(Q + k) * W + t + 3] = ga;
    }
    __syncthreads();
    tile_moment_sums<R>(sd, it, s, Z, tab + L.xi, rtab + sd.tab_off + L.xi, mom, NN);
}

// Isothermal mode, applied after every step to the slabs with T_iso > 0:
// each node's temperature is set back to T_iso with its density, velocity
// and non-equilibrium part kept,
//   F += F_MB(n, u, T_iso) - F_MB(n, u, T),  G += T_iso F_MB(n, u, T_iso) - T F_MB(n, u, T),
// n, u, T from the step's moment sums; F_MB is the projected Maxwellian of
// init_kernel (Hermite coefficients n m_l).  The tile's moment sums are
// rewritten from the updated state.  Blocks of other slabs return at once.
template <typename R>
__global__ void __launch_bounds__(kThreads)
iso_reset_kernel(const SlabDesc* __restrict__ slabs, const WorkItem* __restrict__ items,
                 const double* __restrict__ tables, const R* __restrict__ rtab, R* state, double* mom, long long NF,
                 long long NN, int Z) {
    extern __shared__ __align__(16) double smem[];
    const WorkItem it = items[blockIdx.x];
    const SlabDesc sd = slabs[it.slab];
    if (!(sd.T_iso > 0.0)) return;
    const int Q = sd.Q, W = Z + 6, nz = it.nz;
    Smem<R> s = carve<R>(smem, Q, Z, sd.M);
    TableLayout L(Q);
    const double* tab = tables + sd.tab_off;
    // FP64 coefficient differences [2][Q][Z] in the R blocks C and A
    double* dcoef = reinterpret_cast<double*>(s.C);
    const double* S0 = mom + MOM_S0 * NN + sd.node_off;
    const double* S1 = mom + MOM_S1 * NN + sd.node_off;
    const double* S2 = mom + MOM_S2 * NN + sd.node_off;
    const double* G0 = mom + MOM_G0 * NN + sd.node_off;
    const double Ti = sd.T_iso;
    for (int t = threadIdx.x; t < nz; t += blockDim.x) {
        int i = it.i0 + t;
        double n = S0[i], inv_n = 1.0 / n, u = S1[i] * inv_n;
        double T = (2.0 / 3.0) * ((0.5 * S2[i] + G0[i]) * inv_n - 0.5 * u * u);
        // m_l of N(u, T) and N(u, T_iso) by the recurrence of init_kernel
        double a0 = 1.0, a1 = 0.0, b0 = 1.0, b1 = 0.0, Ta = Ti - 1.0, Tb = T - 1.0;
        for (int l = 0; l < Q; ++l) {
            dcoef[l * Z + t] = n * (a0 - b0);
            dcoef[(Q + l) * Z + t] = n * (Ti * a0 - T * b0);
            double an = fma(u * tab[L.rinv + l], a0, Ta * tab[L.rr + l] * a1);
            double bn = fma(u * tab[L.rinv + l], b0, Tb * tab[L.rr + l] * b1);
            a1 = a0;
            a0 = an;
            b1 = b0;
            b0 = bn;
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < 2 * Q * nz; e += blockDim.x) {
        int t = e % nz, r = e / nz;
        int k = r % Q, d = r / Q;
        const double* c = dcoef + (size_t)d * Q * Z;
        double acc = 0.0;
        for (int l = 0; l < Q; ++l) acc = fma(tab[L.S + k * Q + l], c[l * Z + t], acc);
        long long g = (long long)d * NF + sd.f_off + (long long)k * sd.nx + it.i0 + t;
        R v = (R)((double)state[g] + acc);
        state[g] = v;
        s.F[(size_t)(d * Q + k) * W + t + 3] = v;
    }
    __syncthreads();
    tile_moment_sums<R>(sd, it, s, Z, tab + L.xi, rtab + sd.tab_off + L.xi, mom, NN);
}

// Raw moment sums of an arbitrary state (after set_state); same precision rule
// and summation order as the stage kernel's tile_moment_sums.  The tile's
// 2 Q rows are staged in shared memory with coalesced loads first, so that
// the per-node sums do not wait on Q serial global loads.
template <typename R>
__global__ void __launch_bounds__(kThreads)
sums_kernel(const SlabDesc* __restrict__ slabs, const WorkItem* __restrict__ items,
            const double* __restrict__ tables, const R* __restrict__ rtab, const R* __restrict__ state,
            double* mom, long long NF, long long NN, unsigned* err) {
    const WorkItem it = items[blockIdx.x];
    const SlabDesc sd = slabs[it.slab];
    const int Q = sd.Q, nz = it.nz;
    TableLayout L(Q);
    __shared__ double xp[3 * kQMax];
    __shared__ R xr[2 * kQMax];
    __shared__ R tile[2 * kQMax * kZMax];   // [d][k][t], row length nz
    velocity_powers<R>(Q, tables + sd.tab_off + L.xi, rtab + sd.tab_off + L.xi, xp, xr, threadIdx.x, blockDim.x);
    const int rows = 2 * Q;
#pragma unroll 4
    for (int e = threadIdx.x; e < rows * nz; e += blockDim.x) {
        const int r = e / nz, t = e - r * nz;              // r = d Q + k
        const int d = r >= Q ? 1 : 0, k = r - d * Q;
        tile[e] = state[d * NF + sd.f_off + (long long)k * sd.nx + it.i0 + t];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < kNumMoments * nz; e += blockDim.x) {
        int t = e % nz, which = e / nz;
        int d = which >= MOM_G0 ? 1 : 0;
        double acc = moment_sum<R>(which, Q, tile + (size_t)d * Q * nz + t, nz, xp, xr);
        if (!finite(acc)) atomicOr(err, ERR_NONFINITE);
        mom[which * NN + sd.node_off + it.i0 + t] = acc;
    }
}

// Node fields of the current state (diagnostic).
template <typename R>
__global__ void __launch_bounds__(kThreads)
fields_kernel(const SlabDesc* __restrict__ slabs, const WorkItem* __restrict__ items,
              const R* __restrict__ rtab, const double* __restrict__ taps, const R* __restrict__ rtaps,
              const double* __restrict__ mom, double* fields, long long NN, int Z, unsigned* err) {
    extern __shared__ __align__(16) double smem[];
    const WorkItem it = items[blockIdx.x];
    const SlabDesc sd = slabs[it.slab];
    Smem<R> s = carve<R>(smem, sd.Q, Z, sd.M);
    load_node_inputs<R>(sd, it, s, Z, rtab, mom, NN);
    __syncthreads();
    node_fields<R>(sd, it, s, Z, taps, rtaps, mom, NN, err, fields);
}

// n, u, T, q of node i from its raw sums (null outputs are skipped).
__device__ __forceinline__ void node_moments(const double* __restrict__ mom, long long NN, long long i, double* n,
                                             double* u, double* T, double* q) {
    double S0 = mom[MOM_S0 * NN + i], S1 = mom[MOM_S1 * NN + i], S2 = mom[MOM_S2 * NN + i];
    double S3 = mom[MOM_S3 * NN + i], G0 = mom[MOM_G0 * NN + i], G1 = mom[MOM_G1 * NN + i];
    double uu = S1 / S0;
    if (n) n[i] = S0;
    if (u) u[i] = uu;
    if (T) T[i] = (2.0 / 3.0) * ((0.5 * S2 + G0) / S0 - 0.5 * uu * uu);
    if (q) q[i] = 0.5 * (S3 - 3.0 * uu * S2 + 3.0 * uu * uu * S1 - uu * uu * uu * S0) + G1 - uu * G0;
}

// n, u, T, q per node from the raw sums.
__global__ void moments_kernel(const double* __restrict__ mom, long long NN, double* n, double* u,
                               double* T, double* q) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < NN;
         i += (long long)gridDim.x * blockDim.x)
        node_moments(mom, NN, i, n, u, T, q);
}

// Conserved totals, first pass: per work item (node tile) the sums of S0,
// S1, S2/2 + G0 and of the mean-field energy density (1/2) n_i sum_j e_j
// n_{i+j} (energy taps over a staged density halo), fixed-order tree; the
// tile's n, u, T, q as well where those outputs are given (non-null).
__global__ void __launch_bounds__(kThreads)
totals_part_kernel(const SlabDesc* __restrict__ slabs, const WorkItem* __restrict__ items,
                   const double* __restrict__ taps, const double* __restrict__ mom, long long NN,
                   double* __restrict__ part, double* n, double* u, double* T, double* q) {
    extern __shared__ double sn[];          // S0 on [i0 - M, i0 + nz + M)
    __shared__ double red[4][kThreads];
    const WorkItem it = items[blockIdx.x];
    const SlabDesc sd = slabs[it.slab];
    const int M = sd.M, nz = it.nz;
    const double* S0 = mom + MOM_S0 * NN + sd.node_off;
    const double* S1 = mom + MOM_S1 * NN + sd.node_off;
    const double* S2 = mom + MOM_S2 * NN + sd.node_off;
    const double* G0 = mom + MOM_G0 * NN + sd.node_off;
    const double* etap = taps + sd.tap_off + 2 * sd.M + 1 + 2 * sd.m + 1;
    for (int c = threadIdx.x; c < nz + 2 * M; c += blockDim.x) sn[c] = S0[gidx(it.i0 - M + c, sd.nx, sd.bc)];
    __syncthreads();
    // eight lanes per node split its 2M+1 energy taps (xor-shuffle sum)
    double a0 = 0, a1 = 0, a2 = 0, a3 = 0;
    const int sub = threadIdx.x & 7;
    for (int b = 0; b < nz; b += kThreads / 8) {
        const int t = b + threadIdx.x / 8;
        double acc = 0.0;
        if (t < nz)
            for (int j = -M + sub; j <= M; j += 8) acc = fma(etap[j + M], sn[t + M + j], acc);
        acc += __shfl_xor_sync(0xffffffffu, acc, 4);
        acc += __shfl_xor_sync(0xffffffffu, acc, 2);
        acc += __shfl_xor_sync(0xffffffffu, acc, 1);
        if (t < nz && sub == 0) {
            const int i = it.i0 + t;
            node_moments(mom, NN, sd.node_off + i, n, u, T, q);
            a0 += S0[i];
            a1 += S1[i];
            a2 += 0.5 * S2[i] + G0[i];
            a3 += 0.5 * sn[t + M] * acc;
        }
    }
    red[0][threadIdx.x] = a0;
    red[1][threadIdx.x] = a1;
    red[2][threadIdx.x] = a2;
    red[3][threadIdx.x] = a3;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int c = 0; c < 4; ++c) red[c][threadIdx.x] += red[c][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < 4) part[4 * blockIdx.x + threadIdx.x] = red[threadIdx.x][0];
}

// Per slab: its tiles' partial sums in work-list order (fixed assignment of
// tiles to threads and a fixed tree: deterministic), times dx:
// {mass, momentum, kinetic + internal + mean-field energy, mean-field energy}.
__global__ void __launch_bounds__(kThreads)
totals_kernel(const SlabDesc* __restrict__ slabs, const WorkItem* __restrict__ items, int nitems,
              const double* __restrict__ part, double* out) {
    __shared__ double red[4][kThreads];
    const SlabDesc sd = slabs[blockIdx.x];
    double a[4] = {0, 0, 0, 0};
    for (int j = threadIdx.x; j < nitems; j += blockDim.x)
        if (items[j].slab == (int)blockIdx.x)
            for (int c = 0; c < 4; ++c) a[c] += part[4 * j + c];
    for (int c = 0; c < 4; ++c) red[c][threadIdx.x] = a[c];
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int c = 0; c < 4; ++c) red[c][threadIdx.x] += red[c][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[4 * blockIdx.x + 0] = red[0][0] * sd.dx;
        out[4 * blockIdx.x + 1] = red[1][0] * sd.dx;
        out[4 * blockIdx.x + 3] = red[3][0] * sd.dx;
        out[4 * blockIdx.x + 2] = (red[2][0] + red[3][0]) * sd.dx;
    }
}

// Element-wise precision conversion (state copies in and out of FP32 contexts).
template <typename A, typename B>
__global__ void convert_kernel(const A* __restrict__ in, B* __restrict__ out, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        out[i] = (B)in[i];
}

// ---------------------------------------------------------------------------
// Host-side launch helpers (called from the C-ABI layer).  `prec` selects the
// instantiation: EVFDLB_FP64 (R = double) or EVFDLB_FP32 (R = float); the R
// tables and taps are the FP64 ones for FP64 and float copies for FP32.
// ---------------------------------------------------------------------------
size_t stage_smem_bytes(int Q, int Z, int M) { return smem_bytes_t<double>(Q, Z, M); }

size_t stage_smem_bytes_p(int prec, int Q, int Z, int M) {
    return prec == EVFDLB_FP32 ? smem_bytes_t<float>(Q, Z, M) : smem_bytes_t<double>(Q, Z, M);
}

// The FP64_DF stage keeps its split state tile (2 Q Z float pairs) in the EO
// block (4 H Z >= 2 Q Z doubles).
size_t stage_smem_bytes_df(int Q, int Z, int M) { return smem_bytes_t<double>(Q, Z, M); }

cudaError_t configure_df(size_t smem_bytes) {
    return cudaFuncSetAttribute(stage_kernel<double, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem_bytes);
}

// FP64_DF stage: dftab holds the analysis and synthesis tables as pairs.
void launch_stage_df(int nitems, size_t smem, cudaStream_t st, const SlabDesc* slabs, const WorkItem* items,
                     const double* tables, const double* dftab, const double* taps, const double* src,
                     const double* base, double* out, double* rhs_out, const double* mom_in, double* mom_out,
                     long long NF, long long NN, double alpha, double beta, int mode, int Z, unsigned* err) {
    launch_pdl(stage_kernel<double, true>, nitems, StageThreads<double, true>::value, smem, st, slabs, items, tables,
               dftab, taps, taps, src, base, out, rhs_out, mom_in, mom_out, NF, NN, alpha, beta, mode, Z, err);
}

template <typename R>
static cudaError_t configure_t(size_t smem_bytes) {
    cudaError_t e = cudaFuncSetAttribute(stage_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
    if (e != cudaSuccess) return e;
    if (std::is_same<R, float>::value) {
        e = cudaFuncSetAttribute(stage_kernel<float, false, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem_bytes);
        if (e != cudaSuccess) return e;
    }
    e = cudaFuncSetAttribute(init_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(iso_reset_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
    if (e != cudaSuccess) return e;
    if (std::is_same<R, double>::value) {
        e = cudaFuncSetAttribute(stage_fields_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
        if (e != cudaSuccess) return e;
    }
    return cudaFuncSetAttribute(fields_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
}

cudaError_t configure_kernels_p(int prec, size_t smem_bytes) {
    return prec == EVFDLB_FP32 ? configure_t<float>(smem_bytes) : configure_t<double>(smem_bytes);
}

cudaError_t configure_kernels(size_t smem_bytes) { return configure_t<double>(smem_bytes); }

// Raises (never lowers) the dynamic shared-memory limit of the FP64 stage and
// isothermal-reset kernels on the current device to at least smem_bytes.
cudaError_t ensure_stage_smem(size_t smem_bytes) {
    const void* fns[2] = {(const void*)stage_kernel<double>, (const void*)iso_reset_kernel<double>};
    for (const void* f : fns) {
        cudaFuncAttributes a;
        cudaError_t e = cudaFuncGetAttributes(&a, f);
        if (e != cudaSuccess) return e;
        if ((size_t)a.maxDynamicSharedSizeBytes >= smem_bytes) continue;
        e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// SMs of the current device (cached per device).
static int sm_count() {
    static int cache[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return 1;
    if (!cache[dev]) {
        int n = 0;
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        cache[dev] = n > 0 ? n : 1;
    }
    return cache[dev];
}

// The FP64 stage (8 warps; see StageThreads).
static void launch_stage_fp64(int nitems, size_t smem, cudaStream_t st, const SlabDesc* slabs,
                              const WorkItem* items, const double* tables, const double* rtab, const double* taps,
                              const double* rtaps, const double* src, const double* base, double* out,
                              double* rhs_out, const double* mom_in, double* mom_out, long long NF, long long NN,
                              double alpha, double beta, int mode, int Z, unsigned* err) {
    launch_pdl(stage_kernel<double>, nitems, StageThreads<double>::value, smem, st, slabs, items, tables, rtab, taps,
               rtaps, src, base, out, rhs_out, mom_in, mom_out, NF, NN, alpha, beta, mode, Z, err);
}

void launch_stage_p(int prec, int nitems, size_t smem, cudaStream_t st, const SlabDesc* slabs,
                    const WorkItem* items, const double* tables, const void* rtab, const double* taps,
                    const void* rtaps, const void* src, const void* base, void* out, double* rhs_out,
                    const double* mom_in, double* mom_out, long long NF, long long NN, double alpha, double beta,
                    int mode, int Z, unsigned* err) {
    if (prec == EVFDLB_FP32) {
        // the 16-warp form (one CTA per SM) where the work list fits one wave
        // on the SMs, else the 8-warp form (two CTAs per SM), which finishes
        // up to twice as many tiles in a wave
        if (nitems <= sm_count())
            launch_pdl(stage_kernel<float>, nitems, StageThreads<float>::value, smem, st, slabs, items, tables,
                       (const float*)rtab, taps, (const float*)rtaps, (const float*)src, (const float*)base,
                       (float*)out, rhs_out, mom_in, mom_out, NF, NN, alpha, beta, mode, Z, err);
        else
            launch_pdl(stage_kernel<float, false, 256>, nitems, 256, smem, st, slabs, items, tables,
                       (const float*)rtab, taps, (const float*)rtaps, (const float*)src, (const float*)base,
                       (float*)out, rhs_out, mom_in, mom_out, NF, NN, alpha, beta, mode, Z, err);
    } else
        launch_stage_fp64(nitems, smem, st, slabs, items, tables, (const double*)rtab, taps, (const double*)rtaps,
                          (const double*)src, (const double*)base, (double*)out, rhs_out, mom_in, mom_out, NF, NN,
                          alpha, beta, mode, Z, err);
}

// FP64 stage that also stores the node fields of its input state (the
// adjoint's segment recompute: the reverse sweep reads them instead of
// forming them again).
void launch_stage_fields(int nitems, size_t smem, cudaStream_t st, const SlabDesc* slabs, const WorkItem* items,
                         const double* tables, const double* taps, const double* src, const double* base,
                         double* out, const double* mom_in, double* mom_out, double* fields_out, long long NF,
                         long long NN, double alpha, double beta, int Z, unsigned* err) {
    launch_pdl(stage_fields_kernel, nitems, StageThreads<double>::value, smem, st, slabs, items, tables, taps, src, base,
               out, mom_in, mom_out, fields_out, NF, NN, alpha, beta, Z, err);
}

// FP64 stage (mode 0 writes out; mode 1 writes the right-hand side to out).
void launch_stage(int nitems, size_t smem, cudaStream_t st, const SlabDesc* slabs, const WorkItem* items,
                  const double* tables, const double* taps, const double* src, const double* base,
                  double* out, const double* mom_in, double* mom_out, long long NF, long long NN,
                  double alpha, double beta, int mode, int Z, unsigned* err) {
    launch_stage_fp64(nitems, smem, st, slabs, items, tables, tables, taps, taps, src, base, out, out, mom_in, mom_out,
                      NF, NN, alpha, beta, mode, Z, err);
}

void launch_init_p(int prec, int nitems, size_t smem, cudaStream_t st, const SlabDesc* slabs,
                   const WorkItem* items, const double* tables, const void* rtab, const double* n0,
                   const double* u0, const double* T0, void* state, double* mom, long long NF, long long NN, int Z,
                   unsigned* err) {
    if (prec == EVFDLB_FP32)
        init_kernel<float><<<nitems, kThreads, smem, st>>>(slabs, items, tables, (const float*)rtab, n0, u0, T0,
                                                           (float*)state, mom, NF, NN, Z, err);
    else
        init_kernel<double><<<nitems, kThreads, smem, st>>>(slabs, items, tables, (const double*)rtab, n0, u0, T0,
                                                            (double*)state, mom, NF, NN, Z, err);
}

void launch_iso_reset_p(int prec, int nitems, size_t smem, cudaStream_t st, const SlabDesc* slabs,
                        const WorkItem* items, const double* tables, const void* rtab, void* state, double* mom,
                        long long NF, long long NN, int Z) {
    if (prec == EVFDLB_FP32)
        iso_reset_kernel<float><<<nitems, kThreads, smem, st>>>(slabs, items, tables, (const float*)rtab,
                                                                (float*)state, mom, NF, NN, Z);
    else
        iso_reset_kernel<double><<<nitems, kThreads, smem, st>>>(slabs, items, tables, (const double*)rtab,
                                                                 (double*)state, mom, NF, NN, Z);
}

void launch_sums_p(int prec, int nitems, cudaStream_t st, const SlabDesc* slabs, const WorkItem* items,
                   const double* tables, const void* rtab, const void* state, double* mom, long long NF,
                   long long NN, unsigned* err) {
    if (prec == EVFDLB_FP32)
        sums_kernel<float><<<nitems, kThreads, 0, st>>>(slabs, items, tables, (const float*)rtab,
                                                        (const float*)state, mom, NF, NN, err);
    else
        sums_kernel<double><<<nitems, kThreads, 0, st>>>(slabs, items, tables, (const double*)rtab,
                                                         (const double*)state, mom, NF, NN, err);
}

void launch_sums(int nitems, cudaStream_t st, const SlabDesc* slabs, const WorkItem* items,
                 const double* tables, const double* state, double* mom, long long NF, long long NN,
                 unsigned* err) {
    launch_sums_p(EVFDLB_FP64, nitems, st, slabs, items, tables, tables, state, mom, NF, NN, err);
}

void launch_fields_p(int prec, int nitems, size_t smem, cudaStream_t st, const SlabDesc* slabs,
                     const WorkItem* items, const void* rtab, const double* taps, const void* rtaps,
                     const double* mom, double* fields, long long NN, int Z, unsigned* err) {
    if (prec == EVFDLB_FP32)
        fields_kernel<float><<<nitems, kThreads, smem, st>>>(slabs, items, (const float*)rtab, taps,
                                                             (const float*)rtaps, mom, fields, NN, Z, err);
    else
        fields_kernel<double><<<nitems, kThreads, smem, st>>>(slabs, items, (const double*)rtab, taps,
                                                              (const double*)rtaps, mom, fields, NN, Z, err);
}

void launch_convert_to_f32(cudaStream_t st, const double* in, float* out, long long n) {
    int blocks = (int)std::min<long long>((n + 255) / 256, 4096);
    if (blocks < 1) blocks = 1;
    convert_kernel<double, float><<<blocks, 256, 0, st>>>(in, out, n);
}

void launch_convert_to_f64(cudaStream_t st, const float* in, double* out, long long n) {
    int blocks = (int)std::min<long long>((n + 255) / 256, 4096);
    if (blocks < 1) blocks = 1;
    convert_kernel<float, double><<<blocks, 256, 0, st>>>(in, out, n);
}

void launch_moments(cudaStream_t st, const double* mom, long long NN, double* n, double* u, double* T,
                    double* q) {
    int blocks = (int)((NN + 255) / 256);
    if (blocks > 1024) blocks = 1024;
    moments_kernel<<<blocks, 256, 0, st>>>(mom, NN, n, u, T, q);
}

// Conserved totals: per-tile partial sums (part: 4 per work item), then per
// slab in work-list order.  smem: (Z + 2 Mmax) doubles.
// Conserved totals per slab into out [4 nslabs]; n, u, T, q per node on the
// way (each may be null).
void launch_totals(int nslabs, int nitems, size_t smem, cudaStream_t st, const SlabDesc* slabs,
                   const WorkItem* items, const double* taps, const double* mom, long long NN, double* part,
                   double* out, double* n, double* u, double* T, double* q) {
    totals_part_kernel<<<nitems, kThreads, smem, st>>>(slabs, items, taps, mom, NN, part, n, u, T, q);
    totals_kernel<<<nslabs, kThreads, 0, st>>>(slabs, items, nitems, part, out);
}

}  // namespace evfdlb
