// evfdlb_kernels.cu -- sm_103a kernels of libevfdlb (FP64 forward path).
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
#include <cuda_runtime.h>
#include <math.h>

#include "evfdlb_internal.h"

namespace evfdlb {

__device__ __forceinline__ int gidx(int i, int nx, int bc) {
    if (bc == EVFDLB_BC_PERIODIC) {
        int r = i % nx;
        return r < 0 ? r + nx : r;
    }
    return i < 0 ? 0 : (i >= nx ? nx - 1 : i);
}

// ---------------------------------------------------------------------------
// Shared-memory layout of one CTA (doubles), sized for (Q, Z, M).
// ---------------------------------------------------------------------------
struct Smem {
    double *P, *S;      // analysis / synthesis tables [Q*Q] each
    double *N;          // n on nodes [i0 - M, i0 + Z + M)
    double *U, *T;      // u, T on nodes [i0 - 2, i0 + Z + 2)
    double *X, *Chi;    // X = n^2 chi T and chi on the same nodes
    double *Sc;         // per-node scalars [kNumScalars][Z]
    double *C;          // coefficients [2][Q][Z]
    double *A;          // analysis [2][Q][Z]
    double *F;          // state tile with halo [2][Q][Z+6]
    double *Face;       // WENO face values [2][Q][Z+1]
};

__host__ __device__ inline size_t smem_doubles(int Q, int Z, int M) {
    return (size_t)2 * Q * Q + (Z + 2 * M) + 4 * (Z + 4) + kNumScalars * Z + 2 * (size_t)Q * Z +
           2 * (size_t)Q * Z + 2 * (size_t)Q * (Z + 6) + 2 * (size_t)Q * (Z + 1);
}

__device__ inline Smem carve(double* base, int Q, int Z, int M) {
    Smem s;
    s.P = base;
    s.S = s.P + Q * Q;
    s.N = s.S + Q * Q;
    s.U = s.N + (Z + 2 * M);
    s.T = s.U + (Z + 4);
    s.X = s.T + (Z + 4);
    s.Chi = s.X + (Z + 4);
    s.Sc = s.Chi + (Z + 4);
    s.C = s.Sc + kNumScalars * Z;
    s.A = s.C + 2 * Q * Z;
    s.F = s.A + 2 * Q * Z;
    s.Face = s.F + 2 * Q * (Z + 6);
    return s;
}

enum { SC_N = 0, SC_U, SC_T, SC_NU, SC_FORCE, SC_KQ, SC_K, SC_A, SC_B, SC_D };

__device__ __forceinline__ bool finite(double x) { return isfinite(x); }

// ---------------------------------------------------------------------------
// Phase 0: stage the tables, the density halo, u/T near the tile and the
// state tile (+-3 nodes for WENO-5) into shared memory.
// ---------------------------------------------------------------------------
__device__ void load_node_inputs(const SlabDesc& sd, const WorkItem& it, const Smem& s, int Z,
                                 const double* __restrict__ tables, const double* __restrict__ mom,
                                 long long NN) {
    const int Q = sd.Q, M = sd.M, nx = sd.nx, bc = sd.bc;
    TableLayout L(Q);
    const double* tab = tables + sd.tab_off;
    for (int t = threadIdx.x; t < 2 * Q * Q; t += blockDim.x) s.P[t] = tab[L.P + t];  // P then S
    const double* S0 = mom + MOM_S0 * NN + sd.node_off;
    for (int t = threadIdx.x; t < it.nz + 2 * M; t += blockDim.x)
        s.N[t] = S0[gidx(it.i0 - M + t, nx, bc)];
    const double* S1 = mom + MOM_S1 * NN + sd.node_off;
    const double* S2 = mom + MOM_S2 * NN + sd.node_off;
    const double* G0 = mom + MOM_G0 * NN + sd.node_off;
    for (int t = threadIdx.x; t < it.nz + 4; t += blockDim.x) {
        int i = gidx(it.i0 - 2 + t, nx, bc);
        double n = S0[i], inv_n = 1.0 / n;
        double u = S1[i] * inv_n;
        // (3/2) n T = sum (xi-u)^2/2 F + sum G = S2/2 + G0 - n u^2/2
        s.U[t] = u;
        s.T[t] = (2.0 / 3.0) * ((0.5 * S2[i] + G0[i]) * inv_n - 0.5 * u * u);
    }
}

__device__ void load_state_tile(const SlabDesc& sd, const WorkItem& it, const Smem& s, int Z,
                                const double* __restrict__ src, long long NF) {
    const int Q = sd.Q, nx = sd.nx, bc = sd.bc, W = Z + 6;
    const int cols = it.nz + 6;
    for (int e = threadIdx.x; e < 2 * Q * cols; e += blockDim.x) {
        int c = e % cols, r = e / cols;
        int k = r % Q, d = r / Q;
        int i = gidx(it.i0 - 3 + c, nx, bc);
        s.F[(d * Q + k) * W + c] = src[d * NF + sd.f_off + (long long)k * nx + i];
    }
}

// ---------------------------------------------------------------------------
// Phases 1-2: node fields of the tile.
// ---------------------------------------------------------------------------
__device__ void node_fields(const SlabDesc& sd, const WorkItem& it, const Smem& s, int Z,
                            const double* __restrict__ taps, const double* __restrict__ mom,
                            long long NN, unsigned* err, double* fields_out) {
    const int M = sd.M, m = sd.m;
    const double* ftap = taps + sd.tap_off;          // force [2M+1]
    const double* mtap = ftap + 2 * M + 1;           // Fischer-Methfessel [2m+1]
    // Fischer-Methfessel average (Sec. II.A), chi (Eq. (carnstar)) and
    // X = n^2 chi T on nodes i0-2 .. i0+nz+1.  Under the outflow rule a ghost
    // node copies every node field of the nearest interior node, so the
    // average is centred on the clamped node; under the periodic rule the
    // window around the ghost position is the wrapped node's window.
    for (int t = threadIdx.x; t < it.nz + 4; t += blockDim.x) {
        int pos = it.i0 - 2 + t;
        int shift = (sd.bc == EVFDLB_BC_OUTFLOW) ? gidx(pos, sd.nx, sd.bc) - pos : 0;
        const double* nn = s.N + (t - 2 + M + shift);
        double nb = 0.0;
        for (int j = -m; j <= m; ++j) nb = fma(mtap[j + m], nn[j], nb);
        double eta = sd.eta_coef * nb, om = 1.0 - eta;
        double chi = (2.0 - eta) / (2.0 * om * om * om);
        double n = nn[0];
        s.Chi[t] = chi;
        s.X[t] = n * n * chi * s.T[t];
        if (fields_out && t >= 2 && t < it.nz + 2) {
            long long NNf = NN;
            fields_out[4 * NNf + sd.node_off + it.i0 + t - 2] = nb;
        }
    }
    __syncthreads();
    const double inv12 = sd.inv_dx / 12.0;
    const double* S0 = mom + MOM_S0 * NN + sd.node_off;
    const double* S1 = mom + MOM_S1 * NN + sd.node_off;
    const double* S2 = mom + MOM_S2 * NN + sd.node_off;
    const double* S3 = mom + MOM_S3 * NN + sd.node_off;
    const double* G0 = mom + MOM_G0 * NN + sd.node_off;
    const double* G1 = mom + MOM_G1 * NN + sd.node_off;
    for (int t = threadIdx.x; t < it.nz; t += blockDim.x) {
        const int c = t + 2;                         // index in the +-2 arrays
        const int i = it.i0 + t;
        double n = s.N[t + M], u = s.U[c], T = s.T[c];
        // fourth-order central differences (Sec. III)
        double dX = (s.X[c - 2] - 8.0 * s.X[c - 1] + 8.0 * s.X[c + 1] - s.X[c + 2]) * inv12;
        double dT = (s.T[c - 2] - 8.0 * s.T[c - 1] + 8.0 * s.T[c + 1] - s.T[c + 2]) * inv12;
        double dU = (s.U[c - 2] - 8.0 * s.U[c - 1] + 8.0 * s.U[c + 1] - s.U[c + 2]) * inv12;
        double X = s.X[c], chi = s.Chi[c];
        double A = dX / X, B = dT / T;
        // self-consistent force, Eq. (F1), Simpson taps over |j| <= M
        const double* nn = s.N + (t + M);
        double f1 = 0.0;
        for (int j = -M; j <= M; ++j) f1 = fma(ftap[j + M], nn[j], f1);
        // heat flux from the raw sums: q = (S3 - 3u S2 + 3u^2 S1 - u^3 S0)/2 + G1 - u G0
        double q = 0.5 * (S3[i] - 3.0 * u * S2[i] + 3.0 * u * u * S1[i] - u * u * u * S0[i]) + G1[i] - u * G0[i];
        // transport, Eqs. (viscosity), (tau), (prandtl)
        double bn = sd.b * n, x = bn * chi;
        double mu = sd.mu0_coef * sqrt(T) * (1.0 / chi + 0.8 * bn + (4.0 / 25.0) * (1.0 + 12.0 / M_PI) * bn * bn * chi);
        double tau = mu / (n * T * (1.0 + 0.4 * x));
        double Pr = (2.0 / 3.0) * (1.0 + 0.6 * x) * (1.0 + 0.8 * x + (4.0 / 25.0) * (1.0 + 12.0 / M_PI) * x * x) /
                    ((1.0 + 0.4 * x) * (1.0 + 1.2 * x + (9.0 / 25.0) * (1.0 + 32.0 / (9.0 * M_PI)) * x * x));
        double nu = (sd.relax == EVFDLB_RELAX_INV_TAU) ? 1.0 / tau : chi / tau;
        double* sc = s.Sc;
        sc[SC_N * Z + t] = n;
        sc[SC_U * Z + t] = u;
        sc[SC_T * Z + t] = T;
        sc[SC_NU * Z + t] = nu;
        sc[SC_FORCE * Z + t] = f1;
        sc[SC_KQ * Z + t] = (1.0 - Pr) * q;
        sc[SC_K * Z + t] = -x * n;        // -b n^2 chi, the prefactor of J1
        sc[SC_A * Z + t] = A;
        sc[SC_B * Z + t] = B;
        sc[SC_D * Z + t] = dU;
        if (!(n > 0.0) || !(T > 0.0)) {
            atomicOr(err, (finite(n) && finite(T)) ? ERR_NEGATIVE : ERR_NONFINITE);
        } else if (!finite(f1) || !finite(nu) || !finite(q) || !finite(A) || !finite(B)) {
            atomicOr(err, ERR_NONFINITE);
        }
        if (fields_out) {
            long long o = sd.node_off + i;
            double vals[EVFDLB_NFIELDS] = {n, u, T, q, 0.0, chi, f1, mu, tau, Pr, nu, A, B, dU, X, x};
            for (int f = 0; f < EVFDLB_NFIELDS; ++f)
                if (f != 4) fields_out[f * NN + o] = vals[f];
        }
    }
}

// ---------------------------------------------------------------------------
// Phase 3a: Hermite coefficients of nu F^S + J1_F and nu G^S + J1_G.
// With m_l = E[psi_l(u + c)], c ~ N(0, T) (m_0 = 1,
// m_{l+1} = u m_l / sqrt(l+1) + (T-1) sqrt(l/(l+1)) m_{l-1}) and Stein's
// identity E[c h(c)] = T E[h'(c)], the projections of the reduced Shakhov
// equilibria and of the reduced J1 of Sec. II.B are
//   c_l = c0 m_l + c1 sqrt(l) m_{l-1} + c2 sqrt(l(l-1)) m_{l-2}
//         + c3 sqrt(l(l-1)(l-2)) m_{l-3}
// with per-node constants (K = -b n^2 chi, kq = (1-Pr) q):
//   F: c0 = nu n,             c1 = K A T,
//      c2 = 3/5 K D T,        c3 = nu kq/5 + 3/10 K B T^2
//   G: c0 = nu n T + 2/5 K T D,  c1 = 2/5 nu kq + K T^2 (A + 3/5 B),
//      c2 = 3/5 K T^2 D,         c3 = nu kq T/5 + 3/10 K T^3 B
// ---------------------------------------------------------------------------
__device__ void equilibrium_coefficients(const SlabDesc& sd, const WorkItem& it, const Smem& s, int Z,
                                         const double* __restrict__ tables) {
    const int Q = sd.Q;
    TableLayout L(Q);
    const double* tab = tables + sd.tab_off;
    for (int e = threadIdx.x; e < 2 * it.nz; e += blockDim.x) {
        int t = e % it.nz, d = e / it.nz;
        const double* sc = s.Sc;
        double n = sc[SC_N * Z + t], u = sc[SC_U * Z + t], T = sc[SC_T * Z + t];
        double nu = sc[SC_NU * Z + t], kq = sc[SC_KQ * Z + t], K = sc[SC_K * Z + t];
        double A = sc[SC_A * Z + t], B = sc[SC_B * Z + t], D = sc[SC_D * Z + t];
        double c0, c1, c2, c3;
        if (d == 0) {
            c0 = nu * n;
            c1 = K * A * T;
            c2 = 0.6 * K * D * T;
            c3 = 0.2 * nu * kq + 0.3 * K * B * T * T;
        } else {
            c0 = nu * n * T + 0.4 * K * T * D;
            c1 = 0.4 * nu * kq + K * T * T * (A + 0.6 * B);
            c2 = 0.6 * K * T * T * D;
            c3 = 0.2 * nu * kq * T + 0.3 * K * T * T * T * B;
        }
        double m0 = 1.0, m1 = 0.0, m2 = 0.0, m3 = 0.0, Tm1 = T - 1.0;
        double* out = s.C + (size_t)d * Q * Z + t;
        for (int l = 0; l < Q; ++l) {
            double c = c0 * m0;
            c = fma(c1 * tab[L.r1 + l], m1, c);
            c = fma(c2 * tab[L.r2 + l], m2, c);
            c = fma(c3 * tab[L.r3 + l], m3, c);
            out[l * Z] = c;
            double mn = fma(u * tab[L.rinv + l], m0, Tm1 * tab[L.rr + l] * m1);
            m3 = m2;
            m2 = m1;
            m1 = m0;
            m0 = mn;
        }
    }
}

// Phase 3b: analysis a_l = sum_j psi_l(xi_j) h_j, l <= Q-2 (the force needs
// a_0 .. a_{Q-2}; the l = Q-1 term meets psi_Q(xi_k) = 0).
__device__ void analysis(const SlabDesc& sd, const WorkItem& it, const Smem& s, int Z) {
    const int Q = sd.Q, W = Z + 6, nz = it.nz;
    const int per_d = (Q - 1) * nz;
    for (int e = threadIdx.x; e < 2 * per_d; e += blockDim.x) {
        int d = e / per_d, r = e % per_d;
        int l = r / nz, t = r % nz;
        const double* Pl = s.P + l * Q;
        const double* h = s.F + (size_t)d * Q * W + (t + 3);
        double acc = 0.0;
        for (int j = 0; j < Q; ++j) acc = fma(Pl[j], h[j * W], acc);
        s.A[((size_t)d * Q + l) * Z + t] = acc;
    }
}

// WENO-5 (Jiang & Shu) value at the face between v2 and v3, upwind side v0..v2.
// The nonlinear weights omega_r = (d_r / e_r) / sum_s (d_s / e_s),
// e_r = (eps + beta_r)^2, are formed with a single division.
__device__ __forceinline__ double weno5(double v0, double v1, double v2, double v3, double v4, double eps) {
    const double k6 = 1.0 / 6.0, k1312 = 13.0 / 12.0;
    double q0 = (2.0 * v0 - 7.0 * v1 + 11.0 * v2) * k6;
    double q1 = (-v1 + 5.0 * v2 + 2.0 * v3) * k6;
    double q2 = (2.0 * v2 + 5.0 * v3 - v4) * k6;
    double t0 = v0 - 2.0 * v1 + v2, s0 = v0 - 4.0 * v1 + 3.0 * v2;
    double t1 = v1 - 2.0 * v2 + v3, s1 = v1 - v3;
    double t2 = v2 - 2.0 * v3 + v4, s2 = 3.0 * v2 - 4.0 * v3 + v4;
    double e0 = eps + fma(k1312 * t0, t0, 0.25 * s0 * s0);
    double e1 = eps + fma(k1312 * t1, t1, 0.25 * s1 * s1);
    double e2 = eps + fma(k1312 * t2, t2, 0.25 * s2 * s2);
    e0 *= e0;
    e1 *= e1;
    e2 *= e2;
    double a0 = 0.1 * (e1 * e2), a1 = 0.6 * (e0 * e2), a2 = 0.3 * (e0 * e1);
    return fma(a0, q0, fma(a1, q1, a2 * q2)) / (a0 + a1 + a2);
}

// Phase 3c: face values h_{i-1/2} for faces f = 0..nz (face f lies between
// tile nodes f-1 and f), upwind by the sign of xi_k.
__device__ void faces(const SlabDesc& sd, const WorkItem& it, const Smem& s, int Z,
                      const double* __restrict__ tables) {
    const int Q = sd.Q, W = Z + 6, nf = it.nz + 1;
    TableLayout L(Q);
    const double* xi = tables + sd.tab_off + L.xi;
    for (int e = threadIdx.x; e < 2 * Q * nf; e += blockDim.x) {
        int f = e % nf, r = e / nf;
        int k = r % Q, d = r / Q;
        const double* h = s.F + (size_t)(d * Q + k) * W;
        double x = xi[k], v;
        if (x > 0.0) v = weno5(h[f], h[f + 1], h[f + 2], h[f + 3], h[f + 4], sd.weno_eps);
        else if (x < 0.0) v = weno5(h[f + 5], h[f + 4], h[f + 3], h[f + 2], h[f + 1], sd.weno_eps);
        else v = 0.0;
        s.Face[(size_t)(d * Q + k) * (Z + 1) + f] = v;
    }
}

// Phase 4: add the force term F1 sqrt(l) a_{l-1} to the coefficients
// (d/dxi [omega psi_{l-1}] = -sqrt(l) omega psi_l).
__device__ void add_force(const SlabDesc& sd, const WorkItem& it, const Smem& s, int Z,
                          const double* __restrict__ tables) {
    const int Q = sd.Q, nz = it.nz;
    TableLayout L(Q);
    const double* r1 = tables + sd.tab_off + L.r1;
    for (int e = threadIdx.x; e < 2 * (Q - 1) * nz; e += blockDim.x) {
        int t = e % nz, r = e / nz;
        int l = 1 + r % (Q - 1), d = r / (Q - 1);
        double f1 = s.Sc[SC_FORCE * Z + t];
        s.C[((size_t)d * Q + l) * Z + t] =
            fma(f1 * r1[l], s.A[((size_t)d * Q + l - 1) * Z + t], s.C[((size_t)d * Q + l) * Z + t]);
    }
}

// ---------------------------------------------------------------------------
// Kernels
// ---------------------------------------------------------------------------

// mode 0: out = alpha base + beta (src + dt R);  mode 1: out = R.
__global__ void __launch_bounds__(kThreads)
stage_kernel(const SlabDesc* __restrict__ slabs, const WorkItem* __restrict__ items,
             const double* __restrict__ tables, const double* __restrict__ taps,
             const double* __restrict__ src, const double* base, double* out,
             const double* __restrict__ mom_in, double* __restrict__ mom_out,
             long long NF, long long NN, double alpha, double beta, int mode, int Z, unsigned* err) {
    extern __shared__ double smem[];
    const WorkItem it = items[blockIdx.x];
    const SlabDesc sd = slabs[it.slab];
    const int Q = sd.Q, W = Z + 6, nz = it.nz;
    Smem s = carve(smem, Q, Z, sd.M);

    load_node_inputs(sd, it, s, Z, tables, mom_in, NN);
    load_state_tile(sd, it, s, Z, src, NF);
    __syncthreads();
    node_fields(sd, it, s, Z, taps, mom_in, NN, err, nullptr);
    __syncthreads();
    equilibrium_coefficients(sd, it, s, Z, tables);
    analysis(sd, it, s, Z);
    faces(sd, it, s, Z, tables);
    __syncthreads();
    add_force(sd, it, s, Z, tables);
    __syncthreads();

    // Phase 5: synthesis, advection, relaxation and the RK stage.
    TableLayout L(Q);
    const double* xi = tables + sd.tab_off + L.xi;
    const double dt = sd.dt;
    for (int e = threadIdx.x; e < 2 * Q * nz; e += blockDim.x) {
        int t = e % nz, r = e / nz;
        int k = r % Q, d = r / Q;
        const double* Sk = s.S + k * Q;
        const double* c = s.C + (size_t)d * Q * Z + t;
        double syn = 0.0;
        for (int l = 0; l < Q; ++l) syn = fma(Sk[l], c[l * Z], syn);
        const double* fc = s.Face + (size_t)(d * Q + k) * (Z + 1);
        double h = s.F[(size_t)(d * Q + k) * W + t + 3];
        double R = fma(-xi[k] * sd.inv_dx, fc[t + 1] - fc[t], fma(-s.Sc[SC_NU * Z + t], h, syn));
        long long g = d * NF + sd.f_off + (long long)k * sd.nx + it.i0 + t;
        double o;
        if (mode == 1) {
            o = R;
        } else {
            o = beta * fma(dt, R, h);
            if (alpha != 0.0) o = fma(alpha, base[g], o);
        }
        out[g] = o;
        s.F[(size_t)(d * Q + k) * W + t + 3] = o;
    }
    if (mode == 1) return;
    __syncthreads();

    // Phase 6: raw moment sums of the new stage for the next stage's node fields.
    for (int e = threadIdx.x; e < kNumMoments * nz; e += blockDim.x) {
        int t = e % nz, which = e / nz;
        int d = which >= MOM_G0 ? 1 : 0;
        int p = (which >= MOM_G0) ? which - MOM_G0 : which;   // power of xi
        const double* h = s.F + (size_t)d * Q * W + t + 3;
        double acc = 0.0;
        for (int k = 0; k < Q; ++k) {
            double x = xi[k], wgt = (p == 0) ? 1.0 : (p == 1 ? x : (p == 2 ? x * x : x * x * x));
            acc = fma(wgt, h[k * W], acc);
        }
        mom_out[which * NN + sd.node_off + it.i0 + t] = acc;
    }
}

// Projected Maxwellian pair (F_MB, T F_MB) from node fields:
// F_k = sum_l S_kl n m_l(u, T), G_k = T F_k; also writes the raw moment sums.
__global__ void __launch_bounds__(kThreads)
init_kernel(const SlabDesc* __restrict__ slabs, const WorkItem* __restrict__ items,
            const double* __restrict__ tables, const double* __restrict__ n0,
            const double* __restrict__ u0, const double* __restrict__ T0, double* state,
            double* mom, long long NF, long long NN, int Z, unsigned* err) {
    extern __shared__ double smem[];
    const WorkItem it = items[blockIdx.x];
    const SlabDesc sd = slabs[it.slab];
    const int Q = sd.Q, W = Z + 6, nz = it.nz;
    Smem s = carve(smem, Q, Z, sd.M);
    TableLayout L(Q);
    const double* tab = tables + sd.tab_off;
    for (int t = threadIdx.x; t < 2 * Q * Q; t += blockDim.x) s.P[t] = tab[L.P + t];
    for (int t = threadIdx.x; t < nz; t += blockDim.x) {
        long long o = sd.node_off + it.i0 + t;
        double n = n0[o], u = u0[o], T = T0[o];
        if (!(n > 0.0) || !(T > 0.0) || !finite(u))
            atomicOr(err, (finite(n) && finite(T) && finite(u)) ? ERR_NEGATIVE : ERR_NONFINITE);
        s.Sc[SC_T * Z + t] = T;
        double m0 = 1.0, m1 = 0.0, Tm1 = T - 1.0;
        for (int l = 0; l < Q; ++l) {
            s.C[l * Z + t] = n * m0;
            double mn = fma(u * tab[L.rinv + l], m0, Tm1 * tab[L.rr + l] * m1);
            m1 = m0;
            m0 = mn;
        }
    }
    __syncthreads();
    const double* xi = tab + L.xi;
    for (int e = threadIdx.x; e < Q * nz; e += blockDim.x) {
        int t = e % nz, k = e / nz;
        double acc = 0.0;
        for (int l = 0; l < Q; ++l) acc = fma(s.S[k * Q + l], s.C[l * Z + t], acc);
        double gval = s.Sc[SC_T * Z + t] * acc;
        long long g = sd.f_off + (long long)k * sd.nx + it.i0 + t;
        state[g] = acc;
        state[NF + g] = gval;
        s.F[(size_t)k * W + t + 3] = acc;
        s.F[(size_t)(Q + k) * W + t + 3] = gval;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < kNumMoments * nz; e += blockDim.x) {
        int t = e % nz, which = e / nz;
        int d = which >= MOM_G0 ? 1 : 0;
        int p = (which >= MOM_G0) ? which - MOM_G0 : which;
        const double* h = s.F + (size_t)d * Q * W + t + 3;
        double acc = 0.0;
        for (int k = 0; k < Q; ++k) {
            double x = xi[k], wgt = (p == 0) ? 1.0 : (p == 1 ? x : (p == 2 ? x * x : x * x * x));
            acc = fma(wgt, h[k * W], acc);
        }
        mom[which * NN + sd.node_off + it.i0 + t] = acc;
    }
}

// Raw moment sums of an arbitrary state (after set_state).
__global__ void __launch_bounds__(kThreads)
sums_kernel(const SlabDesc* __restrict__ slabs, const WorkItem* __restrict__ items,
            const double* __restrict__ tables, const double* __restrict__ state, double* mom,
            long long NF, long long NN, unsigned* err) {
    const WorkItem it = items[blockIdx.x];
    const SlabDesc sd = slabs[it.slab];
    const int Q = sd.Q;
    TableLayout L(Q);
    const double* xi = tables + sd.tab_off + L.xi;
    for (int e = threadIdx.x; e < kNumMoments * it.nz; e += blockDim.x) {
        int t = e % it.nz, which = e / it.nz;
        int d = which >= MOM_G0 ? 1 : 0;
        int p = (which >= MOM_G0) ? which - MOM_G0 : which;
        const double* h = state + d * NF + sd.f_off + it.i0 + t;
        double acc = 0.0;
        for (int k = 0; k < Q; ++k) {
            double x = xi[k], wgt = (p == 0) ? 1.0 : (p == 1 ? x : (p == 2 ? x * x : x * x * x));
            acc = fma(wgt, h[(long long)k * sd.nx], acc);
        }
        if (!finite(acc)) atomicOr(err, ERR_NONFINITE);
        mom[which * NN + sd.node_off + it.i0 + t] = acc;
    }
}

// Node fields of the current state (diagnostic).
__global__ void __launch_bounds__(kThreads)
fields_kernel(const SlabDesc* __restrict__ slabs, const WorkItem* __restrict__ items,
              const double* __restrict__ tables, const double* __restrict__ taps,
              const double* __restrict__ mom, double* fields, long long NN, int Z, unsigned* err) {
    extern __shared__ double smem[];
    const WorkItem it = items[blockIdx.x];
    const SlabDesc sd = slabs[it.slab];
    Smem s = carve(smem, sd.Q, Z, sd.M);
    load_node_inputs(sd, it, s, Z, tables, mom, NN);
    __syncthreads();
    node_fields(sd, it, s, Z, taps, mom, NN, err, fields);
}

// n, u, T, q per node from the raw sums.
__global__ void moments_kernel(const double* __restrict__ mom, long long NN, double* n, double* u,
                               double* T, double* q) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < NN;
         i += (long long)gridDim.x * blockDim.x) {
        double S0 = mom[MOM_S0 * NN + i], S1 = mom[MOM_S1 * NN + i], S2 = mom[MOM_S2 * NN + i];
        double S3 = mom[MOM_S3 * NN + i], G0 = mom[MOM_G0 * NN + i], G1 = mom[MOM_G1 * NN + i];
        double uu = S1 / S0;
        if (n) n[i] = S0;
        if (u) u[i] = uu;
        if (T) T[i] = (2.0 / 3.0) * ((0.5 * S2 + G0) / S0 - 0.5 * uu * uu);
        if (q) q[i] = 0.5 * (S3 - 3.0 * uu * S2 + 3.0 * uu * uu * S1 - uu * uu * uu * S0) + G1 - uu * G0;
    }
}

// Per-slab totals {mass, momentum, energy, mean-field energy}; one CTA per
// slab, fixed-order tree reduction (deterministic).
__global__ void __launch_bounds__(kThreads)
totals_kernel(const SlabDesc* __restrict__ slabs, const double* __restrict__ taps,
              const double* __restrict__ mom, long long NN, double* out) {
    __shared__ double red[4][kThreads];
    const SlabDesc sd = slabs[blockIdx.x];
    const double* S0 = mom + MOM_S0 * NN + sd.node_off;
    const double* S1 = mom + MOM_S1 * NN + sd.node_off;
    const double* S2 = mom + MOM_S2 * NN + sd.node_off;
    const double* G0 = mom + MOM_G0 * NN + sd.node_off;
    const double* etap = taps + sd.tap_off + 2 * sd.M + 1 + 2 * sd.m + 1;
    double a0 = 0, a1 = 0, a2 = 0, a3 = 0;
    for (int i = threadIdx.x; i < sd.nx; i += blockDim.x) {
        a0 += S0[i];
        a1 += S1[i];
        a2 += 0.5 * S2[i] + G0[i];
        double acc = 0.0;
        for (int j = -sd.M; j <= sd.M; ++j) acc = fma(etap[j + sd.M], S0[gidx(i + j, sd.nx, sd.bc)], acc);
        a3 += 0.5 * S0[i] * acc;
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
    if (threadIdx.x == 0) {
        out[4 * blockIdx.x + 0] = red[0][0] * sd.dx;
        out[4 * blockIdx.x + 1] = red[1][0] * sd.dx;
        out[4 * blockIdx.x + 3] = red[3][0] * sd.dx;
        out[4 * blockIdx.x + 2] = (red[2][0] + red[3][0]) * sd.dx;
    }
}

// ---------------------------------------------------------------------------
// Host-side launch helpers (called from the C-ABI layer).
// ---------------------------------------------------------------------------
size_t stage_smem_bytes(int Q, int Z, int M) { return smem_doubles(Q, Z, M) * sizeof(double); }

cudaError_t configure_kernels(size_t smem_bytes) {
    cudaError_t e = cudaFuncSetAttribute(stage_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(init_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(fields_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
}

// Raises (never lowers) the stage kernel's dynamic shared-memory limit on the
// current device to at least smem_bytes.
cudaError_t ensure_stage_smem(size_t smem_bytes) {
    cudaFuncAttributes a;
    cudaError_t e = cudaFuncGetAttributes(&a, stage_kernel);
    if (e != cudaSuccess) return e;
    if ((size_t)a.maxDynamicSharedSizeBytes >= smem_bytes) return cudaSuccess;
    return cudaFuncSetAttribute(stage_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
}

void launch_stage(int nitems, size_t smem, cudaStream_t st, const SlabDesc* slabs, const WorkItem* items,
                  const double* tables, const double* taps, const double* src, const double* base,
                  double* out, const double* mom_in, double* mom_out, long long NF, long long NN,
                  double alpha, double beta, int mode, int Z, unsigned* err) {
    stage_kernel<<<nitems, kThreads, smem, st>>>(slabs, items, tables, taps, src, base, out, mom_in, mom_out,
                                                 NF, NN, alpha, beta, mode, Z, err);
}

void launch_init(int nitems, size_t smem, cudaStream_t st, const SlabDesc* slabs, const WorkItem* items,
                 const double* tables, const double* n0, const double* u0, const double* T0,
                 double* state, double* mom, long long NF, long long NN, int Z, unsigned* err) {
    init_kernel<<<nitems, kThreads, smem, st>>>(slabs, items, tables, n0, u0, T0, state, mom, NF, NN, Z, err);
}

void launch_sums(int nitems, cudaStream_t st, const SlabDesc* slabs, const WorkItem* items,
                 const double* tables, const double* state, double* mom, long long NF, long long NN,
                 unsigned* err) {
    sums_kernel<<<nitems, kThreads, 0, st>>>(slabs, items, tables, state, mom, NF, NN, err);
}

void launch_fields(int nitems, size_t smem, cudaStream_t st, const SlabDesc* slabs, const WorkItem* items,
                   const double* tables, const double* taps, const double* mom, double* fields,
                   long long NN, int Z, unsigned* err) {
    fields_kernel<<<nitems, kThreads, smem, st>>>(slabs, items, tables, taps, mom, fields, NN, Z, err);
}

void launch_moments(cudaStream_t st, const double* mom, long long NN, double* n, double* u, double* T,
                    double* q) {
    int blocks = (int)((NN + 255) / 256);
    if (blocks > 1024) blocks = 1024;
    moments_kernel<<<blocks, 256, 0, st>>>(mom, NN, n, u, T, q);
}

void launch_totals(int nslabs, cudaStream_t st, const SlabDesc* slabs, const double* taps, const double* mom,
                   long long NN, double* out) {
    totals_kernel<<<nslabs, kThreads, 0, st>>>(slabs, taps, mom, NN, out);
}

}  // namespace evfdlb
