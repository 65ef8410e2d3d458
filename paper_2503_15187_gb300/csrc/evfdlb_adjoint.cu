// evfdlb_adjoint.cu -- discrete adjoint of the EV1 time step (FP64, periodic
// slabs): vector-Jacobian products of the right-hand side L of Eqs. (ev1) and
// (enskog_approx), of the Shu-Osher RK3 stages, and of the projected initial
// state, for the gradient of a loss of the final state with respect to the
// initial fields (n0, u0, T0), the initial distributions and the well depth
// phi_a of Eq. (sutherland) (through the Eq. (F1) force, which is linear in
// phi_a).
//
// One stage of the reverse sweep, given the adjoint ybar of the stage output
// and the stage input u (recomputed from a checkpoint), forms
//   out     = ca ybar + J(u)^T v + cc acc_in,   v = cb dt ybar,
//   acc_out = cacc acc_in + cy ybar,
// where J(u) is the Jacobian of L at u, in two launches:
//   adj_local_kernel  -- per node tile: the velocity-space part of J^T v
//                        (transposed Hermite synthesis and analysis, the
//                        transposed WENO-5 faces, relaxation) and the adjoints
//                        of the node fields that L reads (n, u, T, q, chi, X,
//                        the three gradients and the force F1);
//   adj_moments_kernel-- per node tile: transposed fourth-order differences,
//                        the chain X = n^2 chi T, chi(nbar) of Eq. (carnstar)
//                        (on the tile and a Fischer-Methfessel halo), the
//                        transposed Fischer-Methfessel average and Eq. (F1)
//                        convolution (correlations), the chain from
//                        (n, u, T, q) to the raw moment sums, and their
//                        transpose onto F and G.
// Forward quantities are recomputed from the stage input and its raw moment
// sums with the same device code as the forward kernels.
#include <cuda_runtime.h>
#include <math.h>

#include "evfdlb_device.cuh"

namespace evfdlb {

// per-node adjoints written by adj_local_kernel ([kNumNodeAdj][NN])
enum { AD_N = 0, AD_U, AD_T, AD_Q, AD_CHI, AD_X, AD_DX, AD_DT, AD_DU, AD_F1, kNumNodeAdj };

constexpr int kHaloH = 5;   // state halo of the transposed WENO-5 faces
constexpr int kHaloV = 3;   // halo of v

struct AdjSmem {
    Smem<double> f;   // S, N, U, T, X, Chi, Sc, Scr of the forward layout; f.P holds
                      // the scaled transposed analysis table PT[l][j] = sqrt(l) psi_{l-1}(xi_j)
    double* H;        // state tile [2][Q][Z + 2 kHaloH]
    double* V;        // v tile [2][Q][Z + 2 kHaloV]
    double* Cb;       // cbar_l = sum_k S_kl v_k, [2][Q][Z]
    double* Ha;       // sum_l PT[l][j] cbar_l, [2][Q][Z]
    double* Hw;       // transposed WENO-5 part, [2][Q][Z]
    double* Red;      // per (distribution, node) sums [2][8][Z]
    // f.Mtap [2M+1] (the 2m+1 Fischer-Methfessel taps) and f.Ftap [2M+1]
    // (the Eq. (F1) taps) follow Red, staged once per CTA
};

__host__ __device__ inline size_t adj_smem_doubles(int Q, int Z, int M) {
    return 2 * (size_t)Q * Q + (Z + 2 * M) + 4 * (size_t)(Z + 4) + (size_t)kNumScalars * Z + 2 * (size_t)Z +
           2 * (size_t)Q * (Z + 2 * kHaloH) + 2 * (size_t)Q * (Z + 2 * kHaloV) + 6 * (size_t)Q * Z + 16 * (size_t)Z +
           2 * (size_t)(2 * M + 1);
}

__device__ inline AdjSmem adj_carve(double* base, int Q, int Z, int M) {
    AdjSmem s;
    s.f.P = base;
    s.f.S = s.f.P + Q * Q;
    s.f.N = s.f.S + Q * Q;
    s.f.Nr = s.f.N;
    s.f.U = s.f.N + (Z + 2 * M);
    s.f.T = s.f.U + (Z + 4);
    s.f.X = s.f.T + (Z + 4);
    s.f.Chi = s.f.X + (Z + 4);
    s.f.Sc = s.f.Chi + (Z + 4);
    s.f.Scr = s.f.Sc + kNumScalars * Z;
    s.f.C = s.f.A = s.f.F = s.f.Face = nullptr;
    s.H = s.f.Scr + 2 * Z;
    s.V = s.H + 2 * Q * (Z + 2 * kHaloH);
    s.Cb = s.V + 2 * Q * (Z + 2 * kHaloV);
    s.Ha = s.Cb + 2 * Q * Z;
    s.Hw = s.Ha + 2 * Q * Z;
    s.Red = s.Hw + 2 * Q * Z;
    s.f.Mtap = s.Red + 16 * Z;
    s.f.Ftap = s.f.Mtap + (2 * M + 1);
    return s;
}

// Gradient of the WENO-5 face value Phi(v0..v4) (upwind side v0..v2), times
// pb: g_r = pb dPhi/dv_r.  Phi is taken in the difference form of the forward
// faces: with d_i = v_{i+1} - v_i, t_0 = d1 - d0, t_1 = d2 - d1, t_2 = d3 - d2,
// s_0 = 3 d1 - d0, s_1 = d1 + d2, s_2 = d3 - 3 d2,
//   e_r = s_r^2 + 13/3 t_r^2 + 4 eps   (= 4 (eps + beta_r)),
//   a_0 = e_1^2 e_2^2, a_1 = e_0^2 e_2^2, a_2 = e_0^2 e_1^2,
//   c_0 = (5 d1 - 2 d0)/60, c_1 = (d1 + 2 d2)/10, c_2 = (4 d2 - d3)/20,
//   Phi = v2 + (sum a_r c_r) / (0.1 a_0 + 0.6 a_1 + 0.3 a_2),
// differentiated in reverse order (one division per face).
__device__ __forceinline__ void weno5_grad(double v0, double v1, double v2, double v3, double v4, double eps,
                                           double pb, double g[5]) {
    const double d0 = v1 - v0, d1 = v2 - v1, d2 = v3 - v2, d3 = v4 - v3;
    const double t0 = d1 - d0, t1 = d2 - d1, t2 = d3 - d2;
    const double s0 = fma(3.0, d1, -d0), s1 = d1 + d2, s2 = fma(-3.0, d2, d3);
    const double e4 = 4.0 * eps, k133 = 13.0 / 3.0;
    const double e0 = fma(s0, s0, fma(k133 * t0, t0, e4));
    const double e1 = fma(s1, s1, fma(k133 * t1, t1, e4));
    const double e2 = fma(s2, s2, fma(k133 * t2, t2, e4));
    const double E0 = e0 * e0, E1 = e1 * e1, E2 = e2 * e2;
    const double a0 = E1 * E2, a1 = E0 * E2, a2 = E0 * E1;
    const double c0 = fma(5.0 / 60.0, d1, (-2.0 / 60.0) * d0);
    const double c1 = fma(0.2, d2, 0.1 * d1);
    const double c2 = fma(0.2, d2, -0.05 * d3);
    const double num = fma(a0, c0, fma(a1, c1, a2 * c2));
    const double den = fma(0.1, a0, fma(0.6, a1, 0.3 * a2));
    const double iden = div_nr(1.0, den);
    const double R = pb * iden;
    const double psi = num * iden;             // Phi - v2
    // adjoints (all times pb)
    const double gc0 = a0 * R, gc1 = a1 * R, gc2 = a2 * R;
    const double gA0 = R * fma(-0.1, psi, c0), gA1 = R * fma(-0.6, psi, c1), gA2 = R * fma(-0.3, psi, c2);
    const double gE0 = fma(gA1, E2, gA2 * E1), gE1 = fma(gA0, E2, gA2 * E0), gE2 = fma(gA0, E1, gA1 * E0);
    const double ge0 = 2.0 * e0 * gE0, ge1 = 2.0 * e1 * gE1, ge2 = 2.0 * e2 * gE2;
    const double gs0 = 2.0 * s0 * ge0, gs1 = 2.0 * s1 * ge1, gs2 = 2.0 * s2 * ge2;
    const double k263 = 26.0 / 3.0;
    const double gt0 = k263 * t0 * ge0, gt1 = k263 * t1 * ge1, gt2 = k263 * t2 * ge2;
    const double gd0 = -gs0 - gt0 + (-2.0 / 60.0) * gc0;
    const double gd1 = fma(3.0, gs0, gs1) + gt0 - gt1 + fma(5.0 / 60.0, gc0, 0.1 * gc1);
    const double gd2 = fma(-3.0, gs2, gs1) + gt1 - gt2 + fma(0.2, gc1, 0.2 * gc2);
    const double gd3 = gs2 + gt2 - 0.05 * gc2;
    g[0] = -gd0;
    g[1] = gd0 - gd1;
    g[2] = pb + gd1 - gd2;
    g[3] = gd2 - gd3;
    g[4] = gd3;
}

__global__ void __launch_bounds__(kThreads)
adj_local_kernel(const SlabDesc* __restrict__ slabs, const WorkItem* __restrict__ items,
                 const double* __restrict__ tables, const double* __restrict__ taps,
                 const double* __restrict__ src, const double* __restrict__ mom, const double* __restrict__ ybar,
                 const double* acc_in, double* acc_out, double* out, double* __restrict__ nadj,
                 double* __restrict__ phis, long long NF, long long NN, double ca, double cb, int use_dt,
                 double cc, double cacc, double cy, int Z, unsigned* err) {
    extern __shared__ double smem[];
    const WorkItem it = items[blockIdx.x];
    const SlabDesc sd = slabs[it.slab];
    const int Q = sd.Q, nz = it.nz, nx = sd.nx, bc = sd.bc;
    const int WH = Z + 2 * kHaloH, WV = Z + 2 * kHaloV;
    AdjSmem s = adj_carve(smem, Q, Z, sd.M);
    TableLayout L(Q);
    const double* tab = tables + sd.tab_off;
    const double* xi = tab + L.xi;
    const double* r1 = tab + L.r1;
    const double* r2 = tab + L.r2;
    const double* r3 = tab + L.r3;

    // phase 0: tables and node inputs, the state tile (+-5) and v (+-3)
    load_node_inputs<double>(sd, it, s.f, Z, tables, mom, NN);
    for (int e = threadIdx.x; e < 2 * Q * (nz + 2 * kHaloH); e += blockDim.x) {
        int c = e % (nz + 2 * kHaloH), r = e / (nz + 2 * kHaloH);
        int k = r % Q, d = r / Q;
        s.H[r * WH + c] = src[d * NF + sd.f_off + (long long)k * nx + gidx(it.i0 - kHaloH + c, nx, bc)];
    }
    const double vscale = cb * (use_dt ? sd.dt : 1.0);
    for (int e = threadIdx.x; e < 2 * Q * (nz + 2 * kHaloV); e += blockDim.x) {
        int c = e % (nz + 2 * kHaloV), r = e / (nz + 2 * kHaloV);
        int k = r % Q, d = r / Q;
        s.V[r * WV + c] = vscale * ybar[d * NF + sd.f_off + (long long)k * nx + gidx(it.i0 - kHaloV + c, nx, bc)];
    }
    for (int j = threadIdx.x; j < 2 * sd.M + 1; j += blockDim.x) s.f.Ftap[j] = taps[sd.tap_off + j];
    for (int j = threadIdx.x; j < 2 * sd.m + 1; j += blockDim.x) s.f.Mtap[j] = taps[sd.tap_off + 2 * sd.M + 1 + j];
    __syncthreads();
    // Warp 0 recomputes the node fields while warps 1-7 run phases 1 and 1b,
    // which need only v and the tables (named barrier 1 joins warps 1-7).
    const bool node_warp = threadIdx.x < 32;
    const int tid7 = threadIdx.x - 32, nth7 = blockDim.x - 32;
    if (node_warp) {
        node_fields_pass1<double>(sd, it, s.f, s.f.Mtap, NN, nullptr, threadIdx.x, 32);
        __syncwarp();
        node_fields_pass2<double>(sd, it, s.f, Z, s.f.Ftap, mom, NN, err, nullptr, threadIdx.x, 32);
    } else {
        // the analysis table is replaced by PT[l][j] = sqrt(l) psi_{l-1}(xi_j) (l >= 1),
        // so that sum_l PT[l][j] cbar_l is the transposed analysis of the force term
        for (int e = tid7; e < Q * Q; e += nth7) {
            int l = e / Q, j = e % Q;
            s.f.P[e] = (l == 0) ? 0.0 : r1[l] * tab[L.P + (l - 1) * Q + j];
        }

        // phase 1: transposed synthesis cbar_l = sum_k S_kl v_k
        for (int e = tid7; e < 2 * Q * nz; e += nth7) {
            int t = e % nz, r = e / nz;
            int l = r % Q, d = r / Q;
            const double* v = s.V + (size_t)d * Q * WV + t + kHaloV;
            double acc = 0.0;
            for (int k = 0; k < Q; ++k) acc = fma(s.f.S[k * Q + l], v[k * WV], acc);
            s.Cb[((size_t)d * Q + l) * Z + t] = acc;
        }
        asm volatile("bar.sync 1, %0;" ::"r"(nth7) : "memory");
        // phase 1b: Ha_j = sum_l sqrt(l) psi_{l-1}(xi_j) cbar_l, the transposed analysis
        // of the force term c_l += F1 sqrt(l) a_{l-1} (times F1 in phase 4); with
        // a_{l-1} = sum_j psi_{l-1}(xi_j) h_j it also gives F1b = sum_j h_j Ha_j.
        for (int e = tid7; e < 2 * Q * nz; e += nth7) {
            int t = e % nz, r = e / nz;
            int j = r % Q, d = r / Q;
            const double* cbar = s.Cb + (size_t)d * Q * Z + t;
            double acc = 0.0;
            for (int l = 1; l < Q; ++l) acc = fma(s.f.P[l * Q + j], cbar[l * Z], acc);
            s.Ha[(size_t)r * Z + t] = acc;
        }
    }
    __syncthreads();

    // Warp 0 runs phases 2 and 3a (per node) while warps 1-7 run phase 3b.
    if (node_warp) {

        // phase 2: per (distribution, node): adjoints of the coefficient
        // constants c0..c3 (c_l = sum_r c_r sqrt(l!/(l-r)!) m_{l-r}), of u and T
        // through m_l (dm_l/du = sqrt(l) m_{l-1}, dm_l/dT = sqrt(l(l-1)) m_{l-2}/2,
        // so dc_l/du = sqrt(l) c_{l-1}, dc_l/dT = sqrt(l(l-1)) c_{l-2}/2), of F1
        // (c_l += F1 sqrt(l) a_{l-1}) and of nu (the -nu h term).
        for (int e = threadIdx.x; e < 2 * nz; e += 32) {
            int t = e % nz, d = e / nz;
            const double* sc = s.f.Sc;
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
            const double* cbar = s.Cb + (size_t)d * Q * Z + t;
            double m0 = 1.0, m1 = 0.0, m2 = 0.0, m3 = 0.0, Tm1 = T - 1.0;
            double cm1 = 0.0, cm2 = 0.0;      // c_{l-1}, c_{l-2}
            double b0 = 0, b1 = 0, b2 = 0, b3 = 0, ub = 0, Tb = 0, fb = 0;
            for (int l = 0; l < Q; ++l) {
                double cl = cbar[l * Z];
                double w1 = r1[l] * m1, w2 = r2[l] * m2, w3 = r3[l] * m3;
                b0 = fma(cl, m0, b0);
                b1 = fma(cl, w1, b1);
                b2 = fma(cl, w2, b2);
                b3 = fma(cl, w3, b3);
                ub = fma(cl * r1[l], cm1, ub);
                Tb = fma(cl * 0.5 * r2[l], cm2, Tb);
                double c = c0 * m0 + c1 * w1 + c2 * w2 + c3 * w3;
                cm2 = cm1;
                cm1 = c;
                double mn = fma(u * tab[L.rinv + l], m0, Tm1 * tab[L.rr + l] * m1);
                m3 = m2;
                m2 = m1;
                m1 = m0;
                m0 = mn;
            }
            double nb = 0.0;
            const double* h = s.H + (size_t)d * Q * WH + t + kHaloH;
            const double* v = s.V + (size_t)d * Q * WV + t + kHaloV;
            const double* ha = s.Ha + (size_t)d * Q * Z + t;
            for (int k = 0; k < Q; ++k) {
                nb = fma(-h[k * WH], v[k * WV], nb);
                fb = fma(h[k * WH], ha[k * Z], fb);
            }
            double* red = s.Red + (size_t)d * 8 * Z + t;
            red[0] = b0;
            red[Z] = b1;
            red[2 * Z] = b2;
            red[3 * Z] = b3;
            red[4 * Z] = ub;
            red[5 * Z] = Tb;
            red[6 * Z] = fb;
            red[7 * Z] = nb;
        }
        __syncwarp();

        // phase 3a: per node, the chain through the coefficient constants, the
        // transport coefficients of Eqs. (viscosity), (tau), (prandtl), and the
        // gradients A = dX/X, B = dT/T, D = du.
        for (int t = threadIdx.x; t < nz; t += 32) {
            const double* sc = s.f.Sc;
            double n = sc[SC_N * Z + t], u = sc[SC_U * Z + t], T = sc[SC_T * Z + t];
            double nu = sc[SC_NU * Z + t], kq = sc[SC_KQ * Z + t], K = sc[SC_K * Z + t];
            double A = sc[SC_A * Z + t], B = sc[SC_B * Z + t], D = sc[SC_D * Z + t];
            double F1 = sc[SC_FORCE * Z + t];
            const double* rF = s.Red + t;
            const double* rG = s.Red + 8 * Z + t;
            double cF0 = rF[0], cF1 = rF[Z], cF2 = rF[2 * Z], cF3 = rF[3 * Z];
            double cG0 = rG[0], cG1 = rG[Z], cG2 = rG[2 * Z], cG3 = rG[3 * Z];
            double ub = rF[4 * Z] + rG[4 * Z];
            double Tb = rF[5 * Z] + rG[5 * Z];
            double F1b = rF[6 * Z] + rG[6 * Z];
            double nub = rF[7 * Z] + rG[7 * Z];
            double nb = 0, Kb = 0, kqb = 0, Ab = 0, Bb = 0, Db = 0, chib = 0, xb = 0, qb = 0;
            // F: c0 = nu n, c1 = K A T, c2 = 3/5 K D T, c3 = nu kq/5 + 3/10 K B T^2
            nub += cF0 * n;
            nb += cF0 * nu;
            Kb += cF1 * A * T;
            Ab += cF1 * K * T;
            Tb += cF1 * K * A;
            Kb += 0.6 * cF2 * D * T;
            Db += 0.6 * cF2 * K * T;
            Tb += 0.6 * cF2 * K * D;
            nub += 0.2 * cF3 * kq;
            kqb += 0.2 * cF3 * nu;
            Kb += 0.3 * cF3 * B * T * T;
            Bb += 0.3 * cF3 * K * T * T;
            Tb += 0.6 * cF3 * K * B * T;
            // G: c0 = nu n T + 2/5 K T D, c1 = 2/5 nu kq + K T^2 (A + 3/5 B),
            //    c2 = 3/5 K T^2 D, c3 = nu kq T/5 + 3/10 K T^3 B
            nub += cG0 * n * T;
            nb += cG0 * nu * T;
            Tb += cG0 * (nu * n + 0.4 * K * D);
            Kb += 0.4 * cG0 * T * D;
            Db += 0.4 * cG0 * K * T;
            nub += 0.4 * cG1 * kq;
            kqb += 0.4 * cG1 * nu;
            Kb += cG1 * T * T * (A + 0.6 * B);
            Tb += 2.0 * cG1 * K * T * (A + 0.6 * B);
            Ab += cG1 * K * T * T;
            Bb += 0.6 * cG1 * K * T * T;
            Kb += 0.6 * cG2 * T * T * D;
            Tb += 1.2 * cG2 * K * T * D;
            Db += 0.6 * cG2 * K * T * T;
            nub += 0.2 * cG3 * kq * T;
            kqb += 0.2 * cG3 * nu * T;
            Tb += cG3 * (0.2 * nu * kq + 0.9 * K * T * T * B);
            Kb += 0.3 * cG3 * T * T * T * B;
            Bb += 0.3 * cG3 * K * T * T * T;
            // transport (recomputed as in node_fields)
            double chi = s.f.Chi[t + 2], X = s.f.X[t + 2];
            double bn = sd.b * n, x = bn * chi;
            const double k1 = (4.0 / 25.0) * (1.0 + 12.0 / M_PI), k2 = (9.0 / 25.0) * (1.0 + 32.0 / (9.0 * M_PI));
            double sqT = sqrt(T);
            double gmu = 1.0 / chi + 0.8 * bn + k1 * bn * bn * chi;
            double mu = sd.mu0_coef * sqT * gmu;
            double den = 1.0 + 0.4 * x;
            double tau = mu / (n * T * den);
            double N1 = 1.0 + 0.6 * x, N2 = 1.0 + 0.8 * x + k1 * x * x, D1 = den, D2 = 1.0 + 1.2 * x + k2 * x * x;
            double Pr = (2.0 / 3.0) * N1 * N2 / (D1 * D2);
            // q from the raw sums (as node_fields forms it)
            long long o = sd.node_off + it.i0 + t;
            double S0 = mom[MOM_S0 * NN + o], S1 = mom[MOM_S1 * NN + o], S2 = mom[MOM_S2 * NN + o];
            double S3 = mom[MOM_S3 * NN + o], G0 = mom[MOM_G0 * NN + o], G1 = mom[MOM_G1 * NN + o];
            double q = 0.5 * (S3 - 3.0 * u * S2 + 3.0 * u * u * S1 - u * u * u * S0) + G1 - u * G0;
            // K = -b n^2 chi
            nb += -2.0 * x * Kb;
            chib += -bn * n * Kb;
            // kq = (1 - Pr) q
            qb += kqb * (1.0 - Pr);
            double Prb = -kqb * q;
            // nu = 1/tau or chi/tau
            double taub;
            if (sd.relax == EVFDLB_RELAX_INV_TAU) {
                taub = -nub / (tau * tau);
            } else {
                chib += nub / tau;
                taub = -nub * chi / (tau * tau);
            }
            // tau = mu / (n T (1 + 2x/5))
            double mub = taub / (n * T * den);
            nb += -taub * tau / n;
            Tb += -taub * tau / T;
            xb += -taub * tau * 0.4 / den;
            // Pr(x)
            xb += Prb * Pr * (0.6 / N1 + (0.8 + 2.0 * k1 * x) / N2 - 0.4 / D1 - (1.2 + 2.0 * k2 * x) / D2);
            // mu = mu0 sqrt(T) (1/chi + 4/5 b n + k1 b^2 n^2 chi)
            Tb += mub * mu / (2.0 * T);
            nb += mub * sd.mu0_coef * sqT * (0.8 * sd.b + 2.0 * k1 * sd.b * bn * chi);
            chib += mub * sd.mu0_coef * sqT * (-1.0 / (chi * chi) + k1 * bn * bn);
            // x = b n chi
            nb += xb * sd.b * chi;
            chib += xb * bn;
            // gradients
            double dXb = Ab / X;
            double Xb = -Ab * A / X;
            double dTb = Bb / T;
            Tb += -Bb * B / T;
            double* na = nadj + sd.node_off + it.i0 + t;
            na[AD_N * NN] = nb;
            na[AD_U * NN] = ub;
            na[AD_T * NN] = Tb;
            na[AD_Q * NN] = qb;
            na[AD_CHI * NN] = chib;
            na[AD_X * NN] = Xb;
            na[AD_DX * NN] = dXb;
            na[AD_DT * NN] = dTb;
            na[AD_DU * NN] = Db;
            na[AD_F1 * NN] = F1b;
            phis[o] += F1b * F1;
        }

        // phase 3b: transposed WENO-5 faces.  A velocity row is cut into chunks of
        // up to 28 tile nodes; a chunk's cn + 4 faces occupy a segment of cn + 4
        // consecutive lanes (one face per lane), and a warp carries as many
        // segments (rows) as fit in 32 lanes.  Each lane forms the five
        // derivatives of its face value times the face adjoint, ordered so that
        // the node at segment lane L' collects g'[s] from segment lane L' + s,
        // s = 0..4 (the five faces that read it).
    } else {
        const int warp = threadIdx.x / 32 - 1, lane = threadIdx.x % 32, nwarps = blockDim.x / 32 - 1;
        const double rdz = sd.inv_dx, eps = sd.weno_eps;
        const int nchunk = (nz + 27) / 28;
        const int cmax = min(28, nz), seg = cmax + 4;
        const int per_warp = 32 / seg;                 // segments per warp
        const int nseg = 2 * Q * nchunk;               // (row, chunk) pairs
        const int sub = lane / seg, sl = lane % seg;
        for (int base = warp * per_warp; base < nseg; base += nwarps * per_warp) {
            const int sid = base + sub;
            const bool active = (sub < per_warp) && (sid < nseg);
            double g[5] = {0, 0, 0, 0, 0};
            int row = 0, c0 = 0, cn = 0;
            double x = 0.0;
            if (active) {
                row = sid / nchunk;
                c0 = (sid % nchunk) * 28;
                cn = min(28, nz - c0);
                x = xi[row % Q];
                const double* h = s.H + (size_t)row * WH + kHaloH;   // h[i], i tile-relative
                const double* v = s.V + (size_t)row * WV + kHaloV;
                if (x != 0.0 && sl < cn + 4) {
                    double gg[5];
                    if (x > 0.0) {
                        int f = c0 - 1 + sl;                     // face between nodes f-1 and f
                        double pb = x * rdz * (v[f] - v[f - 1]);
                        weno5_grad(h[f - 3], h[f - 2], h[f - 1], h[f], h[f + 1], eps, pb, gg);
                        g[0] = gg[4]; g[1] = gg[3]; g[2] = gg[2]; g[3] = gg[1]; g[4] = gg[0];
                    } else {
                        int f = c0 - 2 + sl;
                        double pb = x * rdz * (v[f] - v[f - 1]);
                        weno5_grad(h[f + 2], h[f + 1], h[f], h[f - 1], h[f - 2], eps, pb, gg);
                        g[0] = gg[0]; g[1] = gg[1]; g[2] = gg[2]; g[3] = gg[3]; g[4] = gg[4];
                    }
                }
            }
            const int src = min(lane, 27);               // keeps src + 4 <= 31
            double acc = __shfl_sync(0xffffffffu, g[0], src);
            acc += __shfl_sync(0xffffffffu, g[1], src + 1);
            acc += __shfl_sync(0xffffffffu, g[2], src + 2);
            acc += __shfl_sync(0xffffffffu, g[3], src + 3);
            acc += __shfl_sync(0xffffffffu, g[4], src + 4);
            if (active && sl < cn) s.Hw[(size_t)row * Z + c0 + sl] = (x != 0.0) ? acc : 0.0;
        }
    }
    __syncthreads();

    // phase 4: the distribution-local adjoint and the RK-stage combination
    for (int e = threadIdx.x; e < 2 * Q * nz; e += blockDim.x) {
        int t = e % nz, r = e / nz;
        int j = r % Q, d = r / Q;
        double F1 = s.f.Sc[SC_FORCE * Z + t], nu = s.f.Sc[SC_NU * Z + t];
        double vv = s.V[(size_t)r * WV + t + kHaloV];
        double val = fma(F1, s.Ha[(size_t)r * Z + t], fma(-nu, vv, s.Hw[(size_t)r * Z + t]));
        long long g = d * NF + sd.f_off + (long long)j * nx + it.i0 + t;
        double yb = ybar[g];
        double o = fma(ca, yb, val);
        if (cc != 0.0) o = fma(cc, acc_in[g], o);
        if (acc_out) acc_out[g] = (cacc != 0.0 ? cacc * acc_in[g] : 0.0) + cy * yb;
        out[g] = o;
    }
}

// Per node tile: transposed fourth-order differences of X, T, u, the chain
// X = n^2 chi T, chi = chi(eta), eta = pi sigma^3 nbar / 6 (Eq. (carnstar)) on
// the tile and its Fischer-Methfessel halo, the transposed Fischer-Methfessel
// average and Eq. (F1) convolution (correlations with the same taps), the
// chain (n, u, T, q) <- raw sums, and
// out_{F,k} += S0b + xi S1b + xi^2 S2b + xi^3 S3b, out_{G,k} += G0b + xi G1b.
__host__ __device__ inline size_t adj_moments_smem_doubles(int Z, int m, int M) {
    return 5 * (size_t)(Z + 2 * m) + (size_t)kNumMoments * Z + (size_t)(Z + 4 * m) + (size_t)(Z + 2 * M) +
           (size_t)(Z + 2 * m + 4) + 2 * (size_t)(Z + 4) + (size_t)(2 * M + 1) + (size_t)(2 * m + 1);
}

__global__ void __launch_bounds__(kThreads)
adj_moments_kernel(const SlabDesc* __restrict__ slabs, const WorkItem* __restrict__ items,
                   const double* __restrict__ tables, const double* __restrict__ taps,
                   const double* __restrict__ mom, const double* __restrict__ nadj, double* out, long long NF,
                   long long NN, int Z) {
    extern __shared__ double sm[];
    const WorkItem it = items[blockIdx.x];
    const SlabDesc sd = slabs[it.slab];
    const int nx = sd.nx, bc = sd.bc, M = sd.M, m = sd.m, Q = sd.Q, nz = it.nz;
    const int HW = Z + 2 * m;
    double* sXb = sm;              // X adjoint on [i0 - m, i0 + nz + m)
    double* sNb = sXb + HW;        // nbar adjoint (source of the FM correlation)
    double* sn = sNb + HW;         // n, T, chi on the same nodes
    double* sT = sn + HW;
    double* schi = sT + HW;
    double* sb = schi + HW;        // [kNumMoments][Z] raw-sum adjoints of the tile
    // inputs read by the tap loops, staged once (all threads, coalesced):
    double* sS0 = sb + kNumMoments * Z;    // S0 on [i0 - 2m, i0 + nz + 2m)
    double* sF1 = sS0 + (Z + 4 * m);       // force adjoint on [i0 - M, i0 + nz + M)
    double* sDX = sF1 + (Z + 2 * M);       // X-gradient adjoint on [i0 - m - 2, i0 + nz + m + 2)
    double* sDU = sDX + (Z + 2 * m + 4);   // u- and T-gradient adjoints on [i0 - 2, i0 + nz + 2)
    double* sDT = sDU + (Z + 4);
    double* ftap = sDT + (Z + 4);          // Eq. (F1) taps [2M+1] and FM taps [2m+1]
    double* mtap = ftap + (2 * M + 1);
    const double inv12 = sd.inv_dx / 12.0;
    const double* S0 = mom + MOM_S0 * NN + sd.node_off;
    const double* S1 = mom + MOM_S1 * NN + sd.node_off;
    const double* S2 = mom + MOM_S2 * NN + sd.node_off;
    const double* G0 = mom + MOM_G0 * NN + sd.node_off;
    const double* gF1 = nadj + AD_F1 * NN + sd.node_off;
    const double* gDX = nadj + AD_DX * NN + sd.node_off;
    const double* gDU = nadj + AD_DU * NN + sd.node_off;
    const double* gDT = nadj + AD_DT * NN + sd.node_off;
    for (int c = threadIdx.x; c < nz + 4 * m; c += blockDim.x) sS0[c] = S0[gidx(it.i0 - 2 * m + c, nx, bc)];
    for (int c = threadIdx.x; c < nz + 2 * M; c += blockDim.x) sF1[c] = gF1[gidx(it.i0 - M + c, nx, bc)];
    for (int c = threadIdx.x; c < nz + 2 * m + 4; c += blockDim.x) sDX[c] = gDX[gidx(it.i0 - m - 2 + c, nx, bc)];
    for (int c = threadIdx.x; c < nz + 4; c += blockDim.x) {
        const int i = gidx(it.i0 - 2 + c, nx, bc);
        sDU[c] = gDU[i];
        sDT[c] = gDT[i];
    }
    for (int j = threadIdx.x; j < 2 * M + 1; j += blockDim.x) ftap[j] = taps[sd.tap_off + j];
    for (int j = threadIdx.x; j < 2 * m + 1; j += blockDim.x) mtap[j] = taps[sd.tap_off + 2 * M + 1 + j];
    __syncthreads();
    // transposed fourth-order difference at staged position p (value at p)
    auto d4t = [&](const double* g, int p) { return (g[p + 2] - 8.0 * g[p + 1] + 8.0 * g[p - 1] - g[p - 2]) * inv12; };
    for (int c = threadIdx.x; c < nz + 2 * m; c += blockDim.x) {
        const int i = gidx(it.i0 - m + c, nx, bc);
        double n = S0[i], u = S1[i] / n;
        double T = (2.0 / 3.0) * ((0.5 * S2[i] + G0[i]) / n - 0.5 * u * u);
        double nbF = 0.0;
        const double* s0c = sS0 + c + m;               // S0 at node i0 - m + c
        for (int j = -m; j <= m; ++j) nbF = fma(mtap[j + m], s0c[j], nbF);
        double eta = sd.eta_coef * nbF, om = 1.0 - eta;
        double chi = (2.0 - eta) / (2.0 * om * om * om);
        long long o = sd.node_off + i;
        double Xb = nadj[AD_X * NN + o] + d4t(sDX, c + 2);
        double chib = nadj[AD_CHI * NN + o] + Xb * n * n * T;
        double dchi = (5.0 - 2.0 * eta) / (2.0 * om * om * om * om);
        sXb[c] = Xb;
        sNb[c] = chib * dchi * sd.eta_coef;
        sn[c] = n;
        sT[c] = T;
        schi[c] = chi;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < nz; t += blockDim.x) {
        const int i = it.i0 + t, c = t + m;
        long long o = sd.node_off + i;
        double n = sn[c], T = sT[c], chi = schi[c], Xb = sXb[c];
        double nb = nadj[AD_N * NN + o] + Xb * 2.0 * n * chi * T;
        for (int j = -m; j <= m; ++j) nb = fma(mtap[j + m], sNb[c - j], nb);
        const double* f1c = sF1 + t + M;               // force adjoint at node i
        for (int j = -M; j <= M; ++j) nb = fma(ftap[j + M], f1c[-j], nb);
        double ub = nadj[AD_U * NN + o] + d4t(sDU, t + 2);
        double Tb = nadj[AD_T * NN + o] + d4t(sDT, t + 2) + Xb * n * n * chi;
        double qb = nadj[AD_Q * NN + o];
        double S0v = S0[i], S1v = S1[i], S2v = S2[i], G0v = G0[i];
        double u = S1v / n;
        double E = (0.5 * S2v + G0v) / n;
        // q = (S3 - 3u S2 + 3u^2 S1 - u^3 S0)/2 + G1 - u G0
        double S3b = 0.5 * qb, S2b = -1.5 * u * qb, S1b = 1.5 * u * u * qb, S0b = -0.5 * u * u * u * qb;
        double G1b = qb, G0b = -u * qb;
        ub += qb * (-1.5 * S2v + 3.0 * u * S1v - 1.5 * u * u * S0v - G0v);
        // T = (2/3)(E - u^2/2), E = (S2/2 + G0)/n
        double Eb = (2.0 / 3.0) * Tb;
        ub += -(2.0 / 3.0) * u * Tb;
        S2b += Eb / (2.0 * n);
        G0b += Eb / n;
        nb += -Eb * E / n;
        // u = S1/n
        S1b += ub / n;
        nb += -ub * u / n;
        S0b += nb;
        sb[MOM_S0 * Z + t] = S0b;
        sb[MOM_S1 * Z + t] = S1b;
        sb[MOM_S2 * Z + t] = S2b;
        sb[MOM_S3 * Z + t] = S3b;
        sb[MOM_G0 * Z + t] = G0b;
        sb[MOM_G1 * Z + t] = G1b;
    }
    __syncthreads();
    TableLayout L(Q);
    const double* xi = tables + sd.tab_off + L.xi;
    for (int e = threadIdx.x; e < 2 * Q * nz; e += blockDim.x) {
        int t = e % nz, r = e / nz;
        int k = r % Q, d = r / Q;
        double x = xi[k];
        double add = (d == 0) ? sb[MOM_S0 * Z + t] + x * (sb[MOM_S1 * Z + t] + x * (sb[MOM_S2 * Z + t] + x * sb[MOM_S3 * Z + t]))
                              : sb[MOM_G0 * Z + t] + x * sb[MOM_G1 * Z + t];
        out[d * NF + sd.f_off + (long long)k * nx + it.i0 + t] += add;
    }
}

// Adjoint of the projected initial state F_k = sum_l S_kl n m_l(u, T),
// G_k = T F_k: per node, with W_k = Fb_k + T Gb_k,
//   nb = sum_k W_k F_k / n,  ub = n sum_l (S^T W)_l sqrt(l) m_{l-1},
//   Tb = sum_k Gb_k F_k + n sum_l (S^T W)_l sqrt(l(l-1)) m_{l-2} / 2.
__global__ void __launch_bounds__(kThreads)
adj_init_kernel(const SlabDesc* __restrict__ slabs, const WorkItem* __restrict__ items,
                const double* __restrict__ tables, const double* __restrict__ init_fields,
                const double* __restrict__ lam, double* dn0, double* du0, double* dT0, long long NF, long long NN) {
    const WorkItem it = items[blockIdx.x];
    const SlabDesc sd = slabs[it.slab];
    const int Q = sd.Q, nx = sd.nx;
    TableLayout L(Q);
    const double* tab = tables + sd.tab_off;
    for (int t = threadIdx.x; t < it.nz; t += blockDim.x) {
        const int i = it.i0 + t;
        long long o = sd.node_off + i;
        double n = init_fields[o], u = init_fields[NN + o], T = init_fields[2 * NN + o];
        double m0 = 1.0, m1 = 0.0, m2 = 0.0, Tm1 = T - 1.0;
        double nb = 0.0, ub = 0.0, Tb1 = 0.0, Tb2 = 0.0;
        for (int l = 0; l < Q; ++l) {
            double wl = 0.0, gl = 0.0;
            for (int k = 0; k < Q; ++k) {
                long long g = sd.f_off + (long long)k * nx + i;
                double Fb = lam[g], Gb = lam[NF + g];
                double Skl = tab[L.S + k * Q + l];
                wl = fma(Skl, fma(T, Gb, Fb), wl);
                gl = fma(Skl, Gb, gl);
            }
            nb = fma(wl, m0, nb);
            ub = fma(wl * tab[L.r1 + l], m1, ub);
            Tb1 = fma(gl, m0, Tb1);
            Tb2 = fma(wl * 0.5 * tab[L.r2 + l], m2, Tb2);
            double mn = fma(u * tab[L.rinv + l], m0, Tm1 * tab[L.rr + l] * m1);
            m2 = m1;
            m1 = m0;
            m0 = mn;
        }
        if (dn0) dn0[o] = nb;
        if (du0) du0[o] = n * ub;
        if (dT0) dT0[o] = n * (Tb1 + Tb2);
    }
}

// Per slab: sum of the per-node phi contributions (fixed-order tree), / phi_a.
__global__ void __launch_bounds__(kThreads)
adj_phi_kernel(const SlabDesc* __restrict__ slabs, const double* __restrict__ phis, const double* __restrict__ phi_a,
               double* out) {
    __shared__ double red[kThreads];
    const SlabDesc sd = slabs[blockIdx.x];
    double a = 0.0;
    for (int i = threadIdx.x; i < sd.nx; i += blockDim.x) a += phis[sd.node_off + i];
    red[threadIdx.x] = a;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[blockIdx.x] = red[0] / phi_a[blockIdx.x];
}

// ---------------------------------------------------------------------------
// Host-side launch helpers.
// ---------------------------------------------------------------------------
size_t adj_smem_bytes(int Q, int Z, int M) { return adj_smem_doubles(Q, Z, M) * sizeof(double); }

size_t adj_moments_smem_bytes(int Z, int m, int M) { return adj_moments_smem_doubles(Z, m, M) * sizeof(double); }

cudaError_t configure_adjoint(size_t smem_bytes, size_t smem2_bytes) {
    cudaError_t e = cudaFuncSetAttribute(adj_local_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(adj_moments_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2_bytes);
}

// One stage of the reverse sweep (see the file comment); nadj [10][NN] is a
// work array, phis [NN] accumulates F1b * F1.
void launch_adj_stage(int nitems, size_t smem, size_t smem2, cudaStream_t st, const SlabDesc* slabs,
                      const WorkItem* items, const double* tables, const double* taps, const double* src,
                      const double* mom, const double* ybar, const double* acc_in, double* acc_out, double* out,
                      double* nadj, double* phis, long long NF, long long NN, double ca, double cb, int use_dt,
                      double cc, double cacc, double cy, int Z, unsigned* err) {
    adj_local_kernel<<<nitems, kThreads, smem, st>>>(slabs, items, tables, taps, src, mom, ybar, acc_in, acc_out,
                                                     out, nadj, phis, NF, NN, ca, cb, use_dt, cc, cacc, cy, Z, err);
    adj_moments_kernel<<<nitems, kThreads, smem2, st>>>(slabs, items, tables, taps, mom, nadj, out, NF, NN, Z);
}

// Cotangent of the state for a loss of the final density n = sum_k F_k:
// dL/dF_k = dL/dn at every velocity, dL/dG = 0 (per work item: its nodes).
__global__ void __launch_bounds__(kThreads)
adj_seed_kernel(const SlabDesc* __restrict__ slabs, const WorkItem* __restrict__ items,
                const double* __restrict__ dn, double* __restrict__ barF, double* __restrict__ barG, long long NF) {
    const WorkItem it = items[blockIdx.x];
    const SlabDesc sd = slabs[it.slab];
    for (int e = threadIdx.x; e < sd.Q * it.nz; e += blockDim.x) {
        const int k = e / it.nz, t = e - k * it.nz;
        const long long g = sd.f_off + (long long)k * sd.nx + it.i0 + t;
        barF[g] = dn[sd.node_off + it.i0 + t];
        barG[g] = 0.0;
    }
}

void launch_adj_seed(int nitems, cudaStream_t st, const SlabDesc* slabs, const WorkItem* items, const double* dn,
                     double* barF, double* barG, long long NF) {
    adj_seed_kernel<<<nitems, kThreads, 0, st>>>(slabs, items, dn, barF, barG, NF);
}

void launch_adj_init(int nitems, cudaStream_t st, const SlabDesc* slabs, const WorkItem* items,
                     const double* tables, const double* init_fields, const double* lam, double* dn0, double* du0,
                     double* dT0, long long NF, long long NN) {
    adj_init_kernel<<<nitems, kThreads, 0, st>>>(slabs, items, tables, init_fields, lam, dn0, du0, dT0, NF, NN);
}

void launch_adj_phi(int nslabs, cudaStream_t st, const SlabDesc* slabs, const double* phis, const double* phi_a,
                    double* out) {
    adj_phi_kernel<<<nslabs, kThreads, 0, st>>>(slabs, phis, phi_a, out);
}

}  // namespace evfdlb
