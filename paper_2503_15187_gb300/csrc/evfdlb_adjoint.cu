// evfdlb_adjoint.cu -- discrete adjoint of the EV1 time step (FP64, periodic
// slabs): vector-Jacobian products of the right-hand side L of Eqs. (ev1) and
// (enskog_approx), of the Shu-Osher RK3 stages, and of the projected initial
// state, for the gradient of a loss of the final state with respect to the
// initial fields (n0, u0, T0), the initial distributions and the well depth
// phi_a of Eq. (sutherland) (through the Eq. (F1) force, which is linear in
// phi_a).
//
// One stage of the reverse sweep, given the adjoint ybar of the stage output,
// the stage input u and the node fields of u (both stored by the segment
// recompute), forms
//   out     = ca ybar + J(u)^T v + cc acc_in,   v = cb dt ybar,
//   acc_out = cacc acc_in + cy ybar,
// where J(u) is the Jacobian of L at u, in two launches:
//   adj_local_kernel  -- per node tile: the velocity-space part of J^T v
//                        (transposed WENO-5 faces, each face of the slab
//                        differentiated once by the tile that owns it;
//                        transposed Hermite synthesis and analysis on the
//                        parity-split velocity set; relaxation) and the
//                        adjoints of the node fields that L reads (n, u, T,
//                        q, chi, X, the three gradients and the force F1);
//   adj_moments_kernel-- per node tile: transposed fourth-order differences,
//                        the chain X = n^2 chi T, chi(nbar) of Eq. (carnstar)
//                        (on the tile and a Fischer-Methfessel halo), the
//                        transposed Fischer-Methfessel average and Eq. (F1)
//                        convolution (correlations), the chain from
//                        (n, u, T, q) to the raw moment sums, their transpose
//                        onto F and G, and the face terms that reach the tile
//                        from faces owned by its neighbours.
// FP64 is the GB300's scarcest pipe, and a node tile is small, so the work
// of every phase is spread over all warps of the CTA (lanes on velocities,
// faces or tap chunks), and the per-node chains that remain (the Hermite
// moments of N(u, T), the derivatives of the transport maps) run beside the
// WENO-5 faces, which take most of the pipe.
#include <cuda_runtime.h>
#include <math.h>

#include "evfdlb.h"
#include "evfdlb_device.cuh"

namespace evfdlb {

// per-node adjoints written by adj_local_kernel ([kNumNodeAdj][NN])
enum { AD_N = 0, AD_U, AD_T, AD_Q, AD_CHI, AD_X, AD_DX, AD_DT, AD_DU, AD_F1, kNumNodeAdj };

// slots of the node fields ([EVFDLB_NFIELDS][NN], the layout of evfdlb_fields)
enum { FL_N = 0, FL_U, FL_T, FL_Q, FL_NBAR, FL_CHI, FL_F1, FL_MU, FL_TAU, FL_PR, FL_NU, FL_A, FL_B, FL_DU, FL_X, FL_XX };

// per-node derivatives of the node maps, formed before the adjoints arrive:
// nu(n, T, chi) [NNU, TNU, CNU], kq = (1 - Pr(x)) q [QKQ = dkq/dq, NKQ, CKQ],
// K = -b n^2 chi [NK, CK], and 1/X, A/X, 1/T, B/T for the gradient ratios
enum { J_NNU = 0, J_TNU, J_CNU, J_QKQ, J_NKQ, J_CKQ, J_NK, J_CK, J_IX, J_AIX, J_IT, J_BIT, kNumJac };

constexpr int kZAdj = 32;   // largest node tile of the sweep kernels

// Sign of a velocity by its bit pattern (+1, -1, 0 for +-0): integer
// operations, not compares on the FP64 pipe.
__device__ __forceinline__ int xsign(double x) {
    const long long b = __double_as_longlong(x);
    return (b << 1) == 0 ? 0 : (b < 0 ? -1 : 1);
}
constexpr int kSumChunks = 4;    // lanes per (distribution, node) of the Hermite sums
constexpr int kTapChunks = 8;    // lanes per node of the tap correlations

// Shared-memory layout of adj_local_kernel (doubles).  NP = (Q + 1)/2 rows of
// the parity-split synthesis table and columns of the transposed analysis
// table (node k pairs with Q-1-k; the middle node of an odd Q stands alone).
// The state tile holds nodes i0-3 .. i0+nz+1 (the stencils of the tile's
// own faces), the ybar tile i0-1 .. i0+nz-1 (v = cb dt ybar is formed where
// it is used).  The face gradients G5 are dead once
// gathered; Ha and the per-node sums Red then reuse their block.
struct AdjLay {
    int NP, WH, WV;
    size_t S, PT, xi, r1, r2, r3, rinv, rr, H, V, Fl, J, Cc, Mm, VE, Cl, Cb, Hw, G5, Ha, Red, total;
    __host__ __device__ AdjLay(int Q, int Z) {
        NP = (Q + 1) / 2;
        WH = Z + 5;
        WV = Z + 1;
        size_t o = 0;
        S = o;    o += (size_t)NP * Q;         // S[k][l], k < NP
        PT = o;   o += (size_t)Q * NP;         // PT[l][j] = sqrt(l) psi_{l-1}(xi_j), j < NP
        xi = o;   o += Q;
        r1 = o;   o += Q;
        r2 = o;   o += Q;
        r3 = o;   o += Q;
        rinv = o; o += Q;
        rr = o;   o += Q;
        H = o;    o += 2 * (size_t)Q * WH;     // [2Q][WH]
        V = o;    o += 2 * (size_t)Q * WV;     // ybar [2Q][WV]
        Fl = o;   o += (size_t)EVFDLB_NFIELDS * Z;
        J = o;    o += (size_t)kNumJac * Z;
        Cc = o;   o += 8 * (size_t)Z;          // c0..c3 per distribution [2][4][Z]
        Mm = o;   o += (size_t)Q * Z;          // m_l(u, T) [Q][Z]
        VE = o;   o += 4 * (size_t)NP * Z;     // v_k +- v_{Q-1-k} [2 d][2 parity][NP][Z]
        Cl = o;   o += 2 * (size_t)Q * Z;      // c_l [2Q][Z]
        Cb = o;   o += 2 * (size_t)Q * Z;      // cbar_l [2Q][Z]
        Hw = o;   o += 2 * (size_t)Q * Z;      // transposed WENO-5 part [2Q][Z]
        G5 = o;   o += 10 * (size_t)Q * Z;     // face gradients [5][2Q][Z]
        Ha = G5;                               // [2Q][Z]
        Red = G5 + 2 * (size_t)Q * Z;          // [2][8][Z] (10 Q Z >= 2 Q Z + 16 Z for Q >= 2)
        total = o;
    }
};

__host__ __device__ inline size_t adj_smem_doubles(int Q, int Z) { return AdjLay(Q, Z).total; }

// Gradient of the WENO-5 face value Phi(v0..v4) (upwind side v0..v2), times
// pb: g_r = pb dPhi/dv_r.  Phi is taken in the difference form of the forward
// faces: with d_i = v_{i+1} - v_i, t_0 = d1 - d0, t_1 = d2 - d1, t_2 = d3 - d2,
// s_0 = 3 d1 - d0, s_1 = d1 + d2, s_2 = d3 - 3 d2, k_r = 13/3 t_r,
//   e_r = s_r^2 + k_r t_r + 4 eps   (= 4 (eps + beta_r)),
//   a_0 = e_1^2 e_2^2, a_1 = e_0^2 e_2^2, a_2 = e_0^2 e_1^2,
//   c_0 = (5 d1 - 2 d0)/60, c_1 = (d1 + 2 d2)/10, c_2 = (4 d2 - d3)/20,
//   Phi = v2 + (sum a_r c_r) / (0.1 a_0 + 0.6 a_1 + 0.3 a_2),
// differentiated in reverse order (one division per face).  With
// P_r = 4 e_r dL/dE_r (E_r = e_r^2) the adjoints of s_r and k_r t_r's
// argument are s_r P_r and k_r P_r, so the d-adjoints take the combinations
// s_r +- k_r and 3 s_r + k_r directly.
__device__ __forceinline__ void weno5_grad(double v0, double v1, double v2, double v3, double v4, double eps,
                                           double pb, double g[5]) {
    const double d0 = v1 - v0, d1 = v2 - v1, d2 = v3 - v2, d3 = v4 - v3;
    const double t0 = d1 - d0, t1 = d2 - d1, t2 = d3 - d2;
    const double s0 = fma(3.0, d1, -d0), s1 = d1 + d2, s2 = fma(-3.0, d2, d3);
    const double e4 = 4.0 * eps, k133 = 13.0 / 3.0;
    const double k0 = k133 * t0, k1 = k133 * t1, k2 = k133 * t2;
    const double e0 = fma(s0, s0, fma(k0, t0, e4));
    const double e1 = fma(s1, s1, fma(k1, t1, e4));
    const double e2 = fma(s2, s2, fma(k2, t2, e4));
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
    const double R4 = 4.0 * R;
    // adjoints (all times pb): of c_r, of a_r (times 4), of E_r (times 4)
    const double gc0 = a0 * R, gc1 = a1 * R, gc2 = a2 * R;
    const double gA0 = R4 * fma(-0.1, psi, c0), gA1 = R4 * fma(-0.6, psi, c1), gA2 = R4 * fma(-0.3, psi, c2);
    const double P0 = e0 * fma(gA1, E2, gA2 * E1), P1 = e1 * fma(gA0, E2, gA2 * E0), P2 = e2 * fma(gA0, E1, gA1 * E0);
    const double gd0 = fma(-P0, s0 + k0, (-2.0 / 60.0) * gc0);
    const double gd1 = fma(P0, fma(3.0, s0, k0), fma(P1, s1 - k1, fma(5.0 / 60.0, gc0, 0.1 * gc1)));
    const double gd2 = fma(P1, s1 + k1, fma(-P2, fma(3.0, s2, k2), 0.2 * (gc1 + gc2)));
    const double gd3 = fma(P2, s2 + k2, -0.05 * gc2);
    g[0] = -gd0;
    g[1] = gd0 - gd1;
    g[2] = pb + gd1 - gd2;
    g[3] = gd2 - gd3;
    g[4] = gd3;
}

__global__ void __launch_bounds__(kThreads)
adj_local_kernel(const SlabDesc* __restrict__ slabs, const WorkItem* __restrict__ items,
                 const double* __restrict__ tables, const double* __restrict__ src, const double* __restrict__ fld,
                 const double* __restrict__ ybar, const double* acc_in, double* acc_out, double* out,
                 double* __restrict__ nadj, double* __restrict__ phis, double* __restrict__ gface, long long NF,
                 long long NN, double ca, double cb, int use_dt, double cc, double cacc, double cy, int Z) {
    extern __shared__ __align__(16) double smem[];
    __shared__ int s_next;                       // next warp-sized group of faces
    const WorkItem it = items[blockIdx.x];
    const SlabDesc sd = slabs[it.slab];
    const int Q = sd.Q, nz = it.nz, nx = sd.nx, bc = sd.bc;
    const AdjLay Ly(Q, Z);
    const int NP = Ly.NP, WH = Ly.WH, WV = Ly.WV;
    double *sS = smem + Ly.S, *sPT = smem + Ly.PT, *sxi = smem + Ly.xi, *sr1 = smem + Ly.r1;
    double *sr2 = smem + Ly.r2, *sr3 = smem + Ly.r3, *srinv = smem + Ly.rinv, *srr = smem + Ly.rr;
    double *sH = smem + Ly.H, *sV = smem + Ly.V, *sFl = smem + Ly.Fl, *sJ = smem + Ly.J, *sCc = smem + Ly.Cc;
    double *sMm = smem + Ly.Mm, *sVE = smem + Ly.VE, *sCl = smem + Ly.Cl, *sCb = smem + Ly.Cb;
    double *sHw = smem + Ly.Hw, *sG5 = smem + Ly.G5, *sHa = smem + Ly.Ha, *sRed = smem + Ly.Red;
    TableLayout L(Q);
    const double* tab = tables + sd.tab_off;
    const int tid = threadIdx.x, nth = blockDim.x, lane = tid & 31, warp = tid >> 5;
    const long long row0 = sd.f_off + it.i0;     // + d NF + k nx: velocity k, distribution d, node i0

    // Step 0: tables, the state tile (i0-3 .. i0+nz+1), ybar (i0-1 ..
    // i0+nz-1) and the node fields of the tile, all loads in one phase.
    if (tid == 0) s_next = 0;
    for (int e = tid; e < NP * Q; e += nth) sS[e] = tab[L.S + e];
    for (int e = tid; e < Q * NP; e += nth) {
        const int l = e / NP, j = e - l * NP;
        sPT[e] = (l == 0) ? 0.0 : tab[L.r1 + l] * tab[L.P + (l - 1) * Q + j];
    }
    for (int e = tid; e < Q; e += nth) {
        sxi[e] = tab[L.xi + e];
        sr1[e] = tab[L.r1 + e];
        sr2[e] = tab[L.r2 + e];
        sr3[e] = tab[L.r3 + e];
        srinv[e] = tab[L.rinv + e];
        srr[e] = tab[L.rr + e];
    }
    for (int e = tid; e < 2 * Q * (nz + 5); e += nth) {
        const int c = e % (nz + 5), r = e / (nz + 5);
        const int k = r % Q, d = r / Q;
        sH[r * WH + c] = src[d * NF + sd.f_off + (long long)k * nx + gidx(it.i0 - 3 + c, nx, bc)];
    }
    const double vscale = cb * (use_dt ? sd.dt : 1.0);
    for (int e = tid; e < 2 * Q * (nz + 1); e += nth) {
        const int c = e % (nz + 1), r = e / (nz + 1);
        const int k = r % Q, d = r / Q;
        sV[r * WV + c] = ybar[d * NF + sd.f_off + (long long)k * nx + gidx(it.i0 - 1 + c, nx, bc)];
    }
    for (int e = tid; e < EVFDLB_NFIELDS * nz; e += nth) {
        const int f = e / nz, t = e - f * nz;
        sFl[f * Z + t] = fld[f * NN + sd.node_off + it.i0 + t];
    }
    __syncthreads();

    // Step 1.  Warps 0-2 form the per-node quantities first; then every warp
    // takes warp-sized groups of the tile's own faces from a shared counter.
    //  warp 0: Hermite moments m_l of N(u, T) (m_{l+1} = u m_l / sqrt(l+1)
    //          + (T-1) sqrt(l/(l+1)) m_{l-1});
    //  warp 1: derivatives of the node maps (nu, kq, K, gradient ratios);
    //  warp 2: coefficient constants c0..c3 (c_l = sum_r c_r sqrt(l!/(l-r)!)
    //          m_{l-r}, Eqs. (enskog_approx) and (J1)) and the parity parts
    //          of v = cb dt ybar at the tile nodes.
    auto F = [&](int f, int t) { return sFl[f * Z + t]; };
    if (warp == 0) {
        for (int t = lane; t < nz; t += 32) {
            const double u = F(FL_U, t), Tm1 = F(FL_T, t) - 1.0;
            double m0 = 1.0, m1 = 0.0;
            sMm[t] = 1.0;
            for (int l = 0; l + 1 < Q; ++l) {
                const double mn = fma(u * srinv[l], m0, Tm1 * srr[l] * m1);
                m1 = m0;
                m0 = mn;
                sMm[(l + 1) * Z + t] = mn;
            }
        }
    } else if (warp == 1) {
        const double b = sd.b;
        const double k1 = (4.0 / 25.0) * (1.0 + 12.0 / M_PI), k2 = (9.0 / 25.0) * (1.0 + 32.0 / (9.0 * M_PI));
        for (int t = lane; t < nz; t += 32) {
            const double n = F(FL_N, t), T = F(FL_T, t), chi = F(FL_CHI, t), nu = F(FL_NU, t);
            const double q = F(FL_Q, t), Pr = F(FL_PR, t), x = F(FL_XX, t), X = F(FL_X, t);
            const double bn = b * n;
            const double ichi = div_nr(1.0, chi), in = div_nr(1.0, n), iT = div_nr(1.0, T);
            // nu = 1/tau or chi/tau, tau = mu / (n T (1 + 2x/5)), mu = mu0 sqrt(T) g(n, chi),
            // g = 1/chi + 4/5 b n + k1 b^2 n^2 chi (Eqs. (viscosity), (tau)); both forms give
            // dnu = -nu dln(tau) (+ nu/chi dchi for chi/tau)
            const double den = 1.0 + 0.4 * x;
            const double ig = div_nr(1.0, ichi + 0.8 * bn + k1 * bn * bn * chi), iden = div_nr(1.0, den);
            double* J = sJ + t;
            J[J_NNU * Z] = nu * (in - (0.8 * b + 2.0 * k1 * b * bn * chi) * ig + 0.4 * b * chi * iden);
            J[J_TNU * Z] = 0.5 * nu * iT;
            double cnu = nu * ((ichi * ichi - k1 * bn * bn) * ig + 0.4 * bn * iden);
            if (sd.relax != EVFDLB_RELAX_INV_TAU) cnu += nu * ichi;
            J[J_CNU * Z] = cnu;
            // kq = (1 - Pr(x)) q, Pr of Eq. (prandtl), x = b n chi
            const double N1 = 1.0 + 0.6 * x, N2 = 1.0 + 0.8 * x + k1 * x * x, D2 = 1.0 + 1.2 * x + k2 * x * x;
            const double dPr = Pr * (0.6 * div_nr(1.0, N1) + (0.8 + 2.0 * k1 * x) * div_nr(1.0, N2) - 0.4 * iden -
                                     (1.2 + 2.0 * k2 * x) * div_nr(1.0, D2));
            J[J_QKQ * Z] = 1.0 - Pr;
            J[J_NKQ * Z] = -q * dPr * b * chi;
            J[J_CKQ * Z] = -q * dPr * bn;
            // K = -b n^2 chi
            J[J_NK * Z] = -2.0 * x;
            J[J_CK * Z] = -bn * n;
            // A = dX/X, B = dT/T
            const double iX = div_nr(1.0, X);
            J[J_IX * Z] = iX;
            J[J_AIX * Z] = F(FL_A, t) * iX;
            J[J_IT * Z] = iT;
            J[J_BIT * Z] = F(FL_B, t) * iT;
        }
    } else if (warp == 2) {
        for (int e = lane; e < 2 * nz; e += 32) {
            const int t = e % nz, d = e / nz;
            const double n = F(FL_N, t), T = F(FL_T, t), nu = F(FL_NU, t);
            const double kq = (1.0 - F(FL_PR, t)) * F(FL_Q, t), K = -F(FL_XX, t) * n;
            const double A = F(FL_A, t), B = F(FL_B, t), D = F(FL_DU, t);
            double* c = sCc + d * 4 * Z + t;
            if (d == 0) {
                c[0] = nu * n;
                c[Z] = K * A * T;
                c[2 * Z] = 0.6 * K * D * T;
                c[3 * Z] = 0.2 * nu * kq + 0.3 * K * B * T * T;
            } else {
                c[0] = nu * n * T + 0.4 * K * T * D;
                c[Z] = 0.4 * nu * kq + K * T * T * (A + 0.6 * B);
                c[2 * Z] = 0.6 * K * T * T * D;
                c[3 * Z] = 0.2 * nu * kq * T + 0.3 * K * T * T * T * B;
            }
        }
        for (int e = lane; e < 2 * NP * nz; e += 32) {
            const int t = e % nz, r = e / nz;
            const int k = r % NP, d = r / NP;
            const double* v = sV + (size_t)d * Q * WV + t + 1;
            const double a = v[k * WV];
            const bool pair = (Q - 1 - k != k);
            const double bm = pair ? v[(Q - 1 - k) * WV] : 0.0;
            sVE[((d * 2 + 0) * NP + k) * Z + t] = vscale * (pair ? a + bm : a);
            sVE[((d * 2 + 1) * NP + k) * Z + t] = pair ? vscale * (a - bm) : 0.0;
        }
    }
    // The tile's own faces: face p (tile-relative, between nodes p-1 and p)
    // of row r = d Q + k.  For xi > 0 its WENO-5 stencil is nodes p-3 .. p+1
    // (v0 .. v4), for xi < 0 nodes p+2 .. p-2; its adjoint is
    // pb = xi/dz (v_p - v_{p-1}), v = cb dt ybar.  G5[s][r][p] = pb dPhi/dv_s.  A face whose
    // stencil leaves the tile also goes to gface (global, by face), where the
    // neighbouring tiles' adj_moments_kernel collects its terms.
    {
        const int nface = 2 * Q * nz, ngroup = (nface + 31) / 32;
        const double rdz = sd.inv_dx * vscale, eps = sd.weno_eps;
        for (;;) {
            int g = 0;
            if (lane == 0) g = atomicAdd(&s_next, 1);
            g = __shfl_sync(0xffffffffu, g, 0);
            if (g >= ngroup) break;
            const int e = g * 32 + lane;
            if (e < nface) {
                const int p = e % nz, r = e / nz;
                const int k = r % Q, d = r / Q;
                const double x = sxi[k];
                const int sg = xsign(x);
                double gg[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
                const double* h = sH + (size_t)r * WH + p;      // h[c] = node p - 3 + c
                const double* v = sV + (size_t)r * WV + p;      // ybar at nodes p - 1, p
                if (sg > 0) {
                    weno5_grad(h[0], h[1], h[2], h[3], h[4], eps, x * rdz * (v[1] - v[0]), gg);
                } else if (sg < 0) {
                    weno5_grad(h[5], h[4], h[3], h[2], h[1], eps, x * rdz * (v[1] - v[0]), gg);
                }
#pragma unroll
                for (int s = 0; s < 5; ++s) sG5[((size_t)s * 2 * Q + r) * Z + p] = gg[s];
                const bool edge = (sg > 0) ? (p < 3 || p + 1 >= nz) : (sg < 0 && (p < 2 || p + 2 >= nz));
                if (edge) {
                    double* gf = gface + d * NF + row0 + (long long)k * nx + p;
#pragma unroll
                    for (int s = 0; s < 5; ++s) gf[s * 2 * NF] = gg[s];
                }
            }
        }
    }
    __syncthreads();

    // Step 2, per (distribution d, order or velocity l, node t):
    //  cbar_l = sum_k S_kl v_k on the parity parts (even l: v_k + v_{Q-1-k},
    //           odd l: v_k - v_{Q-1-k});
    //  c_l    = c0 m_l + c1 sqrt(l) m_{l-1} + c2 sqrt(l(l-1)) m_{l-2} + c3 sqrt(l(l-1)(l-2)) m_{l-3};
    //  Hw_l   = the tile's own faces' terms at node t of row (d, l).
    for (int e = tid; e < 2 * Q * nz; e += nth) {
        const int t = e % nz, r = e / nz;
        const int l = r % Q, d = r / Q;
        const double* ve = sVE + ((d * 2 + (l & 1)) * NP) * Z + t;
        double a0 = 0.0, a1 = 0.0;
        int k = 0;
        for (; k + 1 < NP; k += 2) {
            a0 = fma(sS[k * Q + l], ve[k * Z], a0);
            a1 = fma(sS[(k + 1) * Q + l], ve[(k + 1) * Z], a1);
        }
        if (k < NP) a0 = fma(sS[k * Q + l], ve[k * Z], a0);
        sCb[(size_t)r * Z + t] = a0 + a1;
        const double* c = sCc + d * 4 * Z + t;
        const double* m = sMm + t;
        double cl = c[0] * m[l * Z];
        if (l >= 1) cl = fma(c[Z] * sr1[l], m[(l - 1) * Z], cl);
        if (l >= 2) cl = fma(c[2 * Z] * sr2[l], m[(l - 2) * Z], cl);
        if (l >= 3) cl = fma(c[3 * Z] * sr3[l], m[(l - 3) * Z], cl);
        sCl[(size_t)r * Z + t] = cl;
        const int sg = xsign(sxi[l]);
        double hw = 0.0;
        if (sg != 0) {
            // xi > 0: faces p = t-1 .. t+3, node t is v_{t-p+3}; xi < 0: p = t-2 .. t+2, v_{p+2-t}
            const int plo = (sg > 0) ? t - 1 : t - 2;
            for (int p = max(plo, 0); p <= min(plo + 4, nz - 1); ++p) {
                const int s = (sg > 0) ? t - p + 3 : p + 2 - t;
                hw += sG5[((size_t)s * 2 * Q + r) * Z + p];
            }
        }
        sHw[(size_t)r * Z + t] = hw;
    }
    __syncthreads();

    // Step 3.  (a) Per (d, node t, chunk of orders): the sums over l of
    //   b_r = sum cbar_l sqrt(l!/(l-r)!) m_{l-r}  (r = 0..3: adjoints of c0..c3),
    //   ub  = sum cbar_l sqrt(l) c_{l-1}          (dc_l/du = sqrt(l) c_{l-1}),
    //   Tb  = sum cbar_l sqrt(l(l-1)) c_{l-2} / 2 (dc_l/dT),
    //   nub = -sum_k h_k v_k                      (the -nu h term),
    // kSumChunks lanes per (d, t), joined by shuffles.  (b) Per (d, j < NP, t):
    // Ha_j = sum_l sqrt(l) psi_{l-1}(xi_j) cbar_l, the transposed analysis of
    // the force term c_l += F1 sqrt(l) a_{l-1}, on the parity parts (odd l
    // symmetric, even l antisymmetric about j <-> Q-1-j).
    {
        const int nsum = kSumChunks * 2 * nz, nsum_p = (nsum + 31) & ~31;
        const int LQ = (Q + kSumChunks - 1) / kSumChunks;
        for (int base = warp * 32; base < nsum_p + 2 * NP * nz; base += nth) {
            if (base < nsum_p) {
                const int e = base + lane;
                const bool act = e < nsum;
                const int ch = e % kSumChunks, dt = e / kSumChunks;
                const int t = act ? dt % nz : 0, d = act ? dt / nz : 0;
                const double* cbr = sCb + (size_t)d * Q * Z + t;
                const double* clr = sCl + (size_t)d * Q * Z + t;
                const double* m = sMm + t;
                const double* h = sH + (size_t)d * Q * WH + t + 3;
                const double* v = sV + (size_t)d * Q * WV + t + 1;
                double b0 = 0, b1 = 0, b2 = 0, b3 = 0, ub = 0, Tb = 0, nb = 0;
                const int l0 = act ? ch * LQ : Q, l1 = min(Q, l0 + LQ);
                for (int l = l0; l < l1; ++l) {
                    const double cbl = cbr[l * Z];
                    b0 = fma(cbl, m[l * Z], b0);
                    nb = fma(-h[l * WH], v[l * WV], nb);
                    if (l >= 1) {
                        const double p1 = cbl * sr1[l];
                        b1 = fma(p1, m[(l - 1) * Z], b1);
                        ub = fma(p1, clr[(l - 1) * Z], ub);
                    }
                    if (l >= 2) {
                        const double p2 = cbl * sr2[l];
                        b2 = fma(p2, m[(l - 2) * Z], b2);
                        Tb = fma(p2, clr[(l - 2) * Z], Tb);
                    }
                    if (l >= 3) b3 = fma(cbl * sr3[l], m[(l - 3) * Z], b3);
                }
                double acc[7] = {b0, b1, b2, b3, ub, Tb, nb};
#pragma unroll
                for (int s = 0; s < 7; ++s) {
                    acc[s] += __shfl_xor_sync(0xffffffffu, acc[s], 1);
                    acc[s] += __shfl_xor_sync(0xffffffffu, acc[s], 2);
                }
                if (act && ch == 0) {
                    double* red = sRed + (size_t)d * 8 * Z + t;
                    red[0] = acc[0];
                    red[Z] = acc[1];
                    red[2 * Z] = acc[2];
                    red[3 * Z] = acc[3];
                    red[4 * Z] = acc[4];
                    red[5 * Z] = 0.5 * acc[5];
                    red[7 * Z] = vscale * acc[6];
                }
            } else {
                const int e = base - nsum_p + lane;
                if (e < 2 * NP * nz) {
                    const int t = e % nz, r = e / nz;
                    const int j = r % NP, d = r / NP;
                    const double* cbr = sCb + (size_t)d * Q * Z + t;
                    double eo = 0.0, ee = 0.0;      // odd l (symmetric), even l (antisymmetric)
                    int l = 1;
                    for (; l + 1 < Q; l += 2) {
                        eo = fma(sPT[l * NP + j], cbr[l * Z], eo);
                        ee = fma(sPT[(l + 1) * NP + j], cbr[(l + 1) * Z], ee);
                    }
                    if (l < Q) eo = fma(sPT[l * NP + j], cbr[l * Z], eo);
                    double* ha = sHa + (size_t)d * Q * Z + t;
                    ha[j * Z] = eo + ee;
                    if (Q - 1 - j != j) ha[(Q - 1 - j) * Z] = eo - ee;
                }
            }
        }
    }
    __syncthreads();

    // Step 4.  Warp 0: the force adjoint sum F1b_d = sum_k h_k Ha_k, then per
    // node the chain through the coefficient constants, the node maps and the
    // gradient ratios, written as the node adjoints.  Warps 1-7: the
    // distribution-local adjoint and the RK-stage combination.
    if (warp == 0) {
        for (int e = lane; e < 2 * nz; e += 32) {
            const int t = e % nz, d = e / nz;
            const double* h = sH + (size_t)d * Q * WH + t + 3;
            const double* ha = sHa + (size_t)d * Q * Z + t;
            double f0 = 0.0, f1 = 0.0;
            int k = 0;
            for (; k + 1 < Q; k += 2) {
                f0 = fma(h[k * WH], ha[k * Z], f0);
                f1 = fma(h[(k + 1) * WH], ha[(k + 1) * Z], f1);
            }
            if (k < Q) f0 = fma(h[k * WH], ha[k * Z], f0);
            sRed[(size_t)d * 8 * Z + 6 * Z + t] = f0 + f1;
        }
        __syncwarp();
        for (int t = lane; t < nz; t += 32) {
            const double n = F(FL_N, t), T = F(FL_T, t), nu = F(FL_NU, t);
            const double kq = (1.0 - F(FL_PR, t)) * F(FL_Q, t), K = -F(FL_XX, t) * n;
            const double A = F(FL_A, t), B = F(FL_B, t), D = F(FL_DU, t), F1 = F(FL_F1, t);
            const double* rF = sRed + t;
            const double* rG = sRed + 8 * Z + t;
            const double cF0 = rF[0], cF1 = rF[Z], cF2 = rF[2 * Z], cF3 = rF[3 * Z];
            const double cG0 = rG[0], cG1 = rG[Z], cG2 = rG[2 * Z], cG3 = rG[3 * Z];
            double ub = rF[4 * Z] + rG[4 * Z];
            double Tb = rF[5 * Z] + rG[5 * Z];
            const double F1b = rF[6 * Z] + rG[6 * Z];
            double nub = rF[7 * Z] + rG[7 * Z];
            double nb = 0, Kb = 0, kqb = 0, Ab = 0, Bb = 0, Db = 0;
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
            // the node maps nu(n, T, chi), kq(q, n, chi), K(n, chi) and the ratios A, B
            const double* J = sJ + t;
            nb += nub * J[J_NNU * Z] + kqb * J[J_NKQ * Z] + Kb * J[J_NK * Z];
            Tb += nub * J[J_TNU * Z] - Bb * J[J_BIT * Z];
            const double chib = nub * J[J_CNU * Z] + kqb * J[J_CKQ * Z] + Kb * J[J_CK * Z];
            const long long o = sd.node_off + it.i0 + t;
            double* na = nadj + o;
            na[AD_N * NN] = nb;
            na[AD_U * NN] = ub;
            na[AD_T * NN] = Tb;
            na[AD_Q * NN] = kqb * J[J_QKQ * Z];
            na[AD_CHI * NN] = chib;
            na[AD_X * NN] = -Ab * J[J_AIX * Z];
            na[AD_DX * NN] = Ab * J[J_IX * Z];
            na[AD_DT * NN] = Bb * J[J_IT * Z];
            na[AD_DU * NN] = Db;
            na[AD_F1 * NN] = F1b;
            phis[o] += F1b * F1;
        }
    } else {
        for (int e = tid - 32; e < 2 * Q * nz; e += nth - 32) {
            const int t = e % nz, r = e / nz;
            const int j = r % Q, d = r / Q;
            const double F1 = F(FL_F1, t), nu = F(FL_NU, t);
            const double yb = sV[(size_t)r * WV + t + 1];
            const double val = fma(F1, sHa[(size_t)r * Z + t], fma(-nu, vscale * yb, sHw[(size_t)r * Z + t]));
            const long long g = d * NF + row0 + (long long)j * nx + t;
            double o = fma(ca, yb, val);
            if (cc != 0.0) o = fma(cc, acc_in[g], o);
            if (acc_out) acc_out[g] = (cacc != 0.0 ? cacc * acc_in[g] : 0.0) + cy * yb;
            out[g] = o;
        }
    }
}

// Per node tile: transposed fourth-order differences of X, T, u, the chain
// X = n^2 chi T, chi = chi(eta), eta = pi sigma^3 nbar / 6 (Eq. (carnstar)) on
// the tile and its Fischer-Methfessel halo, the transposed Fischer-Methfessel
// average and Eq. (F1) convolution (correlations with the same taps), the
// chain (n, u, T, q) <- raw sums, and
// out_{F,k} += S0b + xi S1b + xi^2 S2b + xi^3 S3b, out_{G,k} += G0b + xi G1b,
// plus the terms of the faces outside the tile whose stencils reach it.
// Every global input is staged in one phase, so that their latencies overlap.
struct AdjMomLay {
    size_t Xb, Nb, n, T, chi, nbar, xa, ca, F1, DX, DU, DT, na, mm, u, sb, part, out, ftap, mtap, total;
    __host__ __device__ AdjMomLay(int Q, int Z, int m, int M) {
        const size_t HW = Z + 2 * m;
        size_t o = 0;
        Xb = o;   o += HW;                      // X adjoint on [i0 - m, i0 + nz + m)
        Nb = o;   o += HW;                      // nbar adjoint (source of the FM correlation)
        n = o;    o += HW;                      // n, T, chi, nbar on the same nodes
        T = o;    o += HW;
        chi = o;  o += HW;
        nbar = o; o += HW;
        xa = o;   o += HW;                      // node adjoints of X and chi there
        ca = o;   o += HW;
        F1 = o;   o += (size_t)Z + 2 * M;       // force adjoint on [i0 - M, i0 + nz + M)
        DX = o;   o += (size_t)Z + 2 * m + 4;   // X-gradient adjoint on [i0 - m - 2, i0 + nz + m + 2)
        DU = o;   o += (size_t)Z + 4;           // u- and T-gradient adjoints on [i0 - 2, i0 + nz + 2)
        DT = o;   o += (size_t)Z + 4;
        na = o;   o += 4 * (size_t)Z;           // node adjoints of n, u, T, q on the tile
        mm = o;   o += 3 * (size_t)Z;           // S1, S2, G0 on the tile
        u = o;    o += (size_t)Z;               // u on the tile
        sb = o;   o += (size_t)kNumMoments * Z; // raw-sum adjoints of the tile
        part = o; o += (size_t)kTapChunks * Z;  // partial tap sums
        out = o;  o += 2 * (size_t)Q * Z;       // out of the tile plus the outside faces' terms
        ftap = o; o += 2 * (size_t)M + 1;       // Eq. (F1) taps
        mtap = o; o += 2 * (size_t)m + 1;       // Fischer-Methfessel taps
        total = o;
    }
};

__host__ __device__ inline size_t adj_moments_smem_doubles(int Q, int Z, int m, int M) {
    return AdjMomLay(Q, Z, m, M).total;
}

__global__ void __launch_bounds__(kThreads)
adj_moments_kernel(const SlabDesc* __restrict__ slabs, const WorkItem* __restrict__ items,
                   const double* __restrict__ tables, const double* __restrict__ taps,
                   const double* __restrict__ mom, const double* __restrict__ fld, const double* __restrict__ nadj,
                   const double* __restrict__ gface, double* out, long long NF, long long NN, int Z) {
    extern __shared__ __align__(16) double sm[];
    const WorkItem it = items[blockIdx.x];
    const SlabDesc sd = slabs[it.slab];
    const int nx = sd.nx, bc = sd.bc, M = sd.M, m = sd.m, Q = sd.Q, nz = it.nz;
    const AdjMomLay Ly(Q, Z, m, M);
    double *sXb = sm + Ly.Xb, *sNb = sm + Ly.Nb, *sn = sm + Ly.n, *sT = sm + Ly.T, *schi = sm + Ly.chi;
    double *snbar = sm + Ly.nbar, *sxa = sm + Ly.xa, *sca = sm + Ly.ca;
    double *sF1 = sm + Ly.F1, *sDX = sm + Ly.DX, *sDU = sm + Ly.DU, *sDT = sm + Ly.DT, *sna = sm + Ly.na;
    double *smm = sm + Ly.mm, *su = sm + Ly.u, *sb = sm + Ly.sb, *spart = sm + Ly.part, *sout = sm + Ly.out;
    double *ftap = sm + Ly.ftap, *mtap = sm + Ly.mtap;
    const int tid = threadIdx.x, nth = blockDim.x;
    const double inv12 = sd.inv_dx / 12.0;
    const long long no = sd.node_off;
    TableLayout L(Q);
    const double* xi = tables + sd.tab_off + L.xi;
    const double* gF1 = nadj + AD_F1 * NN + no;
    const double* gDX = nadj + AD_DX * NN + no;
    const double* gDU = nadj + AD_DU * NN + no;
    const double* gDT = nadj + AD_DT * NN + no;
    for (int j = tid; j < 2 * M + 1; j += nth) ftap[j] = taps[sd.tap_off + j];
    for (int j = tid; j < 2 * m + 1; j += nth) mtap[j] = taps[sd.tap_off + 2 * M + 1 + j];
    for (int c = tid; c < nz + 2 * M; c += nth) sF1[c] = gF1[gidx(it.i0 - M + c, nx, bc)];
    for (int c = tid; c < nz + 2 * m + 4; c += nth) sDX[c] = gDX[gidx(it.i0 - m - 2 + c, nx, bc)];
    for (int c = tid; c < nz + 4; c += nth) {
        const int i = gidx(it.i0 - 2 + c, nx, bc);
        sDU[c] = gDU[i];
        sDT[c] = gDT[i];
    }
    for (int c = tid; c < nz + 2 * m; c += nth) {
        const long long o = no + gidx(it.i0 - m + c, nx, bc);
        sn[c] = fld[FL_N * NN + o];
        sT[c] = fld[FL_T * NN + o];
        schi[c] = fld[FL_CHI * NN + o];
        snbar[c] = fld[FL_NBAR * NN + o];
        sxa[c] = nadj[AD_X * NN + o];
        sca[c] = nadj[AD_CHI * NN + o];
    }
    for (int t = tid; t < nz; t += nth) {
        const long long o = no + it.i0 + t;
        sna[t] = nadj[AD_N * NN + o];
        sna[Z + t] = nadj[AD_U * NN + o];
        sna[2 * Z + t] = nadj[AD_T * NN + o];
        sna[3 * Z + t] = nadj[AD_Q * NN + o];
        smm[t] = mom[MOM_S1 * NN + o];
        smm[Z + t] = mom[MOM_S2 * NN + o];
        smm[2 * Z + t] = mom[MOM_G0 * NN + o];
        su[t] = fld[FL_U * NN + o];
    }
    // out of the tile, plus the terms of the faces outside the tile whose
    // stencils hold node t (see adj_local_kernel): xi > 0: faces p = t-1 ..
    // t+3, node t is v_{t-p+3}; xi < 0: p = t-2 .. t+2, v_{p+2-t}
    for (int e = tid; e < 2 * Q * nz; e += nth) {
        const int t = e % nz, r = e / nz;
        const int k = r % Q, d = r / Q;
        const long long row = d * NF + sd.f_off + (long long)k * nx;
        double v = out[row + it.i0 + t];
        const int sg = xsign(xi[k]);
        if (sg != 0) {
            const int plo = (sg > 0) ? t - 1 : t - 2;
            if (plo < 0 || plo + 4 >= nz) {
                for (int p = plo; p <= plo + 4; ++p) {
                    if (p >= 0 && p < nz) continue;
                    const int s = (sg > 0) ? t - p + 3 : p + 2 - t;
                    v += gface[s * 2 * NF + row + gidx(it.i0 + p, nx, bc)];
                }
            }
        }
        sout[(size_t)r * Z + t] = v;
    }
    __syncthreads();
    // transposed fourth-order difference at staged position p (value at p)
    auto d4t = [&](const double* g, int p) { return (g[p + 2] - 8.0 * g[p + 1] + 8.0 * g[p - 1] - g[p - 2]) * inv12; };
    // the chain to chi on the tile and its Fischer-Methfessel halo
    for (int c = tid; c < nz + 2 * m; c += nth) {
        const double n = sn[c], T = sT[c];
        const double eta = sd.eta_coef * snbar[c], om = 1.0 - eta, om2 = om * om;
        const double Xb = sxa[c] + d4t(sDX, c + 2);
        const double chib = sca[c] + Xb * n * n * T;
        // dchi/deta = (5 - 2 eta) / (2 (1 - eta)^4)
        sXb[c] = Xb;
        sNb[c] = chib * div_nr(5.0 - 2.0 * eta, 2.0 * om2 * om2) * sd.eta_coef;
    }
    __syncthreads();
    // the two correlations, sum_j mtap_j Nb_{i-j} + sum_j ftap_j F1b_{i-j},
    // as one list of 2m+1 + 2M+1 terms cut into kTapChunks chunks per node
    {
        const int LT = 2 * m + 1 + 2 * M + 1, LC = (LT + kTapChunks - 1) / kTapChunks;
        for (int e = tid; e < kTapChunks * nz; e += nth) {
            const int ch = e % kTapChunks, t = e / kTapChunks;
            double a = 0.0;
            for (int j = ch * LC; j < min(LT, (ch + 1) * LC); ++j) {
                if (j < 2 * m + 1) a = fma(mtap[j], sNb[t + 2 * m - j], a);
                else {
                    const int jj = j - (2 * m + 1);
                    a = fma(ftap[jj], sF1[t + 2 * M - jj], a);
                }
            }
            spart[ch * Z + t] = a;
        }
    }
    __syncthreads();
    for (int t = tid; t < nz; t += nth) {
        const int c = t + m;
        const double n = sn[c], T = sT[c], chi = schi[c], Xb = sXb[c];
        double nb = sna[t] + Xb * 2.0 * n * chi * T;
        for (int ch = 0; ch < kTapChunks; ++ch) nb += spart[ch * Z + t];
        double ub = sna[Z + t] + d4t(sDU, t + 2);
        double Tb = sna[2 * Z + t] + d4t(sDT, t + 2) + Xb * n * n * chi;
        const double qb = sna[3 * Z + t];
        const double S0v = n, S1v = smm[t], S2v = smm[Z + t], G0v = smm[2 * Z + t];
        const double in = div_nr(1.0, n);
        const double u = su[t];
        const double E = (0.5 * S2v + G0v) * in;
        // q = (S3 - 3u S2 + 3u^2 S1 - u^3 S0)/2 + G1 - u G0
        double S3b = 0.5 * qb, S2b = -1.5 * u * qb, S1b = 1.5 * u * u * qb, S0b = -0.5 * u * u * u * qb;
        double G1b = qb, G0b = -u * qb;
        ub += qb * (-1.5 * S2v + 3.0 * u * S1v - 1.5 * u * u * S0v - G0v);
        // T = (2/3)(E - u^2/2), E = (S2/2 + G0)/n
        const double Eb = (2.0 / 3.0) * Tb;
        ub += -(2.0 / 3.0) * u * Tb;
        S2b += 0.5 * Eb * in;
        G0b += Eb * in;
        nb += -Eb * E * in;
        // u = S1/n
        S1b += ub * in;
        nb += -ub * u * in;
        S0b += nb;
        sb[MOM_S0 * Z + t] = S0b;
        sb[MOM_S1 * Z + t] = S1b;
        sb[MOM_S2 * Z + t] = S2b;
        sb[MOM_S3 * Z + t] = S3b;
        sb[MOM_G0 * Z + t] = G0b;
        sb[MOM_G1 * Z + t] = G1b;
    }
    __syncthreads();
    for (int e = tid; e < 2 * Q * nz; e += nth) {
        const int t = e % nz, r = e / nz;
        const int k = r % Q, d = r / Q;
        const double x = xi[k];
        const double add = (d == 0) ? sb[MOM_S0 * Z + t] + x * (sb[MOM_S1 * Z + t] + x * (sb[MOM_S2 * Z + t] + x * sb[MOM_S3 * Z + t]))
                                    : sb[MOM_G0 * Z + t] + x * sb[MOM_G1 * Z + t];
        out[d * NF + sd.f_off + (long long)k * nx + it.i0 + t] = sout[(size_t)r * Z + t] + add;
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
int adj_tile_max() { return kZAdj; }

size_t adj_smem_bytes(int Q, int Z) { return adj_smem_doubles(Q, Z) * sizeof(double); }

size_t adj_moments_smem_bytes(int Q, int Z, int m, int M) { return adj_moments_smem_doubles(Q, Z, m, M) * sizeof(double); }

cudaError_t configure_adjoint(size_t smem_bytes, size_t smem2_bytes) {
    cudaError_t e = cudaFuncSetAttribute(adj_local_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(adj_moments_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2_bytes);
}

// One stage of the reverse sweep (see the file comment) over the work items
// of the sweep's node tile Z <= kZAdj.  fld: node fields of src
// [EVFDLB_NFIELDS][NN]; nadj [10][NN] and gface [5][2 NF] are work arrays;
// phis [NN] accumulates F1b * F1.
void launch_adj_stage(int nitems, size_t smem, size_t smem2, cudaStream_t st, const SlabDesc* slabs,
                      const WorkItem* items, const double* tables, const double* taps, const double* src,
                      const double* fld, const double* mom, const double* ybar, const double* acc_in, double* acc_out,
                      double* out, double* nadj, double* phis, double* gface, long long NF, long long NN, double ca,
                      double cb, int use_dt, double cc, double cacc, double cy, int Z) {
    adj_local_kernel<<<nitems, kThreads, smem, st>>>(slabs, items, tables, src, fld, ybar, acc_in, acc_out, out, nadj,
                                                     phis, gface, NF, NN, ca, cb, use_dt, cc, cacc, cy, Z);
    adj_moments_kernel<<<nitems, kThreads, smem2, st>>>(slabs, items, tables, taps, mom, fld, nadj, gface, out, NF,
                                                        NN, Z);
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
