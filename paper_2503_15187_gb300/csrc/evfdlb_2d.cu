// evfdlb_2d.cu -- the two-dimensional tensor-product extension of the EV1
// time step (a plane periodic domain, homogeneous along z), FP32 with FP64
// conserved sums (and an FP64 build for parity checks).  The paper solves a
// 1D slab and names 2D as future work (Sec. IV); the 2D model extends its
// Sec. II-III statement:
//   * reduced distributions over p_z: F = int f dp_z, G = int f p_z^2/2 dp_z,
//     on the tensor product of the full-range Gauss-Hermite set of order Q
//     per axis, projected to order Q-1 per axis;
//   * reduced Shakhov equilibria and J1 (one transverse direction), written
//     as F_MB times a cubic polynomial in the peculiar velocity c, so that
//     their Hermite coefficients are sums of products of one-axis Gaussian
//     moments E[c^a psi_l(u + c)] (Stein's identity);
//   * the Eq. (force) integral over z as the in-plane kernel
//     g2(rho) = rho_vec gamma phi sigma^gamma int_{r > sigma} r^-(gamma+2) dz,
//     summed over the grid offsets inside the r_cut disc (rectangle rule);
//   * the Fischer-Methfessel average with chord weights 2 sqrt(sigma^2 - rho^2),
//     normalised; fourth-order gradients and WENO-5 along each axis.
// One RK stage is four launches:
//   k2_moments  raw moment sums of the stage input per node (the conserved
//               ones -- mass, momentum, energy -- to FP64 accuracy);
//   k2_fields   node fields per 16x16 node tile (force disc, FM average, chi,
//               gradients, transport) and the polynomial coefficients of the
//               equilibria;
//   k2_coll     per group of 8 nodes, all Q^2 velocities: separable Hermite
//               analysis, coefficients (equilibria + force), separable
//               synthesis; writes the local part -nu h + sum S c;
//   k2_adv      per 32x16 node tile and 8 velocity planes: WENO-5 faces along
//               x and y, the full right-hand side and the Shu-Osher combine.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <type_traits>
#include <vector>

#include "evfdlb_internal.h"

namespace evfdlb {

struct Slab2 {
    int nx, ny, Q, relax;
    long long N;          // nodes, nx * ny
    int nft, nfm;         // force and Fischer-Methfessel taps
    int Mf, mfm;          // their radii in nodes
    double dx, inv_dx, dt, weno_eps, b, eta_coef, mu0_coef;
};

// raw moment sums per node ([kNumMom2][N], FP64)
enum { M2_S0 = 0, M2_S1X, M2_S1Y, M2_S2XX, M2_S2YY, M2_G0, M2_S2XY, M2_S3X, M2_S3Y, M2_G1X, M2_G1Y, kNumMom2 };
// node outputs of k2_fields ([kNumFld2][N], precision R): n, ux, uy, T, nu,
// Fx, Fy, then the coefficients P_ab (times n) of the F and G polynomials in
// the order (a,b) = (0,0) (1,0) (0,1) (2,0) (1,1) (0,2) (3,0) (2,1) (1,2) (0,3)
enum { F2_N = 0, F2_UX, F2_UY, F2_T, F2_NU, F2_FX, F2_FY, F2_PF = 7, F2_PG = 17, kNumFld2 = 27 };

constexpr int kTile2 = 16;     // k2_fields tile edge
constexpr int kNB = 8;         // nodes per k2_coll CTA
constexpr int kAdvX = 32, kAdvY = 16, kAdvPlanes = 8;
static_assert(kAdvX == 32 && kAdvY % 8 == 0, "k2_adv maps a warp (256 threads per CTA) to tile rows");

__device__ __forceinline__ int wrapi(int i, int n) {
    int r = i % n;
    return r < 0 ? r + n : r;
}

// ---------------------------------------------------------------------------
// k2_moments: per node, raw sums over the Q^2 velocities.  Conserved sums
// (S0, S1, S2xx, S2yy, G0) are formed from the row and column sums of the
// velocity grid, combined in FP64; for an FP32 state each 16-term row or
// column sum is a compensated (Neumaier) FP32 sum kept as an unevaluated
// pair, accurate to O(Q u^2) of the sum of magnitudes, i.e. FP64 quality at
// FP32-pipe cost.  The heat-flux sums are plain R sums.
// ---------------------------------------------------------------------------
template <typename R>
struct CompSum {                       // R = double: plain accumulation
    double s = 0.0;
    __device__ __forceinline__ void add(R x) { s += (double)x; }
    __device__ __forceinline__ double value() const { return s; }
};
template <>
struct CompSum<float> {                // Neumaier's compensated sum
    float s = 0.0f, c = 0.0f;
    __device__ __forceinline__ void add(float x) {
        float t = s + x;
        c += (fabsf(s) >= fabsf(x)) ? (s - t) + x : (x - t) + s;
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

template <typename R>
__global__ void __launch_bounds__(256)
k2_moments(Slab2 s, const double* __restrict__ tab, const R* __restrict__ st, double* __restrict__ mom,
           unsigned* err) {
    const int Q = s.Q;
    const long long N = s.N, NF = (long long)Q * Q * N;
    TableLayout L(Q);
    const double* xi = tab + L.xi;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        CompSum<R> col[16];
        double s0 = 0, s1x = 0, s2xx = 0, g0 = 0;
        R s2xy = 0, s3x = 0, s3y = 0, g1x = 0, g1y = 0;
        for (int kx = 0; kx < Q; ++kx) {
            const double x = xi[kx];
            CompSum<R> rowF, rowG;
            R ps2xy = 0, ps3x = 0, ps3y = 0, pg1y = 0;
            for (int ky = 0; ky < Q; ++ky) {
                const long long g = (long long)(kx * Q + ky) * N + i;
                R f = st[g], gg = st[NF + g];
                rowF.add(f);
                rowG.add(gg);
                col[ky].add(f);
                const R y = (R)xi[ky], xr = (R)x, v2 = xr * xr + y * y;
                ps2xy = fma(y, f, ps2xy);
                ps3x = fma(v2, f, ps3x);
                ps3y = fma(y * v2, f, ps3y);
                pg1y = fma(y, gg, pg1y);
            }
            const double rf = rowF.value(), rg = rowG.value();
            s0 += rf;
            s1x = fma(x, rf, s1x);
            s2xx = fma(x * x, rf, s2xx);
            g0 += rg;
            s2xy = fma((R)x, ps2xy, s2xy);
            s3x = fma((R)x, ps3x, s3x);
            s3y += ps3y;
            g1x = fma((R)x, (R)rg, g1x);
            g1y += pg1y;
        }
        double s1y = 0, s2yy = 0;
        for (int ky = 0; ky < Q; ++ky) {
            const double cv = col[ky].value();
            s1y = fma(xi[ky], cv, s1y);
            s2yy = fma(xi[ky] * xi[ky], cv, s2yy);
        }
        if (!isfinite(s0) || !isfinite(s2xx + s2yy + g0)) atomicOr(err, ERR_NONFINITE);
        mom[M2_S0 * N + i] = s0;
        mom[M2_S1X * N + i] = s1x;
        mom[M2_S1Y * N + i] = s1y;
        mom[M2_S2XX * N + i] = s2xx;
        mom[M2_S2YY * N + i] = s2yy;
        mom[M2_G0 * N + i] = g0;
        mom[M2_S2XY * N + i] = (double)s2xy;
        mom[M2_S3X * N + i] = (double)s3x;
        mom[M2_S3Y * N + i] = (double)s3y;
        mom[M2_G1X * N + i] = (double)g1x;
        mom[M2_G1Y * N + i] = (double)g1y;
    }
}

// n, u, T of one node from its raw sums
__device__ __forceinline__ void prim2(const double* __restrict__ mom, long long N, long long i, double& n, double& ux,
                                      double& uy, double& T) {
    n = mom[M2_S0 * N + i];
    ux = mom[M2_S1X * N + i] / n;
    uy = mom[M2_S1Y * N + i] / n;
    // (3/2) n T = (S2xx + S2yy)/2 + G0 - n u^2 / 2
    T = (2.0 / 3.0) * ((0.5 * (mom[M2_S2XX * N + i] + mom[M2_S2YY * N + i]) + mom[M2_G0 * N + i]) / n -
                       0.5 * (ux * ux + uy * uy));
}

// ---------------------------------------------------------------------------
// k2_fields: node fields of a 16x16 tile.
// ---------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(256)
k2_fields(Slab2 s, const double* __restrict__ mom, const int* __restrict__ ft_off, const R* __restrict__ ft_g,
          const int* __restrict__ fm_off, const double* __restrict__ fm_w, R* __restrict__ fld, unsigned* err) {
    extern __shared__ double sm2[];
    const int H = max(s.Mf, s.mfm + 2), W = kTile2 + 2 * H, E = kTile2 + 4;
    double* Nh = sm2;                 // n on the tile + H halo, [W][W]
    double* U = Nh + W * W;           // ux, uy, T, X, chi on the tile + 2, [E][E] each
    double* V = U + E * E;
    double* Tt = V + E * E;
    double* Xt = Tt + E * E;
    double* Ct = Xt + E * E;
    R* Nr = reinterpret_cast<R*>(Ct + E * E);   // n in R for the force (FP32)
    const int nx = s.nx, ny = s.ny;
    const long long N = s.N;
    const int x0 = blockIdx.x * kTile2, y0 = blockIdx.y * kTile2;
    for (int e = threadIdx.x; e < W * W; e += blockDim.x) {
        int cy = e / W, cx = e % W;
        long long i = (long long)wrapi(y0 - H + cy, ny) * nx + wrapi(x0 - H + cx, nx);
        double n = mom[M2_S0 * N + i];
        Nh[e] = n;
        Nr[e] = (R)n;
    }
    for (int e = threadIdx.x; e < E * E; e += blockDim.x) {
        int cy = e / E, cx = e % E;
        long long i = (long long)wrapi(y0 - 2 + cy, ny) * nx + wrapi(x0 - 2 + cx, nx);
        double n, ux, uy, T;
        prim2(mom, N, i, n, ux, uy, T);
        U[e] = ux;
        V[e] = uy;
        Tt[e] = T;
    }
    __syncthreads();
    // Fischer-Methfessel average, chi (Eq. (carnstar)) and X = n^2 chi T on the tile + 2
    for (int e = threadIdx.x; e < E * E; e += blockDim.x) {
        int cy = e / E, cx = e % E;
        int hy = cy - 2 + H, hx = cx - 2 + H;   // position in the halo array
        double nb = 0.0;
        for (int t = 0; t < s.nfm; ++t) nb = fma(fm_w[t], Nh[(hy + fm_off[2 * t + 1]) * W + hx + fm_off[2 * t]], nb);
        double eta = s.eta_coef * nb, om = 1.0 - eta;
        double chi = (2.0 - eta) / (2.0 * om * om * om);
        double n = Nh[hy * W + hx];
        Ct[e] = chi;
        Xt[e] = n * n * chi * Tt[e];
    }
    __syncthreads();
    const int tx = threadIdx.x % kTile2, ty = threadIdx.x / kTile2;
    const int x = x0 + tx, y = y0 + ty;
    if (x >= nx || y >= ny) return;
    const long long i = (long long)y * nx + x;
    const int c = (ty + 2) * E + (tx + 2);
    const double k12 = s.inv_dx / 12.0;
    auto d4x = [&](const double* f) { return (f[c - 2] - 8.0 * f[c - 1] + 8.0 * f[c + 1] - f[c + 2]) * k12; };
    auto d4y = [&](const double* f) { return (f[c - 2 * E] - 8.0 * f[c - E] + 8.0 * f[c + E] - f[c + 2 * E]) * k12; };
    const double n = Nh[(ty + H) * W + tx + H], ux = U[c], uy = V[c], T = Tt[c], X = Xt[c], chi = Ct[c];
    const double Ax = d4x(Xt) / X, Ay = d4y(Xt) / X, Bx = d4x(Tt) / T, By = d4y(Tt) / T;
    const double Dxx = d4x(U), Dxy = d4x(V), Dyx = d4y(U), Dyy = d4y(V);
    // force over the disc, rectangle rule (taps carry dx^2 g2)
    R fx = 0, fy = 0;
    const R* nc = Nr + (ty + H) * W + tx + H;
    for (int t = 0; t < s.nft; ++t) {
        R nn = nc[ft_off[2 * t + 1] * W + ft_off[2 * t]];
        fx = fma(ft_g[2 * t], nn, fx);
        fy = fma(ft_g[2 * t + 1], nn, fy);
    }
    // heat flux q_i = sum c_i (c^2/2 F + G)
    const double S0 = mom[M2_S0 * N + i], S1x = mom[M2_S1X * N + i], S1y = mom[M2_S1Y * N + i];
    const double S2xx = mom[M2_S2XX * N + i], S2yy = mom[M2_S2YY * N + i], S2xy = mom[M2_S2XY * N + i];
    const double S3x = mom[M2_S3X * N + i], S3y = mom[M2_S3Y * N + i], G0 = mom[M2_G0 * N + i];
    const double G1x = mom[M2_G1X * N + i], G1y = mom[M2_G1Y * N + i];
    const double u2 = ux * ux + uy * uy, S2 = S2xx + S2yy;
    const double uS1 = ux * S1x + uy * S1y;
    const double qx = 0.5 * (S3x - 2.0 * (ux * S2xx + uy * S2xy) + u2 * S1x - ux * S2 + 2.0 * ux * uS1 - ux * u2 * S0) +
                      G1x - ux * G0;
    const double qy = 0.5 * (S3y - 2.0 * (ux * S2xy + uy * S2yy) + u2 * S1y - uy * S2 + 2.0 * uy * uS1 - uy * u2 * S0) +
                      G1y - uy * G0;
    // transport, Eqs. (viscosity), (tau), (prandtl)
    const double bn = s.b * n, xx = bn * chi;
    const double mu = s.mu0_coef * sqrt(T) * (1.0 / chi + 0.8 * bn + (4.0 / 25.0) * (1.0 + 12.0 / M_PI) * bn * bn * chi);
    const double tau = mu / (n * T * (1.0 + 0.4 * xx));
    const double Pr = (2.0 / 3.0) * (1.0 + 0.6 * xx) * (1.0 + 0.8 * xx + (4.0 / 25.0) * (1.0 + 12.0 / M_PI) * xx * xx) /
                      ((1.0 + 0.4 * xx) * (1.0 + 1.2 * xx + (9.0 / 25.0) * (1.0 + 32.0 / (9.0 * M_PI)) * xx * xx));
    const double nu = (s.relax == EVFDLB_RELAX_INV_TAU) ? 1.0 / tau : chi / tau;
    if (!(n > 0.0) || !(T > 0.0)) atomicOr(err, (isfinite(n) && isfinite(T)) ? ERR_NEGATIVE : ERR_NONFINITE);
    else if (!isfinite((double)fx + (double)fy) || !isfinite(nu) || !isfinite(qx + qy) || !isfinite(Ax + Ay))
        atomicOr(err, ERR_NONFINITE);
    // polynomial coefficients of nu F^S + J1_F and nu G^S + J1_G over F_MB
    // (K = b n chi, sq = nu s with s = (1 - Pr)/(n T^2), div u = Dxx + Dyy)
    const double K = xx, sq = nu * (1.0 - Pr) / (n * T * T), dv = Dxx + Dyy, iT = 1.0 / T;
    double pf[10], pg[10];
    pf[0] = nu + 0.8 * K * dv;
    pf[1] = -0.8 * sq * qx - K * (Ax - 1.2 * Bx);
    pf[2] = -0.8 * sq * qy - K * (Ay - 1.2 * By);
    pf[3] = -0.4 * K * (Dxx + 0.5 * dv) * iT;
    pf[4] = -0.4 * K * (Dxy + Dyx) * iT;
    pf[5] = -0.4 * K * (Dyy + 0.5 * dv) * iT;
    pf[6] = 0.2 * sq * qx * iT - 0.3 * K * Bx * iT;
    pf[7] = 0.2 * sq * qy * iT - 0.3 * K * By * iT;
    pf[8] = 0.2 * sq * qx * iT - 0.3 * K * Bx * iT;
    pf[9] = 0.2 * sq * qy * iT - 0.3 * K * By * iT;
    pg[0] = 0.5 * nu * T + 0.2 * T * K * dv;
    pg[1] = -0.2 * T * sq * qx - 0.5 * T * K * (Ax - 0.6 * Bx);
    pg[2] = -0.2 * T * sq * qy - 0.5 * T * K * (Ay - 0.6 * By);
    pg[3] = -0.2 * K * (Dxx + 0.5 * dv);
    pg[4] = -0.2 * K * (Dxy + Dyx);
    pg[5] = -0.2 * K * (Dyy + 0.5 * dv);
    pg[6] = 0.1 * sq * qx - 0.15 * K * Bx;
    pg[7] = 0.1 * sq * qy - 0.15 * K * By;
    pg[8] = 0.1 * sq * qx - 0.15 * K * Bx;
    pg[9] = 0.1 * sq * qy - 0.15 * K * By;
    R* o = fld + i;
    o[F2_N * N] = (R)n;
    o[F2_UX * N] = (R)ux;
    o[F2_UY * N] = (R)uy;
    o[F2_T * N] = (R)T;
    o[F2_NU * N] = (R)nu;
    o[F2_FX * N] = fx;
    o[F2_FY * N] = fy;
    for (int j = 0; j < 10; ++j) {
        o[(F2_PF + j) * N] = (R)(n * pf[j]);
        o[(F2_PG + j) * N] = (R)(n * pg[j]);
    }
}

// ---------------------------------------------------------------------------
// k2_coll: per group of kNB nodes, the velocity-space part of the RHS.
// With m_l = E[psi_l(u + c)] and mu^a_l = E[c^a psi_l(u + c)] (c ~ N(0, T)):
//   mu^0 = m_l, mu^1 = T sqrt(l) m_{l-1}, mu^2 = T m_l + T^2 sqrt(l(l-1)) m_{l-2},
//   mu^3 = 3T^2 sqrt(l) m_{l-1} + T^3 sqrt(l(l-1)(l-2)) m_{l-3},
// the coefficient of psi_l(xi_x) psi_m(xi_y) of F_MB sum_ab P_ab c_x^a c_y^b is
// n sum_ab P_ab mu^a_l(u_x) mu^b_m(u_y).
// ---------------------------------------------------------------------------
// Shared layout of k2_coll: per distribution and node a Q x Q matrix with
// rows padded to kRow = 20 elements (a multiple of 4, so that rows are
// 16-byte aligned for four-wide loads, and 80 bytes apart, so that rows 4
// apart fall 16 banks apart: the eight threads of a quarter warp then read
// distinct banks in both transform directions), node stride padded by 4 so
// that the eight nodes of a group fall in different banks for the scalar
// state loads.
constexpr int kRow = 20;
__host__ __device__ constexpr int padded_q(int Q) { return (Q + 3) & ~3; }
__host__ __device__ constexpr int node_stride(int Q) { return padded_q(Q) * kRow + 4; }

template <typename R>
__host__ __device__ inline size_t coll_smem_bytes(int Q) {
    size_t X = 2 * (size_t)kNB * node_stride(Q);      // one [2][kNB][Q][kRow] buffer
    return sizeof(R) * (2 * (size_t)padded_q(Q) * kRow + 3 * (size_t)padded_q(Q) + 2 * X + kNumFld2 * kNB +
                        4 * (size_t)Q * kNB +
                        2 * 4 * (size_t)Q * kNB);
}

// Four consecutive elements of a 16-byte aligned shared row.
__device__ __forceinline__ void load4(const float* p, float v[4]) {
    const float4 q = *reinterpret_cast<const float4*>(p);
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
}
__device__ __forceinline__ void load4(const double* p, double v[4]) {
    const double2 a = reinterpret_cast<const double2*>(p)[0], b = reinterpret_cast<const double2*>(p)[1];
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}

// Out[i][j] = sum_k Lt[k][i] In[k][j]  (left contraction, Lt = transposed left matrix)
// or         sum_k In[i][k] Rt[k][j]  (right contraction, Rt = transposed right matrix)
// for the matrices of one (distribution, node); each thread forms a 4 x 4
// block from four-wide row loads: the left form walks k one row of Lt and
// In at a time, the right form four k at a time (four rows of In, four rows
// of Rt; the padded rows and columns Q .. Qp-1 are zero).
template <typename R, bool LEFT, int Q>
__device__ __forceinline__ void block_transform(const R* __restrict__ M, const R* __restrict__ In, R* __restrict__ Out,
                                                int i0, int j0) {
    R acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0;
    if constexpr (LEFT) {
#pragma unroll
        for (int k = 0; k < Q; ++k) {
            R m[4], x[4];
            load4(M + k * kRow + i0, m);       // Lt[k][i0 .. i0+3]
            load4(In + k * kRow + j0, x);      // In[k][j0 .. j0+3]
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] = fma(m[a], x[b], acc[a][b]);
        }
    } else {
        constexpr int Qp = padded_q(Q);
#pragma unroll
        for (int k = 0; k < Qp; k += 4) {
            R m[4][4], x[4][4];
#pragma unroll
            for (int a = 0; a < 4; ++a) load4(In + (i0 + a) * kRow + k, m[a]);   // In[i0 + a][k .. k+3]
#pragma unroll
            for (int q = 0; q < 4; ++q) load4(M + (k + q) * kRow + j0, x[q]);    // Rt[k + q][j0 .. j0+3]
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int b = 0; b < 4; ++b) acc[a][b] = fma(m[a][q], x[q][b], acc[a][b]);
        }
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) Out[(i0 + a) * kRow + j0 + b] = acc[a][b];
}

template <typename R, int Q>
__global__ void __launch_bounds__(256)
k2_coll(Slab2 s, const R* __restrict__ rtab, const R* __restrict__ st, const R* __restrict__ fld, R* __restrict__ RL) {
    extern __shared__ __align__(16) double smc[];
    constexpr int K = Q * Q, NS = node_stride(Q), Qp = padded_q(Q);
    const long long N = s.N, NF = (long long)K * N;
    const long long i0 = (long long)blockIdx.x * kNB;
    const int nb = (int)min((long long)kNB, N - i0);
    TableLayout L(Q);
    R* Pt = reinterpret_cast<R*>(smc);     // Pt[j][l] = psi_l(xi_j)       (transposed analysis table)
    R* St = Pt + Qp * kRow;                // St[l][k] = w_k psi_l(xi_k)   (transposed synthesis table)
    R* r1 = St + Qp * kRow;
    R* r2 = r1 + Qp;
    R* r3 = r2 + Qp;
    R* X0 = r3 + Qp;                       // [2][kNB] matrices, node stride NS (16-byte aligned)
    R* X1 = X0 + 2 * kNB * NS;
    R* sc = X1 + 2 * kNB * NS;             // [kNumFld2][kNB]
    R* mux = sc + kNumFld2 * kNB;          // [4][Q][kNB]
    R* Vy = mux + 4 * Q * kNB;             // [2][4][kNB][Q]
    auto mat = [&](R* X, int d, int t) { return X + (d * kNB + t) * NS; };
    for (int e = threadIdx.x; e < Qp * kRow; e += blockDim.x) {
        int r = e / kRow, c = e % kRow;
        Pt[e] = (c < Q && r < Q) ? rtab[L.P + c * Q + r] : R(0);
        St[e] = (c < Q && r < Q) ? rtab[L.S + c * Q + r] : R(0);
    }
    for (int e = threadIdx.x; e < Q; e += blockDim.x) {
        r1[e] = rtab[L.r1 + e];
        r2[e] = rtab[L.r2 + e];
        r3[e] = rtab[L.r3 + e];
    }
    // state of the group as [d][node][kx][ky] (ky contiguous, rows of kRow);
    // rows and columns Q .. Qp-1 of every matrix stay zero
    for (int e = threadIdx.x; e < 2 * 2 * kNB * NS; e += blockDim.x) X0[e] = R(0);
    __syncthreads();
    for (int e = threadIdx.x; e < 2 * K * kNB; e += blockDim.x) {
        int t = e % kNB, k = (e / kNB) % K, d = e / (kNB * K);
        mat(X0, d, t)[(k / Q) * kRow + k % Q] = (t < nb) ? st[d * NF + (long long)k * N + i0 + t] : R(0);
    }
    for (int e = threadIdx.x; e < kNumFld2 * kNB; e += blockDim.x) {
        int t = e % kNB, f = e / kNB;
        sc[e] = (t < nb) ? fld[f * N + i0 + t] : (f == F2_N || f == F2_T ? R(1) : R(0));
    }
    __syncthreads();
    // one-axis Gaussian moments: x for thread t < kNB, y (folded with the
    // polynomial coefficients) for kNB <= t < 2 kNB
    if (threadIdx.x < 2 * kNB) {
        const int t = threadIdx.x % kNB, axis = threadIdx.x / kNB;
        const R u = sc[(axis ? F2_UY : F2_UX) * kNB + t], T = sc[F2_T * kNB + t], Tm1 = T - R(1);
        R m[4] = {0, 0, 0, 0};   // m_{l}, m_{l-1}, m_{l-2}, m_{l-3}
        R m0 = 1, m1 = 0;
        R PF[4][4], PG[4][4];
        if (axis) {
            // P_ab as a 4x4 table (zero where a + b > 3)
            const int ia[10] = {0, 1, 0, 2, 1, 0, 3, 2, 1, 0}, ib[10] = {0, 0, 1, 0, 1, 2, 0, 1, 2, 3};
            for (int a = 0; a < 4; ++a)
                for (int b = 0; b < 4; ++b) PF[a][b] = PG[a][b] = 0;
            for (int j = 0; j < 10; ++j) {
                PF[ia[j]][ib[j]] = sc[(F2_PF + j) * kNB + t];
                PG[ia[j]][ib[j]] = sc[(F2_PG + j) * kNB + t];
            }
        }
        for (int l = 0; l < Q; ++l) {
            m[3] = m[2];
            m[2] = m[1];
            m[1] = m[0];
            m[0] = m0;
            R mu0 = m[0];
            R mu1 = T * r1[l] * m[1];
            R mu2 = T * m[0] + T * T * r2[l] * m[2];
            R mu3 = R(3) * T * T * r1[l] * m[1] + T * T * T * r3[l] * m[3];
            if (!axis) {
                mux[(0 * Q + l) * kNB + t] = mu0;
                mux[(1 * Q + l) * kNB + t] = mu1;
                mux[(2 * Q + l) * kNB + t] = mu2;
                mux[(3 * Q + l) * kNB + t] = mu3;
            } else {
                const R mb[4] = {mu0, mu1, mu2, mu3};
                for (int a = 0; a < 4; ++a) {
                    R vf = 0, vg = 0;
                    for (int b = 0; b < 4; ++b) {
                        vf = fma(PF[a][b], mb[b], vf);
                        vg = fma(PG[a][b], mb[b], vg);
                    }
                    Vy[((0 * 4 + a) * kNB + t) * Q + l] = vf;
                    Vy[((1 * 4 + a) * kNB + t) * Q + l] = vg;
                }
            }
            R mn = fma(u * rtab[L.rinv + l], m0, Tm1 * rtab[L.rr + l] * m1);
            m1 = m0;
            m0 = mn;
        }
    }
    // the four tensor transforms: one (distribution, node, 4x4 block) per thread
    const int nblk = (Qp / 4) * (Qp / 4);
    const int item = threadIdx.x / nblk, blk = threadIdx.x % nblk;   // item = d * kNB + node
    const bool active = item < 2 * kNB;
    const int d = item / kNB, t = item % kNB;
    const int bi = 4 * (blk / (Qp / 4)), bj = 4 * (blk % (Qp / 4));
    // Two buffers: the state is needed only by the first transform, since
    // -nu h is synthesised from -nu times its own analysis (the tensor
    // Gauss-Hermite transform of order Q per axis is invertible).
    // analysis along xi_x: X1[l][ky] = sum_kx psi_l(xi_kx) X0[kx][ky]
    if (active) block_transform<R, true, Q>(Pt, mat(X0, d, t), mat(X1, d, t), bi, bj);
    __syncthreads();
    // analysis along xi_y: X0[l][m] = sum_ky X1[l][ky] psi_m(xi_ky)
    if (active) block_transform<R, false, Q>(Pt, mat(X1, d, t), mat(X0, d, t), bi, bj);
    __syncthreads();
    // coefficients (relaxation -nu a, equilibria, J1, force terms) into X1: one y-order mm per
    // thread (lanes on consecutive mm: conflict-free rows), looping over the
    // x-order l; the y-moment factors of the thread are loop-invariant
    for (int e = threadIdx.x; e < 2 * kNB * Q; e += blockDim.x) {
        const int mm = e % Q, tt = (e / Q) % kNB, dd = e / (Q * kNB);
        const R* A = mat(X0, dd, tt);
        R* C = mat(X1, dd, tt);
        const R mnu = -sc[F2_NU * kNB + tt];
        R vy[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) vy[a] = Vy[((dd * 4 + a) * kNB + tt) * Q + mm];
        const R fx = sc[F2_FX * kNB + tt], fyr = sc[F2_FY * kNB + tt] * r1[mm];
#pragma unroll
        for (int l = 0; l < Q; ++l) {
            R c = 0;
#pragma unroll
            for (int a = 0; a < 4; ++a) c = fma(mux[(a * Q + l) * kNB + tt], vy[a], c);
            if (l >= 1) c = fma(fx * r1[l], A[(l - 1) * kRow + mm], c);
            if (mm >= 1) c = fma(fyr, A[l * kRow + mm - 1], c);
            c = fma(mnu, A[l * kRow + mm], c);
            C[l * kRow + mm] = c;
        }
    }
    __syncthreads();
    // synthesis along xi_x: X0[kx][m] = sum_l w_kx psi_l(xi_kx) X1[l][m]
    if (active) block_transform<R, true, Q>(St, mat(X1, d, t), mat(X0, d, t), bi, bj);
    __syncthreads();
    // synthesis along xi_y: X1[kx][ky] = sum_m X0[kx][m] w_ky psi_m(xi_ky)
    if (active) block_transform<R, false, Q>(St, mat(X0, d, t), mat(X1, d, t), bi, bj);
    __syncthreads();
    // the local right-hand side -nu h + sum S S c (both in X1)
    for (int e = threadIdx.x; e < 2 * K * kNB; e += blockDim.x) {
        int tt = e % kNB, k = (e / kNB) % K, dd = e / (kNB * K);
        if (tt >= nb) continue;
        const int off = (k / Q) * kRow + k % Q;
        RL[dd * NF + (long long)k * N + i0 + tt] = mat(X1, dd, tt)[off];
    }
}

// ---------------------------------------------------------------------------
// k2_adv: WENO-5 faces along x and y, the right-hand side and the RK combine.
// ---------------------------------------------------------------------------
// One WENO-5 face in difference form (the algebra of the 1D kernels): with
// d_i = v_{i+1} - v_i, the candidates are v2 plus corrections in d, the
// smoothness indicators 4 (eps + beta_r) = s_r^2 + 13/3 t_r^2 + 4 eps from
// first and second differences, and the linear weights are folded into the
// corrections; eps4 = 4 eps.
template <typename R>
__device__ __forceinline__ R weno5_2(R v0, R v1, R v2, R v3, R v4, R eps4) {
    const R d0 = v1 - v0, d1 = v2 - v1, d2 = v3 - v2, d3 = v4 - v3;
    const R t0 = d1 - d0, t1 = d2 - d1, t2 = d3 - d2;
    const R s0 = fma(R(3), d1, -d0), s1 = d1 + d2, s2 = fma(R(-3), d2, d3);
    const R k133 = R(13.0 / 3.0);
    const R e0 = fma(s0, s0, fma(k133 * t0, t0, eps4));
    const R e1 = fma(s1, s1, fma(k133 * t1, t1, eps4));
    const R e2 = fma(s2, s2, fma(k133 * t2, t2, eps4));
    const R E0 = e0 * e0, E1 = e1 * e1, E2 = e2 * e2;
    const R a0 = E1 * E2, a1 = E0 * E2, a2 = E0 * E1;
    const R c0 = fma(R(5.0 / 60.0), d1, R(-2.0 / 60.0) * d0);
    const R c1 = fma(R(0.2), d2, R(0.1) * d1);
    const R c2 = fma(R(0.2), d2, R(-0.05) * d3);
    const R num = fma(a0, c0, fma(a1, c1, a2 * c2));
    const R den = fma(R(0.1), a0, fma(R(0.6), a1, R(0.3) * a2));
    // FP32: the fast reciprocal-based quotient (2 ulp) is far inside the FP32
    // variant's error budget; FP64 keeps the IEEE quotient
    if constexpr (std::is_same<R, float>::value) return v2 + __fdividef(num, den);
    else return v2 + num / den;
}

// The five stencil values of a face from a shared-memory pointer and a
// compile-time stride: upwind for v >= 0 (q[0] .. q[4S]), mirrored for v < 0
// (q[5S] .. q[S]).  The sign is uniform over a plane, so the branch is too.
template <typename R, int S>
__device__ __forceinline__ R face_at(const R* q, bool pos, R eps4) {
    return pos ? weno5_2<R>(q[0], q[S], q[2 * S], q[3 * S], q[4 * S], eps4)
               : weno5_2<R>(q[5 * S], q[4 * S], q[3 * S], q[2 * S], q[S], eps4);
}

// k2_adv: a 32x16 node tile and a run of velocity planes.  Per plane the
// halo (tile +-3) is staged in shared memory (its global offsets computed
// once per CTA); warp w forms the x faces of rows 2w, 2w+1 and the y faces
// of face rows 2w, 2w+1 (lane = face or column); the last x face of each
// row and the last y-face row go to warps 0 and 1.  Stencil offsets are
// compile-time constants and the upwind branch is uniform per plane.  Then
// the right-hand side and the Shu-Osher combine
//   out = alpha base + beta (h + dt R)   (mode 0),   rhs_out = R (mode 1).
template <typename R>
__global__ void __launch_bounds__(256, 5)
k2_adv(Slab2 s, const R* __restrict__ rtab, const R* __restrict__ src, const R* base, R* out,
       const R* __restrict__ RL, double* rhs_out, double alpha, double beta, int mode) {
    constexpr int WX = kAdvX + 6, WY = kAdvY + 6, NH = WX * WY;
    constexpr int NHR = (NH + 255) / 256;                   // halo loads per thread
    constexpr int RPW = kAdvY / 8;                          // rows per warp
    __shared__ R Hs[NH];
    __shared__ R FX[kAdvY * (kAdvX + 1)];
    __shared__ R FY[(kAdvY + 1) * kAdvX];
    __shared__ long long rowoff[WY];
    __shared__ int coloff[WX];
    const int Q = s.Q, K = Q * Q, nx = s.nx, ny = s.ny;
    const long long N = s.N, NF = (long long)K * N;
    const int tilesx = (nx + kAdvX - 1) / kAdvX;
    const int x0 = (blockIdx.x % tilesx) * kAdvX, y0 = (blockIdx.x / tilesx) * kAdvY;
    TableLayout L(Q);
    // wrapped halo coordinates, shared by every plane of this tile
    for (int e = threadIdx.x; e < WY + WX; e += blockDim.x) {
        if (e < WY) rowoff[e] = (long long)wrapi(y0 - 3 + e, ny) * nx;
        else coloff[e - WY] = wrapi(x0 - 3 + (e - WY), nx);
    }
    __syncthreads();
    long long hoff[NHR];
#pragma unroll
    for (int j = 0; j < NHR; ++j) {
        const int e = threadIdx.x + 256 * j;
        hoff[j] = (e < NH) ? rowoff[e / WX] + coloff[e % WX] : 0;
    }
    const R eps4 = R(4) * (R)s.weno_eps, idx = (R)s.inv_dx, dt = (R)s.dt, ralpha = (R)alpha, rbeta = (R)beta;
    const bool with_base = (alpha != 0.0);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // output nodes of this thread (rows warp*RPW + rr, column lane) and
    // their offsets in a velocity plane
    const int x = x0 + lane;
    long long ooff[RPW];
    bool oval[RPW];
#pragma unroll
    for (int rr = 0; rr < RPW; ++rr) {
        const int y = y0 + warp * RPW + rr;
        oval[rr] = (x < nx && y < ny);
        ooff[rr] = (long long)y * nx + x;
    }
    const int p0 = blockIdx.y * kAdvPlanes, p1 = min(p0 + kAdvPlanes, 2 * K);
    for (int plane = p0; plane < p1; ++plane) {
        const int d = plane / K, k = plane % K;
        const R vx = rtab[L.xi + k / Q], vy = rtab[L.xi + k % Q];
        const long long pbase = d * NF + (long long)k * N;
        const R* h = src + pbase;
        __syncthreads();   // previous plane's faces and halo consumed
#pragma unroll
        for (int j = 0; j < NHR; ++j) {
            const int e = threadIdx.x + 256 * j;
            if (e < NH) Hs[e] = h[hoff[j]];
        }
        __syncthreads();
        const bool px = vx >= R(0), py = vy >= R(0);
#pragma unroll
        for (int rr = 0; rr < RPW; ++rr) {
            const int r = warp * RPW + rr;
            // x face `lane` of row r: stencil starts at halo column lane
            FX[r * (kAdvX + 1) + lane] = face_at<R, 1>(Hs + (r + 3) * WX + lane, px, eps4);
            // y face row r, column lane: stencil starts at halo row r
            FY[r * kAdvX + lane] = face_at<R, WX>(Hs + r * WX + lane + 3, py, eps4);
        }
        if (threadIdx.x < kAdvY) {                      // x face kAdvX of row threadIdx.x
            const int r = threadIdx.x;
            FX[r * (kAdvX + 1) + kAdvX] = face_at<R, 1>(Hs + (r + 3) * WX + kAdvX, px, eps4);
        } else if (threadIdx.x >= 32 && threadIdx.x < 32 + kAdvX) {   // y face row kAdvY
            const int c = threadIdx.x - 32;
            FY[kAdvY * kAdvX + c] = face_at<R, WX>(Hs + kAdvY * WX + c + 3, py, eps4);
        }
        __syncthreads();
#pragma unroll
        for (int rr = 0; rr < RPW; ++rr) {
            if (!oval[rr]) continue;
            const int ty = warp * RPW + rr;
            const long long g = pbase + ooff[rr];
            R Rv = RL[g];
            Rv = fma(-vx * idx, FX[ty * (kAdvX + 1) + lane + 1] - FX[ty * (kAdvX + 1) + lane], Rv);
            Rv = fma(-vy * idx, FY[(ty + 1) * kAdvX + lane] - FY[ty * kAdvX + lane], Rv);
            if (mode == 1) {
                rhs_out[g] = (double)Rv;
                continue;
            }
            const R hv = Hs[(ty + 3) * WX + lane + 3];
            R o = rbeta * fma(dt, Rv, hv);
            if (with_base) o = fma(ralpha, base[g], o);
            out[g] = o;
        }
    }
}

// ---------------------------------------------------------------------------
// Initial state, node moments and totals.
// ---------------------------------------------------------------------------
// Projected Maxwellian pair: F_{kx,ky} = n phi_kx(ux) phi_ky(uy) with
// phi_k(u) = sum_l S_kl m_l(u, T) (the 2D Gaussian factorises), G = T/2 F.
template <typename R>
__global__ void k2_init(Slab2 s, const double* __restrict__ tab, const double* __restrict__ n0,
                        const double* __restrict__ u0, const double* __restrict__ T0, R* st, unsigned* err) {
    const int Q = s.Q;
    const long long N = s.N, NF = (long long)Q * Q * N;
    TableLayout L(Q);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        double n = n0[i], ux = u0[i], uy = u0[N + i], T = T0[i];
        if (!(n > 0.0) || !(T > 0.0) || !isfinite(ux) || !isfinite(uy))
            atomicOr(err, (isfinite(n) && isfinite(T) && isfinite(ux) && isfinite(uy)) ? ERR_NEGATIVE : ERR_NONFINITE);
        double px[16], py[16];
        for (int axis = 0; axis < 2; ++axis) {
            double u = axis ? uy : ux, m0 = 1.0, m1 = 0.0, ml[16];
            for (int l = 0; l < Q; ++l) {
                ml[l] = m0;
                double mn = fma(u * tab[L.rinv + l], m0, (T - 1.0) * tab[L.rr + l] * m1);
                m1 = m0;
                m0 = mn;
            }
            for (int k = 0; k < Q; ++k) {
                double acc = 0.0;
                for (int l = 0; l < Q; ++l) acc = fma(tab[L.S + k * Q + l], ml[l], acc);
                (axis ? py : px)[k] = acc;
            }
        }
        for (int kx = 0; kx < Q; ++kx)
            for (int ky = 0; ky < Q; ++ky) {
                double f = n * px[kx] * py[ky];
                long long g = (long long)(kx * Q + ky) * N + i;
                st[g] = (R)f;
                st[NF + g] = (R)(0.5 * T * f);
            }
    }
}

__global__ void k2_prims(Slab2 s, const double* __restrict__ mom, double* n, double* u, double* T, double* q) {
    const long long N = s.N;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        double nn, ux, uy, TT;
        prim2(mom, N, i, nn, ux, uy, TT);
        if (n) n[i] = nn;
        if (u) {
            u[i] = ux;
            u[N + i] = uy;
        }
        if (T) T[i] = TT;
        if (q) {
            const double S0 = mom[M2_S0 * N + i], S1x = mom[M2_S1X * N + i], S1y = mom[M2_S1Y * N + i];
            const double S2xx = mom[M2_S2XX * N + i], S2yy = mom[M2_S2YY * N + i], S2xy = mom[M2_S2XY * N + i];
            const double u2 = ux * ux + uy * uy, S2 = S2xx + S2yy, uS1 = ux * S1x + uy * S1y;
            q[i] = 0.5 * (mom[M2_S3X * N + i] - 2.0 * (ux * S2xx + uy * S2xy) + u2 * S1x - ux * S2 + 2.0 * ux * uS1 -
                          ux * u2 * S0) + mom[M2_G1X * N + i] - ux * mom[M2_G0 * N + i];
            q[N + i] = 0.5 * (mom[M2_S3Y * N + i] - 2.0 * (ux * S2xy + uy * S2yy) + u2 * S1y - uy * S2 + 2.0 * uy * uS1 -
                              uy * u2 * S0) + mom[M2_G1Y * N + i] - uy * mom[M2_G0 * N + i];
        }
    }
}

// {mass, momentum x, momentum y, kinetic + internal energy} x dx^2; one CTA,
// fixed-order tree (deterministic)
__global__ void __launch_bounds__(256) k2_totals(Slab2 s, const double* __restrict__ mom, double* out) {
    __shared__ double red[4][256];
    const long long N = s.N;
    double a[4] = {0, 0, 0, 0};
    for (long long i = threadIdx.x; i < N; i += blockDim.x) {
        a[0] += mom[M2_S0 * N + i];
        a[1] += mom[M2_S1X * N + i];
        a[2] += mom[M2_S1Y * N + i];
        a[3] += 0.5 * (mom[M2_S2XX * N + i] + mom[M2_S2YY * N + i]) + mom[M2_G0 * N + i];
    }
    for (int c = 0; c < 4; ++c) red[c][threadIdx.x] = a[c];
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int c = 0; c < 4; ++c) red[c][threadIdx.x] += red[c][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < 4) out[threadIdx.x] = red[threadIdx.x][0] * s.dx * s.dx;
}

template <typename A, typename B>
__global__ void k2_convert(const A* __restrict__ in, B* __restrict__ out, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = (B)in[i];
}

// ---------------------------------------------------------------------------
// Host side: the 2D context.
// ---------------------------------------------------------------------------
namespace {
const long double kPiL2 = 3.141592653589793238462643383279502884L;

// Gauss-Legendre nodes and weights of order n on [-1, 1] in long double
// (Newton on the Legendre recurrence).
void gauss_legendre_ld(int n, std::vector<long double>& x, std::vector<long double>& w) {
    x.resize(n);
    w.resize(n);
    for (int i = 0; i < n; ++i) {
        long double z = cosl(kPiL2 * (i + 0.75L) / (n + 0.5L)), pp = 0;
        for (int it = 0; it < 100; ++it) {
            long double p1 = 1, p2 = 0;
            for (int j = 1; j <= n; ++j) {
                long double p3 = p2;
                p2 = p1;
                p1 = ((2.0L * j - 1.0L) * z * p2 - (j - 1.0L) * p3) / j;
            }
            pp = n * (z * p1 - p2) / (z * z - 1.0L);
            long double dz = p1 / pp;
            z -= dz;
            if (fabsl(dz) < 1e-19L) break;
        }
        x[i] = z;
        w[i] = 2.0L / ((1.0L - z * z) * pp * pp);
    }
}

// g2 at offset (rx, ry) (components), Eq. (force) integrated over z with
// r = sqrt(rho^2 + z^2) > sigma, gamma = 2(s - 1) even:
//   rho >= sigma: Wallis, int (rho^2 + z^2)^-s dz = rho^(1-2s) pi (2s-3)!!/(2s-2)!!;
//   rho <  sigma: with z = rho cot(psi), 2 rho^(1-2s) int_0^{psi0} sin^(2s-2) psi d psi,
//                 psi0 = atan(rho / z0), by 48-point Gauss-Legendre in long double.
void g2_kernel(const evfdlb_params& p, long double rx, long double ry, long double* gx, long double* gy) {
    long double r = sqrtl(rx * rx + ry * ry), sg = p.sigma;
    *gx = *gy = 0;
    if (r == 0) return;
    int s = (int)llround((p.gamma + 2.0) / 2.0);
    long double J;
    if (r >= sg) {
        long double wallis = kPiL2;
        for (int k = 1; k <= s - 1; ++k) wallis *= (2.0L * k - 1.0L) / (2.0L * k);
        J = wallis * powl(r, 1.0L - 2.0L * s);
    } else {
        static std::vector<long double> gxs, gws;
        if (gxs.empty()) gauss_legendre_ld(48, gxs, gws);
        long double z0 = sqrtl(sg * sg - r * r), psi0 = atanl(r / z0), acc = 0;
        for (int i = 0; i < 48; ++i) {
            long double ps = 0.5L * psi0 * (gxs[i] + 1.0L);
            acc += gws[i] * powl(sinl(ps), 2 * s - 2);
        }
        J = 2.0L * powl(r, 1.0L - 2.0L * s) * 0.5L * psi0 * acc;
    }
    long double c = (long double)p.gamma * p.phi_a * powl(sg, (long double)p.gamma) * J;
    *gx = c * rx;
    *gy = c * ry;
}

struct Taps2 {
    std::vector<int> foff, moff;
    std::vector<double> fg, mw;
    int Mf = 0, mfm = 0;
};

Taps2 taps_2d(const evfdlb_params& p) {
    Taps2 t;
    const double dx = p.dx, rc = p.r_cut, sg = p.sigma;
    t.Mf = (int)floor(rc / dx + 1e-9);
    for (int a = -t.Mf; a <= t.Mf; ++a)
        for (int b = -t.Mf; b <= t.Mf; ++b) {
            double rx = a * dx, ry = b * dx;
            if (rx * rx + ry * ry > rc * rc * (1.0 + 1e-12) || (a == 0 && b == 0)) continue;
            long double gx, gy;
            g2_kernel(p, rx, ry, &gx, &gy);
            t.foff.push_back(a);
            t.foff.push_back(b);
            t.fg.push_back((double)(dx * dx * gx));
            t.fg.push_back((double)(dx * dx * gy));
        }
    t.mfm = (int)ceil(sg / dx);
    long double wsum = 0;
    std::vector<long double> w;
    for (int a = -t.mfm; a <= t.mfm; ++a)
        for (int b = -t.mfm; b <= t.mfm; ++b) {
            long double r2 = (long double)(a * a + b * b) * dx * dx;
            if (r2 >= (long double)sg * sg) continue;
            long double v = 2.0L * sqrtl((long double)sg * sg - r2);
            t.moff.push_back(a);
            t.moff.push_back(b);
            w.push_back(v);
            wsum += v;
        }
    for (long double v : w) t.mw.push_back((double)(v / wsum));
    return t;
}
}  // namespace

bool validate_2d(const evfdlb_params& p) {
    if (p.dim != 2 || p.nx < 8 || p.ny < 8 || !(p.dx > 0) || !(p.sigma > 0) || !(p.phi_a >= 0)) return false;
    if (p.Q < 4 || p.Q > 16 || (p.Q & 1) || p.bc != EVFDLB_BC_PERIODIC) return false;
    if (p.relax_mode != EVFDLB_RELAX_INV_TAU && p.relax_mode != EVFDLB_RELAX_CHI_OVER_TAU) return false;
    if (!(p.weno_eps > 0) || (!(p.dt > 0) && !(p.cfl > 0 && p.cfl <= 1))) return false;
    double g2 = (p.gamma + 2.0) / 2.0;
    if (!(p.gamma > 3) || fabs(g2 - llround(g2)) > 1e-12) return false;   // even integer gamma
    if (!(p.r_cut >= p.sigma + 2 * p.dx)) return false;
    if (p.precision != EVFDLB_FP64 && p.precision != EVFDLB_FP32) return false;
    return true;
}

double resolved_dt_2d(const evfdlb_params& p) {
    if (p.dt > 0) return p.dt;
    double xi[kQMax], w[kQMax];
    velocity_set(p.Q, xi, w);
    // dimension-by-dimension upwind: |xi_x| + |xi_y| <= 2 max|xi| per dx
    return p.cfl * p.dx / (2.0 * fabs(xi[p.Q - 1]));
}

double discrete_a_2d(const evfdlb_params& p) {
    Taps2 t = taps_2d(p);
    long double acc = 0;
    for (size_t j = 0; j < t.fg.size() / 2; ++j) acc += (long double)t.foff[2 * j] * p.dx * t.fg[2 * j];
    return (double)(0.5L * acc);
}

struct Ctx2 {
    evfdlb_params p;
    Slab2 s;
    int prec = EVFDLB_FP32;
    size_t esize = 4;
    cudaStream_t user = nullptr, cap = nullptr;
    void* state[3] = {nullptr, nullptr, nullptr};
    void* RL = nullptr;
    void* fld = nullptr;
    double* mom = nullptr;
    double* tables = nullptr;
    void* rtab = nullptr;
    int* ft_off = nullptr;
    void* ft_g = nullptr;
    int* fm_off = nullptr;
    double* fm_w = nullptr;
    double* scratch = nullptr;   // [2 Q^2 N + 8] doubles
    unsigned* err = nullptr;
    cudaGraphExec_t g_one = nullptr;
    size_t smem_fields = 0, smem_coll = 0;
};

namespace {
// k2_coll is compiled for each even Q of the 2D model (4 .. 16)
template <typename R>
void launch_coll(int Q, int nc, size_t smem, cudaStream_t st, const Slab2& s, const R* rtab, const R* src,
                 const R* fld, R* RL) {
    switch (Q) {
        case 4: k2_coll<R, 4><<<nc, 256, smem, st>>>(s, rtab, src, fld, RL); break;
        case 6: k2_coll<R, 6><<<nc, 256, smem, st>>>(s, rtab, src, fld, RL); break;
        case 8: k2_coll<R, 8><<<nc, 256, smem, st>>>(s, rtab, src, fld, RL); break;
        case 10: k2_coll<R, 10><<<nc, 256, smem, st>>>(s, rtab, src, fld, RL); break;
        case 12: k2_coll<R, 12><<<nc, 256, smem, st>>>(s, rtab, src, fld, RL); break;
        case 14: k2_coll<R, 14><<<nc, 256, smem, st>>>(s, rtab, src, fld, RL); break;
        default: k2_coll<R, 16><<<nc, 256, smem, st>>>(s, rtab, src, fld, RL); break;
    }
}

template <typename R>
cudaError_t coll_attr(int Q, size_t smem) {
    const int v = (int)smem;
    switch (Q) {
        case 4: return cudaFuncSetAttribute(k2_coll<R, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, v);
        case 6: return cudaFuncSetAttribute(k2_coll<R, 6>, cudaFuncAttributeMaxDynamicSharedMemorySize, v);
        case 8: return cudaFuncSetAttribute(k2_coll<R, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, v);
        case 10: return cudaFuncSetAttribute(k2_coll<R, 10>, cudaFuncAttributeMaxDynamicSharedMemorySize, v);
        case 12: return cudaFuncSetAttribute(k2_coll<R, 12>, cudaFuncAttributeMaxDynamicSharedMemorySize, v);
        case 14: return cudaFuncSetAttribute(k2_coll<R, 14>, cudaFuncAttributeMaxDynamicSharedMemorySize, v);
        default: return cudaFuncSetAttribute(k2_coll<R, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, v);
    }
}

template <typename R>
void queue_stage_t(Ctx2* c, cudaStream_t st, const void* src, const void* base, void* out, double* rhs_out,
                   double alpha, double beta, int mode) {
    const Slab2& s = c->s;
    const int Q = s.Q;
    int nb = (int)std::min<long long>((s.N + 255) / 256, 4096);
    k2_moments<R><<<nb, 256, 0, st>>>(s, c->tables, (const R*)src, c->mom, c->err);
    dim3 gf((s.nx + kTile2 - 1) / kTile2, (s.ny + kTile2 - 1) / kTile2);
    k2_fields<R><<<gf, 256, c->smem_fields, st>>>(s, c->mom, c->ft_off, (const R*)c->ft_g, c->fm_off, c->fm_w,
                                                   (R*)c->fld, c->err);
    int nc = (int)((s.N + kNB - 1) / kNB);
    launch_coll<R>(Q, nc, c->smem_coll, st, s, (const R*)c->rtab, (const R*)src, (const R*)c->fld, (R*)c->RL);
    dim3 ga(((s.nx + kAdvX - 1) / kAdvX) * ((s.ny + kAdvY - 1) / kAdvY), (2 * Q * Q + kAdvPlanes - 1) / kAdvPlanes);
    k2_adv<R><<<ga, 256, 0, st>>>(s, (const R*)c->rtab, (const R*)src, (const R*)base, (R*)out, (const R*)c->RL,
                                   rhs_out, alpha, beta, mode);
}

void queue_stage(Ctx2* c, cudaStream_t st, const void* src, const void* base, void* out, double* rhs_out,
                 double alpha, double beta, int mode) {
    if (c->prec == EVFDLB_FP32) queue_stage_t<float>(c, st, src, base, out, rhs_out, alpha, beta, mode);
    else queue_stage_t<double>(c, st, src, base, out, rhs_out, alpha, beta, mode);
}

void queue_step(Ctx2* c, cudaStream_t st) {
    queue_stage(c, st, c->state[0], nullptr, c->state[1], nullptr, 0.0, 1.0, 0);
    queue_stage(c, st, c->state[1], c->state[0], c->state[2], nullptr, 0.75, 0.25, 0);
    queue_stage(c, st, c->state[2], c->state[0], c->state[0], nullptr, 1.0 / 3.0, 2.0 / 3.0, 0);
}

evfdlb_status st2(cudaError_t e) {
    return e == cudaSuccess ? EVFDLB_OK : (e == cudaErrorMemoryAllocation ? EVFDLB_E_OOM : EVFDLB_E_CUDA);
}
}  // namespace

void destroy_2d(Ctx2* c) {
    if (!c) return;
    if (c->g_one) cudaGraphExecDestroy(c->g_one);
    for (int i = 0; i < 3; ++i) cudaFree(c->state[i]);
    cudaFree(c->RL);
    cudaFree(c->fld);
    cudaFree(c->mom);
    cudaFree(c->tables);
    if (c->rtab != c->tables) cudaFree(c->rtab);
    cudaFree(c->ft_off);
    cudaFree(c->ft_g);
    cudaFree(c->fm_off);
    cudaFree(c->fm_w);
    cudaFree(c->scratch);
    cudaFree(c->err);
    if (c->cap) cudaStreamDestroy(c->cap);
    delete c;
}

evfdlb_status create_2d(const evfdlb_params& p, void* stream, Ctx2** out) {
    *out = nullptr;
    if (!validate_2d(p)) return EVFDLB_E_INVALID_ARG;
    if (p.force_model != EVFDLB_EV1 || p.T_iso != 0.0) return EVFDLB_E_UNSUPPORTED;
    Ctx2* c = new (std::nothrow) Ctx2();
    if (!c) return EVFDLB_E_OOM;
    c->p = p;
    c->prec = p.precision;
    c->esize = (c->prec == EVFDLB_FP32) ? sizeof(float) : sizeof(double);
    c->user = (cudaStream_t)stream;
    Slab2& s = c->s;
    s.nx = p.nx;
    s.ny = p.ny;
    s.Q = p.Q;
    s.relax = p.relax_mode;
    s.N = (long long)p.nx * p.ny;
    s.dx = p.dx;
    s.inv_dx = 1.0 / p.dx;
    s.dt = resolved_dt_2d(p);
    s.weno_eps = p.weno_eps;
    s.b = 2.0 * M_PI * p.sigma * p.sigma * p.sigma / 3.0;
    s.eta_coef = M_PI * p.sigma * p.sigma * p.sigma / 6.0;
    s.mu0_coef = 5.0 / (16.0 * p.sigma * p.sigma * sqrt(M_PI));
    Taps2 t = taps_2d(p);
    s.nft = (int)(t.fg.size() / 2);
    s.nfm = (int)t.mw.size();
    s.Mf = t.Mf;
    s.mfm = t.mfm;
    TableLayout L(p.Q);
    std::vector<double> tab(L.total), xi(p.Q), w(p.Q);
    velocity_set(p.Q, xi.data(), w.data());
    build_tables(p.Q, xi.data(), w.data(), tab.data());
    const long long NF = (long long)p.Q * p.Q * s.N;
    cudaError_t e = cudaSuccess;
    auto alloc = [&](void** ptr, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc(ptr, bytes);
    };
    for (int i = 0; i < 3; ++i) alloc(&c->state[i], c->esize * 2 * NF);
    alloc(&c->RL, c->esize * 2 * NF);
    alloc(&c->fld, c->esize * kNumFld2 * s.N);
    alloc((void**)&c->mom, sizeof(double) * kNumMom2 * s.N);
    alloc((void**)&c->tables, sizeof(double) * tab.size());
    alloc((void**)&c->ft_off, sizeof(int) * t.foff.size());
    alloc(&c->ft_g, c->esize * t.fg.size());
    alloc((void**)&c->fm_off, sizeof(int) * t.moff.size());
    alloc((void**)&c->fm_w, sizeof(double) * t.mw.size());
    alloc((void**)&c->scratch, sizeof(double) * (2 * NF + 8));
    alloc((void**)&c->err, sizeof(unsigned));
    std::vector<float> tabf(tab.begin(), tab.end()), fgf(t.fg.begin(), t.fg.end());
    if (c->prec == EVFDLB_FP32) alloc(&c->rtab, sizeof(float) * tab.size());
    else c->rtab = c->tables;
    if (e == cudaSuccess) e = cudaMemcpy(c->tables, tab.data(), sizeof(double) * tab.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && c->prec == EVFDLB_FP32)
        e = cudaMemcpy(c->rtab, tabf.data(), sizeof(float) * tabf.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(c->ft_off, t.foff.data(), sizeof(int) * t.foff.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = (c->prec == EVFDLB_FP32)
                ? cudaMemcpy(c->ft_g, fgf.data(), sizeof(float) * fgf.size(), cudaMemcpyHostToDevice)
                : cudaMemcpy(c->ft_g, t.fg.data(), sizeof(double) * t.fg.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(c->fm_off, t.moff.data(), sizeof(int) * t.moff.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(c->fm_w, t.mw.data(), sizeof(double) * t.mw.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(c->err, 0, sizeof(unsigned));
    const int H = std::max(s.Mf, s.mfm + 2), Wd = kTile2 + 2 * H, Ed = kTile2 + 4;
    c->smem_fields = sizeof(double) * ((size_t)Wd * Wd + 5 * (size_t)Ed * Ed) + c->esize * (size_t)Wd * Wd;
    c->smem_coll = (c->prec == EVFDLB_FP32) ? coll_smem_bytes<float>(p.Q) : coll_smem_bytes<double>(p.Q);
    if (c->smem_fields > 227 * 1024) e = cudaErrorInvalidValue;   // force disc too wide for a tile
    if (e == cudaSuccess) {
        if (c->prec == EVFDLB_FP32) {
            e = cudaFuncSetAttribute(k2_fields<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c->smem_fields);
            if (e == cudaSuccess) e = coll_attr<float>(p.Q, c->smem_coll);
        } else {
            e = cudaFuncSetAttribute(k2_fields<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c->smem_fields);
            if (e == cudaSuccess) e = coll_attr<double>(p.Q, c->smem_coll);
        }
    }
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) {
        cudaGraph_t g = nullptr;
        e = cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            queue_step(c, c->cap);
            e = cudaStreamEndCapture(c->cap, &g);
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&c->g_one, g, 0);
        if (g) cudaGraphDestroy(g);
    }
    if (e != cudaSuccess) {
        evfdlb_status r = (e == cudaErrorInvalidValue) ? EVFDLB_E_INVALID_ARG : st2(e);
        destroy_2d(c);
        return r;
    }
    *out = c;
    return EVFDLB_OK;
}

// Reads and clears the device error word (synchronises the stream).
evfdlb_status check_2d(Ctx2* c) {
    unsigned h = 0;
    cudaError_t e = cudaMemcpyAsync(&h, c->err, sizeof(unsigned), cudaMemcpyDeviceToHost, c->user);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->user);
    if (e != cudaSuccess) return st2(e);
    if (h) {
        cudaMemsetAsync(c->err, 0, sizeof(unsigned), c->user);
        return (h & ERR_NONFINITE) ? EVFDLB_E_NONFINITE : EVFDLB_E_NEGATIVE;
    }
    return EVFDLB_OK;
}

long long nodes_2d(const Ctx2* c) { return c->s.N; }
long long dist_2d(const Ctx2* c) { return (long long)c->s.Q * c->s.Q * c->s.N; }
double dt_2d(const Ctx2* c) { return c->s.dt; }

evfdlb_status init_2d(Ctx2* c, const double* n0, const double* u0, const double* T0, int on_device) {
    const long long N = c->s.N;
    const double *dn = n0, *du = u0, *dT = T0;
    cudaError_t e = cudaSuccess;
    if (!on_device) {
        double* b = c->scratch;   // [4 N] fits: 2 Q^2 N >= 4 N
        e = cudaMemcpyAsync(b, n0, sizeof(double) * N, cudaMemcpyHostToDevice, c->user);
        if (e == cudaSuccess) e = cudaMemcpyAsync(b + N, u0, sizeof(double) * 2 * N, cudaMemcpyHostToDevice, c->user);
        if (e == cudaSuccess) e = cudaMemcpyAsync(b + 3 * N, T0, sizeof(double) * N, cudaMemcpyHostToDevice, c->user);
        dn = b;
        du = b + N;
        dT = b + 3 * N;
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(c->err, 0, sizeof(unsigned), c->user);
    if (e != cudaSuccess) return st2(e);
    int nb = (int)std::min<long long>((N + 255) / 256, 4096);
    if (c->prec == EVFDLB_FP32) k2_init<float><<<nb, 256, 0, c->user>>>(c->s, c->tables, dn, du, dT, (float*)c->state[0], c->err);
    else k2_init<double><<<nb, 256, 0, c->user>>>(c->s, c->tables, dn, du, dT, (double*)c->state[0], c->err);
    if ((e = cudaGetLastError()) != cudaSuccess) return st2(e);
    return check_2d(c);
}

evfdlb_status step_async_2d(Ctx2* c, int64_t nsteps) {
    for (int64_t i = 0; i < nsteps; ++i) {
        cudaError_t e = cudaGraphLaunch(c->g_one, c->user);
        if (e != cudaSuccess) return st2(e);
    }
    return EVFDLB_OK;
}

evfdlb_status get_state_2d(Ctx2* c, double* F, double* G, int on_device) {
    const long long NF = dist_2d(c);
    const double* src = (const double*)c->state[0];
    cudaError_t e = cudaSuccess;
    if (c->prec == EVFDLB_FP32) {
        k2_convert<float, double><<<4096, 256, 0, c->user>>>((const float*)c->state[0], c->scratch, 2 * NF);
        src = c->scratch;
        e = cudaGetLastError();
    }
    cudaMemcpyKind kd = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (e == cudaSuccess) e = cudaMemcpyAsync(F, src, sizeof(double) * NF, kd, c->user);
    if (e == cudaSuccess) e = cudaMemcpyAsync(G, src + NF, sizeof(double) * NF, kd, c->user);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->user);
    return st2(e);
}

evfdlb_status set_state_2d(Ctx2* c, const double* F, const double* G, int on_device) {
    const long long NF = dist_2d(c);
    double* dst = (c->prec == EVFDLB_FP32) ? c->scratch : (double*)c->state[0];
    cudaMemcpyKind kd = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    cudaError_t e = cudaMemcpyAsync(dst, F, sizeof(double) * NF, kd, c->user);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dst + NF, G, sizeof(double) * NF, kd, c->user);
    if (e == cudaSuccess && c->prec == EVFDLB_FP32) {
        k2_convert<double, float><<<4096, 256, 0, c->user>>>(c->scratch, (float*)c->state[0], 2 * NF);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(c->err, 0, sizeof(unsigned), c->user);
    if (e != cudaSuccess) return st2(e);
    return check_2d(c);
}

evfdlb_status rhs_2d(Ctx2* c, double* RF, double* RG, int on_device) {
    const long long NF = dist_2d(c);
    queue_stage(c, c->user, c->state[0], nullptr, nullptr, c->scratch, 0.0, 1.0, 1);
    cudaError_t e = cudaGetLastError();
    cudaMemcpyKind kd = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (e == cudaSuccess) e = cudaMemcpyAsync(RF, c->scratch, sizeof(double) * NF, kd, c->user);
    if (e == cudaSuccess) e = cudaMemcpyAsync(RG, c->scratch + NF, sizeof(double) * NF, kd, c->user);
    if (e != cudaSuccess) return st2(e);
    return check_2d(c);
}

evfdlb_status moments_2d(Ctx2* c, double* n, double* u, double* T, double* q, double* totals, int on_device) {
    const long long N = c->s.N;
    int nb = (int)std::min<long long>((N + 255) / 256, 4096);
    if (c->prec == EVFDLB_FP32) k2_moments<float><<<nb, 256, 0, c->user>>>(c->s, c->tables, (const float*)c->state[0], c->mom, c->err);
    else k2_moments<double><<<nb, 256, 0, c->user>>>(c->s, c->tables, (const double*)c->state[0], c->mom, c->err);
    double* b = c->scratch;   // n [N], u [2N], T [N], q [2N], totals [4]
    double* dn = n ? (on_device ? n : b) : nullptr;
    double* du = u ? (on_device ? u : b + N) : nullptr;
    double* dT = T ? (on_device ? T : b + 3 * N) : nullptr;
    double* dq = q ? (on_device ? q : b + 4 * N) : nullptr;
    k2_prims<<<nb, 256, 0, c->user>>>(c->s, c->mom, dn, du, dT, dq);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && !on_device) {
        if (n) e = cudaMemcpyAsync(n, dn, sizeof(double) * N, cudaMemcpyDeviceToHost, c->user);
        if (e == cudaSuccess && u) e = cudaMemcpyAsync(u, du, sizeof(double) * 2 * N, cudaMemcpyDeviceToHost, c->user);
        if (e == cudaSuccess && T) e = cudaMemcpyAsync(T, dT, sizeof(double) * N, cudaMemcpyDeviceToHost, c->user);
        if (e == cudaSuccess && q) e = cudaMemcpyAsync(q, dq, sizeof(double) * 2 * N, cudaMemcpyDeviceToHost, c->user);
    }
    if (e == cudaSuccess && totals) {
        k2_totals<<<1, 256, 0, c->user>>>(c->s, c->mom, b + 6 * N);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpyAsync(totals, b + 6 * N, sizeof(double) * 4, cudaMemcpyDeviceToHost, c->user);
    }
    if (e != cudaSuccess) return st2(e);
    return check_2d(c);
}

}  // namespace evfdlb
