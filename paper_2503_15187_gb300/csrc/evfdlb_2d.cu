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

#include "evfdlb_device.cuh"
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
constexpr int kNB = 16;        // nodes per k2_coll CTA (half a warp: a lane per node and distribution)
static_assert(kNB == 16, "k2_coll maps the 32 lanes of a warp to 2 distributions x 16 nodes");
constexpr int kAdvX = 32, kAdvY = 16, kAdvPlanes = 8;
static_assert(kAdvX == 32 && kAdvY % 8 == 0, "k2_adv maps a warp (256 threads per CTA) to tile rows");

__device__ __forceinline__ int wrapi(int i, int n) {
    int r = i % n;
    return r < 0 ? r + n : r;
}

// ---------------------------------------------------------------------------
// k2_moments: per node, raw sums over the Q^2 velocities.  Conserved sums
// (S0, S1, S2xx, S2yy, G0) are formed from the row and column sums of the
// velocity grid.  For an FP32 state each 16-term row or column sum is a
// compensated FP32 sum kept as an unevaluated pair (TwoSum, Knuth), and the
// rows and columns are combined in float-float arithmetic (TwoSum and the
// FMA TwoProduct against the velocity powers split into float pairs,
// Ogita-Rump-Oishi): about 2^-44 of the sum of magnitudes, FP64 quality on
// the FP32 pipe (the FP64 pipe of this GPU runs at 1/64 of the FP32 rate).
// The heat-flux sums are plain R sums.  Outputs: the FP64 raw sums (when
// `mom` is given) and, for an FP32 state, the node primitives n, u, T, q in
// FP32 (when `prf` is given: what the stage's field kernel reads).
// ---------------------------------------------------------------------------
enum { P2_N = 0, P2_UX, P2_UY, P2_T, P2_QX, P2_QY, kNumPrf2 };

// velocity powers of the velocity set, passed by value (kernel parameter
// space, read as constant operands once the loops are unrolled)
template <typename R>
struct Pow2 {
    R v[16], v2[16], v3[16];            // xi, xi^2, xi^3 in R
    float h[16], l[16], h2[16], l2[16];  // xi and xi^2 (FP64) as float pairs
};

template <typename R>
struct CompSum {                       // R = double: plain accumulation
    double s = 0.0;
    __device__ __forceinline__ void add(R x) { s += (double)x; }
};
template <>
struct CompSum<float> {                // TwoSum: s + c carries the exact sum to O(n u^2)
    float s = 0.0f, c = 0.0f;
    __device__ __forceinline__ void add(float x) {
        const float t = __fadd_rn(s, x), z = __fsub_rn(t, s);
        c = __fadd_rn(c, __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(x, z)));
        s = t;
    }
};

// float-float accumulator (hi, lo)
struct FF {
    float h = 0.0f, l = 0.0f;
    // += (a + b), a pair
    __device__ __forceinline__ void add(float a, float b) {
        const float t = __fadd_rn(h, a), z = __fsub_rn(t, h);
        const float e = __fadd_rn(__fsub_rn(h, __fsub_rn(t, z)), __fsub_rn(a, z));
        l = __fadd_rn(l, __fadd_rn(e, b));
        h = t;
    }
    // += (xh + xl)(a + b); the xl b term is below the pair's precision
    __device__ __forceinline__ void fma2(float xh, float xl, float a, float b) {
        const float p = __fmul_rn(xh, a), pe = fmaf(xh, a, -p);
        const float t = __fadd_rn(h, p), z = __fsub_rn(t, h);
        const float e = __fadd_rn(__fsub_rn(h, __fsub_rn(t, z)), __fsub_rn(p, z));
        l = __fadd_rn(l, __fadd_rn(e, pe));
        l = fmaf(xh, b, l);
        l = fmaf(xl, a, l);
        h = t;
    }
    __device__ __forceinline__ float value() const { return h + l; }
    __device__ __forceinline__ double value64() const { return (double)h + (double)l; }
};

// Partial raw sums of one node over half of the y velocities (ky = K0 ..
// K0 + Q/2 - 1) and all x velocities.  Conserved sums: float-float pairs for
// an FP32 state (`a*`, `b*`), plain FP64 for an FP64 state (`d*`); heat-flux
// sums in R.  Every sum is linear in the state, so the two halves add.
template <typename R>
struct MomPart {
    FF a0, a1, a2, a3, b1, b2;               // S0, S1x, S2xx, G0, S1y, S2yy (FP32 state)
    double d0 = 0, d1x = 0, d2xx = 0, dg0 = 0, d1y = 0, d2yy = 0;   // (FP64 state)
    R s2xy = 0, s3x = 0, s3y = 0, g1x = 0, g1y = 0;
};
constexpr int kMomX = 17;                    // values exchanged between the halves

template <typename R, int Q, int K0>
__device__ __forceinline__ void moments_half(const R* __restrict__ f, long long N, long long NF, const Pow2<R>& pw,
                                             const R (*sv)[Q], const float (*sh)[Q], MomPart<R>& P) {
    constexpr bool F32 = std::is_same<R, float>::value;
    constexpr int QH = Q / 2;
    CompSum<R> col[QH];
    for (int kx = 0; kx < Q; ++kx) {
        CompSum<R> rowF, rowG;
        R p1 = 0, p2 = 0, p3 = 0, pg = 0;          // sum y f, y^2 f, y^3 f, y g over the half row
#pragma unroll
        for (int j = 0; j < QH; ++j) {
            const long long o = (long long)(kx * Q + K0 + j) * N;
            const R fv = f[o], gv = f[NF + o];
            rowF.add(fv);
            rowG.add(gv);
            col[j].add(fv);
            p1 = fma(pw.v[K0 + j], fv, p1);
            p2 = fma(pw.v2[K0 + j], fv, p2);
            p3 = fma(pw.v3[K0 + j], fv, p3);
            pg = fma(pw.v[K0 + j], gv, pg);
        }
        const R xr = sv[0][kx], x2r = sv[1][kx];
        R rfr, rgr;                                 // half-row sums in R
        if constexpr (F32) {
            P.a0.add(rowF.s, rowF.c);
            P.a1.fma2(sh[0][kx], sh[1][kx], rowF.s, rowF.c);
            P.a2.fma2(sh[2][kx], sh[3][kx], rowF.s, rowF.c);
            P.a3.add(rowG.s, rowG.c);
            rfr = rowF.s + rowF.c;
            rgr = rowG.s + rowG.c;
        } else {
            P.d0 += rowF.s;
            P.d1x = fma((double)xr, rowF.s, P.d1x);
            P.d2xx = fma((double)x2r, rowF.s, P.d2xx);
            P.dg0 += rowG.s;
            rfr = (R)rowF.s;
            rgr = (R)rowG.s;
        }
        // sum (x^2 + y^2) f = x^2 rowF + p2;  sum y (x^2 + y^2) f = x^2 p1 + p3
        P.s2xy = fma(xr, p1, P.s2xy);
        P.s3x = fma(xr, fma(x2r, rfr, p2), P.s3x);
        P.s3y += fma(x2r, p1, p3);
        P.g1x = fma(xr, rgr, P.g1x);
        P.g1y += pg;
    }
#pragma unroll
    for (int j = 0; j < QH; ++j) {
        if constexpr (F32) {
            P.b1.fma2(pw.h[K0 + j], pw.l[K0 + j], col[j].s, col[j].c);
            P.b2.fma2(pw.h2[K0 + j], pw.l2[K0 + j], col[j].s, col[j].c);
        } else {
            P.d1y = fma((double)pw.v[K0 + j], col[j].s, P.d1y);
            P.d2yy = fma((double)pw.v2[K0 + j], col[j].s, P.d2yy);
        }
    }
}

// FP32: four CTAs per SM keep more loads in flight; the FP64 build (parity
// checks) keeps its registers
template <typename R>
constexpr int moments_min_blocks() { return std::is_same<R, float>::value ? 4 : 1; }

// Per CTA pass 128 nodes: warp pair (2p, 2p+1) takes nodes 32p .. 32p+31,
// the even warp the y velocities of the first half, the odd warp the second
// half (each load instruction reads 32 consecutive nodes of one plane); the
// odd warp hands its partial sums to the even one through shared memory.
template <typename R, int Q>
__global__ void __launch_bounds__(256, moments_min_blocks<R>())
k2_moments(Slab2 s, const Pow2<R> pw, const R* __restrict__ st, double* __restrict__ mom, float* __restrict__ prf,
           unsigned* err) {
    constexpr bool F32 = std::is_same<R, float>::value;
    constexpr int kNodes = 128;
    static_assert(Q % 2 == 0, "the y velocities split in two halves");
    const long long N = s.N, NF = (long long)Q * Q * N;
    // the row loop indexes the powers at run time: from shared memory
    __shared__ R sv[2][Q];
    __shared__ float sh[4][Q];
    __shared__ R xch[kMomX][kNodes];
    if (threadIdx.x < Q) {
        const int k = threadIdx.x;
        sv[0][k] = pw.v[k];
        sv[1][k] = pw.v2[k];
        sh[0][k] = pw.h[k];
        sh[1][k] = pw.l[k];
        sh[2][k] = pw.h2[k];
        sh[3][k] = pw.l2[k];
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, half = warp & 1;
    const int slot = (warp >> 1) * 32 + lane;
    for (long long b0 = (long long)blockIdx.x * kNodes; b0 < N; b0 += (long long)gridDim.x * kNodes) {
        const long long i = b0 + slot;
        MomPart<R> P;
        if (i < N) {
            if (half == 0) moments_half<R, Q, 0>(st + i, N, NF, pw, sv, sh, P);
            else moments_half<R, Q, Q / 2>(st + i, N, NF, pw, sv, sh, P);
        }
        if (half == 1) {
            R v[kMomX];
            if constexpr (F32) {
                const float w[12] = {P.a0.h, P.a0.l, P.a1.h, P.a1.l, P.a2.h, P.a2.l,
                                     P.a3.h, P.a3.l, P.b1.h, P.b1.l, P.b2.h, P.b2.l};
#pragma unroll
                for (int q = 0; q < 12; ++q) v[q] = w[q];
            } else {
                const double w[12] = {P.d0, P.d1x, P.d2xx, P.dg0, P.d1y, P.d2yy, 0, 0, 0, 0, 0, 0};
#pragma unroll
                for (int q = 0; q < 12; ++q) v[q] = w[q];
            }
            v[12] = P.s2xy;
            v[13] = P.s3x;
            v[14] = P.s3y;
            v[15] = P.g1x;
            v[16] = P.g1y;
#pragma unroll
            for (int q = 0; q < kMomX; ++q) xch[q][slot] = v[q];
        }
        __syncthreads();
        if (half == 0 && i < N) {
            const R s2xy = P.s2xy + xch[12][slot], s3x = P.s3x + xch[13][slot], s3y = P.s3y + xch[14][slot];
            const R g1x = P.g1x + xch[15][slot], g1y = P.g1y + xch[16][slot];
            double S0, S1x, S1y, S2xx, S2yy, G0;
            float n32 = 0, S1x32 = 0, S1y32 = 0, S2xx32 = 0, S2yy32 = 0, G032 = 0;
            if constexpr (F32) {
                P.a0.add(xch[0][slot], xch[1][slot]);
                P.a1.add(xch[2][slot], xch[3][slot]);
                P.a2.add(xch[4][slot], xch[5][slot]);
                P.a3.add(xch[6][slot], xch[7][slot]);
                P.b1.add(xch[8][slot], xch[9][slot]);
                P.b2.add(xch[10][slot], xch[11][slot]);
                n32 = P.a0.value(); S1x32 = P.a1.value(); S1y32 = P.b1.value();
                S2xx32 = P.a2.value(); S2yy32 = P.b2.value(); G032 = P.a3.value();
                if (!isfinite(n32) || !isfinite(S2xx32 + S2yy32 + G032)) atomicOr(err, ERR_NONFINITE);
                S0 = P.a0.value64(); S1x = P.a1.value64(); S1y = P.b1.value64();
                S2xx = P.a2.value64(); S2yy = P.b2.value64(); G0 = P.a3.value64();
            } else {
                S0 = P.d0 + xch[0][slot]; S1x = P.d1x + xch[1][slot]; S2xx = P.d2xx + xch[2][slot];
                G0 = P.dg0 + xch[3][slot]; S1y = P.d1y + xch[4][slot]; S2yy = P.d2yy + xch[5][slot];
                if (!isfinite(S0) || !isfinite(S2xx + S2yy + G0)) atomicOr(err, ERR_NONFINITE);
            }
            if (mom) {
                mom[M2_S0 * N + i] = S0;
                mom[M2_S1X * N + i] = S1x;
                mom[M2_S1Y * N + i] = S1y;
                mom[M2_S2XX * N + i] = S2xx;
                mom[M2_S2YY * N + i] = S2yy;
                mom[M2_G0 * N + i] = G0;
                mom[M2_S2XY * N + i] = (double)s2xy;
                mom[M2_S3X * N + i] = (double)s3x;
                mom[M2_S3Y * N + i] = (double)s3y;
                mom[M2_G1X * N + i] = (double)g1x;
                mom[M2_G1Y * N + i] = (double)g1y;
            }
            if constexpr (F32) {
                if (prf) {
                    // primitives in FP32: u = S1/n, (3/2) n T = (S2xx + S2yy)/2 + G0 - n u^2/2,
                    // q_i = sum c_i (c^2/2 F + G) expanded in the raw sums
                    const float n = n32, ux = S1x32 / n, uy = S1y32 / n;
                    const float u2 = ux * ux + uy * uy, S2 = S2xx32 + S2yy32;
                    const float T = (2.0f / 3.0f) * ((0.5f * S2 + G032) / n - 0.5f * u2);
                    const float uS1 = ux * S1x32 + uy * S1y32;
                    const float qx = 0.5f * (s3x - 2.0f * (ux * S2xx32 + uy * s2xy) + u2 * S1x32 - ux * S2 +
                                             2.0f * ux * uS1 - ux * u2 * n) + g1x - ux * G032;
                    const float qy = 0.5f * (s3y - 2.0f * (ux * s2xy + uy * S2yy32) + u2 * S1y32 - uy * S2 +
                                             2.0f * uy * uS1 - uy * u2 * n) + g1y - uy * G032;
                    prf[P2_N * N + i] = n;
                    prf[P2_UX * N + i] = ux;
                    prf[P2_UY * N + i] = uy;
                    prf[P2_T * N + i] = T;
                    prf[P2_QX * N + i] = qx;
                    prf[P2_QY * N + i] = qy;
                }
            }
        }
        __syncthreads();                               // xch is reused by the next pass
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
// k2_fields: node fields of a 16x16 tile, computed in the state precision R
// (the FP32 build reads the FP32 primitives of k2_moments; the FP64 build
// derives them from the FP64 raw sums).
//
// Force disc (rectangle rule over the grid offsets inside r_cut; the taps
// carry dx^2 g2): g2 is radial, so g2x(-a, b) = -g2x(a, b) and
// g2y(-a, b) = g2y(a, b) exactly, and one pass over the offset column pair
// (a, -a) adds g2x (n_+ - n_-) and g2y (n_+ + n_-) (column a = 0 with halved
// g2y).  Each warp takes a host-balanced list of column pairs over the whole
// tile: lane = (column, block of 8 rows); the pass walks the rows of the
// column once and keeps the last 8 weight pairs in a register ring, so each
// staged density pair feeds 16 FMAs (8 rows x 2 components).  The per-warp
// partial forces are summed in warp order (deterministic).
// ---------------------------------------------------------------------------
constexpr int kFWarps = 8;           // warps of k2_fields (256 threads)
constexpr int kFRows = 8;            // rows of a force register block (= ring length)
constexpr int kFPlanHead = 12;       // plan header: kFWarps + 1 prefix offsets, padded to 16 bytes
static_assert(kTile2 == 16 && 2 * kFRows == kTile2 && kFWarps * 32 == 256, "force mapping: 16 x 2 lanes x 8 rows");

// pitch of the staged density row: >= W and = 2 (mod 4), so that rows 8
// apart (the two row blocks of a warp) fall 16 banks apart
__host__ __device__ inline int fields_pitch(int W) { return W + ((6 - W % 4) % 4); }

template <typename R>
__host__ __device__ inline size_t fields_smem_bytes(int Mf, int mfm) {
    const int H = Mf > mfm + 2 ? Mf : mfm + 2, W = kTile2 + 2 * H, E = kTile2 + 4, Wr = fields_pitch(W);
    const size_t nr = (size_t)(W + kFRows) * Wr, pf = 2 * (size_t)kFWarps * kTile2 * kTile2;
    return sizeof(R) * ((nr > pf ? nr : pf) + 5 * (size_t)E * E);
}

template <typename R>
__global__ void __launch_bounds__(256)
k2_fields(Slab2 s, const double* __restrict__ mom, const float* __restrict__ prf, const R* __restrict__ ftw,
          const int* __restrict__ fplan, const int* __restrict__ fm_off, const R* __restrict__ fm_w,
          R* __restrict__ fld, unsigned* err) {
    constexpr bool F32 = std::is_same<R, float>::value;
    using R2 = typename std::conditional<F32, float2, double2>::type;
    extern __shared__ __align__(16) unsigned char sm2raw[];
    R* sm2 = reinterpret_cast<R*>(sm2raw);
    const int H = max(s.Mf, s.mfm + 2), W = kTile2 + 2 * H, E = kTile2 + 4, Wr = fields_pitch(W);
    R* Nr = sm2;                      // n on the tile + H halo, [W + 8][Wr]; rows W.. are zero
    R* U = sm2 + max((W + kFRows) * Wr, 2 * kFWarps * kTile2 * kTile2);
    R* V = U + E * E;                 // ux, uy, T, X, chi on the tile + 2, [E][E] each
    R* Tt = V + E * E;
    R* Xt = Tt + E * E;
    R* Ct = Xt + E * E;
    const int nx = s.nx, ny = s.ny;
    const long long N = s.N;
    const int x0 = blockIdx.x * kTile2, y0 = blockIdx.y * kTile2;
    for (int e = threadIdx.x; e < (W + kFRows) * W; e += blockDim.x) {
        const int cy = e / W, cx = e % W;
        R n = R(0);
        if (cy < W) {
            const long long i = (long long)wrapi(y0 - H + cy, ny) * nx + wrapi(x0 - H + cx, nx);
            if constexpr (F32) n = prf[P2_N * N + i];
            else n = mom[M2_S0 * N + i];
        }
        Nr[cy * Wr + cx] = n;
    }
    for (int e = threadIdx.x; e < E * E; e += blockDim.x) {
        const int cy = e / E, cx = e % E;
        const long long i = (long long)wrapi(y0 - 2 + cy, ny) * nx + wrapi(x0 - 2 + cx, nx);
        if constexpr (F32) {
            U[e] = prf[P2_UX * N + i];
            V[e] = prf[P2_UY * N + i];
            Tt[e] = prf[P2_T * N + i];
        } else {
            double n, ux, uy, T;
            prim2(mom, N, i, n, ux, uy, T);
            U[e] = ux;
            V[e] = uy;
            Tt[e] = T;
        }
    }
    __syncthreads();
    // Fischer-Methfessel average, chi (Eq. (carnstar)) and X = n^2 chi T on the tile + 2
    for (int e = threadIdx.x; e < E * E; e += blockDim.x) {
        const int cy = e / E, cx = e % E;
        const int hy = cy - 2 + H, hx = cx - 2 + H;   // position in the halo array
        R nb = R(0);
        for (int t = 0; t < s.nfm; ++t) nb = fma(fm_w[t], Nr[(hy + fm_off[2 * t + 1]) * Wr + hx + fm_off[2 * t]], nb);
        const R eta = (R)s.eta_coef * nb, om = R(1) - eta;
        const R chi = (R(2) - eta) / (R(2) * om * om * om);
        const R n = Nr[hy * Wr + hx];
        Ct[e] = chi;
        Xt[e] = n * n * chi * Tt[e];
    }
    // force over the disc
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int fxl = lane & 15, yb = lane >> 4;
    R ax[kFRows], ay[kFRows];
#pragma unroll
    for (int k = 0; k < kFRows; ++k) ax[k] = ay[k] = R(0);
    {
        const int4* ent = reinterpret_cast<const int4*>(fplan + kFPlanHead);
        const int e1 = fplan[warp + 1];
        for (int e = fplan[warp]; e < e1; ++e) {
            const int4 en = ent[e];          // column a, weight offset, steps (multiple of 8), half height w
            const int a = en.x, steps = en.z, w = en.w;
            const R* pp = Nr + (yb * kFRows - w + H) * Wr + fxl + H + a;   // n(x + a, row of step 0)
            const R* pm = pp - 2 * a;                                       // n(x - a, ...)
            const R2* g = reinterpret_cast<const R2*>(ftw) + en.y;
            // ring: slot (j & 7) holds the weights of step j, i.e. of offset b = j - w
            R gx[kFRows], gy[kFRows];
#pragma unroll
            for (int k = 0; k < kFRows; ++k) gx[k] = gy[k] = R(0);
            for (int j0 = 0; j0 < steps; j0 += kFRows) {
#pragma unroll
                for (int P = 0; P < kFRows; ++P) {
                    const R vp = pp[(j0 + P) * Wr], vm = pm[(j0 + P) * Wr];
                    const R2 gg = __ldg(g + j0 + P);
                    gx[P] = gg.x;
                    gy[P] = gg.y;
                    const R dd = vp - vm, ss = vp + vm;
                    // row k of the block takes offset b = (j - k) - w: the weights of step j - k
#pragma unroll
                    for (int k = 0; k < kFRows; ++k) {
                        ax[k] = fma(gx[(P - k) & (kFRows - 1)], dd, ax[k]);
                        ay[k] = fma(gy[(P - k) & (kFRows - 1)], ss, ay[k]);
                    }
                }
            }
        }
    }
    const int tx = threadIdx.x % kTile2, ty = threadIdx.x / kTile2;
    const R n = Nr[(ty + H) * Wr + tx + H];
    __syncthreads();                  // density reads done: its space takes the partial forces
    R* Pf = sm2;                      // [kFWarps][2][256]
#pragma unroll
    for (int k = 0; k < kFRows; ++k) {
        const int node = (yb * kFRows + k) * kTile2 + fxl;
        Pf[(2 * warp) * 256 + node] = ax[k];
        Pf[(2 * warp + 1) * 256 + node] = ay[k];
    }
    __syncthreads();
    R fx = R(0), fy = R(0);
#pragma unroll
    for (int w = 0; w < kFWarps; ++w) {
        fx += Pf[(2 * w) * 256 + threadIdx.x];
        fy += Pf[(2 * w + 1) * 256 + threadIdx.x];
    }
    const int x = x0 + tx, y = y0 + ty;
    if (x >= nx || y >= ny) return;
    const long long i = (long long)y * nx + x;
    const int c = (ty + 2) * E + (tx + 2);
    const R k12 = (R)(s.inv_dx / 12.0);
    auto d4x = [&](const R* f) { return (f[c - 2] - R(8) * f[c - 1] + R(8) * f[c + 1] - f[c + 2]) * k12; };
    auto d4y = [&](const R* f) { return (f[c - 2 * E] - R(8) * f[c - E] + R(8) * f[c + E] - f[c + 2 * E]) * k12; };
    const R ux = U[c], uy = V[c], T = Tt[c], X = Xt[c], chi = Ct[c];
    const R Ax = d4x(Xt) / X, Ay = d4y(Xt) / X, Bx = d4x(Tt) / T, By = d4y(Tt) / T;
    const R Dxx = d4x(U), Dxy = d4x(V), Dyx = d4y(U), Dyy = d4y(V);
    // heat flux q_i = sum c_i (c^2/2 F + G)
    R qx, qy;
    if constexpr (F32) {
        qx = prf[P2_QX * N + i];
        qy = prf[P2_QY * N + i];
    } else {
        const double S0 = mom[M2_S0 * N + i], S1x = mom[M2_S1X * N + i], S1y = mom[M2_S1Y * N + i];
        const double S2xx = mom[M2_S2XX * N + i], S2yy = mom[M2_S2YY * N + i], S2xy = mom[M2_S2XY * N + i];
        const double S3x = mom[M2_S3X * N + i], S3y = mom[M2_S3Y * N + i], G0 = mom[M2_G0 * N + i];
        const double G1x = mom[M2_G1X * N + i], G1y = mom[M2_G1Y * N + i];
        const double u2 = ux * ux + uy * uy, S2 = S2xx + S2yy;
        const double uS1 = ux * S1x + uy * S1y;
        qx = 0.5 * (S3x - 2.0 * (ux * S2xx + uy * S2xy) + u2 * S1x - ux * S2 + 2.0 * ux * uS1 - ux * u2 * S0) +
             G1x - ux * G0;
        qy = 0.5 * (S3y - 2.0 * (ux * S2xy + uy * S2yy) + u2 * S1y - uy * S2 + 2.0 * uy * uS1 - uy * u2 * S0) +
             G1y - uy * G0;
    }
    // transport, Eqs. (viscosity), (tau), (prandtl)
    const R c16 = R((4.0 / 25.0) * (1.0 + 12.0 / M_PI)), c9 = R((9.0 / 25.0) * (1.0 + 32.0 / (9.0 * M_PI)));
    const R bn = (R)s.b * n, xx = bn * chi;
    const R mu = (R)s.mu0_coef * sqrt(T) * (R(1) / chi + R(0.8) * bn + c16 * bn * bn * chi);
    const R tau = mu / (n * T * (R(1) + R(0.4) * xx));
    const R Pr = R(2.0 / 3.0) * (R(1) + R(0.6) * xx) * (R(1) + R(0.8) * xx + c16 * xx * xx) /
                 ((R(1) + R(0.4) * xx) * (R(1) + R(1.2) * xx + c9 * xx * xx));
    const R nu = (s.relax == EVFDLB_RELAX_INV_TAU) ? R(1) / tau : chi / tau;
    if (!(n > R(0)) || !(T > R(0))) atomicOr(err, (isfinite(n) && isfinite(T)) ? ERR_NEGATIVE : ERR_NONFINITE);
    else if (!isfinite(fx + fy) || !isfinite(nu) || !isfinite(qx + qy) || !isfinite(Ax + Ay))
        atomicOr(err, ERR_NONFINITE);
    // polynomial coefficients of nu F^S + J1_F and nu G^S + J1_G over F_MB
    // (K = b n chi, sq = nu s with s = (1 - Pr)/(n T^2), div u = Dxx + Dyy)
    const R K = xx, sq = nu * (R(1) - Pr) / (n * T * T), dv = Dxx + Dyy, iT = R(1) / T;
    R pf[10], pg[10];
    pf[0] = nu + R(0.8) * K * dv;
    pf[1] = R(-0.8) * sq * qx - K * (Ax - R(1.2) * Bx);
    pf[2] = R(-0.8) * sq * qy - K * (Ay - R(1.2) * By);
    pf[3] = R(-0.4) * K * (Dxx + R(0.5) * dv) * iT;
    pf[4] = R(-0.4) * K * (Dxy + Dyx) * iT;
    pf[5] = R(-0.4) * K * (Dyy + R(0.5) * dv) * iT;
    pf[6] = R(0.2) * sq * qx * iT - R(0.3) * K * Bx * iT;
    pf[7] = R(0.2) * sq * qy * iT - R(0.3) * K * By * iT;
    pf[8] = R(0.2) * sq * qx * iT - R(0.3) * K * Bx * iT;
    pf[9] = R(0.2) * sq * qy * iT - R(0.3) * K * By * iT;
    pg[0] = R(0.5) * nu * T + R(0.2) * T * K * dv;
    pg[1] = R(-0.2) * T * sq * qx - R(0.5) * T * K * (Ax - R(0.6) * Bx);
    pg[2] = R(-0.2) * T * sq * qy - R(0.5) * T * K * (Ay - R(0.6) * By);
    pg[3] = R(-0.2) * K * (Dxx + R(0.5) * dv);
    pg[4] = R(-0.2) * K * (Dxy + Dyx);
    pg[5] = R(-0.2) * K * (Dyy + R(0.5) * dv);
    pg[6] = R(0.1) * sq * qx - R(0.15) * K * Bx;
    pg[7] = R(0.1) * sq * qy - R(0.15) * K * By;
    pg[8] = R(0.1) * sq * qx - R(0.15) * K * Bx;
    pg[9] = R(0.1) * sq * qy - R(0.15) * K * By;
    R* o = fld + i;
    o[F2_N * N] = n;
    o[F2_UX * N] = ux;
    o[F2_UY * N] = uy;
    o[F2_T * N] = T;
    o[F2_NU * N] = nu;
    o[F2_FX * N] = fx;
    o[F2_FY * N] = fy;
#pragma unroll
    for (int j = 0; j < 10; ++j) {
        o[(F2_PF + j) * N] = n * pf[j];
        o[(F2_PG + j) * N] = n * pg[j];
    }
}

// ---------------------------------------------------------------------------
// k2_coll: per group of kNB consecutive nodes, the local (velocity-space)
// part of the right-hand side,
//   RL = -nu h + F_x (D (x) I) h + F_y (I (x) D) h + sum_{a<4} phi^a (x) psi^a.
// D = S diag-shift(sqrt(l)) P is the derivative of the force term on the
// Gauss-Hermite set: the synthesis of its coefficient form F sqrt(l) a_{l-1}
// (S P = I on the set, so the relaxation -nu h needs no transform).  The
// projected Shakhov equilibrium and J1, sum_ab P_ab n mu^a_l(u_x) mu^b_m(u_y)
// in coefficient space (the one-axis Gaussian moments
//   mu^0 = m_l, mu^1 = T sqrt(l) m_{l-1}, mu^2 = T m_l + T^2 sqrt(l(l-1)) m_{l-2},
//   mu^3 = 3T^2 sqrt(l) m_{l-1} + T^3 sqrt(l(l-1)(l-2)) m_{l-3},
// m_l = E[psi_l(u + c)], c ~ N(0, T)), synthesise to the rank-4 sum of
// outer products of phi^a = S mu^a(u_x) and psi^a = sum_b P_ab chi^b,
// chi^b = S mu^b(u_y); a row r of the sum is sum_b pr_b chi^b with
// pr_b = sum_a phi^a_r P_ab.
// The node reflection xi -> -xi maps psi_l to (-1)^l psi_l, so S's rows k and
// Q-1-k differ in the sign of the odd orders, and D anticommutes with it.
// With E_j = h_j + h_{Q-1-j}, O_j = h_j - h_{Q-1-j} (j < Q/2) a line's D h is
//   (D h)_k = (DB E)_k + (DA O)_k,   (D h)_{Q-1-k} = (DA O)_k - (DB E)_k,
// DA_kj = (D_kj - D_{k,Q-1-j})/2, DB_kj = (D_kj + D_{k,Q-1-j})/2: two
// (Q/2)^2 blocks instead of Q^2 products per line, and a synthesis is
// (S c)_k = e_k + o_k, (S c)_{Q-1-k} = e_k - o_k over the even and odd orders.
//
// Work layout: a lane owns one (distribution, node) pair -- the 32 lanes of
// a warp are the 2 x 16 pairs of the group -- and the state sits plane-major
// in shared memory (16 nodes of a plane contiguous, staged by 16-byte
// asynchronous copies), so a warp's shared accesses are conflict-free and its
// global stores are 16 consecutive nodes of one plane per distribution.  A
// warp takes velocity rows w, w + 8, ... (then columns): a line of Q values
// is loaded, split into E and O and multiplied by DA and DB, whose entries
// sit in the constant bank -- uniform across the warp at compile-time
// indices, they are operands of the multiply-adds, with no load instructions
// (the syntheses of phi and chi use S from the constant bank the same way).
//   pass 1 (rows, D along y):  Y = -nu h + F_y (I (x) D) h + sum_b pr_b chi^b
//   pass 2 (columns, along x): RL = Y + F_x (D (x) I) h, to global memory.
// ---------------------------------------------------------------------------
// per even Q of the 2D model (4 .. 16), at coll_coff(Q): DA, DB [(Q/2)^2
// each], then S [Q][Q] (S[k][l] = w_k psi_l(xi_k))
__host__ __device__ constexpr int coll_coff(int Q) {
    int o = 0;
    for (int q = 4; q < Q; q += 2) o += q * q / 2 + q * q;
    return o;
}
constexpr int kCollConst = coll_coff(18);
__constant__ float c_coll_f[kCollConst];
__constant__ double c_coll_d[kCollConst];
template <typename R>
__device__ __forceinline__ R ccoll(int i);
template <>
__device__ __forceinline__ float ccoll<float>(int i) { return c_coll_f[i]; }
template <>
__device__ __forceinline__ double ccoll<double>(int i) { return c_coll_d[i]; }

template <int Q>
struct Coll2Lay {
    static constexpr int K = Q * Q, QH = Q / 2;
    // Xp, Yp [2][K][kNB] (+16 per distribution: the two halves of a warp on
    // opposite bank halves); chi4 [kNB][PS] (chi^b at column k: k 4 + b; PS an
    // odd count of 16-byte units); phi [4][PH] (phi^a_k of node n at k kNB + n;
    // PH = 8 mod 32: the 4 a of 8 nodes on distinct banks); mu [2][Q][kNB][4]
    // (axis, order, node, a); sc [kNumFld2][kNB]; rinv, rr, r1, r2, r3 [Q]
    static constexpr int XD = K * kNB + 16, PS = 4 * (Q + 1), PH = Q * kNB + 8;
};

template <typename R>
__host__ __device__ inline size_t coll_smem_bytes(int Q) {
    const size_t K = (size_t)Q * Q, XD = K * kNB + 16, PS = 4 * ((size_t)Q + 1), PH = (size_t)Q * kNB + 8;
    return sizeof(R) * (4 * XD + kNB * PS + 4 * PH + 2 * (size_t)Q * kNB * 4 + kNumFld2 * kNB + 5 * (size_t)Q);
}

template <typename R>
__device__ __forceinline__ void ld4(const R* p, R& a, R& b, R& c, R& d) {
    if constexpr (std::is_same<R, float>::value) {
        const float4 v = *reinterpret_cast<const float4*>(p);
        a = v.x, b = v.y, c = v.z, d = v.w;
    } else {
        const double2 v0 = reinterpret_cast<const double2*>(p)[0], v1 = reinterpret_cast<const double2*>(p)[1];
        a = v0.x, b = v0.y, c = v1.x, d = v1.y;
    }
}

__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gsrc) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(gsrc) : "memory");
}

// D h along one line of Q values hv: out[k] = sum_j D_kj hv[j]
template <typename R, int Q>
__device__ __forceinline__ void d_line(const R (&hv)[Q], R (&out)[Q]) {
    constexpr int QH = Q / 2, O0 = coll_coff(Q), O1 = O0 + QH * QH;
    R E[QH], Od[QH];
#pragma unroll
    for (int j = 0; j < QH; ++j) {
        E[j] = hv[j] + hv[Q - 1 - j];
        Od[j] = hv[j] - hv[Q - 1 - j];
    }
#pragma unroll
    for (int k = 0; k < QH; ++k) {
        R u = R(0), v = R(0);
#pragma unroll
        for (int j = 0; j < QH; ++j) {
            u = fma(ccoll<R>(O0 + k * QH + j), Od[j], u);
            v = fma(ccoll<R>(O1 + k * QH + j), E[j], v);
        }
        out[k] = v + u;
        out[Q - 1 - k] = u - v;
    }
}

// S c for one vector of Q orders: out[k] = sum_l S_kl c[l]
template <typename R, int Q>
__device__ __forceinline__ void s_line(const R (&c)[Q], R (&out)[Q]) {
    constexpr int QH = Q / 2, OS = coll_coff(Q) + 2 * QH * QH;
#pragma unroll
    for (int k = 0; k < QH; ++k) {
        R e = R(0), o = R(0);
#pragma unroll
        for (int l = 0; l < Q; l += 2) {
            e = fma(ccoll<R>(OS + k * Q + l), c[l], e);
            o = fma(ccoll<R>(OS + k * Q + l + 1), c[l + 1], o);
        }
        out[k] = e + o;
        out[Q - 1 - k] = e - o;
    }
}

// FP32: two CTAs per SM (85 KB of shared memory each at Q = 16); FP64: one
template <typename R>
constexpr int coll_min_blocks() { return std::is_same<R, float>::value ? 2 : 1; }

template <typename R, int Q>
__global__ void __launch_bounds__(256, coll_min_blocks<R>())
k2_coll(Slab2 s, const R* __restrict__ rtab, const R* __restrict__ st, const R* __restrict__ fld,
        R* __restrict__ RL) {
    using Lay = Coll2Lay<Q>;
    constexpr int K = Lay::K, XD = Lay::XD, PS = Lay::PS, PH = Lay::PH, NT = 256;
    extern __shared__ __align__(16) double smc[];
    R* Xp = reinterpret_cast<R*>(smc);                         // [2][K][kNB] (+16 per distribution)
    R* Yp = Xp + 2 * XD;
    R* chi4 = Yp + 2 * XD;                                      // [kNB][PS]
    R* phi = chi4 + kNB * PS;                                   // [4][PH]
    R* mu = phi + 4 * PH;                                       // [2][Q][kNB][4]
    R* sc = mu + 2 * Q * kNB * 4;                               // [kNumFld2][kNB]
    R* rinv = sc + kNumFld2 * kNB;
    R* rr = rinv + Q;
    R* r1 = rr + Q;
    R* r2 = r1 + Q;
    R* r3 = r2 + Q;
    const long long N = s.N, NF = (long long)K * N;
    const long long i0 = (long long)blockIdx.x * kNB;
    const int nb = (int)min((long long)kNB, N - i0);
    TableLayout L(Q);
    // the group's state, plane-major: 16-byte copies when whole aligned
    // chunks of 4 nodes exist (N a multiple of 4, a full group), else per element
    constexpr int CH = 16 / (int)sizeof(R);                     // elements per 16-byte chunk
    if (nb == kNB && (N % CH) == 0) {
        for (int e = threadIdx.x; e < 2 * K * (kNB / CH); e += NT) {
            const int c = e % (kNB / CH), k = (e / (kNB / CH)) % K, d = e / ((kNB / CH) * K);
            cp_async16(Xp + d * XD + k * kNB + c * CH, st + d * NF + (long long)k * N + i0 + c * CH);
        }
    } else {
        for (int e = threadIdx.x; e < 2 * K * kNB; e += NT) {
            const int n = e % kNB, k = (e / kNB) % K, d = e / (kNB * K);
            R* dst = Xp + d * XD + k * kNB + n;
            if (n < nb) cp_async_elem<R>(dst, st + d * NF + (long long)k * N + i0 + n);
            else *dst = R(0);
        }
    }
    cp_async_commit();
    for (int e = threadIdx.x; e < Q; e += NT) {
        rinv[e] = rtab[L.rinv + e];
        rr[e] = rtab[L.rr + e];
        r1[e] = rtab[L.r1 + e];
        r2[e] = rtab[L.r2 + e];
        r3[e] = rtab[L.r3 + e];
    }
    for (int e = threadIdx.x; e < kNumFld2 * kNB; e += NT) {
        const int n = e % kNB, f = e / kNB;
        sc[e] = (n < nb) ? fld[f * N + i0 + n] : (f == F2_N || f == F2_T ? R(1) : R(0));
    }
    __syncthreads();
    // one-axis Gaussian moments mu^a_l, one node and axis per thread
    if (threadIdx.x < 2 * kNB) {
        const int n = threadIdx.x % kNB, axis = threadIdx.x / kNB;
        const R u = sc[(axis ? F2_UY : F2_UX) * kNB + n], T = sc[F2_T * kNB + n], Tm1 = T - R(1);
        R* out = mu + (axis * Q * kNB + n) * 4;
        R m1v = 0, m2v = 0, m3v = 0;                            // m_{l-1}, m_{l-2}, m_{l-3}
        R m0 = 1;                                               // m_l
        for (int l = 0; l < Q; ++l) {
            R* o = out + l * kNB * 4;
            o[0] = m0;
            o[1] = T * r1[l] * m1v;
            o[2] = T * m0 + T * T * r2[l] * m2v;
            o[3] = R(3) * T * T * r1[l] * m1v + T * T * T * r3[l] * m3v;
            const R mn = fma(u * rinv[l], m0, Tm1 * rr[l] * m1v);
            m3v = m2v;
            m2v = m1v;
            m1v = m0;
            m0 = mn;
        }
    }
    __syncthreads();
    // one-axis syntheses, one vector (axis, node, a) per thread:
    // phi^a = S mu^a(u_x) to phi, chi^b = S mu^b(u_y) to chi4
    if (threadIdx.x < 2 * kNB * 4) {
        const int a = threadIdx.x % 4, n = (threadIdx.x / 4) % kNB, axis = threadIdx.x / (4 * kNB);
        R c[Q], out[Q];
#pragma unroll
        for (int l = 0; l < Q; ++l) c[l] = mu[((axis * Q + l) * kNB + n) * 4 + a];
        s_line<R, Q>(c, out);
        if (axis == 0) {
#pragma unroll
            for (int k = 0; k < Q; ++k) phi[a * PH + k * kNB + n] = out[k];
        } else {
#pragma unroll
            for (int k = 0; k < Q; ++k) chi4[n * PS + k * 4 + a] = out[k];
        }
    }
    cp_async_wait_all();
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int d = lane >> 4, n = lane & (kNB - 1);
    const R* h = Xp + d * XD + n;                               // h[k] at k kNB
    R* y = Yp + d * XD + n;
    // pass 1: rows r (fixed kx), D along y
    {
        const R mnu = -sc[F2_NU * kNB + n], fy = sc[F2_FY * kNB + n];
        // P^d_ab (the equilibrium polynomial's coefficient of c_x^a c_y^b,
        // times n) at (a+b)(a+b+1)/2 + b of the order (0,0) (1,0) (0,1)
        // (2,0) (1,1) (0,2) (3,0) (2,1) (1,2) (0,3)
        R P[10];
        const int f0 = d ? F2_PG : F2_PF;
#pragma unroll
        for (int i = 0; i < 10; ++i) P[i] = sc[(f0 + i) * kNB + n];
        const R* ch = chi4 + n * PS;
        for (int r = warp; r < Q; r += NT / 32) {
            R hv[Q], dy[Q];
#pragma unroll
            for (int j = 0; j < Q; ++j) hv[j] = h[(r * Q + j) * kNB];
            d_line<R, Q>(hv, dy);
            const R p0 = phi[0 * PH + r * kNB + n], p1 = phi[1 * PH + r * kNB + n];
            const R p2 = phi[2 * PH + r * kNB + n], p3 = phi[3 * PH + r * kNB + n];
            // pr_b = sum_{a <= 3-b} phi^a_r P_ab
            const R pr0 = fma(p3, P[6], fma(p2, P[3], fma(p1, P[1], p0 * P[0])));
            const R pr1 = fma(p2, P[7], fma(p1, P[4], p0 * P[2]));
            const R pr2 = fma(p1, P[8], p0 * P[5]);
            const R pr3 = p0 * P[9];
#pragma unroll
            for (int c = 0; c < Q; ++c) {
                R q0, q1, q2, q3;
                ld4<R>(ch + c * 4, q0, q1, q2, q3);
                R eq = pr0 * q0;
                eq = fma(pr1, q1, eq);
                eq = fma(pr2, q2, eq);
                eq = fma(pr3, q3, eq);
                const R v = fma(mnu, hv[c], eq);
                y[(r * Q + c) * kNB] = fma(fy, dy[c], v);
            }
        }
    }
    __syncthreads();
    // pass 2: columns c (fixed ky), D along x, and the store
    {
        const R fx = sc[F2_FX * kNB + n];
        R* g = RL + d * NF + i0 + n;
        for (int c = warp; c < Q; c += NT / 32) {
            R hv[Q], dx[Q];
#pragma unroll
            for (int j = 0; j < Q; ++j) hv[j] = h[(j * Q + c) * kNB];
            d_line<R, Q>(hv, dx);
#pragma unroll
            for (int r = 0; r < Q; ++r) {
                const R v = fma(fx, dx[r], y[(r * Q + c) * kNB]);
                if (n < nb) g[(long long)(r * Q + c) * N] = v;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// k2_adv: WENO-5 faces along x and y, the right-hand side and the RK combine.
// ---------------------------------------------------------------------------
// A 32x16 node tile and a run of velocity planes.  Per plane the halo (tile
// +-3) is staged in shared memory (its global offsets computed once per CTA),
// then every thread forms one run of consecutive faces with the difference-
// form WENO-5 of the 1D kernels (Weno5Run: the differences and the t-terms of
// each cell formed once and shared by the run's faces): threads 0-127 the x
// faces (16 rows x runs 5+4+4+4+4+4+4+4 of the 33 faces of a row), threads
// 128-255 the y faces (32 columns x runs 5+4+4+4 of the 17 faces of a
// column); for a negative velocity the stencil is mirrored and the run walked
// down.  Then the right-hand side and the Shu-Osher combine
//   out = alpha base + beta (h + dt R)   (RHS false),   rhs_out = R (RHS true).
// Q is a compile-time parameter: the plane index splits by constants.  So is
// the output form: with a run-time switch the FP32 kernel issued the FP64
// store's conversion (predicated off) for every output of the combine.
template <typename R>
constexpr int adv_min_blocks() { return std::is_same<R, float>::value ? 4 : 2; }

template <typename R, int Q, bool RHS>
__global__ void __launch_bounds__(256, adv_min_blocks<R>())
k2_adv(Slab2 s, const R* __restrict__ rtab, const R* __restrict__ src, const R* base, R* out,
       const R* __restrict__ RL, double* rhs_out, double alpha, double beta) {
    constexpr int WX = kAdvX + 6, WY = kAdvY + 6, NH = WX * WY;
    constexpr int NHR = (NH + 255) / 256;                   // halo loads per thread
    constexpr int RPW = kAdvY / 8;                          // output rows per warp
    constexpr int K = Q * Q;
    static_assert(kAdvX == 32 && kAdvY == 16, "run split: 33 = 5 + 7 x 4 x-faces, 17 = 5 + 3 x 4 y-faces");
    __shared__ R Hs[NH];
    __shared__ R FX[kAdvY * (kAdvX + 1)];
    __shared__ R FY[(kAdvY + 1) * kAdvX];
    __shared__ int rowoff[WY];
    __shared__ int coloff[WX];
    const int nx = s.nx, ny = s.ny;
    const long long N = s.N;
    const int tilesx = (nx + kAdvX - 1) / kAdvX;
    const int x0 = (blockIdx.x % tilesx) * kAdvX, y0 = (blockIdx.x / tilesx) * kAdvY;
    TableLayout L(Q);
    // wrapped halo coordinates, shared by every plane of this tile (node
    // offsets fit 32 bits: the 2D context holds fewer than 2^31 nodes)
    for (int e = threadIdx.x; e < WY + WX; e += blockDim.x) {
        if (e < WY) rowoff[e] = wrapi(y0 - 3 + e, ny) * nx;
        else coloff[e - WY] = wrapi(x0 - 3 + (e - WY), nx);
    }
    __syncthreads();
    int hoff[NHR];
#pragma unroll
    for (int j = 0; j < NHR; ++j) {
        const int e = threadIdx.x + 256 * j;
        hoff[j] = (e < NH) ? rowoff[e / WX] + coloff[e % WX] : 0;
    }
    const R eps = (R)s.weno_eps, idx = (R)s.inv_dx, dt = (R)s.dt, ralpha = (R)alpha, rbeta = (R)beta;
    const bool with_base = (alpha != 0.0);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // this thread's run of faces: along x (threads 0-127) or y (128-255)
    const bool xrun = threadIdx.x < 128;
    const int rj = xrun ? (threadIdx.x >> 4) : ((threadIdx.x - 128) >> 5);   // run index
    const int rl = xrun ? (threadIdx.x & 15) : (threadIdx.x & 31);           // row (x) or column (y)
    const int fa = rj == 0 ? 0 : 4 * rj + 1, nrun = rj == 0 ? 5 : 4, fl = fa + nrun - 1;
    const int hst = xrun ? 1 : WX;                        // halo stride along the run
    // x face f of row r: stencil from halo (r + 3, f); y face f of column c: from halo (f, c + 3)
    const R* hrow = xrun ? Hs + (rl + 3) * WX : Hs + rl + 3;
    R* frow = xrun ? FX + rl * (kAdvX + 1) : FY + rl;
    const int fst = xrun ? 1 : kAdvX;                     // face stride along the run
    // output nodes of this thread (rows warp*RPW + rr, column lane) and
    // their offsets in a velocity plane
    const int x = x0 + lane;
    int ooff[RPW];
    bool oval[RPW];
#pragma unroll
    for (int rr = 0; rr < RPW; ++rr) {
        const int y = y0 + warp * RPW + rr;
        oval[rr] = (x < nx && y < ny);
        ooff[rr] = oval[rr] ? y * nx + x : 0;
    }
    const int p0 = blockIdx.y * kAdvPlanes, p1 = min(p0 + kAdvPlanes, 2 * K);
    // plane p (distribution p / K, velocity p % K) starts at p N: the plane
    // pointers advance by N (no 64-bit products in the loop)
    const long long off0 = (long long)p0 * N;
    const R* hp = src + off0;
    const R* rlp = RL + off0;
    const R* bsp = base + off0;
    R* op = out + off0;
    double* rp = rhs_out ? rhs_out + off0 : nullptr;
    // the halo of the next plane is loaded into registers while this plane's
    // faces are formed, and this plane's RL / base values before them
    R hn[NHR];
#pragma unroll
    for (int j = 0; j < NHR; ++j) hn[j] = (threadIdx.x + 256 * j < NH) ? hp[hoff[j]] : R(0);
    for (int plane = p0; plane < p1; ++plane, hp += N, rlp += N, bsp += N, op += N) {
        const int k = plane % K;
        const R vx = rtab[L.xi + k / Q], vy = rtab[L.xi + k % Q];
        __syncthreads();   // previous plane's faces and halo consumed
#pragma unroll
        for (int j = 0; j < NHR; ++j)
            if (threadIdx.x + 256 * j < NH) Hs[threadIdx.x + 256 * j] = hn[j];
        if (plane + 1 < p1) {
            const R* hq = hp + N;
#pragma unroll
            for (int j = 0; j < NHR; ++j)
                if (threadIdx.x + 256 * j < NH) hn[j] = hq[hoff[j]];
        }
        R rl[RPW], bs[RPW];
#pragma unroll
        for (int rr = 0; rr < RPW; ++rr) {
            rl[rr] = oval[rr] ? rlp[ooff[rr]] : R(0);
            bs[rr] = (oval[rr] && with_base && !RHS) ? bsp[ooff[rr]] : R(0);
        }
        __syncthreads();
        {
            const bool pos = (xrun ? vx : vy) >= R(0);      // uniform per warp
            const int dir = pos ? 1 : -1, f0 = pos ? fa : fl;
            // v >= 0: face f uses halo f .. f+4, walked up; v < 0: f+5 .. f+1, walked down
            const R* hb = hrow + (pos ? fa : fl + 5) * hst;
            const int hs = dir * hst;
            Weno5Run<R> w;
            w.start(hb[0], hb[hs], hb[2 * hs], hb[3 * hs], hb[4 * hs], eps);
#pragma unroll
            for (int q = 0; q < 5; ++q) {
                if (q >= nrun) break;
                frow[(f0 + dir * q) * fst] = w.face();
                if (q + 1 < nrun) w.shift(hb[(q + 5) * hs]);
            }
        }
        __syncthreads();
#pragma unroll
        for (int rr = 0; rr < RPW; ++rr) {
            if (!oval[rr]) continue;
            const int ty = warp * RPW + rr;
            R Rv = rl[rr];
            Rv = fma(-vx * idx, FX[ty * (kAdvX + 1) + lane + 1] - FX[ty * (kAdvX + 1) + lane], Rv);
            Rv = fma(-vy * idx, FY[(ty + 1) * kAdvX + lane] - FY[ty * kAdvX + lane], Rv);
            if constexpr (RHS) {
                rp[(plane - p0) * N + ooff[rr]] = (double)Rv;
                continue;
            }
            const R hv = Hs[(ty + 3) * WX + lane + 3];
            R o = rbeta * fma(dt, Rv, hv);
            if (with_base) o = fma(ralpha, bs[rr], o);
            op[ooff[rr]] = o;
        }
    }
}

// ---------------------------------------------------------------------------
// k2_adv2: the FP32 stage form of k2_adv.  The F and G planes of one
// velocity are carried together as float2 through packed FP32 arithmetic
// (two lanes per instruction): both distributions share the velocity, hence
// the upwind direction of every face, so the pair runs one stencil walk.
// Each packed operation is the IEEE single-precision operation of each lane
// in the order of k2_adv (k2_adv's scalar code may also fuse a product into
// a following add, so the two agree to rounding, not bit for bit).  The
// halo tile, RL and base of velocity k+2 are copied asynchronously into a
// second shared buffer while velocity k is formed (two velocities in
// flight per CTA, no register staging), which keeps enough bytes in flight
// for the kernel to stream.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 f2s(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, f2s(-1.f), a); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }

// Weno5Run on float2 pairs (its operations, lane by lane, none fused)
struct Weno5Run2 {
    float2 v2, v3, v4, d0, d1, d2, d3, u0, u1, u2, eps4;
    __device__ __forceinline__ float2 tterm(float2 t) const {
        return fma2(mul2(f2s(float(13.0 / 3.0)), t), t, eps4);
    }
    __device__ __forceinline__ void start(float2 w0, float2 w1, float2 w2, float2 w3, float2 w4, float eps) {
        eps4 = f2s(4.f * eps);
        v2 = w2;
        v3 = w3;
        v4 = w4;
        d0 = sub2(w1, w0);
        d1 = sub2(w2, w1);
        d2 = sub2(w3, w2);
        d3 = sub2(w4, w3);
        u0 = tterm(sub2(d1, d0));
        u1 = tterm(sub2(d2, d1));
        u2 = tterm(sub2(d3, d2));
    }
    __device__ __forceinline__ float2 face() const {
        const float2 s0 = fma2(f2s(3.f), d1, neg2(d0)), s1 = add2(d1, d2), s2 = fma2(f2s(-3.f), d2, d3);
        const float2 e0 = fma2(s0, s0, u0), e1 = fma2(s1, s1, u1), e2 = fma2(s2, s2, u2);
        const float2 E0 = mul2(e0, e0), E1 = mul2(e1, e1), E2 = mul2(e2, e2);
        const float2 a0 = mul2(E1, E2), a1 = mul2(E0, E2), a2 = mul2(E0, E1);
        const float2 c0 = fma2(f2s(float(5.0 / 60.0)), d1, mul2(f2s(float(-2.0 / 60.0)), d0));
        const float2 p2 = mul2(f2s(0.2f), d2);
        const float2 c1 = fma2(f2s(0.1f), d1, p2);
        const float2 c2 = fma2(f2s(-0.05f), d3, p2);
        const float2 num = fma2(a0, c0, fma2(a1, c1, mul2(a2, c2)));
        const float2 den = fma2(f2s(0.1f), a0, fma2(f2s(0.6f), a1, mul2(f2s(0.3f), a2)));
        return add2(v2, make_float2(__fdividef(num.x, den.x), __fdividef(num.y, den.y)));
    }
    __device__ __forceinline__ void shift(float2 w5) {
        const float2 d4 = sub2(w5, v4);
        u0 = u1;
        u1 = u2;
        u2 = tterm(sub2(d4, d3));
        d0 = d1;
        d1 = d2;
        d2 = d3;
        d3 = d4;
        v2 = v3;
        v3 = v4;
        v4 = w5;
    }
};

// Shared layout of k2_adv2 per buffer (two buffers: velocities k and k+1 in
// flight): the halo tile of F and G, rows y0-3 .. y0+18 with column
// x0-3+i at i + 1 (the interior x0 .. x0+31 at columns 4 .. 35, 16-byte
// aligned, row stride 44: a row's 16 lanes of the x runs on 8 banks apart),
// then RL and base of the tile's nodes.
constexpr int kA2Row = 44, kA2Rows = kAdvY + 6;
constexpr int kA2H = 2 * kA2Rows * kA2Row;                  // halo of F and G
constexpr int kA2T = 2 * kAdvY * kAdvX;                     // RL (or base) of F and G
constexpr int kA2Buf = kA2H + 2 * kA2T;
constexpr size_t kA2Smem = sizeof(float) * 2 * kA2Buf + sizeof(float2) * (kAdvY * (kAdvX + 1) + (kAdvY + 1) * kAdvX) +
                           sizeof(int) * (kA2Rows + kAdvX + 6);

__device__ __forceinline__ void cp_async_wait_1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// A thread's share of the whole-chunk copies of one velocity, the same for
// every velocity of the CTA and so formed once: shared offsets, in-plane
// global offsets (below N < 2^31) and, per copy, whether it reads the G
// plane; a negative shared offset marks an absent copy.
struct Adv2Copies {
    int hs[2], hg[2];   // 16-byte chunks of the halo interior
    int ss[2], sg[2];   // 4-byte elements of the halo side columns
    int rs, rg;         // the 16-byte chunk of RL (and base) every thread copies
    unsigned gmask;     // bit q: hs[q] reads G; bit 2+q: ss[q]; bit 4: the RL chunk
};
static_assert(2 * kAdvY * 8 == 256 && 2 * kA2Rows * 8 <= 512 && 2 * kA2Rows * 6 <= 512,
              "copy shares of a 256-thread CTA");

__device__ __forceinline__ Adv2Copies adv2_plan(const int* rowoff, const int* coloff, int x0, int y0, int nx) {
    Adv2Copies p;
    p.gmask = 0u;
    const int t = threadIdx.x;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const int e = t + 256 * q;
        p.hs[q] = -1;
        p.ss[q] = -1;
        if (e < 2 * kA2Rows * 8) {
            const int c = e % 8, r = (e / 8) % kA2Rows, d = e / (8 * kA2Rows);
            p.hs[q] = (d * kA2Rows + r) * kA2Row + 4 + 4 * c;
            p.hg[q] = rowoff[r] + x0 + 4 * c;
            if (d) p.gmask |= 1u << q;
        }
        if (e < 2 * kA2Rows * 6) {
            const int c = e % 6, r = (e / 6) % kA2Rows, d = e / (6 * kA2Rows);
            const int i = c < 3 ? c : 32 + c;               // halo columns 0..2 and 35..37
            p.ss[q] = (d * kA2Rows + r) * kA2Row + i + 1;
            p.sg[q] = rowoff[r] + coloff[i];
            if (d) p.gmask |= 4u << q;
        }
    }
    const int c = t % 8, r = (t / 8) % kAdvY, d = t / (8 * kAdvY);
    p.rs = (d * kAdvY + r) * kAdvX + 4 * c;
    p.rg = (y0 + r) * nx + x0 + 4 * c;
    if (d) p.gmask |= 16u;
    return p;
}

// Queues the asynchronous copies of velocity k (planes at F + k N and
// F + NF + k N) into buffer `buf`: when `fast`, the thread's whole 16-byte
// chunks of the aligned interior and its side-column elements (plan `cp`);
// otherwise element copies of everything (wrapped columns, a ragged tile
// edge, nx not a multiple of 4).
__device__ __forceinline__ void adv2_issue(float* buf, const float* src, const float* RL, const float* base,
                                           long long kN, long long NF, const int* rowoff, const int* coloff,
                                           int x0, int y0, int nx, int ny, bool fast, bool with_base,
                                           const Adv2Copies& cp) {
    float* H = buf;
    float* Rs = buf + kA2H;
    float* Bs = Rs + kA2T;
    const int t = threadIdx.x;
    if (fast) {
        const float* sF = src + kN;
        const float* sG = sF + NF;
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            if (cp.hs[q] >= 0) cp_async16(H + cp.hs[q], ((cp.gmask >> q) & 1u ? sG : sF) + cp.hg[q]);
            if (cp.ss[q] >= 0) cp_async_elem<float>(H + cp.ss[q], ((cp.gmask >> (2 + q)) & 1u ? sG : sF) + cp.sg[q]);
        }
        const long long g = kN + ((cp.gmask & 16u) ? NF : 0) + cp.rg;
        cp_async16(Rs + cp.rs, RL + g);
        if (with_base) cp_async16(Bs + cp.rs, base + g);
    } else {
        for (int e = t; e < 2 * kA2Rows * (kAdvX + 6); e += 256) {
            const int i = e % (kAdvX + 6), r = (e / (kAdvX + 6)) % kA2Rows, d = e / ((kAdvX + 6) * kA2Rows);
            cp_async_elem<float>(H + (d * kA2Rows + r) * kA2Row + i + 1, src + d * NF + kN + rowoff[r] + coloff[i]);
        }
        for (int e = t; e < 2 * kAdvY * kAdvX; e += 256) {
            const int c = e % kAdvX, r = (e / kAdvX) % kAdvY, d = e / (kAdvX * kAdvY);
            if (x0 + c < nx && y0 + r < ny) {
                const long long g = d * NF + kN + (long long)(y0 + r) * nx + x0 + c;
                cp_async_elem<float>(Rs + (d * kAdvY + r) * kAdvX + c, RL + g);
                if (with_base) cp_async_elem<float>(Bs + (d * kAdvY + r) * kAdvX + c, base + g);
            }
        }
    }
}

// three CTAs per SM: with up to 85 registers the constants of the packed
// arithmetic and the copy plan stay in registers (with the 64 of four CTAs
// per SM the kernel executed 9 % more instructions and took 10 % longer)
template <int Q>
__global__ void __launch_bounds__(256, 3)
k2_adv2(Slab2 s, const float* __restrict__ rtab, const float* __restrict__ src, const float* base, float* out,
        const float* __restrict__ RL, double alpha, double beta) {
    constexpr int K = Q * Q, RPW = kAdvY / 8;
    static_assert(kAdvX == 32 && kAdvY == 16, "run split: 33 = 5 + 7 x 4 x-faces, 17 = 5 + 3 x 4 y-faces");
    extern __shared__ __align__(16) double sma[];
    float* buf0 = reinterpret_cast<float*>(sma);
    float2* FX = reinterpret_cast<float2*>(buf0 + 2 * kA2Buf);
    float2* FY = FX + kAdvY * (kAdvX + 1);
    int* rowoff = reinterpret_cast<int*>(FY + (kAdvY + 1) * kAdvX);
    int* coloff = rowoff + kA2Rows;
    const int nx = s.nx, ny = s.ny;
    const long long N = s.N, NF = (long long)K * N;
    const int tilesx = (nx + kAdvX - 1) / kAdvX;
    const int x0 = (blockIdx.x % tilesx) * kAdvX, y0 = (blockIdx.x / tilesx) * kAdvY;
    TableLayout L(Q);
    for (int e = threadIdx.x; e < kA2Rows + kAdvX + 6; e += blockDim.x) {
        if (e < kA2Rows) rowoff[e] = wrapi(y0 - 3 + e, ny) * nx;
        else coloff[e - kA2Rows] = wrapi(x0 - 3 + (e - kA2Rows), nx);
    }
    __syncthreads();
    const bool fast = (nx % 4 == 0) && (x0 + kAdvX <= nx) && (y0 + kAdvY <= ny);
    const Adv2Copies cplan = adv2_plan(rowoff, coloff, x0, y0, nx);
    const float eps = (float)s.weno_eps, idx = (float)s.inv_dx, dt = (float)s.dt, ralpha = (float)alpha,
                rbeta = (float)beta;
    const bool with_base = (alpha != 0.0);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const bool xrun = threadIdx.x < 128;
    const int rj = xrun ? (threadIdx.x >> 4) : ((threadIdx.x - 128) >> 5);
    const int rl = xrun ? (threadIdx.x & 15) : (threadIdx.x & 31);
    const int fa = rj == 0 ? 0 : 4 * rj + 1, nrun = rj == 0 ? 5 : 4, fl = fa + nrun - 1;
    const int hst = xrun ? 1 : kA2Row;
    // x face f of row r: stencil from halo (r + 3, f); y face f of column c: from halo (f, c + 3)
    const int hrow = xrun ? (rl + 3) * kA2Row + 1 : rl + 3 + 1;
    float2* frow = xrun ? FX + rl * (kAdvX + 1) : FY + rl;
    const int fst = xrun ? 1 : kAdvX;
    const int x = x0 + lane;
    int ooff[RPW];
    bool oval[RPW];
#pragma unroll
    for (int rr = 0; rr < RPW; ++rr) {
        const int y = y0 + warp * RPW + rr;
        oval[rr] = (x < nx && y < ny);
        ooff[rr] = oval[rr] ? y * nx + x : 0;
    }
    const int k0 = blockIdx.y * kAdvPlanes, k1 = min(k0 + kAdvPlanes, K);
    constexpr int HG = kA2Rows * kA2Row;                    // G's halo after F's
    adv2_issue(buf0, src, RL, base, (long long)k0 * N, NF, rowoff, coloff, x0, y0, nx, ny, fast, with_base, cplan);
    cp_async_commit();
    if (k0 + 1 < k1)
        adv2_issue(buf0 + kA2Buf, src, RL, base, (long long)(k0 + 1) * N, NF, rowoff, coloff, x0, y0, nx, ny, fast,
                   with_base, cplan);
    cp_async_commit();
    for (int k = k0; k < k1; ++k) {
        float* buf = buf0 + ((k - k0) & 1) * kA2Buf;
        const float* H = buf;
        const float* Rs = buf + kA2H;
        const float* Bs = Rs + kA2T;
        const float vx = rtab[L.xi + k / Q], vy = rtab[L.xi + k % Q];
        cp_async_wait_1();                                  // velocity k's copies (all but the newest group)
        __syncthreads();
        {
            const bool pos = (xrun ? vx : vy) >= 0.f;       // uniform per warp
            const int dir = pos ? 1 : -1, f0 = pos ? fa : fl;
            const float* hb = H + hrow + (pos ? fa : fl + 5) * hst;
            const int hs = dir * hst;
            auto at = [&](int o) { return make_float2(hb[o], hb[HG + o]); };
            Weno5Run2 w;
            w.start(at(0), at(hs), at(2 * hs), at(3 * hs), at(4 * hs), eps);
#pragma unroll
            for (int q = 0; q < 5; ++q) {
                if (q >= nrun) break;
                frow[(f0 + dir * q) * fst] = w.face();
                if (q + 1 < nrun) w.shift(at((q + 5) * hs));
            }
        }
        __syncthreads();
        const float2 cx = f2s(-vx * idx), cy = f2s(-vy * idx);
        float* op = out + (long long)k * N;
#pragma unroll
        for (int rr = 0; rr < RPW; ++rr) {
            if (!oval[rr]) continue;
            const int ty = warp * RPW + rr;
            float2 Rv = make_float2(Rs[ty * kAdvX + lane], Rs[(kAdvY + ty) * kAdvX + lane]);
            Rv = fma2(cx, sub2(FX[ty * (kAdvX + 1) + lane + 1], FX[ty * (kAdvX + 1) + lane]), Rv);
            Rv = fma2(cy, sub2(FY[(ty + 1) * kAdvX + lane], FY[ty * kAdvX + lane]), Rv);
            const int hc = (ty + 3) * kA2Row + lane + 4;
            const float2 hv = make_float2(H[hc], H[HG + hc]);
            float2 o = mul2(f2s(rbeta), fma2(f2s(dt), Rv, hv));
            if (with_base)
                o = fma2(f2s(ralpha), make_float2(Bs[ty * kAdvX + lane], Bs[(kAdvY + ty) * kAdvX + lane]), o);
            op[ooff[rr]] = o.x;
            op[NF + ooff[rr]] = o.y;
        }
        __syncthreads();                                    // this buffer and the faces consumed
        if (k + 2 < k1)
            adv2_issue(buf, src, RL, base, (long long)(k + 2) * N, NF, rowoff, coloff, x0, y0, nx, ny, fast,
                       with_base, cplan);
        cp_async_commit();
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

// Force plan of k2_fields: the disc's offset columns a = 0 .. Mf, each as a
// run of `steps` weight pairs (a multiple of 8: offsets b = -w .. w, then
// zeros), column 0 with halved g2y (its pass adds n(x) twice); the columns
// are dealt to the kFWarps warps longest first, each to the least loaded
// warp (deterministic).  Layout of `plan`: kFWarps + 1 prefix offsets
// (padded to kFPlanHead ints), then per entry {a, weight offset, steps, w}.
struct ForcePlan {
    std::vector<int> plan;
    std::vector<double> w;     // (g2x, g2y) pairs
    bool ok = true;
};

ForcePlan force_plan(const Taps2& t) {
    ForcePlan fp;
    const int Mf = t.Mf, D = 2 * Mf + 1;
    std::vector<double> gx((size_t)D * D, 0.0), gy((size_t)D * D, 0.0);
    std::vector<char> in((size_t)D * D, 0);
    for (size_t j = 0; j < t.fg.size() / 2; ++j) {
        const size_t k = (size_t)(t.foff[2 * j] + Mf) * D + (t.foff[2 * j + 1] + Mf);
        gx[k] = t.fg[2 * j];
        gy[k] = t.fg[2 * j + 1];
        in[k] = 1;
    }
    auto at = [&](int a, int b) { return (size_t)(a + Mf) * D + (b + Mf); };
    struct Col { int a, w, steps, off; };
    std::vector<Col> cols;
    for (int a = 0; a <= Mf; ++a) {
        int w = -1;
        for (int b = -Mf; b <= Mf; ++b)
            if (in[at(a, b)] || in[at(-a, b)]) w = std::max(w, std::abs(b));
        if (w < 0) continue;
        for (int b = -w; b <= w; ++b)   // the pairing needs the disc's mirror symmetry, exactly
            if (in[at(a, b)] != in[at(-a, b)] || gx[at(a, b)] != -gx[at(-a, b)] || gy[at(a, b)] != gy[at(-a, b)])
                fp.ok = false;
        const int steps = (2 * w + 8 + 7) & ~7;
        cols.push_back({a, w, steps, (int)(fp.w.size() / 2)});
        for (int j = 0; j < steps; ++j) {
            const int b = j - w;
            double x = 0.0, y = 0.0;
            if (b <= w) {
                x = (a == 0) ? 0.0 : gx[at(a, b)];
                y = (a == 0) ? 0.5 * gy[at(a, b)] : gy[at(a, b)];
            }
            fp.w.push_back(x);
            fp.w.push_back(y);
        }
    }
    std::vector<int> order(cols.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
    std::stable_sort(order.begin(), order.end(), [&](int p, int q) { return cols[p].steps > cols[q].steps; });
    std::vector<std::vector<int>> bins(kFWarps);
    std::vector<long long> load(kFWarps, 0);
    for (int ci : order) {
        int best = 0;
        for (int k = 1; k < kFWarps; ++k)
            if (load[k] < load[best]) best = k;
        bins[best].push_back(ci);
        load[best] += cols[ci].steps;
    }
    fp.plan.assign(kFPlanHead, 0);
    int n = 0;
    for (int k = 0; k < kFWarps; ++k) {
        fp.plan[k] = n;
        n += (int)bins[k].size();
    }
    fp.plan[kFWarps] = n;
    for (int k = 0; k < kFWarps; ++k)
        for (int ci : bins[k]) {
            const Col& c = cols[ci];
            fp.plan.insert(fp.plan.end(), {c.a, c.off, c.steps, c.w});
        }
    return fp;
}

// Parity blocks of the force term's derivative on the velocity set,
// D_kj = sum_{l=1}^{Q-1} w_k psi_l(xi_k) sqrt(l) psi_{l-1}(xi_j) (D = S shift P,
// the synthesis of the coefficient form F sqrt(l) a_{l-1}), in long double:
// DA_kj = (D_kj - D_{k,Q-1-j}) / 2 and DB_kj = (D_kj + D_{k,Q-1-j}) / 2 for
// k, j < Q/2, as [QH][QH] each (DA then DB).
std::vector<double> d_blocks(int Q, const double* xi, const double* w) {
    const int QH = Q / 2;
    std::vector<long double> ps((size_t)Q * (Q + 1));
    for (int k = 0; k < Q; ++k) {
        long double* p = ps.data() + (size_t)k * (Q + 1);
        const long double x = xi[k];
        p[0] = 1;
        p[1] = x;
        for (int l = 1; l < Q; ++l) p[l + 1] = (x * p[l] - sqrtl((long double)l) * p[l - 1]) / sqrtl((long double)(l + 1));
    }
    auto D = [&](int k, int j) {
        long double acc = 0;
        for (int l = 1; l < Q; ++l)
            acc += (long double)w[k] * ps[(size_t)k * (Q + 1) + l] * sqrtl((long double)l) * ps[(size_t)j * (Q + 1) + l - 1];
        return acc;
    };
    std::vector<double> out(2 * (size_t)QH * QH);
    for (int k = 0; k < QH; ++k)
        for (int j = 0; j < QH; ++j) {
            const long double a = D(k, j), b = D(k, Q - 1 - j);
            out[k * QH + j] = (double)(0.5L * (a - b));
            out[QH * QH + k * QH + j] = (double)(0.5L * (a + b));
        }
    return out;
}

template <typename R>
Pow2<R> make_pow2(int Q, const double* xi) {
    Pow2<R> p{};
    for (int k = 0; k < Q && k < 16; ++k) {
        const double x = xi[k], x2 = x * x;
        p.v[k] = (R)x;
        p.v2[k] = (R)x2;
        p.v3[k] = (R)(x2 * x);
        p.h[k] = (float)x;
        p.l[k] = (float)(x - (double)p.h[k]);
        p.h2[k] = (float)x2;
        p.l2[k] = (float)(x2 - (double)p.h2[k]);
    }
    return p;
}
}  // namespace

bool validate_2d(const evfdlb_params& p) {
    if (p.dim != 2 || p.nx < 8 || p.ny < 8 || !(p.dx > 0) || !(p.sigma > 0) || !(p.phi_a >= 0)) return false;
    if ((long long)p.nx * p.ny >= (1LL << 31)) return false;   // node offsets are 32-bit in k2_adv
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
    int* fplan = nullptr;        // force plan: per-warp column lists (k2_fields)
    void* ftw = nullptr;         // force weight pairs per column step, precision R
    int* fm_off = nullptr;
    void* fm_w = nullptr;        // Fischer-Methfessel weights, precision R
    float* prf = nullptr;        // FP32 build: node primitives [kNumPrf2][N] of the stage input
    Pow2<float> pwf{};
    Pow2<double> pwd{};
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

// k2_adv is compiled for each even Q of the 2D model (4 .. 16) and both
// output forms
template <typename R, bool RHS>
void launch_adv_t(int Q, dim3 g, cudaStream_t st, const Slab2& s, const R* rtab, const R* src, const R* base,
                  R* out, const R* RL, double* rhs_out, double alpha, double beta) {
    switch (Q) {
        case 4: k2_adv<R, 4, RHS><<<g, 256, 0, st>>>(s, rtab, src, base, out, RL, rhs_out, alpha, beta); break;
        case 6: k2_adv<R, 6, RHS><<<g, 256, 0, st>>>(s, rtab, src, base, out, RL, rhs_out, alpha, beta); break;
        case 8: k2_adv<R, 8, RHS><<<g, 256, 0, st>>>(s, rtab, src, base, out, RL, rhs_out, alpha, beta); break;
        case 10: k2_adv<R, 10, RHS><<<g, 256, 0, st>>>(s, rtab, src, base, out, RL, rhs_out, alpha, beta); break;
        case 12: k2_adv<R, 12, RHS><<<g, 256, 0, st>>>(s, rtab, src, base, out, RL, rhs_out, alpha, beta); break;
        case 14: k2_adv<R, 14, RHS><<<g, 256, 0, st>>>(s, rtab, src, base, out, RL, rhs_out, alpha, beta); break;
        default: k2_adv<R, 16, RHS><<<g, 256, 0, st>>>(s, rtab, src, base, out, RL, rhs_out, alpha, beta); break;
    }
}

// the FP32 stage form: F and G of a velocity as float2 pairs
void launch_adv2(int Q, dim3 g, cudaStream_t st, const Slab2& s, const float* rtab, const float* src,
                 const float* base, float* out, const float* RL, double alpha, double beta) {
    switch (Q) {
        case 4: k2_adv2<4><<<g, 256, kA2Smem, st>>>(s, rtab, src, base, out, RL, alpha, beta); break;
        case 6: k2_adv2<6><<<g, 256, kA2Smem, st>>>(s, rtab, src, base, out, RL, alpha, beta); break;
        case 8: k2_adv2<8><<<g, 256, kA2Smem, st>>>(s, rtab, src, base, out, RL, alpha, beta); break;
        case 10: k2_adv2<10><<<g, 256, kA2Smem, st>>>(s, rtab, src, base, out, RL, alpha, beta); break;
        case 12: k2_adv2<12><<<g, 256, kA2Smem, st>>>(s, rtab, src, base, out, RL, alpha, beta); break;
        case 14: k2_adv2<14><<<g, 256, kA2Smem, st>>>(s, rtab, src, base, out, RL, alpha, beta); break;
        default: k2_adv2<16><<<g, 256, kA2Smem, st>>>(s, rtab, src, base, out, RL, alpha, beta); break;
    }
}

template <typename R>
void launch_adv(int Q, dim3 g, cudaStream_t st, const Slab2& s, const R* rtab, const R* src, const R* base, R* out,
                const R* RL, double* rhs_out, double alpha, double beta, int mode) {
    if (mode == 1) launch_adv_t<R, true>(Q, g, st, s, rtab, src, base, out, RL, rhs_out, alpha, beta);
    else launch_adv_t<R, false>(Q, g, st, s, rtab, src, base, out, RL, rhs_out, alpha, beta);
}

// k2_moments: 128 nodes per CTA pass (grid-stride beyond 8192 CTAs)
int moments_grid(long long N) { return (int)std::min<long long>((N + 127) / 128, 8192); }

// k2_moments is compiled for each even Q of the 2D model (4 .. 16)
template <typename R>
void launch_moments(int Q, int nb, cudaStream_t st, const Slab2& s, const Pow2<R>& pw, const R* src, double* mom,
                    float* prf, unsigned* err) {
    switch (Q) {
        case 4: k2_moments<R, 4><<<nb, 256, 0, st>>>(s, pw, src, mom, prf, err); break;
        case 6: k2_moments<R, 6><<<nb, 256, 0, st>>>(s, pw, src, mom, prf, err); break;
        case 8: k2_moments<R, 8><<<nb, 256, 0, st>>>(s, pw, src, mom, prf, err); break;
        case 10: k2_moments<R, 10><<<nb, 256, 0, st>>>(s, pw, src, mom, prf, err); break;
        case 12: k2_moments<R, 12><<<nb, 256, 0, st>>>(s, pw, src, mom, prf, err); break;
        case 14: k2_moments<R, 14><<<nb, 256, 0, st>>>(s, pw, src, mom, prf, err); break;
        default: k2_moments<R, 16><<<nb, 256, 0, st>>>(s, pw, src, mom, prf, err); break;
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
    constexpr bool F32 = std::is_same<R, float>::value;
    // FP32: the field kernel reads the FP32 primitives; the FP64 raw sums are
    // only needed by the FP64 build and by the diagnostics
    const int nbm = moments_grid(s.N);
    if constexpr (F32) launch_moments<float>(Q, nbm, st, s, c->pwf, (const float*)src, nullptr, c->prf, c->err);
    else launch_moments<double>(Q, nbm, st, s, c->pwd, (const double*)src, c->mom, nullptr, c->err);
    dim3 gf((s.nx + kTile2 - 1) / kTile2, (s.ny + kTile2 - 1) / kTile2);
    k2_fields<R><<<gf, 256, c->smem_fields, st>>>(s, c->mom, c->prf, (const R*)c->ftw, c->fplan, c->fm_off,
                                                   (const R*)c->fm_w, (R*)c->fld, c->err);
    int nc = (int)((s.N + kNB - 1) / kNB);
    launch_coll<R>(Q, nc, c->smem_coll, st, s, (const R*)c->rtab, (const R*)src, (const R*)c->fld, (R*)c->RL);
    const int tiles = ((s.nx + kAdvX - 1) / kAdvX) * ((s.ny + kAdvY - 1) / kAdvY);
    if (F32 && mode == 0) {   // the FP32 stage form: one CTA column per group of velocities, F and G paired
        dim3 ga(tiles, (Q * Q + kAdvPlanes - 1) / kAdvPlanes);
        launch_adv2(Q, ga, st, s, (const float*)c->rtab, (const float*)src, (const float*)base, (float*)out,
                    (const float*)c->RL, alpha, beta);
    } else {
        dim3 ga(tiles, (2 * Q * Q + kAdvPlanes - 1) / kAdvPlanes);
        launch_adv<R>(Q, ga, st, s, (const R*)c->rtab, (const R*)src, (const R*)base, (R*)out, (const R*)c->RL,
                      rhs_out, alpha, beta, mode);
    }
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
    cudaFree(c->fplan);
    cudaFree(c->ftw);
    cudaFree(c->fm_off);
    cudaFree(c->fm_w);
    cudaFree(c->prf);
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
    const ForcePlan fp = force_plan(t);
    if (!fp.ok) e = cudaErrorInvalidValue;      // the tap set lost its mirror symmetry
    const bool f32 = (c->prec == EVFDLB_FP32);
    alloc((void**)&c->fplan, sizeof(int) * fp.plan.size());
    alloc(&c->ftw, c->esize * fp.w.size());
    alloc((void**)&c->fm_off, sizeof(int) * t.moff.size());
    alloc(&c->fm_w, c->esize * t.mw.size());
    if (f32) alloc((void**)&c->prf, sizeof(float) * kNumPrf2 * s.N);
    std::vector<double> dbl = d_blocks(p.Q, xi.data(), w.data());
    {   // k2_coll's constant block: DA, DB, then S[k][l] = w_k psi_l(xi_k)
        const TableLayout L(p.Q);
        dbl.insert(dbl.end(), tab.begin() + L.S, tab.begin() + L.S + p.Q * p.Q);
    }
    const std::vector<float> dblf(dbl.begin(), dbl.end());
    alloc((void**)&c->scratch, sizeof(double) * (2 * NF + 8));
    alloc((void**)&c->err, sizeof(unsigned));
    std::vector<float> tabf(tab.begin(), tab.end()), ftwf(fp.w.begin(), fp.w.end()), mwf(t.mw.begin(), t.mw.end());
    if (f32) alloc(&c->rtab, sizeof(float) * tab.size());
    else c->rtab = c->tables;
    c->pwf = make_pow2<float>(p.Q, xi.data());
    c->pwd = make_pow2<double>(p.Q, xi.data());
    if (e == cudaSuccess) e = cudaMemcpy(c->tables, tab.data(), sizeof(double) * tab.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && c->prec == EVFDLB_FP32)
        e = cudaMemcpy(c->rtab, tabf.data(), sizeof(float) * tabf.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(c->fplan, fp.plan.data(), sizeof(int) * fp.plan.size(), cudaMemcpyHostToDevice);
    // the parity blocks and the synthesis matrix of this Q into k2_coll's
    // constant bank (every context of the same Q writes the same values)
    if (e == cudaSuccess)
        e = f32 ? cudaMemcpyToSymbol(c_coll_f, dblf.data(), sizeof(float) * dblf.size(),
                                     sizeof(float) * coll_coff(p.Q))
                : cudaMemcpyToSymbol(c_coll_d, dbl.data(), sizeof(double) * dbl.size(),
                                     sizeof(double) * coll_coff(p.Q));
    if (e == cudaSuccess)
        e = f32 ? cudaMemcpy(c->ftw, ftwf.data(), sizeof(float) * ftwf.size(), cudaMemcpyHostToDevice)
                : cudaMemcpy(c->ftw, fp.w.data(), sizeof(double) * fp.w.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(c->fm_off, t.moff.data(), sizeof(int) * t.moff.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = f32 ? cudaMemcpy(c->fm_w, mwf.data(), sizeof(float) * mwf.size(), cudaMemcpyHostToDevice)
                : cudaMemcpy(c->fm_w, t.mw.data(), sizeof(double) * t.mw.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(c->err, 0, sizeof(unsigned));
    c->smem_fields = f32 ? fields_smem_bytes<float>(s.Mf, s.mfm) : fields_smem_bytes<double>(s.Mf, s.mfm);
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
    const int nbm = moments_grid(N);
    if (c->prec == EVFDLB_FP32)
        launch_moments<float>(c->s.Q, nbm, c->user, c->s, c->pwf, (const float*)c->state[0], c->mom, nullptr, c->err);
    else
        launch_moments<double>(c->s.Q, nbm, c->user, c->s, c->pwd, (const double*)c->state[0], c->mom, nullptr, c->err);
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
