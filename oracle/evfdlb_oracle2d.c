/*
 * evfdlb_oracle2d.c -- plain, slow FP64 CPU reference ("the oracle") for one
 * time step of the two-dimensional extension of the EV1 Enskog-Vlasov FDLB
 * model of Busuioc & Sofonea (arXiv:2503.15187).  The paper solves a 1D
 * slab and leaves 2D as future work (Sec. IV); this file states the
 * tensor-product extension of its equations written out from Sec. II-III.
 *
 * TEST INFRASTRUCTURE ONLY, like evfdlb_oracle.c: only the test suite may
 * load it.  It shares nothing with the CUDA library; the 1D velocity set and
 * projection rule arrive as arrays from the caller (numpy's Gauss-Hermite).
 *
 * Model (READINGS, each a plain extension of the 1D statement):
 *  - homogeneity along z; reduced distributions over p_z:
 *      F(x, y, xi_x, xi_y) = int f dp_z,  G = int f p_z^2/2 dp_z;
 *  - velocity set: tensor product of the 1D full-range Gauss-Hermite set of
 *    order Q per axis; projections to order Q-1 per axis;
 *  - moments: n = sum F, n u = sum xi F, (3/2) n T = sum [(xi-u)^2/2 F + G],
 *    q = sum c [c^2/2 F + G], c = xi - u (in-plane);
 *  - reduced Shakhov equilibria and J1 (one transverse direction,
 *    <c_z^2> = T, <c_z^4> = 3 T^2), with s = (1 - Pr)/(n T^2):
 *      F^S = F_MB [1 + s (c.q)(c^2/(5T) - 4/5)]
 *      G^S = T/2 F_MB [1 + s (c.q)(c^2/(5T) - 2/5)]
 *      J1_F = -b n chi F_MB { c.A + 3/5 (c^2/(2T) - 2) c.B
 *                             + 2/5 [ c.D.c / T + (c^2/(2T) - 2) div u ] }
 *      J1_G = -b n chi F_MB { T/2 c.A + 3/10 (c^2/2 - T) c.B
 *                             + 1/5 [ c.D.c + (c^2/2 - T) div u ] }
 *    with A = grad(n^2 chi T)/(n^2 chi T), B = grad T / T, D_ij = d_i u_j,
 *    F_MB = n (2 pi T)^-1 exp(-c^2/(2T));
 *  - force: the Eq. (force) integral over z gives the in-plane kernel
 *      g2(rho) = rho_vec gamma phi sigma^gamma int (rho^2 + z^2)^(-(gamma+2)/2) dz
 *    over the z where rho^2 + z^2 > sigma^2 (all z for rho >= sigma; for
 *    gamma = 6 and rho >= sigma, (15 pi/8) phi sigma^6 rho_vec / rho^7);
 *    F = sum over grid offsets with |rho| <= r_cut of dx^2 g2(rho) n(r + rho)
 *    (the rectangle rule over the disc);
 *  - Fischer-Methfessel average: the sphere average reduced to the plane,
 *    weights 2 sqrt(sigma^2 - rho^2) on offsets with rho < sigma, normalised
 *    to sum 1 (so that a uniform density is its own average);
 *  - advection: WENO-5 along x and along y (dimension by dimension);
 *    gradients: fourth-order central differences along each axis;
 *  - boundaries: periodic in x and y;
 *  - chi, the transport coefficients and the time integrator as in 1D.
 * Layout: F[k * N + y * nx + x], k = kx * Q + ky, N = nx * ny.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int nx, ny, Q;
    double dx, dt;
    double sigma, phi, gamma, rcut, weno_eps;
    int relax;            /* 0: rate 1/tau; 1: rate chi/tau                */
    const double *xi;     /* [Q] 1D velocity nodes                          */
    const double *w;      /* [Q] weights, sum 1                             */
    int nq;               /* points per axis of the projection rule          */
    const double *zq, *wq;
} orc2_params;

#define ORC2_NFIELDS 22   /* see orc2_node_fields */

static const double PI2D = 3.14159265358979323846;

double orc_weno5(double v0, double v1, double v2, double v3, double v4, double eps);  /* evfdlb_oracle.c */

static int wrap(int i, int n)
{
    int r = i % n;
    return r < 0 ? r + n : r;
}

static void hermite_all2(int L, double x, double *he)
{
    he[0] = 1.0;
    if (L >= 1) he[1] = x;
    for (int l = 1; l < L; l++) he[l + 1] = x * he[l] - l * he[l - 1];
}

/* ------------------------------------------------------------------ */
/* In-plane force kernel                                               */
/* ------------------------------------------------------------------ */

/* Gauss-Legendre rule of order 32 on [-1, 1] (Newton on P_32, textbook). */
static void gauss_legendre32(double *x, double *w)
{
    const int n = 32;
    for (int i = 0; i < n; i++) {
        double z = cos(PI2D * (i + 0.75) / (n + 0.5)), pp = 0.0;
        for (int it = 0; it < 100; it++) {
            double p1 = 1.0, p2 = 0.0;
            for (int j = 1; j <= n; j++) {
                double p3 = p2;
                p2 = p1;
                p1 = ((2.0 * j - 1.0) * z * p2 - (j - 1.0) * p3) / j;
            }
            pp = n * (z * p1 - p2) / (z * z - 1.0);
            double dz = p1 / pp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * pp * pp);
    }
}

/* int_{|z| > z0} (a^2 + z^2)^(-s) dz with z = a tan(theta):
 * 2 a^(1-2s) int_0^{phi0} sin^(2s-2)(phi) d phi, phi0 = atan(a / z0) (pi/2 for
 * z0 = 0), by the 32-point Gauss-Legendre rule on [0, phi0]; no cancellation
 * for small a. */
static double line_integral(int s, double a, double z0)
{
    static double gx[32], gw[32];
    static int ready = 0;
#pragma omp critical(orc2_gauss_legendre)
    {
        if (!ready) {
            gauss_legendre32(gx, gw);
            ready = 1;
        }
    }
    double phi0 = (z0 > 0.0) ? atan(a / z0) : 0.5 * PI2D;
    double acc = 0.0;
    for (int i = 0; i < 32; i++) {
        double ph = 0.5 * phi0 * (gx[i] + 1.0);
        acc += gw[i] * pow(sin(ph), 2 * s - 2);
    }
    return 2.0 * pow(a, 1.0 - 2.0 * s) * 0.5 * phi0 * acc;
}

/* g2 at in-plane offset (rx, ry): out[0], out[1].  gamma must be even. */
void orc2_force_kernel(const orc2_params *p, double rx, double ry, double *out)
{
    double r = sqrt(rx * rx + ry * ry);
    out[0] = out[1] = 0.0;
    if (r == 0.0) return;
    int s = (int)lround((p->gamma + 2.0) / 2.0);
    double z0 = (r < p->sigma) ? sqrt(p->sigma * p->sigma - r * r) : 0.0;
    double J = line_integral(s, r, z0);
    double c = p->gamma * p->phi * pow(p->sigma, p->gamma) * J;
    out[0] = c * rx;
    out[1] = c * ry;
}

/* discrete force constant a_d = (1/2) sum dx^2 rho_x g2_x over the disc:
 * for n = n0 + G x the discrete force is F_x = 2 a_d G */
double orc2_discrete_a(const orc2_params *p)
{
    int M = (int)floor(p->rcut / p->dx + 1e-9);
    double acc = 0.0, g[2];
    for (int a = -M; a <= M; a++)
        for (int b = -M; b <= M; b++) {
            double rx = a * p->dx, ry = b * p->dx;
            if (rx * rx + ry * ry > p->rcut * p->rcut * (1.0 + 1e-12)) continue;
            orc2_force_kernel(p, rx, ry, g);
            acc += p->dx * p->dx * rx * g[0];
        }
    return 0.5 * acc;
}

static double chi_cs(const orc2_params *p, double n)
{
    double eta = PI2D * p->sigma * p->sigma * p->sigma * n / 6.0;
    double om = 1.0 - eta;
    return (2.0 - eta) / (2.0 * om * om * om);
}

/* ------------------------------------------------------------------ */
/* Moments                                                             */
/* ------------------------------------------------------------------ */

void orc2_moments(const orc2_params *p, const double *F, const double *G, double *n,
                  double *ux, double *uy, double *T, double *qx, double *qy)
{
    int N = p->nx * p->ny, Q = p->Q;
#pragma omp parallel for schedule(static)
    for (int i = 0; i < N; i++) {
        double sn = 0.0, sx = 0.0, sy = 0.0;
        for (int kx = 0; kx < Q; kx++)
            for (int ky = 0; ky < Q; ky++) {
                double f = F[(kx * Q + ky) * N + i];
                sn += f;
                sx += p->xi[kx] * f;
                sy += p->xi[ky] * f;
            }
        double u = sx / sn, v = sy / sn;
        double se = 0.0, sqx = 0.0, sqy = 0.0;
        for (int kx = 0; kx < Q; kx++)
            for (int ky = 0; ky < Q; ky++) {
                int k = kx * Q + ky;
                double cx = p->xi[kx] - u, cy = p->xi[ky] - v;
                double e = 0.5 * (cx * cx + cy * cy) * F[k * N + i] + G[k * N + i];
                se += e;
                sqx += cx * e;
                sqy += cy * e;
            }
        n[i] = sn;
        ux[i] = u;
        uy[i] = v;
        T[i] = 2.0 * se / (3.0 * sn);
        qx[i] = sqx;
        qy[i] = sqy;
    }
}

/* ------------------------------------------------------------------ */
/* Node fields                                                         */
/* ------------------------------------------------------------------ */

static double d4x(const orc2_params *p, const double *f, int x, int y)
{
    int nx = p->nx, ny = p->ny;
    (void)ny;
    return (f[y * nx + wrap(x - 2, nx)] - 8.0 * f[y * nx + wrap(x - 1, nx)]
            + 8.0 * f[y * nx + wrap(x + 1, nx)] - f[y * nx + wrap(x + 2, nx)]) / (12.0 * p->dx);
}

static double d4y(const orc2_params *p, const double *f, int x, int y)
{
    int nx = p->nx, ny = p->ny;
    return (f[wrap(y - 2, ny) * nx + x] - 8.0 * f[wrap(y - 1, ny) * nx + x]
            + 8.0 * f[wrap(y + 1, ny) * nx + x] - f[wrap(y + 2, ny) * nx + x]) / (12.0 * p->dx);
}

/* Per-node fields as [ORC2_NFIELDS][N]:
 *  0 n  1 ux  2 uy  3 T  4 qx  5 qy  6 nbar  7 chi  8 Fx  9 Fy
 * 10 mu 11 tau 12 Pr 13 nu 14 Ax 15 Ay 16 Bx 17 By
 * 18 Dxx = d_x ux  19 Dxy = d_x uy  20 Dyx = d_y ux  21 Dyy = d_y uy */
void orc2_node_fields(const orc2_params *p, const double *n, const double *ux, const double *uy,
                      const double *T, const double *qx, const double *qy, double *out)
{
    int nx = p->nx, ny = p->ny, N = nx * ny;
    double b = 2.0 * PI2D * p->sigma * p->sigma * p->sigma / 3.0;
    for (int f = 0; f < ORC2_NFIELDS; f++) memset(out + (size_t)f * N, 0, N * sizeof(double));
    memcpy(out + 0 * N, n, N * sizeof(double));
    memcpy(out + 1 * N, ux, N * sizeof(double));
    memcpy(out + 2 * N, uy, N * sizeof(double));
    memcpy(out + 3 * N, T, N * sizeof(double));
    memcpy(out + 4 * N, qx, N * sizeof(double));
    memcpy(out + 5 * N, qy, N * sizeof(double));
    double *nbar = out + 6 * N, *chi = out + 7 * N, *Fx = out + 8 * N, *Fy = out + 9 * N;
    double *mu = out + 10 * N, *tau = out + 11 * N, *Pr = out + 12 * N, *nu = out + 13 * N;
    double *Ax = out + 14 * N, *Ay = out + 15 * N, *Bx = out + 16 * N, *By = out + 17 * N;
    double *Dxx = out + 18 * N, *Dxy = out + 19 * N, *Dyx = out + 20 * N, *Dyy = out + 21 * N;

    /* Fischer-Methfessel average with normalised chord weights */
    int m = (int)ceil(p->sigma / p->dx);
    double wsum = 0.0;
    for (int a = -m; a <= m; a++)
        for (int c = -m; c <= m; c++) {
            double r2 = (a * a + c * c) * p->dx * p->dx;
            if (r2 < p->sigma * p->sigma) wsum += 2.0 * sqrt(p->sigma * p->sigma - r2);
        }
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; y++)
        for (int x = 0; x < nx; x++) {
            double acc = 0.0;
            for (int a = -m; a <= m; a++)
                for (int c = -m; c <= m; c++) {
                    double r2 = (a * a + c * c) * p->dx * p->dx;
                    if (r2 >= p->sigma * p->sigma) continue;
                    acc += 2.0 * sqrt(p->sigma * p->sigma - r2) * n[wrap(y + c, ny) * nx + wrap(x + a, nx)];
                }
            nbar[y * nx + x] = acc / wsum;
            chi[y * nx + x] = chi_cs(p, nbar[y * nx + x]);
        }

    /* force over the disc |rho| <= rcut (kernel values tabulated once) */
    int M = (int)floor(p->rcut / p->dx + 1e-9), W = 2 * M + 1;
    double *gt = (double *)calloc(2 * (size_t)W * W, sizeof(double));
    for (int a = -M; a <= M; a++)
        for (int c = -M; c <= M; c++) {
            double rx = a * p->dx, ry = c * p->dx;
            if (rx * rx + ry * ry > p->rcut * p->rcut * (1.0 + 1e-12)) continue;
            orc2_force_kernel(p, rx, ry, gt + 2 * ((a + M) * W + (c + M)));
        }
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; y++)
        for (int x = 0; x < nx; x++) {
            double sx = 0.0, sy = 0.0;
            for (int a = -M; a <= M; a++)
                for (int c = -M; c <= M; c++) {
                    const double *g = gt + 2 * ((a + M) * W + (c + M));
                    double nn = n[wrap(y + c, ny) * nx + wrap(x + a, nx)];
                    sx += p->dx * p->dx * g[0] * nn;
                    sy += p->dx * p->dx * g[1] * nn;
                }
            Fx[y * nx + x] = sx;
            Fy[y * nx + x] = sy;
        }
    free(gt);

    /* gradients (READING as in 1D: A = grad X / X, B = grad T / T) */
    double *X = (double *)malloc(N * sizeof(double));
    for (int i = 0; i < N; i++) X[i] = n[i] * n[i] * chi[i] * T[i];
    for (int y = 0; y < ny; y++)
        for (int x = 0; x < nx; x++) {
            int i = y * nx + x;
            Ax[i] = d4x(p, X, x, y) / X[i];
            Ay[i] = d4y(p, X, x, y) / X[i];
            Bx[i] = d4x(p, T, x, y) / T[i];
            By[i] = d4y(p, T, x, y) / T[i];
            Dxx[i] = d4x(p, ux, x, y);
            Dxy[i] = d4x(p, uy, x, y);
            Dyx[i] = d4y(p, ux, x, y);
            Dyy[i] = d4y(p, uy, x, y);
        }
    free(X);

    /* transport, Eqs. (viscosity), (tau), (prandtl) */
    for (int i = 0; i < N; i++) {
        double bn = b * n[i], xx = bn * chi[i];
        double mu0 = 5.0 / (16.0 * p->sigma * p->sigma) * sqrt(T[i] / PI2D);
        mu[i] = mu0 * (1.0 / chi[i] + 0.8 * bn + 4.0 / 25.0 * (1.0 + 12.0 / PI2D) * bn * bn * chi[i]);
        tau[i] = mu[i] / (n[i] * T[i] * (1.0 + 0.4 * xx));
        Pr[i] = 2.0 / 3.0 * (1.0 + 0.6 * xx) / (1.0 + 0.4 * xx)
              * (1.0 + 0.8 * xx + 4.0 / 25.0 * (1.0 + 12.0 / PI2D) * xx * xx)
              / (1.0 + 1.2 * xx + 9.0 / 25.0 * (1.0 + 32.0 / (9.0 * PI2D)) * xx * xx);
        nu[i] = (p->relax == 0) ? 1.0 / tau[i] : chi[i] / tau[i];
    }
}

/* ------------------------------------------------------------------ */
/* Projected equilibria and J1 of one node                             */
/* ------------------------------------------------------------------ */

/* Tensor-product projection: h_{kx,ky} = w_kx w_ky sum_{l,m<Q} a_lm He_l(xi_kx) He_m(xi_ky)/(l! m!),
 * a_lm = int h He_l(xi_x) He_m(xi_y) d^2 xi. */
static void project2(const orc2_params *p, const double *a, double *h)
{
    int Q = p->Q;
    double *hx = (double *)malloc((Q + 1) * sizeof(double));
    double *hy = (double *)malloc((Q + 1) * sizeof(double));
    for (int kx = 0; kx < Q; kx++) {
        hermite_all2(Q, p->xi[kx], hx);
        for (int ky = 0; ky < Q; ky++) {
            hermite_all2(Q, p->xi[ky], hy);
            double acc = 0.0, fl = 1.0;
            for (int l = 0; l < Q; l++) {
                if (l > 0) fl *= l;
                double fm = 1.0;
                for (int m = 0; m < Q; m++) {
                    if (m > 0) fm *= m;
                    acc += a[l * Q + m] * hx[l] * hy[m] / (fl * fm);
                }
            }
            h[kx * Q + ky] = p->w[kx] * p->w[ky] * acc;
        }
    }
    free(hx);
    free(hy);
}

/* fl: the node's fields (see orc2_node_fields), one value each */
void orc2_equilibria_node(const orc2_params *p, const double *fl, double *FS, double *GS,
                          double *JF, double *JG)
{
    int Q = p->Q;
    double n = fl[0], ux = fl[1], uy = fl[2], T = fl[3], qx = fl[4], qy = fl[5];
    double chi = fl[7], Pr = fl[12];
    double Ax = fl[14], Ay = fl[15], Bx = fl[16], By = fl[17];
    double Dxx = fl[18], Dxy = fl[19], Dyx = fl[20], Dyy = fl[21];
    double b = 2.0 * PI2D * p->sigma * p->sigma * p->sigma / 3.0;
    double bnchi = b * n * chi, divu = Dxx + Dyy;
    double s = (1.0 - Pr) / (n * T * T);
    double *aS = (double *)calloc(Q * Q, sizeof(double));
    double *bS = (double *)calloc(Q * Q, sizeof(double));
    double *aJ = (double *)calloc(Q * Q, sizeof(double));
    double *bJ = (double *)calloc(Q * Q, sizeof(double));
    double *hx = (double *)malloc((Q + 1) * sizeof(double));
    double *hy = (double *)malloc((Q + 1) * sizeof(double));
    double sqT = sqrt(T);
    for (int i = 0; i < p->nq; i++) {
        double cx = sqT * p->zq[i];
        hermite_all2(Q, ux + cx, hx);
        for (int j = 0; j < p->nq; j++) {
            double cy = sqT * p->zq[j];
            hermite_all2(Q, uy + cy, hy);
            double W = p->wq[i] * p->wq[j] * n;
            double c2 = cx * cx + cy * cy, cq = cx * qx + cy * qy;
            double cA = cx * Ax + cy * Ay, cB = cx * Bx + cy * By;
            double cDc = cx * cx * Dxx + cx * cy * (Dxy + Dyx) + cy * cy * Dyy;
            double pS = 1.0 + s * cq * (c2 / (5.0 * T) - 0.8);
            double pG = 0.5 * T * (1.0 + s * cq * (c2 / (5.0 * T) - 0.4));
            double pJF = -bnchi * (cA + 0.6 * (c2 / (2.0 * T) - 2.0) * cB
                                   + 0.4 * (cDc / T + (c2 / (2.0 * T) - 2.0) * divu));
            double pJG = -bnchi * (0.5 * T * cA + 0.3 * (0.5 * c2 - T) * cB
                                   + 0.2 * (cDc + (0.5 * c2 - T) * divu));
            for (int l = 0; l < Q; l++)
                for (int m = 0; m < Q; m++) {
                    double hh = W * hx[l] * hy[m];
                    aS[l * Q + m] += pS * hh;
                    bS[l * Q + m] += pG * hh;
                    aJ[l * Q + m] += pJF * hh;
                    bJ[l * Q + m] += pJG * hh;
                }
        }
    }
    project2(p, aS, FS);
    project2(p, bS, GS);
    project2(p, aJ, JF);
    project2(p, bJ, JG);
    free(aS); free(bS); free(aJ); free(bJ); free(hx); free(hy);
}

/* Projected Maxwellian pair (F_MB, T/2 F_MB) of (n, ux, uy, T) per node. */
void orc2_equilibrium(const orc2_params *p, const double *n, const double *ux, const double *uy,
                      const double *T, double *F, double *G)
{
    int N = p->nx * p->ny, Q = p->Q;
#pragma omp parallel
    {
        double fl[ORC2_NFIELDS];
        double *FS = (double *)malloc(Q * Q * sizeof(double));
        double *GS = (double *)malloc(Q * Q * sizeof(double));
        double *JF = (double *)malloc(Q * Q * sizeof(double));
        double *JG = (double *)malloc(Q * Q * sizeof(double));
#pragma omp for schedule(static)
        for (int i = 0; i < N; i++) {
            memset(fl, 0, sizeof(fl));
            fl[0] = n[i]; fl[1] = ux[i]; fl[2] = uy[i]; fl[3] = T[i];
            fl[7] = 1.0; fl[12] = 1.0;   /* q = 0, Pr = 1: the Shakhov factor is 1 */
            orc2_equilibria_node(p, fl, FS, GS, JF, JG);
            for (int k = 0; k < Q * Q; k++) {
                F[k * N + i] = FS[k];
                G[k * N + i] = GS[k];
            }
        }
        free(FS); free(GS); free(JF); free(JG);
    }
}

/* ------------------------------------------------------------------ */
/* Velocity derivatives on the tensor-product set                      */
/* ------------------------------------------------------------------ */

/* 1D operator of Sec. II-III on one axis: (dh)_k = -w_k sum_{l<=Q-2} He_{l+1}(xi_k)/l! sum_j h_j He_l(xi_j) */
static void dxi_1d(const orc2_params *p, const double *h, int stride, double *dh, int ostride)
{
    int Q = p->Q;
    double *a = (double *)calloc(Q, sizeof(double));
    double *he = (double *)malloc((Q + 1) * sizeof(double));
    for (int j = 0; j < Q; j++) {
        hermite_all2(Q, p->xi[j], he);
        for (int l = 0; l < Q; l++) a[l] += h[j * stride] * he[l];
    }
    for (int k = 0; k < Q; k++) {
        hermite_all2(Q, p->xi[k], he);
        double acc = 0.0, fact = 1.0;
        for (int l = 0; l <= Q - 2; l++) {
            if (l > 0) fact *= l;
            acc += he[l + 1] / fact * a[l];
        }
        dh[k * ostride] = -p->w[k] * acc;
    }
    free(a);
    free(he);
}

/* d/dxi_x and d/dxi_y of a node's h[kx * Q + ky] */
void orc2_dxi(const orc2_params *p, const double *h, double *dhx, double *dhy)
{
    int Q = p->Q;
    for (int ky = 0; ky < Q; ky++) dxi_1d(p, h + ky, Q, dhx + ky, Q);
    for (int kx = 0; kx < Q; kx++) dxi_1d(p, h + kx * Q, 1, dhy + kx * Q, 1);
}

/* ------------------------------------------------------------------ */
/* Right-hand side and time step                                       */
/* ------------------------------------------------------------------ */

/* -xi_x dh/dx - xi_y dh/dy by WENO-5 along each axis (flux form, upwind by sign) */
static void advect_plane(const orc2_params *p, double vx, double vy, const double *h, double *out)
{
    int nx = p->nx, ny = p->ny;
    double e = p->weno_eps;
    for (int y = 0; y < ny; y++)
        for (int x = 0; x < nx; x++) {
            double r = 0.0;
            if (vx != 0.0) {
                const double *row = h + y * nx;
                double fr, fl;
                if (vx > 0.0) {
                    fr = orc_weno5(row[wrap(x - 2, nx)], row[wrap(x - 1, nx)], row[x], row[wrap(x + 1, nx)],
                                   row[wrap(x + 2, nx)], e);
                    fl = orc_weno5(row[wrap(x - 3, nx)], row[wrap(x - 2, nx)], row[wrap(x - 1, nx)], row[x],
                                   row[wrap(x + 1, nx)], e);
                } else {
                    fr = orc_weno5(row[wrap(x + 3, nx)], row[wrap(x + 2, nx)], row[wrap(x + 1, nx)], row[x],
                                   row[wrap(x - 1, nx)], e);
                    fl = orc_weno5(row[wrap(x + 2, nx)], row[wrap(x + 1, nx)], row[x], row[wrap(x - 1, nx)],
                                   row[wrap(x - 2, nx)], e);
                }
                r += -vx * (fr - fl) / p->dx;
            }
            if (vy != 0.0) {
#define HY(j) h[wrap(j, ny) * nx + x]
                double fr, fl;
                if (vy > 0.0) {
                    fr = orc_weno5(HY(y - 2), HY(y - 1), HY(y), HY(y + 1), HY(y + 2), e);
                    fl = orc_weno5(HY(y - 3), HY(y - 2), HY(y - 1), HY(y), HY(y + 1), e);
                } else {
                    fr = orc_weno5(HY(y + 3), HY(y + 2), HY(y + 1), HY(y), HY(y - 1), e);
                    fl = orc_weno5(HY(y + 2), HY(y + 1), HY(y), HY(y - 1), HY(y - 2), e);
                }
#undef HY
                r += -vy * (fr - fl) / p->dx;
            }
            out[y * nx + x] = r;
        }
}

void orc2_rhs(const orc2_params *p, const double *F, const double *G, double *RF, double *RG,
              double *fields)
{
    int N = p->nx * p->ny, Q = p->Q, K = Q * Q;
    double *mom = (double *)malloc(6 * (size_t)N * sizeof(double));
    double *fl = (double *)malloc((size_t)ORC2_NFIELDS * N * sizeof(double));
    orc2_moments(p, F, G, mom, mom + N, mom + 2 * N, mom + 3 * N, mom + 4 * N, mom + 5 * N);
    orc2_node_fields(p, mom, mom + N, mom + 2 * N, mom + 3 * N, mom + 4 * N, mom + 5 * N, fl);
#pragma omp parallel for collapse(2) schedule(static)
    for (int kx = 0; kx < Q; kx++)
        for (int ky = 0; ky < Q; ky++) {
            int k = kx * Q + ky;
            advect_plane(p, p->xi[kx], p->xi[ky], F + (size_t)k * N, RF + (size_t)k * N);
            advect_plane(p, p->xi[kx], p->xi[ky], G + (size_t)k * N, RG + (size_t)k * N);
        }
    /* node by node (nodes are independent; with OpenMP each thread has its
     * own scratch) */
#pragma omp parallel
    {
        double *FS = (double *)malloc(K * sizeof(double)), *GS = (double *)malloc(K * sizeof(double));
        double *JF = (double *)malloc(K * sizeof(double)), *JG = (double *)malloc(K * sizeof(double));
        double *h = (double *)malloc(K * sizeof(double));
        double *dx_ = (double *)malloc(K * sizeof(double)), *dy_ = (double *)malloc(K * sizeof(double));
        double node[ORC2_NFIELDS];
#pragma omp for schedule(static)
        for (int i = 0; i < N; i++) {
            for (int f = 0; f < ORC2_NFIELDS; f++) node[f] = fl[(size_t)f * N + i];
            orc2_equilibria_node(p, node, FS, GS, JF, JG);
            double Fx = node[8], Fy = node[9], nu = node[13];
            for (int k = 0; k < K; k++) h[k] = F[(size_t)k * N + i];
            orc2_dxi(p, h, dx_, dy_);
            for (int k = 0; k < K; k++)
                RF[(size_t)k * N + i] += -Fx * dx_[k] - Fy * dy_[k] - nu * (h[k] - FS[k]) + JF[k];
            for (int k = 0; k < K; k++) h[k] = G[(size_t)k * N + i];
            orc2_dxi(p, h, dx_, dy_);
            for (int k = 0; k < K; k++)
                RG[(size_t)k * N + i] += -Fx * dx_[k] - Fy * dy_[k] - nu * (h[k] - GS[k]) + JG[k];
        }
        free(FS); free(GS); free(JF); free(JG); free(h); free(dx_); free(dy_);
    }
    if (fields) memcpy(fields, fl, (size_t)ORC2_NFIELDS * N * sizeof(double));
    free(mom); free(fl);
}

/* Shu-Osher RK3, in place */
void orc2_step(const orc2_params *p, double *F, double *G, int nsteps)
{
    size_t M = (size_t)p->Q * p->Q * p->nx * p->ny;
    double *F1 = (double *)malloc(M * sizeof(double)), *G1 = (double *)malloc(M * sizeof(double));
    double *F2 = (double *)malloc(M * sizeof(double)), *G2 = (double *)malloc(M * sizeof(double));
    double *RF = (double *)malloc(M * sizeof(double)), *RG = (double *)malloc(M * sizeof(double));
    double dt = p->dt;
    for (int s = 0; s < nsteps; s++) {
        orc2_rhs(p, F, G, RF, RG, NULL);
#pragma omp parallel for schedule(static)
        for (size_t e = 0; e < M; e++) {
            F1[e] = F[e] + dt * RF[e];
            G1[e] = G[e] + dt * RG[e];
        }
        orc2_rhs(p, F1, G1, RF, RG, NULL);
#pragma omp parallel for schedule(static)
        for (size_t e = 0; e < M; e++) {
            F2[e] = 0.75 * F[e] + 0.25 * (F1[e] + dt * RF[e]);
            G2[e] = 0.75 * G[e] + 0.25 * (G1[e] + dt * RG[e]);
        }
        orc2_rhs(p, F2, G2, RF, RG, NULL);
#pragma omp parallel for schedule(static)
        for (size_t e = 0; e < M; e++) {
            F[e] = F[e] / 3.0 + 2.0 / 3.0 * (F2[e] + dt * RF[e]);
            G[e] = G[e] / 3.0 + 2.0 / 3.0 * (G2[e] + dt * RG[e]);
        }
    }
    free(F1); free(G1); free(F2); free(G2); free(RF); free(RG);
}

/* {mass, momentum x, momentum y, kinetic + internal energy} times dx^2 */
void orc2_totals(const orc2_params *p, const double *F, const double *G, double *out)
{
    int N = p->nx * p->ny, Q = p->Q;
    double m = 0.0, px = 0.0, py = 0.0, e = 0.0;
    for (int kx = 0; kx < Q; kx++)
        for (int ky = 0; ky < Q; ky++) {
            int k = kx * Q + ky;
            double vx = p->xi[kx], vy = p->xi[ky];
            for (int i = 0; i < N; i++) {
                double f = F[(size_t)k * N + i];
                m += f;
                px += vx * f;
                py += vy * f;
                e += 0.5 * (vx * vx + vy * vy) * f + G[(size_t)k * N + i];
            }
        }
    double a = p->dx * p->dx;
    out[0] = m * a;
    out[1] = px * a;
    out[2] = py * a;
    out[3] = e * a;
}
