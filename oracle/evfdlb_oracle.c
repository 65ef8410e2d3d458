/*
 * evfdlb_oracle.c -- plain, slow FP64 CPU reference ("the oracle") for one
 * time step of the Enskog-Vlasov finite-difference lattice Boltzmann model of
 * Busuioc & Sofonea, "Thermal Enskog-Vlasov Lattice Boltzmann model with
 * phase separation" (arXiv:2503.15187), in its one-dimensional EV1 form.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this file.  It shares no code,
 * header, table or constant generator with the CUDA library: the velocity set
 * and the projection rule arrive as arrays from the caller (oracle/__init__.py
 * builds them with numpy's Gauss-Hermite routine), and everything else is
 * computed here from the paper's formulas.
 *
 * Every routine follows the paper's statement in the paper's order, in plain
 * loops; nothing is blocked, fused or reordered for speed.  Built with
 * OpenMP, the independent node loops (and velocity rows) are shared among
 * threads; each node's arithmetic, and so every result bit, is the same for
 * any thread count.
 *
 * Notation (reduced units of Sec. III: m = k_B = 1):
 *   F(z, xi) = integral of f over the transverse momenta,
 *   G(z, xi) = integral of f p_perp^2 / 2 over the transverse momenta
 *   (reduced distributions of the 1D reduction, Sec. III), stored as
 *   F[k * nz + i] at velocity node xi_k and grid node z_i.
 * Readings of passages the paper leaves open are marked READING.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Scalar type of everything that depends on the state.  The file is compiled
 * twice: as plain FP64 (real = double, entry points orc_*), and with
 * ORC_COMPLEX (real = double complex, entry points orc_cs_*) for
 * complex-step differentiation (Squire & Trapp 1998): evaluating the same
 * arithmetic at x + i h v gives the tangent-linear map J v = Im f / h to
 * rounding, with no subtractive cancellation.  Nothing in the arithmetic
 * differs between the two builds. */
#ifdef ORC_COMPLEX
#include <complex.h>
typedef double _Complex real;
#define R_SQRT csqrt
#define ORC(name) orc_cs_##name
#define ORC_CONST static
#else
typedef double real;
#define R_SQRT sqrt
#define ORC(name) orc_##name
#define ORC_CONST
#endif

typedef struct {
    int nz;            /* grid nodes                                        */
    int Q;             /* velocity nodes (full-range Gauss-Hermite order)   */
    double dz;         /* grid spacing (units of sigma)                     */
    double dt;         /* time step                                         */
    double sigma;      /* hard-sphere diameter, Eq. (sutherland)            */
    double phi;        /* well depth phi_sigma, Eq. (sutherland)            */
    double gamma;      /* tail exponent, Eq. (sutherland)                   */
    double rcut;       /* truncation radius of the force integral           */
    int bc;            /* 0: periodic, 1: outflow (zero-gradient ghosts)    */
    int relax;         /* 0: rate 1/tau; 1: rate chi/tau (Sec. II.B)        */
    double weno_eps;   /* WENO-5 smoothness regulariser                     */
    const double *xi;  /* [Q] velocity nodes                                */
    const double *w;   /* [Q] weights, sum 1                                */
    int nq;            /* points of the projection rule                     */
    const double *zq;  /* [nq] nodes of a normalised Gauss-Hermite rule     */
    const double *wq;  /* [nq] its weights, sum 1                           */
    double phi_tl;     /* complex-step build only: imaginary part of phi    */
    int force_model;   /* 0: EV1, Eq. (F1); 1: EV2, Eq. (F2)                */
    double T_iso;      /* > 0: temperature reset to T_iso after every step  */
} orc_params;

/* number of per-node fields returned by orc_node_fields */
#define ORC_NFIELDS 16

static const double PI = 3.14159265358979323846;

/* ------------------------------------------------------------------ */
/* grid index with the boundary rule (periodic wrap or outflow clamp)  */
/* ------------------------------------------------------------------ */
static int gidx(const orc_params *p, int i)
{
    if (p->bc == 0) {
        int r = i % p->nz;
        return r < 0 ? r + p->nz : r;
    }
    if (i < 0) return 0;
    if (i >= p->nz) return p->nz - 1;
    return i;
}

/* probabilists' Hermite polynomials He_0..He_L at x by their three-term
 * recurrence He_{l+1} = x He_l - l He_{l-1}. */
static void hermite_all(int L, real x, real *he)
{
    he[0] = 1.0;
    if (L >= 1) he[1] = x;
    for (int l = 1; l < L; l++) he[l + 1] = x * he[l] - l * he[l - 1];
}

/* composite Simpson 1/3 weight of node j in -M..M (2M panels of width dz) */
static double simpson_w(int j, int M, double dz)
{
    int t = j + M;
    double c;
    if (t == 0 || t == 2 * M) c = 1.0;
    else if (t % 2 == 1) c = 4.0;
    else c = 2.0;
    return c * dz / 3.0;
}

/* ------------------------------------------------------------------ */
/* Sec. II: interaction kernels                                        */
/* ------------------------------------------------------------------ */

/* Kernel of the 1D self-consistent force, Eq. (F1):
 *   F1(x) = integral g(x'-x) n(x') dx',
 *   g(z) = 2 pi phi z              for |z| <  sigma,
 *        = 2 pi phi sigma^g z/|z|^g for |z| >= sigma.            */
ORC_CONST double orc_force_kernel(const orc_params *p, double z)
{
    double az = fabs(z);
    if (az < p->sigma) return 2.0 * PI * p->phi * z;
    return 2.0 * PI * p->phi * pow(p->sigma, p->gamma) * z / pow(az, p->gamma);
}

/* Even potential Phi_F with Phi_F' = g and Phi_F -> 0 at infinity; the
 * mean-field energy of the F1 dynamics is (1/2) sum n Phi_F n.
 * READING: energy bookkeeping is not printed in the paper; Phi_F is the
 * unique even antiderivative of the Eq. (F1) kernel that vanishes at infinity. */
ORC_CONST double orc_force_potential(const orc_params *p, double z)
{
    double az = fabs(z), s = p->sigma, g = p->gamma;
    if (az < s) return PI * p->phi * (z * z - s * s * g / (g - 2.0));
    return -2.0 * PI * p->phi * pow(s, g) * pow(az, 2.0 - g) / (g - 2.0);
}

/* Sutherland tail integrated over a plane at distance z, restricted to
 * rho > sigma (Eq. (sutherland)):
 *   -2 pi phi sigma^2/(g-2)                for |z| < sigma,
 *   -2 pi phi sigma^g |z|^(2-g)/(g-2)       beyond.               */
ORC_CONST double orc_plane_potential(const orc_params *p, double z)
{
    double az = fabs(z), s = p->sigma, g = p->gamma;
    if (az < s) return -2.0 * PI * p->phi * s * s / (g - 2.0);
    return -2.0 * PI * p->phi * pow(s, g) * pow(az, 2.0 - g) / (g - 2.0);
}

/* Carnahan-Starling contact value, Eq. (carnstar): chi = (2-eta)/(2(1-eta)^3),
 * eta = pi sigma^3 n / 6. */
real ORC(chi)(const orc_params *p, real n)
{
    real eta = PI * p->sigma * p->sigma * p->sigma * n / 6.0;
    real om = 1.0 - eta;
    return (2.0 - eta) / (2.0 * om * om * om);
}

/* ------------------------------------------------------------------ */
/* Sec. II.B: macroscopic moments                                      */
/* ------------------------------------------------------------------ */

/* n = int F; n u = int xi F; (3/2) n T = int [(xi-u)^2/2 F + G];
 * q = int (xi-u)[(xi-u)^2/2 F + G]  (moment definitions of Sec. II.B and the
 * heat flux under the Shakhov term, written for the reduced distributions). */
void ORC(moments)(const orc_params *p, const real *F, const real *G,
                  real *n, real *u, real *T, real *q)
{
    int nz = p->nz, Q = p->Q;
#pragma omp parallel for schedule(static)
    for (int i = 0; i < nz; i++) {
        real sn = 0.0, sj = 0.0;
        for (int k = 0; k < Q; k++) {
            sn += F[k * nz + i];
            sj += p->xi[k] * F[k * nz + i];
        }
        real ui = sj / sn;
        real se = 0.0, sq = 0.0;
        for (int k = 0; k < Q; k++) {
            real c = p->xi[k] - ui;
            real e = 0.5 * c * c * F[k * nz + i] + G[k * nz + i];
            se += e;
            sq += c * e;
        }
        n[i] = sn;
        u[i] = ui;
        T[i] = 2.0 * se / (3.0 * sn);
        q[i] = sq;
    }
}

/* ------------------------------------------------------------------ */
/* Node-level fields                                                   */
/* ------------------------------------------------------------------ */

/* Fischer-Methfessel average over a sphere of radius sigma (Sec. II.A),
 * reduced to 1D: nbar(z) = 3/(4 sigma^3) int_{|s|<sigma} (sigma^2 - s^2) n(z+s) ds,
 * the factor pi(sigma^2 - s^2) being the area of the slice of the sphere at
 * offset s; composite Simpson 1/3 over 2m panels, m = sigma/dz. */
static void fm_average(const orc_params *p, const real *n, real *nbar)
{
    int m = (int)lround(p->sigma / p->dz);
    double s3 = p->sigma * p->sigma * p->sigma;
    for (int i = 0; i < p->nz; i++) {
        real acc = 0.0;
        for (int j = -m; j <= m; j++) {
            double z = j * p->dz;
            acc += simpson_w(j, m, p->dz) * (p->sigma * p->sigma - z * z) * n[gidx(p, i + j)];
        }
        nbar[i] = 3.0 / (4.0 * s3) * acc;
    }
}

/* EV1 force, Eq. (F1), by the composite Simpson 1/3 rule on the grid,
 * truncated at |x'-x| <= rcut (M = rcut/dz panels each side). */
static void ev1_force(const orc_params *p, const real *n, real *force)
{
    int M = (int)lround(p->rcut / p->dz);
    for (int i = 0; i < p->nz; i++) {
        real acc = 0.0;
        for (int j = -M; j <= M; j++)
            acc += simpson_w(j, M, p->dz) * orc_force_kernel(p, j * p->dz) * n[gidx(p, i + j)];
#ifdef ORC_COMPLEX
        /* the kernel is linear in phi: a complex phi scales the integral */
        acc = acc * (1.0 + I * (p->phi_tl / p->phi));
#endif
        force[i] = acc;
    }
}

static void grad4(const orc_params *p, const real *f, real *df);
static void d3_5pt(const orc_params *p, const real *f, real *d3);

/* EV2 force, Eq. (F2): F2 = 2a dn/dz + kappa d^3n/dz^3 with
 * a = (2 pi sigma^3/3) phi gamma/(gamma-3), kappa = (2 pi sigma^5/15) phi gamma/(gamma-5);
 * dn/dz by the fourth-order central difference and d^3n/dz^3 by the five-point
 * stencil (Sec. III). */
static void ev2_force(const orc_params *p, const real *n, real *force)
{
    double s = p->sigma, g = p->gamma;
    double a = 2.0 * PI * s * s * s / 3.0 * p->phi * g / (g - 3.0);
    double kappa = 2.0 * PI * pow(s, 5.0) / 15.0 * p->phi * g / (g - 5.0);
    real *dn = (real *)malloc(p->nz * sizeof(real));
    real *d3 = (real *)malloc(p->nz * sizeof(real));
    grad4(p, n, dn);
    d3_5pt(p, n, d3);
    for (int i = 0; i < p->nz; i++) {
        real f = 2.0 * a * dn[i] + kappa * d3[i];
#ifdef ORC_COMPLEX
        f = f * (1.0 + I * (p->phi_tl / p->phi));
#endif
        force[i] = f;
    }
    free(dn);
    free(d3);
}

/* five-point third derivative: (f_{i+2} - 2 f_{i+1} + 2 f_{i-1} - f_{i-2}) / (2 dz^3) */
static void d3_5pt(const orc_params *p, const real *f, real *d3)
{
    double h3 = p->dz * p->dz * p->dz;
    for (int i = 0; i < p->nz; i++)
        d3[i] = (f[gidx(p, i + 2)] - 2.0 * f[gidx(p, i + 1)] + 2.0 * f[gidx(p, i - 1)] - f[gidx(p, i - 2)]) / (2.0 * h3);
}

/* fourth-order central difference (Sec. III):
 * f'_i = (f_{i-2} - 8 f_{i-1} + 8 f_{i+1} - f_{i+2}) / (12 dz) */
static void grad4(const orc_params *p, const real *f, real *df)
{
    for (int i = 0; i < p->nz; i++) {
        df[i] = (f[gidx(p, i - 2)] - 8.0 * f[gidx(p, i - 1)]
                 + 8.0 * f[gidx(p, i + 1)] - f[gidx(p, i + 2)]) / (12.0 * p->dz);
    }
}

/* Per-node fields of one right-hand-side evaluation, as [ORC_NFIELDS][nz]:
 *  0 n   1 u   2 T   3 q   4 nbar   5 chi   6 force F1
 *  7 mu  8 tau 9 Pr 10 rate nu
 * 11 A = d ln(n^2 chi T)/dz   12 B = d ln T/dz   13 D = du/dz
 * 14 X = n^2 chi T            15 b n chi
 * READING (gradients): A = D4(X)/X and B = D4(T)/T, the logarithmic
 * derivatives of Eq. (J1) taken as derivative over value. */
void ORC(node_fields)(const orc_params *p, const real *n, const real *u,
                      const real *T, const real *q, real *out)
{
    int nz = p->nz;
    real *nbar = out + 4 * nz, *chi = out + 5 * nz, *force = out + 6 * nz;
    real *mu = out + 7 * nz, *tau = out + 8 * nz, *Pr = out + 9 * nz;
    real *rate = out + 10 * nz, *A = out + 11 * nz, *B = out + 12 * nz;
    real *D = out + 13 * nz, *X = out + 14 * nz, *bnchi = out + 15 * nz;
    double b = 2.0 * PI * p->sigma * p->sigma * p->sigma / 3.0;   /* Eq. (carnstar) */

    memcpy(out + 0 * nz, n, nz * sizeof(real));
    memcpy(out + 1 * nz, u, nz * sizeof(real));
    memcpy(out + 2 * nz, T, nz * sizeof(real));
    memcpy(out + 3 * nz, q, nz * sizeof(real));

    /* chi at the Fischer-Methfessel averaged density (Sec. II.A) */
    fm_average(p, n, nbar);
    for (int i = 0; i < nz; i++) chi[i] = ORC(chi)(p, nbar[i]);

    /* self-consistent force, Eq. (F1) or Eq. (F2) */
    if (p->force_model == 1) ev2_force(p, n, force);
    else ev1_force(p, n, force);

    /* gradients entering J1, Eq. (J1) */
    for (int i = 0; i < nz; i++) X[i] = n[i] * n[i] * chi[i] * T[i];
    real *dX = (real *)malloc(nz * sizeof(real));
    real *dT = (real *)malloc(nz * sizeof(real));
    grad4(p, X, dX);
    grad4(p, T, dT);
    grad4(p, u, D);
    for (int i = 0; i < nz; i++) {
        A[i] = dX[i] / X[i];
        B[i] = dT[i] / T[i];
    }
    free(dX);
    free(dT);

    /* transport coefficients, Eqs. (viscosity), (tau), (prandtl) */
    for (int i = 0; i < nz; i++) {
        real bn = b * n[i];
        real x = bn * chi[i];
        real mu0 = 5.0 / (16.0 * p->sigma * p->sigma) * R_SQRT(T[i] / PI);
        mu[i] = mu0 * (1.0 / chi[i] + 0.8 * bn + 4.0 / 25.0 * (1.0 + 12.0 / PI) * bn * bn * chi[i]);
        real Pi = n[i] * T[i];
        tau[i] = mu[i] / (Pi * (1.0 + 0.4 * x));
        Pr[i] = 2.0 / 3.0 * (1.0 + 0.6 * x) / (1.0 + 0.4 * x)
              * (1.0 + 0.8 * x + 4.0 / 25.0 * (1.0 + 12.0 / PI) * x * x)
              / (1.0 + 1.2 * x + 9.0 / 25.0 * (1.0 + 32.0 / (9.0 * PI)) * x * x);
        rate[i] = (p->relax == 0) ? 1.0 / tau[i] : chi[i] / tau[i];
        bnchi[i] = x;
    }
}

/* ------------------------------------------------------------------ */
/* Sec. II.B: Shakhov equilibrium and J1, reduced and Hermite-projected */
/* ------------------------------------------------------------------ */

/* Projection of a velocity function h(xi) on the discrete set, to order Q-1:
 * h_k = w_k sum_{l<Q} a_l He_l(xi_k)/l!,  a_l = int h He_l dxi.
 * For h = F_MB * poly(c), c = xi - u, a_l = n E[poly(c) He_l(u + c)],
 * c ~ N(0, T), computed with the nq-point normalised Gauss-Hermite rule at
 * c = sqrt(T) z (exact for the polynomial degrees involved). */
static void project(const orc_params *p, const real *coef_l, real *h)
{
    int Q = p->Q;
    real *he = (real *)malloc((Q + 1) * sizeof(real));
    for (int k = 0; k < Q; k++) {
        hermite_all(Q, p->xi[k], he);
        real acc = 0.0;
        double fact = 1.0;
        for (int l = 0; l < Q; l++) {
            if (l > 0) fact *= l;
            acc += coef_l[l] * he[l] / fact;
        }
        h[k] = p->w[k] * acc;
    }
    free(he);
}

/* For one node: the projected reduced Shakhov equilibria F^S, G^S and the
 * projected reduced J1 terms J1_F, J1_G (each [Q]).
 *
 * Reduction over the transverse momenta (Sec. III cites reduced distributions
 * without printing them; READING: integrate f^S and J1 of Sec. II.B over
 * p_y, p_z with weights 1 and p_perp^2/2, using <c_perp^2> = 2T and
 * <c_perp^4> = 8T^2):
 *   s    = (1 - Pr) q / (n T^2)
 *   F^S  = F_MB [1 + s c (c^2/(5T) - 3/5)]
 *   G^S  = T F_MB [1 + s c (c^2/(5T) - 1/5)]
 *   J1_F = -b n chi F_MB { c [A + 3/5 (c^2/(2T) - 3/2) B] + 2/5 (3c^2/(2T) - 3/2) D }
 *   J1_G = -b n chi F_MB { c [T A + 3/5 (c^2/2 - T/2) B] + 2/5 (3c^2/2 - T/2) D }
 * with F_MB = n (2 pi T)^(-1/2) exp(-c^2/(2T)). */
void ORC(equilibria_node)(const orc_params *p, real n, real u, real T,
                          real q, real Pr, real bnchi, real A, real B,
                          real D, real *FS, real *GS, real *JF, real *JG)
{
    int Q = p->Q;
    real *aS = (real *)calloc(Q, sizeof(real));
    real *bS = (real *)calloc(Q, sizeof(real));
    real *aJ = (real *)calloc(Q, sizeof(real));
    real *bJ = (real *)calloc(Q, sizeof(real));
    real *he = (real *)malloc((Q + 1) * sizeof(real));
    real s = (1.0 - Pr) * q / (n * T * T);
    real sqT = R_SQRT(T);
    for (int m = 0; m < p->nq; m++) {
        real c = sqT * p->zq[m];
        real W = p->wq[m] * n;
        hermite_all(Q, u + c, he);
        real pS = 1.0 + s * c * (c * c / (5.0 * T) - 0.6);
        real pG = T * (1.0 + s * c * (c * c / (5.0 * T) - 0.2));
        real pJF = -bnchi * (c * (A + 0.6 * (c * c / (2.0 * T) - 1.5) * B)
                             + 0.4 * (3.0 * c * c / (2.0 * T) - 1.5) * D);
        real pJG = -bnchi * (c * (T * A + 0.6 * (c * c / 2.0 - T / 2.0) * B)
                             + 0.4 * (3.0 * c * c / 2.0 - T / 2.0) * D);
        for (int l = 0; l < Q; l++) {
            aS[l] += W * pS * he[l];
            bS[l] += W * pG * he[l];
            aJ[l] += W * pJF * he[l];
            bJ[l] += W * pJG * he[l];
        }
    }
    project(p, aS, FS);
    project(p, bS, GS);
    project(p, aJ, JF);
    project(p, bJ, JG);
    free(aS); free(bS); free(aJ); free(bJ); free(he);
}

/* Projected Maxwellian pair (F_MB, T F_MB) for initial data. */
void ORC(equilibrium)(const orc_params *p, const real *n, const real *u,
                      const real *T, real *F, real *G)
{
    int nz = p->nz, Q = p->Q;
#pragma omp parallel
    {
        real *FS = (real *)malloc(Q * sizeof(real));
        real *GS = (real *)malloc(Q * sizeof(real));
        real *JF = (real *)malloc(Q * sizeof(real));
        real *JG = (real *)malloc(Q * sizeof(real));
#pragma omp for schedule(static)
        for (int i = 0; i < nz; i++) {
            ORC(equilibria_node)(p, n[i], u[i], T[i], 0.0, 1.0, 0.0, 0.0, 0.0, 0.0, FS, GS, JF, JG);
            for (int k = 0; k < Q; k++) {
                F[k * nz + i] = FS[k];
                G[k * nz + i] = GS[k];
            }
        }
        free(FS); free(GS); free(JF); free(JG);
    }
}

/* ------------------------------------------------------------------ */
/* Velocity derivative on the Gauss-Hermite set                        */
/* ------------------------------------------------------------------ */

/* (d/dxi h)_k for a projected h: since d/dxi [omega He_l] = -omega He_{l+1},
 * (dh)_k = -w_k sum_{l=0}^{Q-2} He_{l+1}(xi_k)/l! sum_j h_j He_l(xi_j);
 * the l = Q-1 term vanishes at the nodes because He_Q(xi_k) = 0. */
void ORC(dxi)(const orc_params *p, const real *h, real *dh)
{
    int Q = p->Q;
    real *a = (real *)calloc(Q, sizeof(real));
    real *he = (real *)malloc((Q + 1) * sizeof(real));
    for (int j = 0; j < Q; j++) {
        hermite_all(Q, p->xi[j], he);
        for (int l = 0; l < Q; l++) a[l] += h[j] * he[l];
    }
    for (int k = 0; k < Q; k++) {
        hermite_all(Q, p->xi[k], he);
        real acc = 0.0;
        double fact = 1.0;
        for (int l = 0; l <= Q - 2; l++) {
            if (l > 0) fact *= l;
            acc += he[l + 1] / fact * a[l];
        }
        dh[k] = -p->w[k] * acc;
    }
    free(a);
    free(he);
}

/* ------------------------------------------------------------------ */
/* WENO-5 (Jiang-Shu) upwind reconstruction                            */
/* ------------------------------------------------------------------ */

/* Value at the face between the third and fourth of five upwind-ordered
 * points v0..v4 (v2 is the upwind cell of the face). */
real ORC(weno5)(real v0, real v1, real v2, real v3, real v4, double eps)
{
    real q0 = (2.0 * v0 - 7.0 * v1 + 11.0 * v2) / 6.0;
    real q1 = (-v1 + 5.0 * v2 + 2.0 * v3) / 6.0;
    real q2 = (2.0 * v2 + 5.0 * v3 - v4) / 6.0;
    real b0 = 13.0 / 12.0 * (v0 - 2.0 * v1 + v2) * (v0 - 2.0 * v1 + v2)
              + 0.25 * (v0 - 4.0 * v1 + 3.0 * v2) * (v0 - 4.0 * v1 + 3.0 * v2);
    real b1 = 13.0 / 12.0 * (v1 - 2.0 * v2 + v3) * (v1 - 2.0 * v2 + v3)
              + 0.25 * (v1 - v3) * (v1 - v3);
    real b2 = 13.0 / 12.0 * (v2 - 2.0 * v3 + v4) * (v2 - 2.0 * v3 + v4)
              + 0.25 * (3.0 * v2 - 4.0 * v3 + v4) * (3.0 * v2 - 4.0 * v3 + v4);
    real a0 = 0.1 / ((eps + b0) * (eps + b0));
    real a1 = 0.6 / ((eps + b1) * (eps + b1));
    real a2 = 0.3 / ((eps + b2) * (eps + b2));
    real sa = a0 + a1 + a2;
    return (a0 * q0 + a1 * q1 + a2 * q2) / sa;
}

/* -xi (h_{i+1/2} - h_{i-1/2}) / dz for one velocity row h[0..nz) with the
 * boundary rule; upwind side by the sign of xi (flux xi h is linear in h).
 * READING: the reconstruction acts on the stored F_k, G_k (weights included). */
static void advect_row(const orc_params *p, double xi, const real *h, real *out)
{
    int nz = p->nz;
    double e = p->weno_eps;
    for (int i = 0; i < nz; i++) {
        if (xi == 0.0) { out[i] = 0.0; continue; }
        real fr, fl;   /* faces i+1/2 and i-1/2 */
        if (xi > 0.0) {
            fr = ORC(weno5)(h[gidx(p, i - 2)], h[gidx(p, i - 1)], h[gidx(p, i)],
                            h[gidx(p, i + 1)], h[gidx(p, i + 2)], e);
            fl = ORC(weno5)(h[gidx(p, i - 3)], h[gidx(p, i - 2)], h[gidx(p, i - 1)],
                            h[gidx(p, i)], h[gidx(p, i + 1)], e);
        } else {
            fr = ORC(weno5)(h[gidx(p, i + 3)], h[gidx(p, i + 2)], h[gidx(p, i + 1)],
                            h[gidx(p, i)], h[gidx(p, i - 1)], e);
            fl = ORC(weno5)(h[gidx(p, i + 2)], h[gidx(p, i + 1)], h[gidx(p, i)],
                            h[gidx(p, i - 1)], h[gidx(p, i - 2)], e);
        }
        out[i] = -xi * (fr - fl) / p->dz;
    }
}

/* exported form of the free-streaming term of one velocity row */
void ORC(advect_row)(const orc_params *p, double xi, const real *h, real *out)
{
    advect_row(p, xi, h, out);
}

/* ------------------------------------------------------------------ */
/* Right-hand side of Eq. (ev1) for the reduced pair (F, G)            */
/* ------------------------------------------------------------------ */

/* dF/dt = -xi dF/dz - F1 dF/dxi - nu (F - F^S) + J1_F, and the same for G,
 * Eqs. (enskog_approx) and (ev1).  Writes RF, RG ([Q][nz]); fields (optional,
 * may be NULL) receives the node fields of orc_node_fields. */
void ORC(rhs)(const orc_params *p, const real *F, const real *G,
              real *RF, real *RG, real *fields)
{
    int nz = p->nz, Q = p->Q;
    real *n = (real *)malloc(nz * sizeof(real));
    real *u = (real *)malloc(nz * sizeof(real));
    real *T = (real *)malloc(nz * sizeof(real));
    real *q = (real *)malloc(nz * sizeof(real));
    real *fl = (real *)malloc((size_t)ORC_NFIELDS * nz * sizeof(real));

    /* moments, then node fields */
    ORC(moments)(p, F, G, n, u, T, q);
    ORC(node_fields)(p, n, u, T, q, fl);
    const real *force = fl + 6 * nz, *Pr = fl + 9 * nz, *rate = fl + 10 * nz;
    const real *A = fl + 11 * nz, *B = fl + 12 * nz, *D = fl + 13 * nz;
    const real *bnchi = fl + 15 * nz;

    /* free streaming term (velocity rows are independent) */
#pragma omp parallel for schedule(static)
    for (int k = 0; k < Q; k++) {
        advect_row(p, p->xi[k], F + (size_t)k * nz, RF + (size_t)k * nz);
        advect_row(p, p->xi[k], G + (size_t)k * nz, RG + (size_t)k * nz);
    }
    /* force, collision and J1 terms, node by node (nodes are independent;
     * with OpenMP each thread has its own scratch) */
#pragma omp parallel
    {
        real *hk = (real *)malloc(Q * sizeof(real));
        real *dh = (real *)malloc(Q * sizeof(real));
        real *FS = (real *)malloc(Q * sizeof(real));
        real *GS = (real *)malloc(Q * sizeof(real));
        real *JF = (real *)malloc(Q * sizeof(real));
        real *JG = (real *)malloc(Q * sizeof(real));
#pragma omp for schedule(static)
        for (int i = 0; i < nz; i++) {
            ORC(equilibria_node)(p, n[i], u[i], T[i], q[i], Pr[i], bnchi[i],
                                 A[i], B[i], D[i], FS, GS, JF, JG);
            for (int k = 0; k < Q; k++) hk[k] = F[k * nz + i];
            ORC(dxi)(p, hk, dh);
            for (int k = 0; k < Q; k++)
                RF[k * nz + i] += -force[i] * dh[k] - rate[i] * (hk[k] - FS[k]) + JF[k];
            for (int k = 0; k < Q; k++) hk[k] = G[k * nz + i];
            ORC(dxi)(p, hk, dh);
            for (int k = 0; k < Q; k++)
                RG[k * nz + i] += -force[i] * dh[k] - rate[i] * (hk[k] - GS[k]) + JG[k];
        }
        free(hk); free(dh); free(FS); free(GS); free(JF); free(JG);
    }
    if (fields) memcpy(fields, fl, (size_t)ORC_NFIELDS * nz * sizeof(real));
    free(n); free(u); free(T); free(q); free(fl);
}

/* ------------------------------------------------------------------ */
/* Isothermal mode (Sec. III.A)                                        */
/* ------------------------------------------------------------------ */

/* READING: Sec. III.A keeps the fluid temperature constant without saying
 * how.  Here, after every time step, each node's temperature is set back to
 * T_iso while its density, velocity and non-equilibrium part are kept:
 *   F <- F + F_MB(n, u, T_iso) - F_MB(n, u, T),
 *   G <- G + T_iso F_MB(n, u, T_iso) - T F_MB(n, u, T),
 * with n, u, T the moments of the state and F_MB the Hermite-projected
 * Maxwellian (the pair the initial state uses). */
static void isothermal_reset(const orc_params *p, real *F, real *G)
{
    int nz = p->nz, Q = p->Q;
    size_t N = (size_t)Q * nz;
    real *n = (real *)malloc(nz * sizeof(real));
    real *u = (real *)malloc(nz * sizeof(real));
    real *T = (real *)malloc(nz * sizeof(real));
    real *q = (real *)malloc(nz * sizeof(real));
    real *Ti = (real *)malloc(nz * sizeof(real));
    real *Fa = (real *)malloc(N * sizeof(real)), *Ga = (real *)malloc(N * sizeof(real));
    real *Fb = (real *)malloc(N * sizeof(real)), *Gb = (real *)malloc(N * sizeof(real));
    ORC(moments)(p, F, G, n, u, T, q);
    for (int i = 0; i < nz; i++) Ti[i] = p->T_iso;
    ORC(equilibrium)(p, n, u, Ti, Fa, Ga);
    ORC(equilibrium)(p, n, u, T, Fb, Gb);
    for (size_t e = 0; e < N; e++) {
        F[e] += Fa[e] - Fb[e];
        G[e] += Ga[e] - Gb[e];
    }
    free(n); free(u); free(T); free(q); free(Ti); free(Fa); free(Ga); free(Fb); free(Gb);
}

/* ------------------------------------------------------------------ */
/* Third-order TVD Runge-Kutta of Shu and Osher (Sec. III)             */
/* ------------------------------------------------------------------ */

/* u1 = u + dt L(u); u2 = 3/4 u + 1/4 (u1 + dt L(u1));
 * u_new = 1/3 u + 2/3 (u2 + dt L(u2)).  Advances (F, G) in place. */
void ORC(step)(const orc_params *p, real *F, real *G, int nsteps)
{
    size_t N = (size_t)p->Q * p->nz;
    real *F1 = (real *)malloc(N * sizeof(real));
    real *G1 = (real *)malloc(N * sizeof(real));
    real *F2 = (real *)malloc(N * sizeof(real));
    real *G2 = (real *)malloc(N * sizeof(real));
    real *RF = (real *)malloc(N * sizeof(real));
    real *RG = (real *)malloc(N * sizeof(real));
    double dt = p->dt;
    for (int s = 0; s < nsteps; s++) {
        ORC(rhs)(p, F, G, RF, RG, NULL);
#pragma omp parallel for schedule(static)
        for (size_t e = 0; e < N; e++) {
            F1[e] = F[e] + dt * RF[e];
            G1[e] = G[e] + dt * RG[e];
        }
        ORC(rhs)(p, F1, G1, RF, RG, NULL);
#pragma omp parallel for schedule(static)
        for (size_t e = 0; e < N; e++) {
            F2[e] = 0.75 * F[e] + 0.25 * (F1[e] + dt * RF[e]);
            G2[e] = 0.75 * G[e] + 0.25 * (G1[e] + dt * RG[e]);
        }
        ORC(rhs)(p, F2, G2, RF, RG, NULL);
#pragma omp parallel for schedule(static)
        for (size_t e = 0; e < N; e++) {
            F[e] = F[e] / 3.0 + 2.0 / 3.0 * (F2[e] + dt * RF[e]);
            G[e] = G[e] / 3.0 + 2.0 / 3.0 * (G2[e] + dt * RG[e]);
        }
        if (p->T_iso > 0.0) isothermal_reset(p, F, G);
    }
    free(F1); free(G1); free(F2); free(G2); free(RF); free(RG);
}

#ifndef ORC_COMPLEX
/* ------------------------------------------------------------------ */
/* Threads                                                             */
/* ------------------------------------------------------------------ */

/* Node loops (and the velocity rows of the free-streaming term) run in
 * parallel when the oracle is built with OpenMP; every node's arithmetic is
 * the same in any thread, so results do not depend on the thread count.
 * Sets the thread count (n > 0) and returns the count in effect (1 without
 * OpenMP). */
int orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

/* ------------------------------------------------------------------ */
/* Conserved totals                                                    */
/* ------------------------------------------------------------------ */

/* out = {mass, momentum, energy, E_mf}:
 *   mass = dz sum n, momentum = dz sum n u,
 *   energy = dz sum_i sum_k (xi_k^2/2 F_k + G_k) + E_mf,
 *   E_mf = (dz/2) sum_i n_i sum_j s_j [Phi_F(j dz) - Phi_F(rcut)] n_{i+j}
 * (Simpson taps and cut as in the force).  READING: the paper prints no
 * energy bookkeeping; this is the energy the truncated EV1 dynamics exchanges
 * with the kinetic part through the force term.  The shift by Phi_F(rcut)
 * makes the potential vanish at the cut, so that minus its convolution's
 * derivative is exactly the truncated Eq. (F1) integral. */
void orc_totals(const orc_params *p, const double *F, const double *G, double *out)
{
    int nz = p->nz, Q = p->Q;
    int M = (int)lround(p->rcut / p->dz);
    double *n = (double *)calloc(nz, sizeof(double));
    double mass = 0.0, mom = 0.0, kin = 0.0, emf = 0.0;
    double phiR = orc_force_potential(p, p->rcut);
    for (int i = 0; i < nz; i++) {
        for (int k = 0; k < Q; k++) {
            double f = F[k * nz + i];
            n[i] += f;
            mom += p->xi[k] * f;
            kin += 0.5 * p->xi[k] * p->xi[k] * f + G[k * nz + i];
        }
        mass += n[i];
    }
    if (p->force_model == 1) {
        /* EV2: the field psi = -2a n - kappa d2n/dz2 has -dpsi/dz = F2 of Eq. (F2);
         * E_mf = sum dz (1/2) n psi with the fourth-order second difference */
        double s = p->sigma, g = p->gamma;
        double a = 2.0 * PI * s * s * s / 3.0 * p->phi * g / (g - 3.0);
        double kappa = 2.0 * PI * pow(s, 5.0) / 15.0 * p->phi * g / (g - 5.0);
        for (int i = 0; i < nz; i++) {
            double d2 = (-n[gidx(p, i - 2)] + 16.0 * n[gidx(p, i - 1)] - 30.0 * n[i] + 16.0 * n[gidx(p, i + 1)]
                         - n[gidx(p, i + 2)]) / (12.0 * p->dz * p->dz);
            emf += 0.5 * n[i] * (-2.0 * a * n[i] - kappa * d2);
        }
    } else {
        for (int i = 0; i < nz; i++) {
            double acc = 0.0;
            for (int j = -M; j <= M; j++)
                acc += simpson_w(j, M, p->dz) * (orc_force_potential(p, j * p->dz) - phiR) * n[gidx(p, i + j)];
            emf += 0.5 * n[i] * acc;
        }
    }
    out[0] = mass * p->dz;
    out[1] = mom * p->dz;
    out[3] = emf * p->dz;
    out[2] = kin * p->dz + out[3];
    free(n);
}

/* Discrete force constant a_d = (1/2) sum_j s_j (j dz) g(j dz): for a linear
 * density the Simpson force of Eq. (F1) is exactly 2 a_d dn/dz. */
double orc_discrete_a(const orc_params *p)
{
    if (p->force_model == 1)   /* EV2: the printed a of Eq. (F2) */
        return 2.0 * PI * p->sigma * p->sigma * p->sigma / 3.0 * p->phi * p->gamma / (p->gamma - 3.0);
    int M = (int)lround(p->rcut / p->dz);
    double acc = 0.0;
    for (int j = -M; j <= M; j++)
        acc += simpson_w(j, M, p->dz) * (j * p->dz) * orc_force_kernel(p, j * p->dz);
    return 0.5 * acc;
}
#endif /* ORC_COMPLEX */
