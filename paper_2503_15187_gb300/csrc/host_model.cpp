// host_model.cpp -- host-side model constants of libevfdlb: the Gauss-Hermite
// velocity set and its Hermite tables, the Simpson taps of the force and of
// the Fischer-Methfessel average, parameter validation, and the equation of
// state with its critical point and Maxwell construction.
//
// Paper: Busuioc & Sofonea, arXiv:2503.15187.  Equations cited by label.
#include <math.h>

#include <algorithm>
#include <vector>

#include "evfdlb_internal.h"

namespace evfdlb {

namespace {
const long double kPiL = 3.141592653589793238462643383279502884L;
const double kPi = 3.14159265358979323846;

// Orthonormal probabilists' Hermite functions psi_l = He_l / sqrt(l!) at x,
// l = 0..L, by psi_{l+1} = (x psi_l - sqrt(l) psi_{l-1}) / sqrt(l+1).
template <typename R>
void psi_all(int L, R x, R* psi) {
    psi[0] = 1;
    if (L >= 1) psi[1] = x;
    for (int l = 1; l < L; ++l)
        psi[l + 1] = (x * psi[l] - sqrtl((long double)l) * psi[l - 1]) / sqrtl((long double)(l + 1));
}

// Number of eigenvalues below x of the Jacobi matrix of the probabilists'
// Hermite recurrence (zero diagonal, off-diagonal sqrt(k)), by the Sturm
// count of the LDL^T pivots.
int sturm_count(int Q, long double x) {
    int count = 0;
    long double d = -x;
    if (d < 0) ++count;
    for (int k = 1; k < Q; ++k) {
        long double piv = (d == 0) ? 1e-300L : d;
        d = -x - (long double)k / piv;
        if (d < 0) ++count;
    }
    return count;
}
}  // namespace

// Roots of He_Q (the velocity nodes of the full-range Gauss-Hermite rule) by
// bisection on the Sturm count, polished by Newton on psi_Q with
// psi_Q' = sqrt(Q) psi_{Q-1}; weights w = 1 / (Q psi_{Q-1}(x)^2), which sum to 1.
// Fixed-size storage (no heap), so that the allocation-free step can call it.
bool velocity_set(int Q, double* xi, double* w) {
    if (Q < 1 || Q > kVelocitySetMax) return false;
    long double psi[kVelocitySetMax + 1];
    long double bound = sqrtl(4.0L * Q + 2.0L) + 1.0L;
    for (int k = 0; k < Q; ++k) {
        long double lo = -bound, hi = bound;   // k-th smallest: count(x) >= k+1
        for (int it = 0; it < 200 && hi - lo > 1e-18L * (1 + fabsl(lo)); ++it) {
            long double mid = 0.5L * (lo + hi);
            if (sturm_count(Q, mid) >= k + 1) hi = mid; else lo = mid;
        }
        long double x = 0.5L * (lo + hi);
        for (int it = 0; it < 3; ++it) {
            psi_all<long double>(Q, x, psi);
            long double dpsi = sqrtl((long double)Q) * psi[Q - 1];
            if (dpsi == 0) break;
            x -= psi[Q] / dpsi;
        }
        psi_all<long double>(Q, x, psi);
        xi[k] = (double)x;
        w[k] = (double)(1.0L / ((long double)Q * psi[Q - 1] * psi[Q - 1]));
    }
    // He_Q has the parity of Q: its roots are symmetric about 0.  Make the
    // stored set exactly so (xi_{Q-1-k} = -xi_k, w_{Q-1-k} = w_k, a zero node
    // for odd Q), which the parity-split transforms rely on.
    for (int k = 0; k < Q / 2; ++k) {
        const long double a = 0.5L * ((long double)xi[Q - 1 - k] - (long double)xi[k]);
        const long double b = 0.5L * ((long double)w[Q - 1 - k] + (long double)w[k]);
        xi[k] = (double)(-a);
        xi[Q - 1 - k] = (double)a;
        w[k] = w[Q - 1 - k] = (double)b;
    }
    if (Q & 1) xi[Q / 2] = 0.0;
    return true;
}

// Fixed-size storage (no heap), like velocity_set.
void build_tables(int Q, const double* xi, const double* w, double* out) {
    TableLayout L(Q);
    long double psi[kVelocitySetMax + 1];
    for (int k = 0; k < Q; ++k) {
        out[L.xi + k] = xi[k];
        out[L.w + k] = w[k];
        psi_all<long double>(Q, (long double)xi[k], psi);
        for (int l = 0; l < Q; ++l) {
            out[L.P + l * Q + k] = (double)psi[l];
            out[L.S + k * Q + l] = (double)((long double)w[k] * psi[l]);
        }
    }
    // parity-split tables (the nodes are symmetric: see velocity_set)
    const ParitySplit ps(Q);
    for (int g = 0; g < ps.GE + ps.GO; ++g) {
        const int l = (g < ps.GE) ? 4 * g : 4 * (g - ps.GE) + 1;
        for (int j = 0; j < ps.H; ++j) {
            out[L.Pp + 2 * (g * ps.H + j)] = (l <= Q - 2) ? out[L.P + l * Q + j] : 0.0;
            out[L.Pp + 2 * (g * ps.H + j) + 1] = (l + 2 <= Q - 2) ? out[L.P + (l + 2) * Q + j] : 0.0;
        }
    }
    for (int k = 0; k < ps.H; ++k)
        for (int l = 0; l < ps.QE; ++l) out[L.Sp + k * ps.QE + l] = (l < Q) ? out[L.S + k * Q + l] : 0.0;
    for (int l = 0; l < Q; ++l) {
        long double ll = l;
        out[L.rinv + l] = (double)(1.0L / sqrtl(ll + 1));
        out[L.rr + l] = (double)(sqrtl(ll) / sqrtl(ll + 1));
        out[L.r1 + l] = (double)sqrtl(ll);
        out[L.r2 + l] = (double)sqrtl(ll * (ll - 1 > 0 ? ll - 1 : 0));
        out[L.r3 + l] = (double)sqrtl(ll * (ll - 1 > 0 ? ll - 1 : 0) * (ll - 2 > 0 ? ll - 2 : 0));
    }
}

int tap_halfwidth(double len, double dx) {
    double r = len / dx;
    long long n = llround(r);
    if (n < 1 || fabs(r - (double)n) > 1e-9 * (1.0 + r)) return -1;
    return (int)n;
}

bool validate(const evfdlb_params& p, const char** why) {
    const char* w = nullptr;
    if (p.dim != 1) w = "dim must be 1";
    else if (p.ny != 1) w = "ny must be 1 for a 1D slab";
    else if (p.nx < 8) w = "nx must be >= 8";
    else if (!(p.dx > 0)) w = "dx must be > 0";
    else if (!(p.sigma > 0)) w = "sigma must be > 0";
    else if (!(p.phi_a >= 0)) w = "phi_a must be >= 0";
    else if (!(p.gamma > 3)) w = "gamma must be > 3";
    else if (p.Q < 4 || p.Q > kQMax) w = "Q must be in [4, 32]";
    else if (p.bc < EVFDLB_BC_PERIODIC || p.bc > EVFDLB_BC_HALO_OUTFLOW_HI) w = "bad bc";
    else if (p.relax_mode != EVFDLB_RELAX_INV_TAU && p.relax_mode != EVFDLB_RELAX_CHI_OVER_TAU) w = "bad relax_mode";
    else if (!(p.weno_eps > 0)) w = "weno_eps must be > 0";
    else if (!(p.T_iso >= 0) || !isfinite(p.T_iso)) w = "T_iso must be 0 (thermal) or > 0";
    else if (!(p.dt > 0) && !(p.cfl > 0 && p.cfl <= 1)) w = "need dt > 0 or 0 < cfl <= 1";
    else if (p.force_model != EVFDLB_EV1 && p.force_model != EVFDLB_EV2) w = "bad force_model";
    else if (p.force_model == EVFDLB_EV2 && !(p.gamma > 5)) w = "EV2 needs gamma > 5 (kappa of Eq. (F2))";
    else {
        int m = tap_halfwidth(p.sigma, p.dx);
        int M = tap_halfwidth(p.r_cut, p.dx);
        if (m < 1) w = "sigma/dx must be a positive integer";
        else if (p.force_model == EVFDLB_EV2) w = nullptr;      // r_cut unused
        else if (M < 1) w = "r_cut/dx must be a positive integer";
        else if (M < m + 2) w = "r_cut must be >= sigma + 2 dx";
        else if ((M - m) % 2) w = "(r_cut - sigma)/dx must be even (Simpson panels end at +-sigma)";
    }
    // a HALO slab sends its first and last G interior nodes: it holds >= G of
    // them besides its ghost bands
    if (!w && is_halo_bc(p.bc) && p.nx < (p.bc == EVFDLB_BC_HALO ? 3 : 2) * halo_width(p))
        w = "HALO needs at least halo_width interior nodes";
    if (why) *why = w;
    return w == nullptr;
}

// Ghost nodes per side of a HALO slab: the widest read of the stage about a
// node, i.e. the density sums over +-M (force / energy taps) and F, G over
// +-3 (the WENO-5 stencil of the face fluxes).
int halo_width(const evfdlb_params& p) { return std::max(3, force_halfwidth(p)); }

namespace {
double simpson(int j, int M, double dx) {
    int t = j + M;
    double c = (t == 0 || t == 2 * M) ? 1.0 : ((t & 1) ? 4.0 : 2.0);
    return c * dx / 3.0;
}
// Eq. (F1) kernel: the 3D force of Eq. (force) integrated over a plane at offset z.
double g_kernel(double z, double s, double phi, double gam) {
    double az = fabs(z);
    if (az < s) return 2.0 * kPi * phi * z;
    return 2.0 * kPi * phi * pow(s / az, gam) * z;
}
// Even potential whose derivative is g, vanishing at infinity.
double g_potential(double z, double s, double phi, double gam) {
    double az = fabs(z);
    if (az < s) return kPi * phi * (z * z - s * s * gam / (gam - 2.0));
    return -2.0 * kPi * phi * s * s * pow(s / az, gam - 2.0) / (gam - 2.0);
}
}  // namespace

// Half-width of the force and energy tap blocks, which is also the density
// halo a node tile stages.  EV1: r_cut/dx (the Simpson range of Eq. (F1)).
// EV2: sigma/dx + 2, the halo the Fischer-Methfessel average of the +-2
// gradient neighbours needs; the EV2 stencils reach +-2 and the taps beyond
// are zero.
int force_halfwidth(const evfdlb_params& p) {
    int m = tap_halfwidth(p.sigma, p.dx);
    if (p.force_model == EVFDLB_EV2) return m < 1 ? -1 : m + 2;
    return tap_halfwidth(p.r_cut, p.dx);
}

// Taps of one slab: [force 2M+1 | Fischer-Methfessel 2m+1 | energy 2M+1],
// M = force_halfwidth.  Without heap use; returns the count, or -1 when it
// exceeds cap.
//  fm_j     = 3/(4 sigma^3) s_j (sigma^2 - (j dx)^2)     (sphere average, Sec. II.A)
// EV1, Eq. (F1) with Simpson 1/3 weights s_j:
//  force_j  = s_j g(j dx)
//  energy_j = s_j [Phi(j dx) - Phi(r_cut)]               (mean-field energy)
// EV2, Eq. (F2): F2 = 2a dn/dz + kappa d3n/dz3 with the fourth-order first
// difference (1, -8, 0, 8, -1)/(12 dx) and the five-point third difference
// (-1, 2, 0, -2, 1)/(2 dx^3), merged into one antisymmetric stencil:
//  force_{+-1} = +-(16a/(12 dx) - kappa/dx^3),  force_{+-2} = +-(-2a/(12 dx) + kappa/(2 dx^3))
// and the energy field psi = -2a n - kappa d2n/dz2 (fourth-order second
// difference (-1, 16, -30, 16, -1)/(12 dx^2)), whose -dpsi/dz is F2:
//  energy_0 = -2a + 30 kappa/(12 dx^2), energy_{+-1} = -16 kappa/(12 dx^2),
//  energy_{+-2} = kappa/(12 dx^2)
int fill_taps(const evfdlb_params& p, double* out, int cap) {
    int M = force_halfwidth(p), m = tap_halfwidth(p.sigma, p.dx);
    if (M < 1 || m < 1) return -1;
    int need = 2 * (2 * M + 1) + 2 * m + 1;
    if (need > cap) return -1;
    double* force = out;
    double* fm = out + 2 * M + 1;
    double* energy = fm + 2 * m + 1;
    double s3 = p.sigma * p.sigma * p.sigma;
    for (int j = -m; j <= m; ++j) {
        double z = j * p.dx;
        fm[j + m] = 3.0 / (4.0 * s3) * simpson(j, m, p.dx) * (p.sigma * p.sigma - z * z);
    }
    if (p.force_model == EVFDLB_EV2) {
        double a = ev2_a(p), kappa = ev2_kappa(p), h = p.dx;
        for (int j = 0; j < 2 * M + 1; ++j) force[j] = energy[j] = 0.0;
        double t1 = 16.0 * a / (12.0 * h) - kappa / (h * h * h);
        double t2 = -2.0 * a / (12.0 * h) + kappa / (2.0 * h * h * h);
        force[M + 1] = t1;
        force[M - 1] = -t1;
        force[M + 2] = t2;
        force[M - 2] = -t2;
        double k12 = kappa / (12.0 * h * h);
        energy[M] = -2.0 * a + 30.0 * k12;
        energy[M + 1] = energy[M - 1] = -16.0 * k12;
        energy[M + 2] = energy[M - 2] = k12;
        return need;
    }
    for (int j = -M; j <= M; ++j) force[j + M] = simpson(j, M, p.dx) * g_kernel(j * p.dx, p.sigma, p.phi_a, p.gamma);
    double phiR = g_potential(p.r_cut, p.sigma, p.phi_a, p.gamma);
    for (int j = -M; j <= M; ++j)
        energy[j + M] = simpson(j, M, p.dx) * (g_potential(j * p.dx, p.sigma, p.phi_a, p.gamma) - phiR);
    return need;
}

void build_taps(const evfdlb_params& p, std::vector<double>& out) {
    int M = force_halfwidth(p), m = tap_halfwidth(p.sigma, p.dx);
    out.assign(M < 1 || m < 1 ? 0 : 2 * (2 * M + 1) + 2 * m + 1, 0.0);
    if (!out.empty()) fill_taps(p, out.data(), (int)out.size());
}

// Eq. (F2) constants: a = (2 pi sigma^3/3) phi gamma/(gamma-3) and
// kappa = (2 pi sigma^5/15) phi gamma/(gamma-5), the first and third moments
// (2a = int s g, 6 kappa = int s^3 g) of the Eq. (F1) plane kernel g.
double ev2_a(const evfdlb_params& p) {
    double s = p.sigma;
    return 2.0 * kPi * s * s * s / 3.0 * p.phi_a * p.gamma / (p.gamma - 3.0);
}
double ev2_kappa(const evfdlb_params& p) {
    double s = p.sigma;
    return 2.0 * kPi * s * s * s * s * s / 15.0 * p.phi_a * p.gamma / (p.gamma - 5.0);
}

double discrete_a(const evfdlb_params& p) {
    if (p.force_model == EVFDLB_EV2) return ev2_a(p);
    int M = tap_halfwidth(p.r_cut, p.dx);
    if (M < 1) return NAN;
    long double acc = 0;
    for (int j = -M; j <= M; ++j)
        acc += (long double)simpson(j, M, p.dx) * (j * p.dx) * g_kernel(j * p.dx, p.sigma, p.phi_a, p.gamma);
    return (double)(0.5L * acc);
}

double resolved_dt(const evfdlb_params& p) {
    if (p.dt > 0) return p.dt;
    double xi[kQMax], w[kQMax];
    velocity_set(p.Q, xi, w);
    return p.cfl * p.dx / fabs(xi[p.Q - 1]);
}

// ---------------------------------------------------------------------------
// Equation of state, Eq. (EOSS): P = n T Z(eta) - a n^2 with the
// Carnahan-Starling Z = (1 + eta + eta^2 - eta^3)/(1 - eta)^3, eta = pi s^3 n/6.
// With y(eta) = eta Z(eta):
//   y'  = (1 + 4 eta + 4 eta^2 - 4 eta^3 + eta^4) / (1 - eta)^4
//   y'' = [N'(1 - eta) + 4 N] / (1 - eta)^5,  N the numerator of y'.
// ---------------------------------------------------------------------------
namespace {
struct Eos {
    double a, s, k;  // k = 6 / (pi s^3): n = k eta
    double eta(double n) const { return n / k; }
    double P(double n, double T) const {
        double e = eta(n), om = 1 - e;
        return n * T * (1 + e + e * e - e * e * e) / (om * om * om) - a * n * n;
    }
    static double y1(double e) {
        double om = 1 - e;
        return (1 + 4 * e + 4 * e * e - 4 * e * e * e + e * e * e * e) / (om * om * om * om);
    }
    static double y2(double e) {
        double om = 1 - e;
        double N = 1 + 4 * e + 4 * e * e - 4 * e * e * e + e * e * e * e;
        double dN = 4 + 8 * e - 12 * e * e + 4 * e * e * e;
        return (dN * om + 4 * N) / (om * om * om * om * om);
    }
    double dPdn(double n, double T) const { return T * y1(eta(n)) - 2 * a * n; }
    // chemical potential up to a function of T: n dmu/dn = dP/dn
    double mu(double n, double T) const {
        double e = eta(n), om = 1 - e;
        return T * (log(n) + (8 * e - 9 * e * e + 3 * e * e * e) / (om * om * om)) - 2 * a * n;
    }
};

template <typename Fn>
double bisect(Fn f, double lo, double hi, int iters = 400) {
    double flo = f(lo);
    for (int it = 0; it < iters; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid == lo || mid == hi) break;
        double fm = f(mid);
        if ((fm < 0) == (flo < 0)) { lo = mid; flo = fm; } else { hi = mid; }
    }
    return 0.5 * (lo + hi);
}
}  // namespace

// Critical point: dP/dn = d2P/dn2 = 0, i.e. y'(eta) = eta y''(eta) and
// T_c = 2 a k / y''(eta_c).
double critical_T_of_a(double a, double sigma, double* n_c) {
    Eos E{a, sigma, 6.0 / (kPi * sigma * sigma * sigma)};
    double ec = bisect([](double e) { return Eos::y1(e) - e * Eos::y2(e); }, 0.01, 0.4);
    if (n_c) *n_c = E.k * ec;
    return 2.0 * a * E.k / Eos::y2(ec);
}

// Maxwell construction at temperature T (Sec. III.A): find the saturation
// pressure at which the vapour and liquid branches have equal chemical potential.
bool coexistence_of(double a, double sigma, double T, double* nv, double* nl) {
    double n_c;
    double Tc = critical_T_of_a(a, sigma, &n_c);
    if (!(T > 0) || !(T < Tc)) return false;
    Eos E{a, sigma, 6.0 / (kPi * sigma * sigma * sigma)};
    double n_max = 0.99 * E.k;
    double s_lo = bisect([&](double n) { return E.dPdn(n, T); }, 1e-12, n_c);
    double s_hi = bisect([&](double n) { return E.dPdn(n, T); }, n_c, n_max);
    double p_hi = E.P(s_lo, T);
    double p_lo = E.P(s_hi, T);
    if (p_lo < 0) p_lo = 0;
    auto branches = [&](double Ps, double* v, double* l) {
        // vapour branch is increasing on (0, s_lo), liquid on (s_hi, n_max)
        *v = bisect([&](double n) { return E.P(n, T) - Ps; }, 1e-300, s_lo);
        *l = bisect([&](double n) { return E.P(n, T) - Ps; }, s_hi, n_max);
    };
    double Ps = bisect([&](double P) {
        double v, l;
        branches(P, &v, &l);
        return E.mu(l, T) - E.mu(v, T);
    }, p_lo + 1e-300, p_hi, 200);
    branches(Ps, nv, nl);
    return true;
}

}  // namespace evfdlb
