// evfdlb_internal.h -- structures shared by the host model code, the kernels
// and the C-ABI layer of libevfdlb.  Not part of the public interface.
#pragma once

#include <stdint.h>

#include <vector>

#include "evfdlb.h"

#ifdef __CUDACC__
#define EVF_HD __host__ __device__
#else
#define EVF_HD
#endif

namespace evfdlb {

constexpr int kQMax = 32;          // largest Gauss-Hermite order of a slab
constexpr int kZMax = 64;          // largest node tile of one CTA
constexpr int kThreads = 256;      // threads of the per-tile kernels
// Threads of the RK-stage kernel (warp 0 forms the node work).  The FP64 pipe
// of this part accepts one warp instruction per scheduler every 64 cycles
// whatever the number of active lanes, so the FP64 kernels run 8 warps (two
// worker warps beside the node warp per scheduler, and two CTAs of at most
// 128 registers per SM when the work list spans several waves); the FP32
// variant's per-velocity work is cheap and latency-bound, so it runs 16.
template <typename R, bool DF = false> struct StageThreads { static constexpr int value = 256; };
template <> struct StageThreads<float, false> { static constexpr int value = 512; };
constexpr int kNumMoments = 6;     // raw moment sums kept per node
constexpr int kNumScalars = 10;    // per-node scalars feeding the synthesis

// Raw moment sums of a state, per node: S0 = sum F, S1 = sum xi F,
// S2 = sum xi^2 F, S3 = sum xi^3 F, G0 = sum G, G1 = sum xi G.
enum { MOM_S0 = 0, MOM_S1, MOM_S2, MOM_S3, MOM_G0, MOM_G1 };

// Error bits latched by the kernels.
enum : unsigned { ERR_NONFINITE = 1u, ERR_NEGATIVE = 2u, ERR_TIMEOUT = 4u };

// Parity split of the Gauss-Hermite transforms.  The nodes are symmetric,
// xi_{Q-1-j} = -xi_j (w likewise), and psi_l(-x) = (-1)^l psi_l(x), so with
// E_j = h_j + h_{Q-1-j}, O_j = h_j - h_{Q-1-j} (j < H = (Q+1)/2; for odd Q the
// middle node has E = h, O = 0) the analysis is
//   a_l = sum_{j<H} psi_l(xi_j) (l even ? E_j : O_j),
// and a synthesis sum_l w_k psi_l(xi_k) c_l = E_k + O_k at k < H, E_k - O_k at
// Q-1-k, with E_k, O_k its even- and odd-order parts: half the products.
struct ParitySplit {
    int H;        // nodes with xi <= 0
    int GE, GO;   // analysis groups of two even / two odd orders (orders <= Q-2)
    int QE;       // Q rounded up to even: the synthesis row length
    EVF_HD explicit ParitySplit(int Q) {
        H = (Q + 1) / 2;
        const int ne = (Q - 2) / 2 + 1, no = (Q - 3) / 2 + 1;   // even / odd orders <= Q-2
        GE = (ne + 1) / 2;
        GO = (no + 1) / 2;
        QE = Q + (Q & 1);
    }
    EVF_HD int analysis_len() const { return 2 * (GE + GO) * H; }   // Pp
    EVF_HD int synthesis_len() const { return H * QE; }             // Sp
};

// Offsets inside the table block of one velocity order Q (doubles).
struct TableLayout {
    int xi, w, P, S, rinv, rr, r1, r2, r3, Pp, Sp, total;
    EVF_HD explicit TableLayout(int Q) {
        const ParitySplit ps(Q);
        xi = 0;
        w = xi + Q;
        P = w + Q;          // P[l*Q + j] = psi_l(xi_j)          (analysis)
        S = P + Q * Q;      // S[k*Q + l] = w_k psi_l(xi_k)      (synthesis)
        rinv = S + Q * Q;   // 1/sqrt(l+1)
        rr = rinv + Q;      // sqrt(l)/sqrt(l+1)
        r1 = rr + Q;        // sqrt(l)
        r2 = r1 + Q;        // sqrt(l(l-1))
        r3 = r2 + Q;        // sqrt(l(l-1)(l-2))
        // parity-split analysis pairs Pp[g][j] = (psi_l(xi_j), psi_{l+2}(xi_j)), j < H,
        // groups g: even orders l = 4g (g < GE), then odd orders l = 4(g - GE) + 1
        // (a missing second order is 0)
        Pp = r3 + Q;
        // parity-split synthesis rows Sp[k][l] = S[k][l], k < H, rows padded to
        // an even length QE with zeros (orders l, l+1 in one two-wide load)
        Sp = Pp + ps.analysis_len();
        total = Sp + ps.synthesis_len();
    }
};

// One slab as the kernels see it.
struct SlabDesc {
    int nx, Q, bc, relax;
    int M, m;            // half-widths of the force and Fischer-Methfessel taps
    int tab_off;         // offset of this slab's velocity tables (doubles)
    int tap_off;         // offset of this slab's taps: force[2M+1], fm[2m+1], energy[2M+1]
    long long f_off;     // offset of this slab in the F (and G) arrays (elements)
    long long node_off;  // offset of this slab in per-node arrays
    double dx, inv_dx, dt, weno_eps;
    double b;            // 2 pi sigma^3 / 3, Eq. (carnstar)
    double eta_coef;     // pi sigma^3 / 6
    double mu0_coef;     // 5 / (16 sigma^2 sqrt(pi)), Eq. (viscosity)
    double T_iso;        // > 0: node fields formed at this temperature (isothermal mode)
};

// One CTA's share of work: nodes [i0, i0 + nz) of slab `slab`.
struct WorkItem {
    int slab, i0, nz, pad;
};

// Arguments of the persistent step (by value): nsteps Shu-Osher steps of
// every slab as 3 nsteps x nitems queued work items.
struct PersistArgs {
    const SlabDesc* slabs;
    const WorkItem* items;   // the work list, one entry per slab tile
    const int* tiles;        // work items per slab
    const double* tables;
    const double* taps;
    double* st[3];           // u, u1, u2: [2][NF] each
    double* mom[3];          // their raw moment sums [6][NN]
    unsigned* err;           // error word (ERR_* bits)
    unsigned* queue;         // next work item (zeroed before the launch)
    unsigned* done;          // completed items per slab (zeroed before the launch)
    const unsigned* gate;    // 1: open; 0: every wait waits on a flag nothing sets
    long long NF, NN;
    long long spin_limit;    // polls of a dependency wait before it gives up
    int nitems, nstages, Z;
};

// ---- host model code (host_model.cpp) ----
constexpr int kVelocitySetMax = 64;                              // largest order of evfdlb_velocity_set
bool velocity_set(int Q, double* xi, double* w);                 // ascending, sum w = 1; no heap
void build_tables(int Q, const double* xi, const double* w, double* out);  // TableLayout(Q); no heap
bool validate(const evfdlb_params& p, const char** why);
int tap_halfwidth(double len, double dx);                        // len/dx if integral, else -1
int force_halfwidth(const evfdlb_params& p);                     // force/energy taps and density halo
int halo_width(const evfdlb_params& p);                          // ghost nodes per side of a HALO slab
inline bool is_halo_bc(int bc) { return bc >= EVFDLB_BC_HALO && bc <= EVFDLB_BC_HALO_OUTFLOW_HI; }
int fill_taps(const evfdlb_params& p, double* out, int cap);     // force, fm, energy; no heap
void build_taps(const evfdlb_params& p, std::vector<double>& out);  // force, fm, energy
double ev2_a(const evfdlb_params& p);                            // Eq. (F2) a
double ev2_kappa(const evfdlb_params& p);                        // Eq. (F2) kappa
double discrete_a(const evfdlb_params& p);
double critical_T_of_a(double a, double sigma, double* n_c);
bool coexistence_of(double a, double sigma, double T, double* nv, double* nl);
double resolved_dt(const evfdlb_params& p);

}  // namespace evfdlb
