/*
 * evfdlb.h -- C ABI of libevfdlb, a GB300 (sm_103a) implementation of the
 * time step of the Enskog-Vlasov finite-difference lattice Boltzmann model
 * (EV-FDLB, EV1 force) of Busuioc & Sofonea, "Thermal Enskog-Vlasov Lattice
 * Boltzmann model with phase separation", arXiv:2503.15187.
 *
 * The model (paper Sec. II-III): a fluid of hard spheres of diameter sigma
 * with a Sutherland attractive tail -phi_a (r/sigma)^-gamma, Eq. (sutherland),
 * homogeneous across the slab, described by the reduced distributions
 *   F(z, xi) = int f dp_y dp_z,   G(z, xi) = int f (p_y^2 + p_z^2)/2 dp_y dp_z
 * on the full-range Gauss-Hermite velocity set xi_k (k < Q) and a uniform grid
 * z_i = i dx (i < nx).  One time step is the third-order TVD Runge-Kutta
 * scheme of Shu and Osher applied to
 *   dF/dt = -xi dF/dz - F1[n] dF/dxi - nu (F - F^S) + J1_F      (Eqs. (ev1),
 *   dG/dt = -xi dG/dz - F1[n] dG/dxi - nu (G - G^S) + J1_G       (enskog_approx))
 * with WENO-5 advection, the Simpson-integrated self-consistent force of
 * Eq. (F1), the Shakhov equilibrium and the simplified Enskog term J1 of
 * Sec. II.B evaluated with chi at the Fischer-Methfessel average density,
 * and the transport coefficients of Eqs. (viscosity), (tau), (prandtl).
 * Units are the reduced units of Sec. III (m = k_B = 1).
 *
 * Conventions for every entry point
 *  - Returns an evfdlb_status; nothing else crosses the ABI (no exceptions,
 *    no aborts).  A device-side error (non-finite value, n <= 0, T <= 0) is
 *    latched by the kernels and reported by the next call that synchronises
 *    (step, moments, get_state, rhs, fields); the context then refuses to step
 *    (EVFDLB_E_STATE) until init or set_state is called again.
 *  - Array arguments are borrowed for the duration of the call only.  With
 *    on_device = 0 they are host pointers (any host memory); with
 *    on_device = 1 they are device pointers on the context's device, read or
 *    written in order on the context's stream.  Calls that return data to
 *    host memory synchronise the stream before returning.
 *  - Distributions are laid out velocity-major: F[k * nx + i] (k < Q, i < nx),
 *    float64; for a batch, slab s occupies Q_s * nx_s consecutive entries in
 *    slab order.  Per-node arrays are [nx] per slab, concatenated.
 *  - A context is bound to one CUDA stream and is not thread-safe.
 */
#ifndef EVFDLB_H
#define EVFDLB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct evfdlb_ctx evfdlb_ctx;

typedef enum {
    EVFDLB_OK = 0,
    EVFDLB_E_INVALID_ARG = -1, /* a parameter or pointer fails validation       */
    EVFDLB_E_CUDA = -2,        /* a CUDA runtime call failed                     */
    EVFDLB_E_OOM = -3,         /* device allocation failed                       */
    EVFDLB_E_NONFINITE = -4,   /* a kernel met a NaN/Inf in the state            */
    EVFDLB_E_NEGATIVE = -5,    /* a kernel met n <= 0 or T <= 0                  */
    EVFDLB_E_TIMEOUT = -6,     /* a bounded device wait ran out                  */
    EVFDLB_E_STATE = -7,       /* call out of order (e.g. step before init)      */
    EVFDLB_E_UNSUPPORTED = -8  /* valid request this build does not implement    */
} evfdlb_status;

/* Boundary of a slab.  PERIODIC: the slab wraps.  OUTFLOW: ghost nodes copy
 * the nearest interior node.  HALO: the slab is one rank's part of a larger
 * z-split domain; its first and last G = evfdlb_halo_width(params) of the nx
 * nodes are ghost nodes that only the caller's halo exchange writes
 * (evfdlb_halo_pack / evfdlb_halo_unpack), and each RK stage (evfdlb_stage)
 * updates the interior nodes alone.  HALO_OUTFLOW_LO / _HI: the same, for the
 * first / last part of a split OUTFLOW slab: that end has no ghost band and
 * is the slab's outflow boundary (node 0 / nx-1 is a boundary node). */
enum {
    EVFDLB_BC_PERIODIC = 0,
    EVFDLB_BC_OUTFLOW = 1,
    EVFDLB_BC_HALO = 2,
    EVFDLB_BC_HALO_OUTFLOW_LO = 3,
    EVFDLB_BC_HALO_OUTFLOW_HI = 4
};
/* Precision.  FP64: every step in FP64.  FP32: FP32 state and per-velocity
 * work, FP64 chi / transport / gradients / conserved sums.  FP64_DF: FP64
 * state and FP64 arithmetic except the Hermite analysis and synthesis of the
 * stage, which run as double-float pairs (hi, lo floats, ~48 bits) on the
 * FP32 pipe with the compensated dot product Dot2 of Ogita, Rump & Oishi
 * (2005); the adjoint returns E_UNSUPPORTED for it. */
enum { EVFDLB_FP64 = 0, EVFDLB_FP32 = 1, EVFDLB_FP64_DF = 2 };
/* Force model (Sec. II.A).  EV1: the convolution of Eq. (F1), Simpson taps
 * over |z| <= r_cut.  EV2: its gradient expansion, Eq. (F2),
 * F2 = 2a dn/dz + kappa d3n/dz3 with a = (2 pi sigma^3/3) phi_a gamma/(gamma-3)
 * and kappa = (2 pi sigma^5/15) phi_a gamma/(gamma-5); dn/dz by the
 * fourth-order central difference and d3n/dz3 by the five-point stencil
 * (-1, 2, 0, -2, 1)/(2 dx^3) (Sec. III).  EV2 ignores r_cut and needs
 * gamma > 5; dim = 2 is EV1 only. */
enum { EVFDLB_EV1 = 0, EVFDLB_EV2 = 1 };
/* Relaxation rate of the Shakhov term J0 (Sec. II.B).  The paper writes
 * J0 = -(chi/tau)(f - f^S) with tau of Eq. (tau); the Chapman-Enskog
 * argument that fixes Eq. (tau) reproduces the Enskog viscosity only with
 * rate 1/tau.  Both readings are selectable; 1/tau is the default. */
enum { EVFDLB_RELAX_INV_TAU = 0, EVFDLB_RELAX_CHI_OVER_TAU = 1 };

/* Problem statement of one slab (paper Sec. III: sigma = phi_a = 1, gamma = 6),
 * or, with dim = 2, of one plane periodic domain of the two-dimensional
 * tensor-product extension (the paper names 2D as future work, Sec. IV):
 * reduced distributions over p_z on the tensor product of the order-Q
 * Gauss-Hermite set per axis (Q even, 4..16), the Eq. (force) integral over
 * z as the in-plane kernel summed over the grid offsets inside the r_cut
 * disc, the Fischer-Methfessel average with chord weights, WENO-5 and
 * fourth-order gradients along each axis; periodic only, EV1, FP32 or FP64,
 * gamma an even integer, nx * ny < 2^31, dt = cfl dx / (2 max|xi|) when
 * dt <= 0 (otherwise E_INVALID_ARG).  A 2D
 * context has nbatch = 1; evfdlb_fields, evfdlb_tune, evfdlb_rhs_vjp and the
 * adjoint return E_UNSUPPORTED for it. */
typedef struct {
    int32_t dim;          /* 1 (slab) or 2 (plane, see above)                          */
    int32_t nx;           /* grid nodes along x, >= 8                                  */
    int32_t ny;           /* 1 for a slab; nodes along y (>= 8) for dim = 2            */
    double  dx;           /* grid spacing; sigma/dx and (EV1) r_cut/dx must be integers*/
                          /* and (r_cut - sigma)/dx even (Simpson panels end at sigma) */
    double  sigma;        /* hard-sphere diameter, Eq. (sutherland)                    */
    double  phi_a;        /* depth of the attractive tail, Eq. (sutherland)            */
    double  gamma;        /* tail exponent (> 3), Eq. (sutherland)                     */
    double  r_cut;        /* EV1: cut of the Eq. (F1) integral (>= sigma + 2dx)        */
    int32_t Q;            /* Gauss-Hermite order, 4 <= Q <= 32                         */
    int32_t bc;           /* EVFDLB_BC_* (above)                                       */
    int32_t precision;    /* EVFDLB_FP64, EVFDLB_FP32 or EVFDLB_FP64_DF (see above);   */
                          /* one precision per context (the ABI stays float64)         */
    int32_t force_model;  /* EVFDLB_EV1 or EVFDLB_EV2 (see above)                      */
    int32_t relax_mode;   /* EVFDLB_RELAX_INV_TAU or EVFDLB_RELAX_CHI_OVER_TAU         */
    double  dt;           /* > 0: time step; <= 0: dt = cfl * dx / max|xi_k|           */
    double  cfl;          /* used when dt <= 0; 0 < cfl <= 1                           */
    int32_t ckpt_every;   /* > 0: the context keeps the state every ckpt_every steps   */
                          /* (the checkpoints of evfdlb_adjoint / adjoint_state, which */
                          /* recompute each segment from them); 0: no checkpoints, and */
                          /* the trajectory adjoint returns E_STATE.  One value per    */
                          /* context (that of slab 0)                                   */
    double  weno_eps;     /* WENO-5 smoothness regulariser (> 0), e.g. 1e-6            */
    double  T_iso;        /* 0: thermal (default).  > 0: isothermal mode -- after every */
                          /* step each node's temperature is set back to T_iso, its    */
                          /* density, velocity and non-equilibrium part kept:          */
                          /* F += F_MB(n,u,T_iso) - F_MB(n,u,T), G likewise with the   */
                          /* pair (F_MB, T F_MB) (Sec. III.A keeps T constant; the     */
                          /* mechanism is this library's reading).  evfdlb_rhs is the  */
                          /* thermal right-hand side.  dim = 1 only; the adjoint       */
                          /* returns E_UNSUPPORTED for it.                             */
} evfdlb_params;

/* Fills p with the defaults of Sec. III: dim 1, sigma = phi_a = 1, gamma = 6,
 * r_cut = 6, Q = 16, periodic, FP64, EV1, rate 1/tau, cfl 0.5, weno_eps 1e-6,
 * thermal (T_iso = 0).
 * nx and dx are left for the caller (set to 0). */
void evfdlb_default_params(evfdlb_params* p);

/* Creates a context for nbatch >= 1 independent slabs.  With nbatch == 1 the
 * slab is *p and per_slab may be NULL; with nbatch > 1, per_slab[s] gives slab
 * s (p may be NULL) and all slabs advance together in evfdlb_step.
 * cuda_stream is a cudaStream_t (NULL = the legacy default stream).  The
 * context owns all device memory it uses.  On success *out is set; on failure
 * *out is NULL and nothing is leaked.
 * Errors: E_INVALID_ARG (validation, see evfdlb_params), E_UNSUPPORTED,
 * E_OOM, E_CUDA. */
evfdlb_status evfdlb_create(const evfdlb_params* p, int32_t nbatch,
                            const evfdlb_params* per_slab, void* cuda_stream,
                            evfdlb_ctx** out);

/* Sets the state to the Hermite-projected Maxwellian pair (F_MB, T F_MB) of
 * the fields n0 > 0, u0, T0 > 0 ([sum nx], slab order).  For dim = 2 the
 * arrays are [nx * ny] (index y * nx + x), u0 is [2][nx * ny] (u_x then
 * u_y) and the pair is (F_MB, T/2 F_MB).  Errors: E_INVALID_ARG (NULL
 * pointer), E_NONFINITE / E_NEGATIVE (checked on the device), E_CUDA. */
evfdlb_status evfdlb_init(evfdlb_ctx* ctx, const double* n0, const double* u0,
                          const double* T0, int32_t on_device);

/* Advances every slab by nsteps >= 0 Shu-Osher RK3 steps (3 right-hand-side
 * evaluations each).  Work is queued on the context's stream as CUDA graphs;
 * the call synchronises once at the end to read the device error word.
 * Errors: E_STATE (no valid state), E_NONFINITE, E_NEGATIVE, E_CUDA. */
evfdlb_status evfdlb_step(evfdlb_ctx* ctx, int64_t nsteps);

/* Queues nsteps steps without synchronising and without reading the error
 * word (for timing and for callers that overlap work); a later synchronising
 * call reports any latched device error. */
evfdlb_status evfdlb_step_async(evfdlb_ctx* ctx, int64_t nsteps);

/* Macroscopic fields of the current state (Sec. II.B): n, u, T and heat flux
 * q per node ([sum nx] each; any may be NULL) and, if totals != NULL, per
 * slab four totals {mass, momentum, energy incl. mean-field energy, mean-field
 * energy} ([4 * nbatch], always host memory).  For dim = 2: u and q are
 * [2][nx * ny] and the totals are {mass, momentum x, momentum y, kinetic +
 * internal energy}: the second momentum component takes the fourth slot,
 * and the 2D mean-field energy is not formed (it would need the potential
 * of the z-integrated plane kernel on the force disc's taps, a second
 * convolution per call, and a fifth slot).  Mean-field energy:
 * EV1: (dx/2) sum_i n_i sum_j s_j [Phi(j dx) - Phi(r_cut)] n_{i+j} with Phi the
 * even potential whose derivative is the Eq. (F1) kernel and s_j Simpson
 * weights; EV2: (dx/2) sum_i n_i psi_i with psi = -2a n - kappa d2n/dz2 (the
 * fourth-order second difference), whose -dpsi/dz is F2. */
evfdlb_status evfdlb_moments(evfdlb_ctx* ctx, double* n, double* u, double* T,
                             double* q, double* totals, int32_t on_device);

/* Copies the state (F, G; [sum Q nx] each, layout above) out of / into the
 * context.  set_state also clears a latched device error; it returns once
 * host arrays have been read (device arrays: once the copies are queued), and
 * a state that the kernels reject (a non-finite moment sum) is reported by
 * the next call that synchronises (for dim = 2, set_state itself, which
 * synchronises).  For dim = 2 the state is
 * [Q * Q][ny][nx] per distribution, velocity index kx * Q + ky. */
evfdlb_status evfdlb_get_state(evfdlb_ctx* ctx, double* F, double* G, int32_t on_device);
evfdlb_status evfdlb_set_state(evfdlb_ctx* ctx, const double* F, const double* G,
                               int32_t on_device);

/* One evaluation of the right-hand side L(F, G) of Eq. (ev1) at the current
 * state, written to RF, RG (layout of the state).  Diagnostic; the state is
 * not changed. */
evfdlb_status evfdlb_rhs(evfdlb_ctx* ctx, double* RF, double* RG, int32_t on_device);

/* Node fields of one right-hand-side evaluation at the current state, as
 * [EVFDLB_NFIELDS][sum nx]: n, u, T, q, nbar (Fischer-Methfessel average,
 * Sec. II.A), chi (Eq. (carnstar) at nbar), F1 (Eq. (F1)), mu (Eq. (viscosity)),
 * tau (Eq. (tau)), Pr (Eq. (prandtl)), nu (relaxation rate), A = d ln(n^2 chi T)/dz,
 * B = d ln T/dz, D = du/dz (Eq. (J1)), X = n^2 chi T, b n chi. */
#define EVFDLB_NFIELDS 16
evfdlb_status evfdlb_fields(evfdlb_ctx* ctx, double* fields, int32_t on_device);

/* Number of slabs, and the nodes / velocity order / time step of slab s. */
evfdlb_status evfdlb_slab_info(const evfdlb_ctx* ctx, int32_t s, int32_t* nx,
                               int32_t* Q, double* dt);

/* Number of the library's own kernel launches queued per time step (all
 * slabs), for launch accounting. */
int32_t evfdlb_launches_per_step(const evfdlb_ctx* ctx);

/* Node tile of the work decomposition: each CTA of a stage kernel advances
 * all velocities of tile_nodes consecutive nodes of one slab (1..64).  The
 * context picks one wave of CTAs over the SMs by default; evfdlb_tune
 * re-partitions (and re-captures the step graphs), e.g. for an autotuner.
 * Synchronises the stream.  Errors: E_INVALID_ARG, E_CUDA. */
evfdlb_status evfdlb_tune(evfdlb_ctx* ctx, int32_t tile_nodes);
int32_t evfdlb_tile_nodes(const evfdlb_ctx* ctx);

/* ---- Discrete adjoint (FP64, periodic, thermal, one-dimensional contexts) ----
 * The reverse mode of the FP64 step above: exact discrete vector-Jacobian
 * products of the right-hand side L of Eqs. (ev1), (enskog_approx) and of the
 * Shu-Osher stages (Sec. III), for the gradient of a loss of the final state.
 * phi_a enters through the Eq. (F1) force, which is linear in it (the kernel
 * g of Eq. (F1) integrates the Sutherland tail of Eq. (sutherland)), and
 * through nothing else; the initial fields enter through the projected
 * Maxwellian pair of evfdlb_init.  The trajectory is the one since the last
 * evfdlb_init or evfdlb_set_state: it is rebuilt segment by segment from the
 * checkpoints kept every ckpt_every steps (checkpoint-and-recompute; the
 * recompute of one segment runs on a second stream of the context beside the
 * reverse sweep of the next, with identical results).  Work buffers are
 * allocated on the first adjoint call.  Per-slab outputs (dL_dphi_a, dphi)
 * are always host memory ([nbatch]); the others follow on_device.
 * Errors: E_INVALID_ARG (NULL context or cotangent), E_STATE (no state; for
 * the trajectory calls also a context without checkpoints, ckpt_every = 0,
 * a poisoned context, or field gradients asked of a trajectory that began
 * at set_state), E_UNSUPPORTED (dim = 2, FP32, FP64_DF, outflow ends,
 * isothermal mode, phi_a = 0), E_OOM, E_CUDA, and the latched device errors.
 *
 * evfdlb_rhs_vjp: at the current state u, (outF, outG) = J(u)^T (WF, WG) with
 *   J = dL/du (one right-hand side), and dphi[s] = sum W . dL/dphi_a of slab s
 *   (may be NULL).  WF, WG, outF, outG: [sum Q nx] each, the state layout. */
evfdlb_status evfdlb_rhs_vjp(evfdlb_ctx* ctx, const double* WF, const double* WG, int32_t on_device,
                             double* outF, double* outG, double* dphi);

/* evfdlb_adjoint_state: given the cotangent (barF, barG) = dL/d(F, G) of the
 * current state, sweeps the trajectory back to its origin and returns (each
 * output may be NULL) dL/dphi_a per slab, dL/dF0 and dL/dG0 of the origin
 * state ([sum Q nx] each) and, for a trajectory that began at evfdlb_init,
 * the gradients with respect to the initial fields dL/dn0, dL/du0, dL/dT0
 * ([sum nx] each, per node: a uniform T0 has dL/dT = sum_i dL/dT0_i). */
evfdlb_status evfdlb_adjoint_state(evfdlb_ctx* ctx, const double* barF, const double* barG, int32_t on_device,
                                   double* dL_dphi_a, double* dL_dF0, double* dL_dG0, double* dL_dn0,
                                   double* dL_du0, double* dL_dT0);

/* evfdlb_adjoint: the density-profile form of the above for a loss L(n_end)
 * of the final density n = sum_k F_k (Sec. II.B): given dL/dn_end ([sum nx]),
 * dL/dF_k = dL/dn for every k and dL/dG = 0; returns dL/dphi_a per slab
 * (host, [nbatch]) and dL/dT0, dL/dn0 per node ([sum nx], on_device; any
 * output may be NULL).  The trajectory must begin at evfdlb_init. */
evfdlb_status evfdlb_adjoint(evfdlb_ctx* ctx, const double* dL_dn_end, int32_t on_device, double* dL_dphi_a,
                             double* dL_dT0, double* dL_dn0);

/* Time step without any device allocation.  The paper has no counterpart.
 * It serves callers that cannot call cudaMalloc: a plugin whose host
 * application owns all device memory through its own pool and hands out
 * only pointers; a process held to a fixed device-memory budget fixed at
 * start-up, where a later allocation may fail; and latency-bound loops, where
 * cudaMalloc / cudaFree may synchronise the device and take unbounded time.
 *
 * Advances the slab described by *p (validated as for evfdlb_create; FP64,
 * EV1 or EV2) by nsteps Shu-Osher RK3 steps, in place.  state is a DEVICE pointer to
 * 2 * Q * nx doubles: F (velocity-major, [k * nx + i]) followed by G, owned
 * by the caller.  All working memory (the two intermediate stages, moment
 * sums, velocity tables, taps, work list and error word) lives in one
 * file-scope __device__ array of about 3.4 MiB that every GPU loading the
 * library holds until the process exits; no cudaMalloc, cudaFree or other
 * allocating routine is called.
 * Limits: nx <= EVFDLB_STATIC_MAX_NODES, Q * nx <= EVFDLB_STATIC_MAX_ELEMENTS,
 * force tap half-width (EV1: r_cut / dx; EV2: sigma / dx + 2)
 * <= EVFDLB_STATIC_MAX_HALFWIDTH; larger requests return
 * EVFDLB_E_INVALID_ARG before any CUDA call.
 * Set-up: the first call on a device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current) and raises the stage
 * kernel's shared-memory limit; make that first call before any stream
 * capture.  Every call shares the one array and leaves its contents behind
 * (the error word is cleared at the start of each call; everything else is
 * written before it is read), so calls that overlap on the GPU -- on
 * different streams or host threads of one device -- race: the caller must
 * serialise them (calls from host threads of one process are serialised by
 * the library; a lock is held for the whole call).  Work is queued on
 * cuda_stream (a cudaStream_t, NULL = the legacy default stream); every call
 * copies its small parameter block from static host memory and synchronises
 * that stream before it returns, to read the error word.
 * Errors: E_INVALID_ARG, E_UNSUPPORTED (precision other than FP64, or bc =
 * EVFDLB_BC_HALO), E_NONFINITE, E_NEGATIVE, E_CUDA (also
 * when a CUDA error is already pending in the calling thread: it is returned,
 * not cleared, and nothing is queued). */
#define EVFDLB_STATIC_MAX_NODES 8192
#define EVFDLB_STATIC_MAX_ELEMENTS 65536
#define EVFDLB_STATIC_MAX_HALFWIDTH 500
evfdlb_status evfdlb_step_static(const evfdlb_params* p, double* state, int64_t nsteps,
                                 void* cuda_stream);

/* ---- Measurement and self-test (no counterpart in the paper) ----
 * evfdlb_probe_fp64_fma: FP64 fused multiply-add throughput of the current
 *   device in GFLOP/s (2 flops per FMA): independent FMA chains on every SM,
 *   timed with CUDA events on cuda_stream; best of reps >= 1 timed launches
 *   after one warm-up.  The FP64 step is bound by this pipe, so this is the
 *   measured peak of its roofline.  Synchronises the stream.
 * evfdlb_divide_fp64: q[i] = a[i] / b[i] (n >= 0 DEVICE arrays) as the
 *   kernels form FP64 quotients on the hot path (a Newton-refined reciprocal
 *   with a final residual correction, Markstein's scheme: within about one
 *   ulp for numerators of magnitude >= 2^-920, within 2^8 ulp below, where
 *   the residual leaves the normal range; not correctly rounded; divisors
 *   outside the float exponent range use
 *   the IEEE quotient; a quotient that overflows, or an infinite numerator,
 *   gives NaN where IEEE gives +-inf -- both non-finite, which is what the
 *   kernels check), and, if q_ieee != NULL, the IEEE quotient beside it.
 *   Synchronises the stream.
 * evfdlb_profile_stage: queues stage s (0, 1, 2) of one Shu-Osher step of a
 *   one-dimensional context on its stream, as evfdlb_step runs it, without
 *   touching the context's state: stage 2 writes the first intermediate
 *   buffer instead of the state.  For timing the stage kernel by itself (the
 *   caller brackets the call with events on the context's stream).  Errors:
 *   E_INVALID_ARG, E_STATE (no state), E_UNSUPPORTED (dim = 2), E_CUDA. */
evfdlb_status evfdlb_probe_fp64_fma(int32_t reps, void* cuda_stream, double* gflops);
evfdlb_status evfdlb_divide_fp64(const double* a, const double* b, double* q, double* q_ieee, int64_t n,
                                 void* cuda_stream);
evfdlb_status evfdlb_profile_stage(evfdlb_ctx* ctx, int32_t stage);

/* Persistent form of the step for a batch of slabs (FP64, thermal, dim = 1).
 * enable = 1: every evfdlb_step / step_async advances all slabs by one
 * launch per graph of steps: the CTAs stay resident and take work items
 * (RK stage, slab tile) from a queue in stage order; an item of stage g of
 * slab s waits, on the device, until every item of stage g-1 of slab s is
 * complete, so slabs of different lengths move through their stages
 * independently instead of meeting at a grid-wide launch boundary after
 * every stage.  Results are bit-identical to the launch-per-stage form.
 * Every such wait is bounded: after spin_limit polls (each sleeps about
 * 0.1 us; spin_limit <= 0: 2^23, about a second) the kernel records a timeout
 * and all its CTAs return; the next synchronising call reports
 * EVFDLB_E_TIMEOUT and the context refuses to step until init / set_state.
 * enable = 0: back to one launch per RK stage.  Re-captures the step graphs
 * and synchronises the stream.
 * Errors: E_INVALID_ARG, E_UNSUPPORTED (dim = 2, FP32, FP64_DF, isothermal
 * mode), E_OOM, E_CUDA. */
evfdlb_status evfdlb_set_persistent(evfdlb_ctx* ctx, int32_t enable, int64_t spin_limit);

/* Testing hook of the persistent form: with open = 0 every dependency wait
 * also waits for a gate flag that nothing sets, so that each wait runs to
 * its spin limit and the launch ends with EVFDLB_E_TIMEOUT (the bounded-wait
 * path, exercised without faulting the GPU); open = 1 (the default)
 * restores normal operation.  Synchronises the stream.  Errors:
 * E_INVALID_ARG, E_STATE (the persistent form was never enabled), E_CUDA. */
evfdlb_status evfdlb_debug_gate(evfdlb_ctx* ctx, int32_t open);

/* --- z-split slab (domain decomposition across ranks) ---------------------
 * The method is an explicit stencil in z (Sec. III): one RK stage of a node
 * reads F and G over +-3 nodes (WENO-5) and the density sums over +-M nodes
 * (the Eq. (F1) integral; M = r_cut/dx for EV1).  A slab is split along z by
 * giving each rank a context with bc = EVFDLB_BC_HALO over its part plus G
 * ghost nodes per side, and by exchanging, before every RK stage, one
 * message per side with each neighbour:
 *   init (ghost entries of n0, u0, T0 are ignored; ghosts hold 0)
 *   repeat: pack -> exchange -> unpack -> evfdlb_stage(s), s = 0, 1, 2
 * where the message a rank sends to its left neighbour becomes that
 * neighbour's from_right (and the right-going one its from_left).  A
 * periodic slab splits into HALO parts on a ring; an outflow slab into
 * HALO_OUTFLOW_LO (first part), HALO (middle parts) and HALO_OUTFLOW_HI
 * (last part) on a line.  The interior nodes then evolve bit-identically to
 * the same nodes of the unsplit slab.  evfdlb_step and evfdlb_rhs return E_UNSUPPORTED for a HALO
 * context; moments / totals cover its interior nodes for the totals, every
 * node for the per-node fields. */

/* Ghost nodes per side of a HALO slab with these parameters:
 * max(3, force half-width), or -1 when the parameters fail validation or
 * dim != 1.  A split part needs at least G interior nodes besides its ghost
 * bands (nx >= 3 G for HALO, nx >= 2 G for the outflow ends). */
int32_t evfdlb_halo_width(const evfdlb_params* params);

/* Length, in doubles, of one halo message of this context:
 * 6 Q + 6 G (F and G over 3 columns, the six raw moment sums over G columns,
 * FP64 whatever the state precision); 0 for a context that is not HALO. */
int64_t evfdlb_halo_len(const evfdlb_ctx* ctx);

/* Runs RK stage `stage` (0, 1, 2 of the Shu-Osher step) of every slab,
 * queued on the context's stream without synchronising (errors in the
 * kernels show at the next synchronising call).  Stages must come in order,
 * starting at 0 after init / set_state; after stage 2 the state is one step
 * further, exactly as evfdlb_step(ctx, 1) leaves it.  Works for every 1D
 * context; the only way to advance a HALO context.  Errors: E_INVALID_ARG,
 * E_STATE (no state, poisoned, or stage out of order), E_UNSUPPORTED (dim 2,
 * or ckpt_every > 0), E_CUDA. */
evfdlb_status evfdlb_stage(evfdlb_ctx* ctx, int32_t stage);

/* Writes the two halo messages of the state the next stage reads, with
 * lo / hi the ghost nodes below / above the interior (G, or 0 at an outflow
 * end): to_left from the first interior nodes (F, G at nodes lo .. lo+2,
 * moments at lo .. lo+G-1), to_right from the last ones (F, G at
 * nx-hi-3 .. nx-hi-1, moments at nx-hi-G .. nx-hi-1).  Both are device
 * buffers of evfdlb_halo_len(ctx) doubles owned by the caller; the one of an
 * outflow end is not touched and may be NULL.  Queued on the context's
 * stream.  Errors: E_INVALID_ARG, E_UNSUPPORTED (not HALO), E_STATE, E_CUDA. */
evfdlb_status evfdlb_halo_pack(evfdlb_ctx* ctx, double* to_left, double* to_right);

/* Writes the neighbours' messages into the ghost nodes of the state the next
 * stage reads: from_left (the left neighbour's to_right) into F, G at nodes
 * lo-3 .. lo-1 and moments at lo-G .. lo-1; from_right (the right
 * neighbour's to_left) into F, G at nx-hi .. nx-hi+2 and moments at
 * nx-hi .. nx-hi+G-1.  Device buffers as for pack (NULL at an outflow end);
 * queued on the context's stream.  Errors as pack. */
evfdlb_status evfdlb_halo_unpack(evfdlb_ctx* ctx, const double* from_left, const double* from_right);

/* Releases the context and its device memory (NULL is a no-op). */
void evfdlb_destroy(evfdlb_ctx* ctx);

/* Static description of a status code. */
const char* evfdlb_status_string(evfdlb_status s);

/* Host-side model constants (no GPU needed).
 *  evfdlb_discrete_a: a_d = (1/2) sum_j s_j (j dx) g(j dx), the constant the
 *    Simpson-integrated Eq. (F1) force gives for a linear density (F1 = 2 a_d dn/dz);
 *    for EV2 the a of Eq. (F2), which its stencils reproduce on a linear density;
 *  evfdlb_critical_T: critical temperature of Eq. (EOSS) with a = a_d
 *    (Carnahan-Starling repulsion, mean-field attraction);
 *  evfdlb_coexistence: Maxwell construction (Sec. III.A) at temperature T:
 *    vapour and liquid densities with equal pressure and chemical potential.
 * All return NaN / E_INVALID_ARG on invalid parameters. */
double evfdlb_discrete_a(const evfdlb_params* p);
double evfdlb_critical_T(const evfdlb_params* p);
evfdlb_status evfdlb_coexistence(const evfdlb_params* p, double T, double* n_vapour,
                                 double* n_liquid);

/* Full-range Gauss-Hermite velocity set of order Q (4 <= Q <= 64): roots of
 * the probabilists' He_Q and weights summing to 1, ascending. */
evfdlb_status evfdlb_velocity_set(int32_t Q, double* xi, double* w);

#ifdef __cplusplus
}
#endif
#endif /* EVFDLB_H */
