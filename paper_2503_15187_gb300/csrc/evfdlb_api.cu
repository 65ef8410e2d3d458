// evfdlb_api.cu -- the C ABI of libevfdlb (see include/evfdlb.h): context
// set-up, device buffers, CUDA-graph capture of the time step, transfers and
// error reporting.
#include <cuda_runtime.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <new>
#include <vector>

#include "evfdlb_internal.h"

namespace evfdlb {
size_t stage_smem_bytes_p(int prec, int Q, int Z, int M);
cudaError_t configure_kernels_p(int prec, size_t smem_bytes);
void launch_stage_p(int prec, int nitems, size_t smem, cudaStream_t st, const SlabDesc* slabs,
                    const WorkItem* items, const double* tables, const void* rtab, const double* taps,
                    const void* rtaps, const void* src, const void* base, void* out, double* rhs_out,
                    const double* mom_in, double* mom_out, long long NF, long long NN, double alpha, double beta,
                    int mode, int Z, unsigned* err);
void launch_stage_fields(int nitems, size_t smem, cudaStream_t st, const SlabDesc* slabs, const WorkItem* items,
                         const double* tables, const double* taps, const double* src, const double* base,
                         double* out, const double* mom_in, double* mom_out, double* fields_out, long long NF,
                         long long NN, double alpha, double beta, int Z, unsigned* err);
void launch_init_p(int prec, int nitems, size_t smem, cudaStream_t st, const SlabDesc* slabs,
                   const WorkItem* items, const double* tables, const void* rtab, const double* n0,
                   const double* u0, const double* T0, void* state, double* mom, long long NF, long long NN, int Z,
                   unsigned* err);
void launch_sums_p(int prec, int nitems, cudaStream_t st, const SlabDesc* slabs, const WorkItem* items,
                   const double* tables, const void* rtab, const void* state, double* mom, long long NF,
                   long long NN, unsigned* err);
size_t stage_smem_bytes_df(int Q, int Z, int M);
cudaError_t configure_df(size_t smem_bytes);
void launch_stage_df(int nitems, size_t smem, cudaStream_t st, const SlabDesc* slabs, const WorkItem* items,
                     const double* tables, const double* dftab, const double* taps, const double* src,
                     const double* base, double* out, double* rhs_out, const double* mom_in, double* mom_out,
                     long long NF, long long NN, double alpha, double beta, int mode, int Z, unsigned* err);
void launch_iso_reset_p(int prec, int nitems, size_t smem, cudaStream_t st, const SlabDesc* slabs,
                        const WorkItem* items, const double* tables, const void* rtab, void* state, double* mom,
                        long long NF, long long NN, int Z);
void launch_fields_p(int prec, int nitems, size_t smem, cudaStream_t st, const SlabDesc* slabs,
                     const WorkItem* items, const void* rtab, const double* taps, const void* rtaps,
                     const double* mom, double* fields, long long NN, int Z, unsigned* err);
cudaError_t configure_persist(size_t smem_bytes);
int persist_grid(size_t smem_bytes);
void launch_persist(int grid, size_t smem, cudaStream_t st, const PersistArgs& a);
void launch_convert_to_f32(cudaStream_t st, const double* in, float* out, long long n);
long long halo_message_len(int Q, int G);
void launch_halo_pack(int prec, cudaStream_t st, const void* state, const double* mom, long long NF, long long NN,
                      int nx, int Q, int G, int lo, int hi, double* to_left, double* to_right);
void launch_halo_unpack(int prec, cudaStream_t st, void* state, double* mom, long long NF, long long NN, int nx, int Q,
                        int G, int lo, int hi, const double* from_left, const double* from_right);
void launch_convert_to_f64(cudaStream_t st, const float* in, double* out, long long n);
void launch_moments(cudaStream_t st, const double* mom, long long NN, double* n, double* u, double* T,
                    double* q);
void launch_totals(int nslabs, int nitems, size_t smem, cudaStream_t st, const SlabDesc* slabs,
                   const WorkItem* items, const double* taps, const double* mom, long long NN, double* part,
                   double* out, double* n, double* u, double* T, double* q);
int adj_tile_max();
size_t adj_smem_bytes(int Q, int Z);
size_t adj_moments_smem_bytes(int Q, int Z, int m, int M);
cudaError_t configure_adjoint(size_t smem_bytes, size_t smem2_bytes);
void launch_adj_stage(int nitems, size_t smem, size_t smem2, cudaStream_t st, const SlabDesc* slabs,
                      const WorkItem* items, const double* tables, const double* taps, const double* src,
                      const double* fld, const double* mom, const double* ybar, const double* acc_in, double* acc_out,
                      double* out, double* nadj, double* phis, double* gface, long long NF, long long NN, double ca,
                      double cb, int use_dt, double cc, double cacc, double cy, int Z);
void launch_adj_init(int nitems, cudaStream_t st, const SlabDesc* slabs, const WorkItem* items,
                     const double* tables, const double* init_fields, const double* lam, double* dn0, double* du0,
                     double* dT0, long long NF, long long NN);
void launch_adj_phi(int nslabs, cudaStream_t st, const SlabDesc* slabs, const double* phis, const double* phi_a,
                    double* out);
void launch_adj_seed(int nitems, cudaStream_t st, const SlabDesc* slabs, const WorkItem* items, const double* dn,
                     double* barF, double* barG, long long NF);
// two-dimensional model (evfdlb_2d.cu)
struct Ctx2;
evfdlb_status create_2d(const evfdlb_params& p, void* stream, Ctx2** out);
void destroy_2d(Ctx2* c);
evfdlb_status init_2d(Ctx2* c, const double* n0, const double* u0, const double* T0, int on_device);
evfdlb_status step_async_2d(Ctx2* c, int64_t nsteps);
evfdlb_status check_2d(Ctx2* c);
evfdlb_status get_state_2d(Ctx2* c, double* F, double* G, int on_device);
evfdlb_status set_state_2d(Ctx2* c, const double* F, const double* G, int on_device);
evfdlb_status rhs_2d(Ctx2* c, double* RF, double* RG, int on_device);
evfdlb_status moments_2d(Ctx2* c, double* n, double* u, double* T, double* q, double* totals, int on_device);
long long nodes_2d(const Ctx2* c);
double dt_2d(const Ctx2* c);
double discrete_a_2d(const evfdlb_params& p);
bool validate_2d(const evfdlb_params& p);
}  // namespace evfdlb

using namespace evfdlb;

struct evfdlb_ctx {
    Ctx2* c2 = nullptr;          // set for a two-dimensional context (the rest unused)
    bool c2_state = false;
    int nbatch = 0;
    std::vector<evfdlb_params> params;
    std::vector<SlabDesc> slabs_h;
    std::vector<WorkItem> items_h;
    long long NF = 0;           // elements of F (= of G) over all slabs
    long long NN = 0;           // nodes over all slabs
    int Z = 1;                  // node tile of the work items
    size_t smem = 0;
    int device = 0;
    cudaStream_t user = nullptr;
    cudaStream_t cap = nullptr;  // private stream used only for graph capture
    int prec = EVFDLB_FP64;      // storage / per-velocity precision of the state
    size_t esize = sizeof(double);
    void* state[3] = {nullptr, nullptr, nullptr};    // each [2][NF] of esize: F then G
    double* mom[3] = {nullptr, nullptr, nullptr};    // each [6][NN]
    double* tables = nullptr;
    double* taps = nullptr;
    void* rtables = nullptr;     // tables / taps in the state precision (aliases for FP64)
    void* rtaps = nullptr;
    double* scratch = nullptr;   // [2 NF + 16 NN + 4 nbatch]
    SlabDesc* slabs = nullptr;
    WorkItem* items = nullptr;
    unsigned* err = nullptr;
    unsigned* err_h = nullptr;   // pinned host copy of the error word
    cudaEvent_t ev_in = nullptr; // end of set_state's host-to-device copies
    cudaGraphExec_t g_chunk = nullptr;
    cudaGraphExec_t g_one = nullptr;
    int chunk = 16;
    int Qmax = 0, Mmax = 0, mmax = 0;
    size_t items_cap = 0;        // capacity of the device work list
    bool have_state = false;
    bool poisoned = false;
    bool iso = false;            // some slab has T_iso > 0 (reset after every step)
    bool df = false;             // FP64_DF: FP64 context whose stages use double-float transforms
    // z-split slab (EVFDLB_BC_HALO): G ghost nodes per side, and the RK stage
    // that evfdlb_stage runs next (0 after init / set_state / a whole step)
    bool halo = false;
    int halo_G = 0;
    int halo_lo = 0, halo_hi = 0;   // ghost nodes below / above the interior (0: an outflow end)
    int rk_next = 0;
    double* dftables = nullptr;  // analysis / synthesis tables as float pairs (FP64_DF)
    size_t smem_df = 0;          // stage shared memory of the FP64_DF kernel
    // adjoint: checkpoints of the trajectory since the last init / set_state
    int ckpt_every = 0;          // 0: no tracking (no adjoint)
    int64_t steps = 0;           // steps since the trajectory origin
    bool origin_init = false;    // origin set by evfdlb_init (fields known)
    double* init_fields = nullptr;           // [3][NN]: n0, u0, T0
    std::vector<double*> ckpts;              // state at steps 0, K, 2K, ...
    double* seg[2] = {nullptr, nullptr};   // recomputed segments (two: the recompute of one overlaps
                                           // the reverse sweep of the other); each (3K+1) states [2 NF],
                                           // then (3K+1) moment sets [6 NN], then (3K+1) node-field
                                           // sets [EVFDLB_NFIELDS NN] (of the stage inputs)
    cudaStream_t aux = nullptr;            // the adjoint's recompute stream
    cudaEvent_t ev_fork = nullptr, ev_rec[2] = {nullptr, nullptr}, ev_sweep[2] = {nullptr, nullptr};
    double* adj = nullptr;       // see AdjBuf
    // the sweep's work items (node tile aZ <= the sweep kernels' largest tile)
    WorkItem* aitems = nullptr;
    std::vector<WorkItem> aitems_h;
    int aZ = 0;
    // persistent form of the step (evfdlb_set_persistent)
    bool persistent = false;
    long long spin_limit = 0;
    unsigned* pq = nullptr;      // [0] queue head, [1] gate, [2 ..] completed items per slab
    int* tiles_d = nullptr;      // work items per slab
    std::vector<int> tiles_h;
    int pgrid = 1;               // resident CTAs of the persistent kernel
};

namespace {

evfdlb_status cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return EVFDLB_OK;
    if (e == cudaErrorMemoryAllocation) return EVFDLB_E_OOM;
    return EVFDLB_E_CUDA;
}

#define TRY_CUDA(x)                                  \
    do {                                             \
        cudaError_t e_ = (x);                        \
        if (e_ != cudaSuccess) return cuda_status(e_); \
    } while (0)

void free_ctx(evfdlb_ctx* c) {
    if (!c) return;
    if (c->c2) destroy_2d(c->c2);
    if (c->g_chunk) cudaGraphExecDestroy(c->g_chunk);
    if (c->g_one) cudaGraphExecDestroy(c->g_one);
    for (int i = 0; i < 3; ++i) {
        cudaFree(c->state[i]);
        cudaFree(c->mom[i]);
    }
    if (c->rtables != c->tables) cudaFree(c->rtables);
    cudaFree(c->dftables);
    if (c->rtaps != c->taps) cudaFree(c->rtaps);
    cudaFree(c->tables);
    cudaFree(c->taps);
    cudaFree(c->scratch);
    cudaFree(c->init_fields);
    for (double* p : c->ckpts) cudaFree(p);
    for (int i = 0; i < 2; ++i) {
        cudaFree(c->seg[i]);
        if (c->ev_rec[i]) cudaEventDestroy(c->ev_rec[i]);
        if (c->ev_sweep[i]) cudaEventDestroy(c->ev_sweep[i]);
    }
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->aux) cudaStreamDestroy(c->aux);
    cudaFree(c->adj);
    cudaFree(c->aitems);
    cudaFree(c->pq);
    cudaFree(c->tiles_d);
    cudaFree(c->slabs);
    cudaFree(c->items);
    cudaFree(c->err);
    if (c->err_h) cudaFreeHost(c->err_h);
    if (c->ev_in) cudaEventDestroy(c->ev_in);
    if (c->cap) cudaStreamDestroy(c->cap);
    delete c;
}

// One RK stage kernel of the context's step: out = a base + b (src + dt L(src)).
void queue_stage(evfdlb_ctx* c, cudaStream_t st, const void* src, const void* base, void* out, const double* mi,
                 double* mo, double a, double b) {
    const int n = (int)c->items_h.size();
    if (c->df)
        launch_stage_df(n, c->smem_df, st, c->slabs, c->items, c->tables, c->dftables, c->taps, (const double*)src,
                        (const double*)base, (double*)out, nullptr, mi, mo, c->NF, c->NN, a, b, 0, c->Z, c->err);
    else
        launch_stage_p(c->prec, n, c->smem, st, c->slabs, c->items, c->tables, c->rtables, c->taps, c->rtaps, src,
                       base, out, nullptr, mi, mo, c->NF, c->NN, a, b, 0, c->Z, c->err);
}

// Queues nsteps steps of every slab as one persistent launch (after zeroing
// the queue head and the per-slab counters).
void queue_persist(evfdlb_ctx* c, cudaStream_t st, int nsteps) {
    cudaMemsetAsync(c->pq, 0, sizeof(unsigned), st);
    cudaMemsetAsync(c->pq + 2, 0, sizeof(unsigned) * c->nbatch, st);
    PersistArgs a;
    a.slabs = c->slabs;
    a.items = c->items;
    a.tiles = c->tiles_d;
    a.tables = c->tables;
    a.taps = c->taps;
    for (int i = 0; i < 3; ++i) {
        a.st[i] = (double*)c->state[i];
        a.mom[i] = c->mom[i];
    }
    a.err = c->err;
    a.queue = c->pq;
    a.gate = c->pq + 1;
    a.done = c->pq + 2;
    a.NF = c->NF;
    a.NN = c->NN;
    a.spin_limit = c->spin_limit;
    a.nitems = (int)c->items_h.size();
    a.nstages = 3 * nsteps;
    a.Z = c->Z;
    launch_persist(c->pgrid, c->smem, st, a);
}

// Queues one time step (three stages) on stream st.
void queue_step(evfdlb_ctx* c, cudaStream_t st) {
    const int n = (int)c->items_h.size();
    void *f0 = c->state[0], *f1 = c->state[1], *f2 = c->state[2];
    double *m0 = c->mom[0], *m1 = c->mom[1], *m2 = c->mom[2];
    auto stage = [&](const void* src, const void* base, void* out, const double* mi, double* mo, double a,
                     double b) { queue_stage(c, st, src, base, out, mi, mo, a, b); };
    stage(f0, nullptr, f1, m0, m1, 0.0, 1.0);              // u1 = u + dt L(u)
    stage(f1, f0, f2, m1, m2, 0.75, 0.25);                 // u2 = 3/4 u + 1/4 (u1 + dt L(u1))
    stage(f2, f0, f0, m2, m0, 1.0 / 3.0, 2.0 / 3.0);       // u_new = 1/3 u + 2/3 (u2 + dt L(u2)), over u
    if (c->iso)                                            // isothermal slabs: T back to T_iso
        launch_iso_reset_p(c->prec, n, c->smem, st, c->slabs, c->items, c->tables, c->rtables, f0, m0, c->NF,
                           c->NN, c->Z);
}

// Splits every slab into node tiles of Z nodes (the last tile of a slab may
// be shorter); the device work list is sized for the finest split (Z = 1).
void partition(evfdlb_ctx* c, int Z) {
    c->Z = Z;
    c->items_h.clear();
    for (int s = 0; s < c->nbatch; ++s) {
        // a HALO slab's work covers its interior nodes alone
        const int lo = c->halo_lo, hi = c->params[s].nx - c->halo_hi;
        for (int i0 = lo; i0 < hi; i0 += Z) c->items_h.push_back(WorkItem{s, i0, std::min(Z, hi - i0), 0});
    }
    c->smem = stage_smem_bytes_p(c->prec, c->Qmax, Z, c->Mmax);
    c->smem_df = stage_smem_bytes_df(c->Qmax, Z, c->Mmax);
    if (c->items_cap == 0) c->items_cap = (size_t)c->NN;
    c->tiles_h.assign(c->nbatch, 0);
    for (const WorkItem& w : c->items_h) ++c->tiles_h[w.slab];
}

evfdlb_status capture(evfdlb_ctx* c, int steps, cudaGraphExec_t* out) {
    cudaGraph_t g = nullptr;
    TRY_CUDA(cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal));
    if (c->persistent) queue_persist(c, c->cap, steps);
    else
        for (int s = 0; s < steps; ++s) queue_step(c, c->cap);
    cudaError_t e = cudaStreamEndCapture(c->cap, &g);
    if (e != cudaSuccess) return cuda_status(e);
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    return cuda_status(e);
}

// Reads and clears the device error word (synchronises the user stream).
evfdlb_status check_device(evfdlb_ctx* c) {
    unsigned hs = 0;
    unsigned* hp = c->err_h ? c->err_h : &hs;
    TRY_CUDA(cudaMemcpyAsync(hp, c->err, sizeof(unsigned), cudaMemcpyDeviceToHost, c->user));
    TRY_CUDA(cudaStreamSynchronize(c->user));
    const unsigned h = *hp;
    if (h) {
        c->poisoned = true;
        TRY_CUDA(cudaMemsetAsync(c->err, 0, sizeof(unsigned), c->user));
        if (h & ERR_TIMEOUT) return EVFDLB_E_TIMEOUT;
        return (h & ERR_NONFINITE) ? EVFDLB_E_NONFINITE : EVFDLB_E_NEGATIVE;
    }
    return EVFDLB_OK;
}

evfdlb_status copy_in(evfdlb_ctx* c, double* dst, const double* src, size_t bytes, int on_device) {
    TRY_CUDA(cudaMemcpyAsync(dst, src, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                             c->user));
    return EVFDLB_OK;
}

evfdlb_status copy_out(evfdlb_ctx* c, double* dst, const double* src, size_t bytes, int on_device) {
    TRY_CUDA(cudaMemcpyAsync(dst, src, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                             c->user));
    return EVFDLB_OK;
}

// Slots of the adjoint's work buffer c->adj (doubles).
struct AdjBuf {
    double *lam, *y1, *y2, *acc;   // [2 NF] each
    double* gface;                 // face gradients of the tiles' edge faces [5][2 NF]
    double* nadj;                  // node adjoints [10][NN]
    double* fld;                   // node fields of the state (evfdlb_rhs_vjp) [EVFDLB_NFIELDS][NN]
    double* phis;                  // per-node phi_a terms [NN]
    double* phi;                   // phi_a per slab [nbatch]
    double* dphi;                  // dL/dphi_a per slab [nbatch]
    size_t total;
    AdjBuf(double* base, long long NF, long long NN, int nbatch) {
        double* p = base;
        auto take = [&](size_t n) { double* q = p; p += n; return q; };
        lam = take(2 * NF);
        y1 = take(2 * NF);
        y2 = take(2 * NF);
        acc = take(2 * NF);
        gface = take(10 * (size_t)NF);
        nadj = take(10 * (size_t)NN);
        fld = take((size_t)EVFDLB_NFIELDS * NN);
        phis = take(NN);
        phi = take(nbatch);
        dphi = take(nbatch);
        total = (size_t)(p - base);
    }
};

AdjBuf adj_buf(const evfdlb_ctx* c) { return AdjBuf(c->adj, c->NF, c->NN, c->nbatch); }

// Work buffers of the adjoint, allocated on first use.
evfdlb_status ensure_adjoint_buffers(evfdlb_ctx* c) {
    if (!c->adj) {
        TRY_CUDA(cudaMalloc((void**)&c->adj, sizeof(double) * AdjBuf(nullptr, c->NF, c->NN, c->nbatch).total));
        std::vector<double> phi(c->nbatch);
        for (int s = 0; s < c->nbatch; ++s) phi[s] = c->params[s].phi_a;
        TRY_CUDA(cudaMemcpy(adj_buf(c).phi, phi.data(), sizeof(double) * c->nbatch, cudaMemcpyHostToDevice));
        TRY_CUDA(configure_adjoint(adj_smem_bytes(c->Qmax, adj_tile_max()),
                                   adj_moments_smem_bytes(c->Qmax, adj_tile_max(), c->mmax, c->Mmax)));
        TRY_CUDA(cudaMalloc((void**)&c->aitems, sizeof(WorkItem) * (size_t)c->NN));
    }
    // the sweep's work items: the step's node tile, capped at the sweep
    // kernels' largest tile (rebuilt when the step's tile changes; the
    // previous sweep may still read the list)
    const int aZ = std::min(c->Z, adj_tile_max());
    if (aZ != c->aZ) {
        TRY_CUDA(cudaStreamSynchronize(c->user));
        c->aitems_h.clear();
        for (int s = 0; s < c->nbatch; ++s)
            for (int i0 = 0; i0 < c->params[s].nx; i0 += aZ)
                c->aitems_h.push_back(WorkItem{s, i0, std::min(aZ, c->params[s].nx - i0), 0});
        TRY_CUDA(cudaMemcpy(c->aitems, c->aitems_h.data(), sizeof(WorkItem) * c->aitems_h.size(),
                            cudaMemcpyHostToDevice));
        c->aZ = aZ;
    }
    if (!c->seg[1] && c->ckpt_every > 0) {
        size_t nst = 3 * (size_t)c->ckpt_every + 1;
        for (int i = 0; i < 2; ++i)
            if (!c->seg[i])
                TRY_CUDA(cudaMalloc((void**)&c->seg[i],
                                    sizeof(double) * nst *
                                        (2 * (size_t)c->NF + (kNumMoments + EVFDLB_NFIELDS) * (size_t)c->NN)));
    }
    if (!c->aux) {
        TRY_CUDA(cudaStreamCreateWithFlags(&c->aux, cudaStreamNonBlocking));
        TRY_CUDA(cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming));
        for (int i = 0; i < 2; ++i) {
            TRY_CUDA(cudaEventCreateWithFlags(&c->ev_rec[i], cudaEventDisableTiming));
            TRY_CUDA(cudaEventCreateWithFlags(&c->ev_sweep[i], cudaEventDisableTiming));
        }
    }
    return EVFDLB_OK;
}

evfdlb_status adjoint_supported(evfdlb_ctx* c) {
    if (c->prec != EVFDLB_FP64 || c->df) return EVFDLB_E_UNSUPPORTED;
    for (auto& q : c->params) {
        if (q.bc != EVFDLB_BC_PERIODIC) return EVFDLB_E_UNSUPPORTED;
        if (q.T_iso > 0.0) return EVFDLB_E_UNSUPPORTED;       // T does not follow the state
        if (!(q.phi_a != 0.0)) return EVFDLB_E_UNSUPPORTED;   // the phi gradient divides by phi_a
    }
    return EVFDLB_OK;
}

// One stage of the reverse sweep on the context's stream; fld: the node
// fields of src.
void adj_stage(evfdlb_ctx* c, const double* src, const double* fld, const double* mom, const double* ybar,
               const double* acc_in, double* acc_out, double* out, double ca, double cb, int use_dt, double cc,
               double cacc, double cy) {
    const AdjBuf a = adj_buf(c);
    launch_adj_stage((int)c->aitems_h.size(), adj_smem_bytes(c->Qmax, c->aZ),
                     adj_moments_smem_bytes(c->Qmax, c->aZ, c->mmax, c->Mmax), c->user, c->slabs, c->aitems, c->tables,
                     c->taps, src, fld, mom, ybar, acc_in, acc_out, out, a.nadj, a.phis, a.gface, c->NF, c->NN, ca, cb,
                     use_dt, cc, cacc, cy, c->aZ);
}

}  // namespace

extern "C" {

void evfdlb_default_params(evfdlb_params* p) {
    if (!p) return;
    memset(p, 0, sizeof(*p));
    p->dim = 1;
    p->ny = 1;
    p->sigma = 1.0;
    p->phi_a = 1.0;
    p->gamma = 6.0;
    p->r_cut = 6.0;
    p->Q = 16;
    p->bc = EVFDLB_BC_PERIODIC;
    p->precision = EVFDLB_FP64;
    p->force_model = EVFDLB_EV1;
    p->relax_mode = EVFDLB_RELAX_INV_TAU;
    p->dt = 0.0;
    p->cfl = 0.5;
    p->ckpt_every = 0;
    p->weno_eps = 1e-6;
}

const char* evfdlb_status_string(evfdlb_status s) {
    switch (s) {
        case EVFDLB_OK: return "ok";
        case EVFDLB_E_INVALID_ARG: return "invalid argument";
        case EVFDLB_E_CUDA: return "CUDA runtime error";
        case EVFDLB_E_OOM: return "out of device memory";
        case EVFDLB_E_NONFINITE: return "non-finite value in the state";
        case EVFDLB_E_NEGATIVE: return "non-positive density or temperature";
        case EVFDLB_E_TIMEOUT: return "bounded device wait timed out";
        case EVFDLB_E_STATE: return "call out of order (no valid state)";
        case EVFDLB_E_UNSUPPORTED: return "not supported by this build";
    }
    return "unknown status";
}

double evfdlb_discrete_a(const evfdlb_params* p) {
    if (p && p->dim == 2) return validate_2d(*p) ? discrete_a_2d(*p) : NAN;
    if (!p || !validate(*p, nullptr)) return NAN;
    return discrete_a(*p);
}

double evfdlb_critical_T(const evfdlb_params* p) {
    if (p && p->dim == 2) return validate_2d(*p) ? critical_T_of_a(discrete_a_2d(*p), p->sigma, nullptr) : NAN;
    if (!p || !validate(*p, nullptr)) return NAN;
    return critical_T_of_a(discrete_a(*p), p->sigma, nullptr);
}

evfdlb_status evfdlb_coexistence(const evfdlb_params* p, double T, double* nv, double* nl) {
    if (!p || !nv || !nl) return EVFDLB_E_INVALID_ARG;
    const bool two = (p->dim == 2);
    if (two ? !validate_2d(*p) : !validate(*p, nullptr)) return EVFDLB_E_INVALID_ARG;
    if (!coexistence_of(two ? discrete_a_2d(*p) : discrete_a(*p), p->sigma, T, nv, nl)) return EVFDLB_E_INVALID_ARG;
    return EVFDLB_OK;
}

evfdlb_status evfdlb_velocity_set(int32_t Q, double* xi, double* w) {
    if (!xi || !w || Q < 4 || Q > 64) return EVFDLB_E_INVALID_ARG;
    return velocity_set(Q, xi, w) ? EVFDLB_OK : EVFDLB_E_INVALID_ARG;
}

evfdlb_status evfdlb_create(const evfdlb_params* p, int32_t nbatch, const evfdlb_params* per_slab,
                            void* cuda_stream, evfdlb_ctx** out) {
    if (!out) return EVFDLB_E_INVALID_ARG;
    *out = nullptr;
    if (nbatch < 1) return EVFDLB_E_INVALID_ARG;
    {
        const evfdlb_params* q0 = p ? p : per_slab;
        if (q0 && q0->dim == 2) {     // one plane periodic domain per context
            if (nbatch != 1) return EVFDLB_E_UNSUPPORTED;
            evfdlb_ctx* c = new (std::nothrow) evfdlb_ctx();
            if (!c) return EVFDLB_E_OOM;
            evfdlb_status st = create_2d(*q0, cuda_stream, &c->c2);
            if (st != EVFDLB_OK) {
                delete c;
                return st;
            }
            c->nbatch = 1;
            c->params.push_back(*q0);
            c->user = (cudaStream_t)cuda_stream;
            *out = c;
            return EVFDLB_OK;
        }
    }
    if (nbatch == 1 && !p && !per_slab) return EVFDLB_E_INVALID_ARG;
    if (nbatch > 1 && !per_slab) return EVFDLB_E_INVALID_ARG;
    std::vector<evfdlb_params> ps(nbatch);
    for (int s = 0; s < nbatch; ++s) {
        ps[s] = (nbatch == 1) ? (p ? *p : per_slab[0]) : per_slab[s];
        if (!validate(ps[s], nullptr)) return EVFDLB_E_INVALID_ARG;
        if (ps[s].precision != EVFDLB_FP64 && ps[s].precision != EVFDLB_FP32 && ps[s].precision != EVFDLB_FP64_DF)
            return EVFDLB_E_INVALID_ARG;
        if (ps[s].precision != ps[0].precision) return EVFDLB_E_INVALID_ARG;   // one precision per context
        if (is_halo_bc(ps[s].bc) && nbatch != 1) return EVFDLB_E_UNSUPPORTED;   // one split slab per context
    }
    evfdlb_ctx* c = new (std::nothrow) evfdlb_ctx();
    if (!c) return EVFDLB_E_OOM;
    c->nbatch = nbatch;
    c->params = ps;
    c->halo = is_halo_bc(ps[0].bc);
    c->halo_G = c->halo ? halo_width(ps[0]) : 0;
    c->halo_lo = (c->halo && ps[0].bc != EVFDLB_BC_HALO_OUTFLOW_LO) ? c->halo_G : 0;
    c->halo_hi = (c->halo && ps[0].bc != EVFDLB_BC_HALO_OUTFLOW_HI) ? c->halo_G : 0;
    c->user = (cudaStream_t)cuda_stream;
    c->df = (ps[0].precision == EVFDLB_FP64_DF);
    c->prec = c->df ? EVFDLB_FP64 : ps[0].precision;   // FP64_DF is an FP64 context but for its stages
    c->ckpt_every = ps[0].ckpt_every > 0 ? ps[0].ckpt_every : 0;
    c->esize = (c->prec == EVFDLB_FP32) ? sizeof(float) : sizeof(double);
    if (cudaGetDevice(&c->device) != cudaSuccess) { free_ctx(c); return EVFDLB_E_CUDA; }
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
    if (sms <= 0) sms = 1;

    // velocity tables, one block per distinct Q
    std::map<int, int> tab_off;
    std::vector<double> tables;
    for (auto& q : ps) {
        if (tab_off.count(q.Q)) continue;
        TableLayout L(q.Q);
        std::vector<double> xi(q.Q), w(q.Q);
        velocity_set(q.Q, xi.data(), w.data());
        tab_off[q.Q] = (int)tables.size();
        tables.resize(tables.size() + L.total);
        build_tables(q.Q, xi.data(), w.data(), tables.data() + tab_off[q.Q]);
    }
    // taps, slab descriptors, work items
    std::vector<double> taps;
    long long NF = 0, NN = 0;
    int Qmax = 0, Mmax = 0, mmax = 0;
    for (int s = 0; s < nbatch; ++s) {
        const evfdlb_params& q = ps[s];
        SlabDesc d;
        memset(&d, 0, sizeof(d));
        d.nx = q.nx;
        d.Q = q.Q;
        // a split slab reads with the outflow rule: inside a ghost band the
        // clamp never acts, and at an outflow end it is that end's boundary
        d.bc = is_halo_bc(q.bc) ? EVFDLB_BC_OUTFLOW : q.bc;
        d.relax = q.relax_mode;
        d.M = force_halfwidth(q);
        d.m = tap_halfwidth(q.sigma, q.dx);
        d.tab_off = tab_off[q.Q];
        d.tap_off = (int)taps.size();
        std::vector<double> t;
        build_taps(q, t);
        taps.insert(taps.end(), t.begin(), t.end());
        d.f_off = NF;
        d.node_off = NN;
        d.dx = q.dx;
        d.inv_dx = 1.0 / q.dx;
        d.dt = resolved_dt(q);
        d.weno_eps = q.weno_eps;
        d.b = 2.0 * M_PI * q.sigma * q.sigma * q.sigma / 3.0;
        d.eta_coef = M_PI * q.sigma * q.sigma * q.sigma / 6.0;
        d.mu0_coef = 5.0 / (16.0 * q.sigma * q.sigma * sqrt(M_PI));
        d.T_iso = q.T_iso;
        if (q.T_iso > 0.0) c->iso = true;
        NF += (long long)q.Q * q.nx;
        NN += q.nx;
        Qmax = std::max(Qmax, q.Q);
        Mmax = std::max(Mmax, d.M);
        mmax = std::max(mmax, d.m);
        c->slabs_h.push_back(d);
    }
    c->NF = NF;
    c->NN = NN;
    c->Qmax = Qmax;
    c->Mmax = Mmax;
    c->mmax = mmax;
    // node tile: one wave of CTAs over the SMs when possible
    long long z = (NN + sms - 1) / sms;
    partition(c, (int)std::min<long long>(std::max<long long>(z, 1), kZMax));

    cudaError_t e = cudaSuccess;
    auto alloc = [&](void** ptr, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc(ptr, bytes);
    };
    for (int i = 0; i < 3; ++i) {
        alloc((void**)&c->state[i], c->esize * 2 * NF);
        alloc((void**)&c->mom[i], sizeof(double) * kNumMoments * NN);
    }
    alloc((void**)&c->tables, sizeof(double) * tables.size());
    alloc((void**)&c->taps, sizeof(double) * taps.size());
    std::vector<float> tables_f(tables.begin(), tables.end()), taps_f(taps.begin(), taps.end());
    if (c->prec == EVFDLB_FP32) {
        alloc((void**)&c->rtables, sizeof(float) * tables_f.size());
        alloc((void**)&c->rtaps, sizeof(float) * taps_f.size());
    } else {
        c->rtables = c->tables;
        c->rtaps = c->taps;
    }
    alloc((void**)&c->scratch, sizeof(double) * (2 * NF + EVFDLB_NFIELDS * NN + 4 * nbatch));
    alloc((void**)&c->slabs, sizeof(SlabDesc) * nbatch);
    alloc((void**)&c->items, sizeof(WorkItem) * c->items_cap);
    alloc((void**)&c->err, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaHostAlloc((void**)&c->err_h, sizeof(unsigned), cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_in, cudaEventDisableTiming);
    if (c->ckpt_every > 0) alloc((void**)&c->init_fields, sizeof(double) * 3 * NN);
    if (e == cudaSuccess) e = cudaMemcpy(c->tables, tables.data(), sizeof(double) * tables.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(c->taps, taps.data(), sizeof(double) * taps.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && c->prec == EVFDLB_FP32)
        e = cudaMemcpy(c->rtables, tables_f.data(), sizeof(float) * tables_f.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && c->prec == EVFDLB_FP32)
        e = cudaMemcpy(c->rtaps, taps_f.data(), sizeof(float) * taps_f.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(c->slabs, c->slabs_h.data(), sizeof(SlabDesc) * nbatch, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(c->items, c->items_h.data(), sizeof(WorkItem) * c->items_h.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(c->err, 0, sizeof(unsigned));
    if (e == cudaSuccess) e = configure_kernels_p(c->prec, stage_smem_bytes_p(c->prec, Qmax, kZMax, Mmax));
    if (e == cudaSuccess && c->df) {
        // analysis and synthesis tables as (hi, lo) float pairs in 8-byte slots
        std::vector<double> dft(tables.size());
        for (size_t i = 0; i < tables.size(); ++i) {
            float pr[2];
            pr[0] = (float)tables[i];
            pr[1] = (float)(tables[i] - (double)pr[0]);
            memcpy(&dft[i], pr, sizeof(pr));
        }
        alloc((void**)&c->dftables, sizeof(double) * dft.size());
        if (e == cudaSuccess)
            e = cudaMemcpy(c->dftables, dft.data(), sizeof(double) * dft.size(), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = configure_df(stage_smem_bytes_df(Qmax, kZMax, Mmax));
    }
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        evfdlb_status st = cuda_status(e);
        free_ctx(c);
        return st;
    }
    evfdlb_status st = capture(c, 1, &c->g_one);
    if (st == EVFDLB_OK) st = capture(c, c->chunk, &c->g_chunk);
    if (st != EVFDLB_OK) {
        free_ctx(c);
        return st;
    }
    *out = c;
    return EVFDLB_OK;
}

void evfdlb_destroy(evfdlb_ctx* c) {
    if (!c) return;
    if (c->user) cudaStreamSynchronize(c->user);
    else cudaDeviceSynchronize();
    free_ctx(c);
}

evfdlb_status evfdlb_init(evfdlb_ctx* c, const double* n0, const double* u0, const double* T0, int32_t on_device) {
    if (!c || !n0 || !u0 || !T0) return EVFDLB_E_INVALID_ARG;
    if (c->c2) {
        evfdlb_status s = init_2d(c->c2, n0, u0, T0, on_device);
        c->c2_state = (s == EVFDLB_OK);
        c->poisoned = false;
        return s;
    }
    const double* dn = n0;
    const double* du = u0;
    const double* dT = T0;
    size_t bytes = sizeof(double) * c->NN;
    if (!on_device) {
        double* buf = c->scratch;   // [3 NN] fits inside the scratch block
        evfdlb_status s;
        if ((s = copy_in(c, buf, n0, bytes, 0)) != EVFDLB_OK) return s;
        if ((s = copy_in(c, buf + c->NN, u0, bytes, 0)) != EVFDLB_OK) return s;
        if ((s = copy_in(c, buf + 2 * c->NN, T0, bytes, 0)) != EVFDLB_OK) return s;
        dn = buf;
        du = buf + c->NN;
        dT = buf + 2 * c->NN;
    }
    TRY_CUDA(cudaMemsetAsync(c->err, 0, sizeof(unsigned), c->user));
    if (c->halo) {   // ghost columns hold zeros until the first exchange
        const size_t es = (c->prec == EVFDLB_FP32) ? sizeof(float) : sizeof(double);
        for (int i = 0; i < 3; ++i) {
            TRY_CUDA(cudaMemsetAsync(c->state[i], 0, es * 2 * c->NF, c->user));
            TRY_CUDA(cudaMemsetAsync(c->mom[i], 0, sizeof(double) * kNumMoments * c->NN, c->user));
        }
    }
    launch_init_p(c->prec, (int)c->items_h.size(), c->smem, c->user, c->slabs, c->items, c->tables, c->rtables, dn,
                  du, dT, c->state[0], c->mom[0], c->NF, c->NN, c->Z, c->err);
    TRY_CUDA(cudaGetLastError());
    if (c->ckpt_every > 0) {   // trajectory origin for the adjoint
        TRY_CUDA(cudaMemcpyAsync(c->init_fields, dn, bytes, cudaMemcpyDeviceToDevice, c->user));
        TRY_CUDA(cudaMemcpyAsync(c->init_fields + c->NN, du, bytes, cudaMemcpyDeviceToDevice, c->user));
        TRY_CUDA(cudaMemcpyAsync(c->init_fields + 2 * c->NN, dT, bytes, cudaMemcpyDeviceToDevice, c->user));
    }
    c->steps = 0;
    c->rk_next = 0;
    c->origin_init = true;
    c->poisoned = false;
    evfdlb_status s = check_device(c);
    c->have_state = (s == EVFDLB_OK);
    return s;
}

evfdlb_status evfdlb_step_async(evfdlb_ctx* c, int64_t nsteps) {
    if (!c || nsteps < 0) return EVFDLB_E_INVALID_ARG;
    if (c->c2) {
        if (!c->c2_state || c->poisoned) return EVFDLB_E_STATE;
        return step_async_2d(c->c2, nsteps);
    }
    if (!c->have_state || c->poisoned) return EVFDLB_E_STATE;
    if (c->halo) return EVFDLB_E_UNSUPPORTED;   // a split slab advances by evfdlb_stage + halo exchange
    if (c->rk_next != 0) return EVFDLB_E_STATE;   // a step started by evfdlb_stage is unfinished
    while (nsteps > 0) {
        int64_t n = nsteps;
        if (c->ckpt_every > 0) {
            // the state at every multiple of ckpt_every steps is kept for the adjoint
            const int64_t K = c->ckpt_every;
            if (c->steps % K == 0) {
                size_t idx = (size_t)(c->steps / K);
                while (c->ckpts.size() <= idx) {
                    double* p = nullptr;
                    TRY_CUDA(cudaMalloc((void**)&p, sizeof(double) * 2 * c->NF));
                    c->ckpts.push_back(p);
                }
                TRY_CUDA(cudaMemcpyAsync(c->ckpts[idx], c->state[0], sizeof(double) * 2 * c->NF,
                                         cudaMemcpyDeviceToDevice, c->user));
            }
            n = std::min<int64_t>(nsteps, K - c->steps % K);
        }
        int64_t full = n / c->chunk, rest = n % c->chunk;
        for (int64_t i = 0; i < full; ++i) TRY_CUDA(cudaGraphLaunch(c->g_chunk, c->user));
        for (int64_t i = 0; i < rest; ++i) TRY_CUDA(cudaGraphLaunch(c->g_one, c->user));
        c->steps += n;
        nsteps -= n;
    }
    return EVFDLB_OK;
}

evfdlb_status evfdlb_step(evfdlb_ctx* c, int64_t nsteps) {
    evfdlb_status s = evfdlb_step_async(c, nsteps);
    if (s != EVFDLB_OK) return s;
    if (c->c2) {
        s = check_2d(c->c2);
        if (s != EVFDLB_OK) c->poisoned = true;
        return s;
    }
    return check_device(c);
}

evfdlb_status evfdlb_get_state(evfdlb_ctx* c, double* F, double* G, int32_t on_device) {
    if (!c || !F || !G) return EVFDLB_E_INVALID_ARG;
    if (c->c2) return c->c2_state ? get_state_2d(c->c2, F, G, on_device) : EVFDLB_E_STATE;
    if (!c->have_state) return EVFDLB_E_STATE;
    size_t bytes = sizeof(double) * c->NF;
    const double* src = (const double*)c->state[0];
    if (c->prec == EVFDLB_FP32) {   // widen into the scratch block first
        launch_convert_to_f64(c->user, (const float*)c->state[0], c->scratch, 2 * c->NF);
        TRY_CUDA(cudaGetLastError());
        src = c->scratch;
    }
    evfdlb_status s;
    if ((s = copy_out(c, F, src, bytes, on_device)) != EVFDLB_OK) return s;
    if ((s = copy_out(c, G, src + c->NF, bytes, on_device)) != EVFDLB_OK) return s;
    TRY_CUDA(cudaStreamSynchronize(c->user));
    return EVFDLB_OK;
}

evfdlb_status evfdlb_set_state(evfdlb_ctx* c, const double* F, const double* G, int32_t on_device) {
    if (!c || !F || !G) return EVFDLB_E_INVALID_ARG;
    if (c->c2) {
        evfdlb_status s = set_state_2d(c->c2, F, G, on_device);
        c->c2_state = (s == EVFDLB_OK);
        c->poisoned = false;
        return s;
    }
    size_t bytes = sizeof(double) * c->NF;
    double* dst = (c->prec == EVFDLB_FP32) ? c->scratch : (double*)c->state[0];
    evfdlb_status s;
    if ((s = copy_in(c, dst, F, bytes, on_device)) != EVFDLB_OK) return s;
    if ((s = copy_in(c, dst + c->NF, G, bytes, on_device)) != EVFDLB_OK) return s;
    if (!on_device) TRY_CUDA(cudaEventRecord(c->ev_in, c->user));
    if (c->prec == EVFDLB_FP32) {   // round to the state precision
        launch_convert_to_f32(c->user, c->scratch, (float*)c->state[0], 2 * c->NF);
        TRY_CUDA(cudaGetLastError());
    }
    TRY_CUDA(cudaMemsetAsync(c->err, 0, sizeof(unsigned), c->user));
    launch_sums_p(c->prec, (int)c->items_h.size(), c->user, c->slabs, c->items, c->tables, c->rtables, c->state[0],
                  c->mom[0], c->NF, c->NN, c->err);
    TRY_CUDA(cudaGetLastError());
    c->steps = 0;
    c->rk_next = 0;
    c->origin_init = false;
    c->poisoned = false;
    c->have_state = true;
    // Host arrays are released once their copies have run; the moment sums
    // stay queued, and a state they reject is reported by the next call that
    // synchronises.
    if (!on_device) TRY_CUDA(cudaEventSynchronize(c->ev_in));
    return EVFDLB_OK;
}

evfdlb_status evfdlb_rhs(evfdlb_ctx* c, double* RF, double* RG, int32_t on_device) {
    if (!c || !RF || !RG) return EVFDLB_E_INVALID_ARG;
    if (c->c2) return c->c2_state ? rhs_2d(c->c2, RF, RG, on_device) : EVFDLB_E_STATE;
    if (!c->have_state) return EVFDLB_E_STATE;
    if (c->halo) return EVFDLB_E_UNSUPPORTED;
    if (c->df)
        launch_stage_df((int)c->items_h.size(), c->smem_df, c->user, c->slabs, c->items, c->tables, c->dftables,
                        c->taps, (const double*)c->state[0], nullptr, nullptr, c->scratch, c->mom[0], nullptr, c->NF,
                        c->NN, 0.0, 1.0, 1, c->Z, c->err);
    else
        launch_stage_p(c->prec, (int)c->items_h.size(), c->smem, c->user, c->slabs, c->items, c->tables,
                       c->rtables, c->taps, c->rtaps, c->state[0], nullptr, nullptr, c->scratch, c->mom[0], nullptr,
                       c->NF, c->NN, 0.0, 1.0, 1, c->Z, c->err);
    TRY_CUDA(cudaGetLastError());
    size_t bytes = sizeof(double) * c->NF;
    evfdlb_status s;
    if ((s = copy_out(c, RF, c->scratch, bytes, on_device)) != EVFDLB_OK) return s;
    if ((s = copy_out(c, RG, c->scratch + c->NF, bytes, on_device)) != EVFDLB_OK) return s;
    return check_device(c);
}

evfdlb_status evfdlb_fields(evfdlb_ctx* c, double* fields, int32_t on_device) {
    if (!c || !fields) return EVFDLB_E_INVALID_ARG;
    if (c->c2) return EVFDLB_E_UNSUPPORTED;
    if (!c->have_state) return EVFDLB_E_STATE;
    double* buf = c->scratch;
    launch_fields_p(c->prec, (int)c->items_h.size(), c->smem, c->user, c->slabs, c->items, c->rtables, c->taps,
                    c->rtaps, c->mom[0], buf, c->NN, c->Z, c->err);
    TRY_CUDA(cudaGetLastError());
    evfdlb_status s = copy_out(c, fields, buf, sizeof(double) * EVFDLB_NFIELDS * c->NN, on_device);
    if (s != EVFDLB_OK) return s;
    return check_device(c);
}

evfdlb_status evfdlb_moments(evfdlb_ctx* c, double* n, double* u, double* T, double* q, double* totals,
                             int32_t on_device) {
    if (!c) return EVFDLB_E_INVALID_ARG;
    if (c->c2) return c->c2_state ? moments_2d(c->c2, n, u, T, q, totals, on_device) : EVFDLB_E_STATE;
    if (!c->have_state) return EVFDLB_E_STATE;
    double* buf = c->scratch;
    double* outs[4] = {n, u, T, q};
    double* dptr[4];
    for (int i = 0; i < 4; ++i) dptr[i] = outs[i] ? (on_device ? outs[i] : buf + i * c->NN) : nullptr;
    double* dt = buf + EVFDLB_NFIELDS * c->NN;
    if (totals) {   // the totals' first pass writes n, u, T, q as well
        double* part = dt + 4 * c->nbatch;   // 4 per work item (<= 4 NN <= 2 NF)
        launch_totals(c->nbatch, (int)c->items_h.size(), sizeof(double) * (c->Z + 2 * c->Mmax), c->user, c->slabs,
                      c->items, c->taps, c->mom[0], c->NN, part, dt, dptr[0], dptr[1], dptr[2], dptr[3]);
    } else {
        launch_moments(c->user, c->mom[0], c->NN, dptr[0], dptr[1], dptr[2], dptr[3]);
    }
    TRY_CUDA(cudaGetLastError());
    if (!on_device)
        for (int i = 0; i < 4; ++i)
            if (outs[i]) {
                evfdlb_status s = copy_out(c, outs[i], dptr[i], sizeof(double) * c->NN, 0);
                if (s != EVFDLB_OK) return s;
            }
    if (totals) {
        evfdlb_status s = copy_out(c, totals, dt, sizeof(double) * 4 * c->nbatch, 0);
        if (s != EVFDLB_OK) return s;
    }
    return check_device(c);
}

evfdlb_status evfdlb_slab_info(const evfdlb_ctx* c, int32_t s, int32_t* nx, int32_t* Q, double* dt) {
    if (!c || s < 0 || s >= c->nbatch) return EVFDLB_E_INVALID_ARG;
    if (c->c2) {
        if (nx) *nx = c->params[0].nx;
        if (Q) *Q = c->params[0].Q;
        if (dt) *dt = dt_2d(c->c2);
        return EVFDLB_OK;
    }
    if (nx) *nx = c->slabs_h[s].nx;
    if (Q) *Q = c->slabs_h[s].Q;
    if (dt) *dt = c->slabs_h[s].dt;
    return EVFDLB_OK;
}

int32_t evfdlb_launches_per_step(const evfdlb_ctx* c) {
    return c ? (c->c2 ? 12 : (c->persistent ? 1 : (c->iso ? 4 : 3))) : 0;
}

int32_t evfdlb_tile_nodes(const evfdlb_ctx* c) { return c ? (c->c2 ? 0 : c->Z) : 0; }

evfdlb_status evfdlb_tune(evfdlb_ctx* c, int32_t tile_nodes) {
    if (!c || tile_nodes < 1 || tile_nodes > kZMax) return EVFDLB_E_INVALID_ARG;
    if (c->c2) return EVFDLB_E_UNSUPPORTED;
    TRY_CUDA(cudaStreamSynchronize(c->user));
    partition(c, tile_nodes);
    TRY_CUDA(cudaMemcpy(c->items, c->items_h.data(), sizeof(WorkItem) * c->items_h.size(), cudaMemcpyHostToDevice));
    if (c->tiles_d)
        TRY_CUDA(cudaMemcpy(c->tiles_d, c->tiles_h.data(), sizeof(int) * c->nbatch, cudaMemcpyHostToDevice));
    if (c->persistent) {
        TRY_CUDA(configure_persist(c->smem));
        c->pgrid = persist_grid(c->smem);
    }
    if (c->g_chunk) cudaGraphExecDestroy(c->g_chunk);
    if (c->g_one) cudaGraphExecDestroy(c->g_one);
    c->g_chunk = c->g_one = nullptr;
    evfdlb_status st = capture(c, 1, &c->g_one);
    if (st == EVFDLB_OK) st = capture(c, c->chunk, &c->g_chunk);
    return st;
}

evfdlb_status evfdlb_profile_stage(evfdlb_ctx* c, int32_t stage) {
    if (!c || stage < 0 || stage > 2) return EVFDLB_E_INVALID_ARG;
    if (c->c2) return EVFDLB_E_UNSUPPORTED;
    if (!c->have_state || c->poisoned) return EVFDLB_E_STATE;
    void *f0 = c->state[0], *f1 = c->state[1], *f2 = c->state[2];
    double *m0 = c->mom[0], *m1 = c->mom[1], *m2 = c->mom[2];
    if (stage == 0) queue_stage(c, c->user, f0, nullptr, f1, m0, m1, 0.0, 1.0);
    else if (stage == 1) queue_stage(c, c->user, f1, f0, f2, m1, m2, 0.75, 0.25);
    else queue_stage(c, c->user, f2, f0, f1, m2, m1, 1.0 / 3.0, 2.0 / 3.0);   // the state stays untouched
    TRY_CUDA(cudaGetLastError());
    return EVFDLB_OK;
}

evfdlb_status evfdlb_set_persistent(evfdlb_ctx* c, int32_t enable, int64_t spin_limit) {
    if (!c || (enable != 0 && enable != 1)) return EVFDLB_E_INVALID_ARG;
    if (c->c2) return EVFDLB_E_UNSUPPORTED;
    if (enable && (c->prec != EVFDLB_FP64 || c->df || c->iso || c->halo)) return EVFDLB_E_UNSUPPORTED;
    TRY_CUDA(cudaStreamSynchronize(c->user));
    if (enable && !c->pq) {
        TRY_CUDA(cudaMalloc((void**)&c->pq, sizeof(unsigned) * (2 + (size_t)c->nbatch)));
        TRY_CUDA(cudaMalloc((void**)&c->tiles_d, sizeof(int) * (size_t)c->nbatch));
        TRY_CUDA(cudaMemset(c->pq, 0, sizeof(unsigned) * (2 + (size_t)c->nbatch)));
        const unsigned open = 1u;
        TRY_CUDA(cudaMemcpy(c->pq + 1, &open, sizeof(unsigned), cudaMemcpyHostToDevice));
    }
    if (enable)
        TRY_CUDA(cudaMemcpy(c->tiles_d, c->tiles_h.data(), sizeof(int) * c->nbatch, cudaMemcpyHostToDevice));
    c->persistent = (enable == 1);
    // about a second of polling by default (each poll sleeps ~0.1 us)
    c->spin_limit = spin_limit > 0 ? spin_limit : (1LL << 23);
    if (c->persistent) {
        TRY_CUDA(configure_persist(c->smem));
        c->pgrid = persist_grid(c->smem);
    }
    if (c->g_chunk) cudaGraphExecDestroy(c->g_chunk);
    if (c->g_one) cudaGraphExecDestroy(c->g_one);
    c->g_chunk = c->g_one = nullptr;
    evfdlb_status st = capture(c, 1, &c->g_one);
    if (st == EVFDLB_OK) st = capture(c, c->chunk, &c->g_chunk);
    return st;
}

evfdlb_status evfdlb_debug_gate(evfdlb_ctx* c, int32_t open) {
    if (!c || (open != 0 && open != 1)) return EVFDLB_E_INVALID_ARG;
    if (!c->pq) return EVFDLB_E_STATE;
    const unsigned v = (unsigned)open;
    TRY_CUDA(cudaStreamSynchronize(c->user));
    TRY_CUDA(cudaMemcpy(c->pq + 1, &v, sizeof(unsigned), cudaMemcpyHostToDevice));
    return EVFDLB_OK;
}

int32_t evfdlb_halo_width(const evfdlb_params* p) {
    if (!p || p->dim != 1 || !validate(*p, nullptr)) return -1;
    return halo_width(*p);
}

int64_t evfdlb_halo_len(const evfdlb_ctx* c) {
    return (c && c->halo) ? halo_message_len(c->params[0].Q, c->halo_G) : 0;
}

evfdlb_status evfdlb_stage(evfdlb_ctx* c, int32_t stage) {
    if (!c || stage < 0 || stage > 2) return EVFDLB_E_INVALID_ARG;
    if (c->c2 || c->ckpt_every > 0) return EVFDLB_E_UNSUPPORTED;
    if (!c->have_state || c->poisoned || stage != c->rk_next) return EVFDLB_E_STATE;
    void *f0 = c->state[0], *f1 = c->state[1], *f2 = c->state[2];
    double *m0 = c->mom[0], *m1 = c->mom[1], *m2 = c->mom[2];
    // the three stages of queue_step, one per call
    if (stage == 0) queue_stage(c, c->user, f0, nullptr, f1, m0, m1, 0.0, 1.0);
    else if (stage == 1) queue_stage(c, c->user, f1, f0, f2, m1, m2, 0.75, 0.25);
    else {
        queue_stage(c, c->user, f2, f0, f0, m2, m0, 1.0 / 3.0, 2.0 / 3.0);
        if (c->iso)
            launch_iso_reset_p(c->prec, (int)c->items_h.size(), c->smem, c->user, c->slabs, c->items, c->tables,
                               c->rtables, f0, m0, c->NF, c->NN, c->Z);
        ++c->steps;
    }
    TRY_CUDA(cudaGetLastError());
    c->rk_next = (stage + 1) % 3;
    return EVFDLB_OK;
}

evfdlb_status evfdlb_halo_pack(evfdlb_ctx* c, double* to_left, double* to_right) {
    if (!c) return EVFDLB_E_INVALID_ARG;
    if (!c->halo) return EVFDLB_E_UNSUPPORTED;
    if ((c->halo_lo && !to_left) || (c->halo_hi && !to_right)) return EVFDLB_E_INVALID_ARG;
    if (!c->have_state || c->poisoned) return EVFDLB_E_STATE;
    const int b = c->rk_next;   // the buffers the next stage reads
    launch_halo_pack(c->prec, c->user, c->state[b], c->mom[b], c->NF, c->NN, c->params[0].nx, c->params[0].Q,
                     c->halo_G, c->halo_lo, c->halo_hi, to_left, to_right);
    TRY_CUDA(cudaGetLastError());
    return EVFDLB_OK;
}

evfdlb_status evfdlb_halo_unpack(evfdlb_ctx* c, const double* from_left, const double* from_right) {
    if (!c) return EVFDLB_E_INVALID_ARG;
    if (!c->halo) return EVFDLB_E_UNSUPPORTED;
    if ((c->halo_lo && !from_left) || (c->halo_hi && !from_right)) return EVFDLB_E_INVALID_ARG;
    if (!c->have_state || c->poisoned) return EVFDLB_E_STATE;
    const int b = c->rk_next;
    launch_halo_unpack(c->prec, c->user, c->state[b], c->mom[b], c->NF, c->NN, c->params[0].nx, c->params[0].Q,
                       c->halo_G, c->halo_lo, c->halo_hi, from_left, from_right);
    TRY_CUDA(cudaGetLastError());
    return EVFDLB_OK;
}

evfdlb_status evfdlb_rhs_vjp(evfdlb_ctx* c, const double* WF, const double* WG, int32_t on_device, double* outF,
                             double* outG, double* dphi) {
    if (!c || !WF || !WG || !outF || !outG) return EVFDLB_E_INVALID_ARG;
    if (c->c2) return EVFDLB_E_UNSUPPORTED;
    if (!c->have_state) return EVFDLB_E_STATE;
    evfdlb_status st = adjoint_supported(c);
    if (st != EVFDLB_OK) return st;
    if ((st = ensure_adjoint_buffers(c)) != EVFDLB_OK) return st;
    size_t bytes = sizeof(double) * c->NF;
    const AdjBuf a = adj_buf(c);
    double* w = a.y1;
    double* o = a.lam;
    if ((st = copy_in(c, w, WF, bytes, on_device)) != EVFDLB_OK) return st;
    if ((st = copy_in(c, w + c->NF, WG, bytes, on_device)) != EVFDLB_OK) return st;
    TRY_CUDA(cudaMemsetAsync(a.phis, 0, sizeof(double) * c->NN, c->user));
    // the node fields of the state, then one transposed right-hand side
    launch_fields_p(EVFDLB_FP64, (int)c->items_h.size(), c->smem, c->user, c->slabs, c->items, c->tables, c->taps,
                    c->taps, c->mom[0], a.fld, c->NN, c->Z, c->err);
    adj_stage(c, (const double*)c->state[0], a.fld, c->mom[0], w, nullptr, nullptr, o, 0.0, 1.0, 0, 0.0, 0.0, 0.0);
    launch_adj_phi(c->nbatch, c->user, c->slabs, a.phis, a.phi, a.dphi);
    TRY_CUDA(cudaGetLastError());
    if ((st = copy_out(c, outF, o, bytes, on_device)) != EVFDLB_OK) return st;
    if ((st = copy_out(c, outG, o + c->NF, bytes, on_device)) != EVFDLB_OK) return st;
    if (dphi) TRY_CUDA(cudaMemcpyAsync(dphi, a.dphi, sizeof(double) * c->nbatch, cudaMemcpyDeviceToHost, c->user));
    return check_device(c);
}

evfdlb_status evfdlb_adjoint_state(evfdlb_ctx* c, const double* barF, const double* barG, int32_t on_device,
                                   double* dL_dphi_a, double* dL_dF0, double* dL_dG0, double* dL_dn0,
                                   double* dL_du0, double* dL_dT0) {
    if (!c || !barF || !barG) return EVFDLB_E_INVALID_ARG;
    if (c->c2) return EVFDLB_E_UNSUPPORTED;
    if (!c->have_state || c->poisoned || c->ckpt_every <= 0) return EVFDLB_E_STATE;
    if ((dL_dn0 || dL_du0 || dL_dT0) && !c->origin_init) return EVFDLB_E_STATE;
    evfdlb_status st = adjoint_supported(c);
    if (st != EVFDLB_OK) return st;
    if ((st = ensure_adjoint_buffers(c)) != EVFDLB_OK) return st;
    const long long NF = c->NF, NN = c->NN;
    const size_t sbytes = sizeof(double) * NF;
    const AdjBuf a = adj_buf(c);
    double *lam = a.lam, *y1 = a.y1, *y2 = a.y2, *acc = a.acc, *phis = a.phis;
    if ((st = copy_in(c, lam, barF, sbytes, on_device)) != EVFDLB_OK) return st;
    if ((st = copy_in(c, lam + NF, barG, sbytes, on_device)) != EVFDLB_OK) return st;
    TRY_CUDA(cudaMemsetAsync(phis, 0, sizeof(double) * NN, c->user));
    const int K = c->ckpt_every;
    const size_t nst = 3 * (size_t)K + 1;
    const int n = (int)c->items_h.size();
    const int64_t nseg = (c->steps + K - 1) / K;
    // Segments are swept last to first.  The recompute of segment sg - 1
    // (from its checkpoint, on the aux stream, into the other segment buffer)
    // runs while the user stream sweeps segment sg; the buffer is reused once
    // the sweep of segment sg + 1 has finished with it.  Every kernel computes
    // the same values as in a serial order: the overlap changes no result.
    auto segp = [&](int64_t sg) { return c->seg[sg & 1]; };
    // slot j of a segment buffer: state, raw moment sums, node fields
    auto sst_of = [&](double* base, size_t j) { return base + j * 2 * NF; };
    auto smo_of = [&](double* base, size_t j) { return base + nst * 2 * NF + j * kNumMoments * NN; };
    auto sfl_of = [&](double* base, size_t j) {
        return base + nst * (2 * NF + kNumMoments * NN) + j * EVFDLB_NFIELDS * NN;
    };
    // the recompute of a segment from its checkpoint; every stage also
    // stores the node fields of its input for the sweep
    auto recompute = [&](int64_t sg) -> cudaError_t {
        double* base = segp(sg);
        auto sst = [&](size_t j) { return sst_of(base, j); };
        auto smo = [&](size_t j) { return smo_of(base, j); };
        const int ns = (int)std::min<int64_t>(K, c->steps - sg * K);
        cudaError_t e = cudaMemcpyAsync(sst(0), c->ckpts[sg], sizeof(double) * 2 * NF, cudaMemcpyDeviceToDevice, c->aux);
        if (e != cudaSuccess) return e;
        launch_sums_p(EVFDLB_FP64, n, c->aux, c->slabs, c->items, c->tables, c->tables, sst(0), smo(0), NF, NN, c->err);
        auto stage = [&](size_t j, const double* sbase, double alpha, double beta) {
            launch_stage_fields(n, c->smem, c->aux, c->slabs, c->items, c->tables, c->taps, sst(j), sbase, sst(j + 1),
                                smo(j), smo(j + 1), sfl_of(base, j), NF, NN, alpha, beta, c->Z, c->err);
        };
        for (int t = 0; t < ns; ++t) {
            size_t b = 3 * (size_t)t;
            stage(b, nullptr, 0.0, 1.0);
            stage(b + 1, sst(b), 0.75, 0.25);
            stage(b + 2, sst(b), 1.0 / 3.0, 2.0 / 3.0);
        }
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventRecord(c->ev_rec[sg & 1], c->aux);
        return e;
    };
    TRY_CUDA(cudaEventRecord(c->ev_fork, c->user));      // the checkpoints and lam are ready
    TRY_CUDA(cudaStreamWaitEvent(c->aux, c->ev_fork, 0));
    TRY_CUDA(recompute(nseg - 1));
    for (int64_t sg = nseg - 1; sg >= 0; --sg) {
        if (sg >= 1) {
            if (sg + 1 <= nseg - 1) TRY_CUDA(cudaStreamWaitEvent(c->aux, c->ev_sweep[(sg + 1) & 1], 0));
            TRY_CUDA(recompute(sg - 1));
        }
        TRY_CUDA(cudaStreamWaitEvent(c->user, c->ev_rec[sg & 1], 0));
        double* base = segp(sg);
        auto sstate = [&](size_t j) { return sst_of(base, j); };
        auto smom = [&](size_t j) { return smo_of(base, j); };
        auto sfld = [&](size_t j) { return sfl_of(base, j); };
        const int ns = (int)std::min<int64_t>(K, c->steps - sg * K);
        // reverse sweep of the segment (Shu-Osher stages in reverse order):
        //   y2  = 2/3 lam + J(u2)^T (2/3 dt lam),   acc = 1/3 lam
        //   y1  = 1/4 y2  + J(u1)^T (1/4 dt y2),    acc += 3/4 y2
        //   lam = y1 + J(u)^T (dt y1) + acc
        for (int t = ns - 1; t >= 0; --t) {
            size_t b = 3 * (size_t)t;
            adj_stage(c, sstate(b + 2), sfld(b + 2), smom(b + 2), lam, nullptr, acc, y2, 2.0 / 3.0, 2.0 / 3.0, 1,
                      0.0, 0.0, 1.0 / 3.0);
            adj_stage(c, sstate(b + 1), sfld(b + 1), smom(b + 1), y2, acc, acc, y1, 0.25, 0.25, 1, 0.0, 1.0, 0.75);
            adj_stage(c, sstate(b), sfld(b), smom(b), y1, acc, nullptr, lam, 1.0, 1.0, 1, 1.0, 0.0, 0.0);
        }
        TRY_CUDA(cudaGetLastError());
        TRY_CUDA(cudaEventRecord(c->ev_sweep[sg & 1], c->user));
    }
    evfdlb_status s2;
    if (dL_dF0 && (s2 = copy_out(c, dL_dF0, lam, sbytes, on_device)) != EVFDLB_OK) return s2;
    if (dL_dG0 && (s2 = copy_out(c, dL_dG0, lam + NF, sbytes, on_device)) != EVFDLB_OK) return s2;
    if (dL_dn0 || dL_du0 || dL_dT0) {
        double* f = y1;   // [3][NN] fits in the y1 slot (2 NF >= 3 NN for Q >= 2)
        launch_adj_init(n, c->user, c->slabs, c->items, c->tables, c->init_fields, lam, f, f + NN, f + 2 * NN, NF, NN);
        TRY_CUDA(cudaGetLastError());
        size_t nb = sizeof(double) * NN;
        if (dL_dn0 && (s2 = copy_out(c, dL_dn0, f, nb, on_device)) != EVFDLB_OK) return s2;
        if (dL_du0 && (s2 = copy_out(c, dL_du0, f + NN, nb, on_device)) != EVFDLB_OK) return s2;
        if (dL_dT0 && (s2 = copy_out(c, dL_dT0, f + 2 * NN, nb, on_device)) != EVFDLB_OK) return s2;
    }
    if (dL_dphi_a) {
        launch_adj_phi(c->nbatch, c->user, c->slabs, phis, a.phi, a.dphi);
        TRY_CUDA(cudaGetLastError());
        TRY_CUDA(cudaMemcpyAsync(dL_dphi_a, a.dphi, sizeof(double) * c->nbatch, cudaMemcpyDeviceToHost, c->user));
    }
    return check_device(c);
}

evfdlb_status evfdlb_adjoint(evfdlb_ctx* c, const double* dL_dn_end, int32_t on_device, double* dL_dphi_a,
                             double* dL_dT0, double* dL_dn0) {
    if (!c || !dL_dn_end) return EVFDLB_E_INVALID_ARG;
    if (c->c2) return EVFDLB_E_UNSUPPORTED;
    if (!c->have_state) return EVFDLB_E_STATE;
    // n = sum_k F_k, so dL/dF_k = dL/dn for every k and dL/dG = 0: the
    // cotangent is formed on the device, in the scratch block [2 NF]
    const double* g = dL_dn_end;
    if (!on_device) {
        double* gd = c->scratch + 2 * c->NF;     // [NN] after the cotangent (scratch holds 2 NF + 16 NN)
        evfdlb_status s = copy_in(c, gd, dL_dn_end, sizeof(double) * c->NN, 0);
        if (s != EVFDLB_OK) return s;
        g = gd;
    }
    launch_adj_seed((int)c->items_h.size(), c->user, c->slabs, c->items, g, c->scratch, c->scratch + c->NF, c->NF);
    TRY_CUDA(cudaGetLastError());
    // host outputs pass through device homes in the scratch block
    double* tn = c->scratch + 2 * c->NF + c->NN;
    double* tT = tn + c->NN;
    double* on = dL_dn0 ? (on_device ? dL_dn0 : tn) : nullptr;
    double* oT = dL_dT0 ? (on_device ? dL_dT0 : tT) : nullptr;
    evfdlb_status s = evfdlb_adjoint_state(c, c->scratch, c->scratch + c->NF, 1, dL_dphi_a, nullptr, nullptr, on,
                                           nullptr, oT);
    if (s != EVFDLB_OK || on_device) return s;
    const size_t nb = sizeof(double) * c->NN;
    if (dL_dn0 && (s = copy_out(c, dL_dn0, tn, nb, 0)) != EVFDLB_OK) return s;
    if (dL_dT0 && (s = copy_out(c, dL_dT0, tT, nb, 0)) != EVFDLB_OK) return s;
    TRY_CUDA(cudaStreamSynchronize(c->user));
    return EVFDLB_OK;
}

}  // extern "C"
