// evfdlb_static.cu -- evfdlb_step_static: the time step for callers that
// cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: a plugin whose host application owns
// all device memory through its own pool and hands out only pointers, a
// process held to a device-memory budget fixed at start-up, and latency-bound
// loops in which cudaMalloc / cudaFree may synchronise the device.  For them
// this entry point advances a caller-owned state with all of its working
// memory (the two intermediate Runge-Kutta stages, the moment sums, the
// velocity tables, the taps, the work list and the error word) in one
// file-scope __device__ array of fixed size.  Every GPU that loads the
// library holds that array (about 3.4 MiB) until the process exits.
//
// The state buffer, the only data the caller passes, is advanced in place.
// Calls share the array, so calls that overlap on the GPU race.  The mutex
// below is held for a whole call, through its final stream synchronisation,
// so calls from different host threads of one process are serialised; calls
// from different processes, or work the caller queues on other streams
// against the same state, are not.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <mutex>

#include "evfdlb_internal.h"

namespace evfdlb {
size_t stage_smem_bytes(int Q, int Z, int M);
cudaError_t ensure_stage_smem(size_t smem_bytes);
void launch_stage(int nitems, size_t smem, cudaStream_t st, const SlabDesc* slabs, const WorkItem* items,
                  const double* tables, const double* taps, const double* src, const double* base,
                  double* out, const double* mom_in, double* mom_out, long long NF, long long NN,
                  double alpha, double beta, int mode, int Z, unsigned* err);
void launch_iso_reset_p(int prec, int nitems, size_t smem, cudaStream_t st, const SlabDesc* slabs,
                        const WorkItem* items, const double* tables, const void* rtab, void* state, double* mom,
                        long long NF, long long NN, int Z);
void launch_sums(int nitems, cudaStream_t st, const SlabDesc* slabs, const WorkItem* items,
                 const double* tables, const double* state, double* mom, long long NF, long long NN,
                 unsigned* err);
}  // namespace evfdlb

using namespace evfdlb;

namespace {

// Limits of the static working memory.
constexpr long long kMaxElems = EVFDLB_STATIC_MAX_ELEMENTS;  // Q * nx
constexpr int kMaxNodes = EVFDLB_STATIC_MAX_NODES;           // nx
constexpr int kMaxHalfWidth = EVFDLB_STATIC_MAX_HALFWIDTH;   // force tap half-width
constexpr int kMaxTaps = 3 * (2 * kMaxHalfWidth + 1);         // force, FM (m <= M), energy
constexpr int kTableDoubles = 7 * kQMax + 4 * kQMax * kQMax; // >= TableLayout(Q).total, Q <= 32
constexpr int kDescDoubles = (sizeof(SlabDesc) + 7) / 8;
constexpr int kItemDoubles = (sizeof(WorkItem) + 7) / 8;

// Layout of the array, in doubles.
constexpr long long kOffU1 = 0;
constexpr long long kOffU2 = kOffU1 + 2 * kMaxElems;
constexpr long long kOffMom = kOffU2 + 2 * kMaxElems;                 // 3 x [6][kMaxNodes]
constexpr long long kOffTab = kOffMom + 3LL * kNumMoments * kMaxNodes;
constexpr long long kOffTaps = kOffTab + kTableDoubles;
constexpr long long kOffDesc = kOffTaps + kMaxTaps;
constexpr long long kOffItems = kOffDesc + kDescDoubles;
constexpr long long kOffErr = kOffItems + (long long)kItemDoubles * kMaxNodes;
constexpr long long kTotal = kOffErr + 32;   // keeps the error word 256-byte padded

__device__ __align__(256) double g_static_scratch[kTotal];

// Device address of g_static_scratch per device, looked up once per device.
constexpr int kMaxDevices = 64;
double* g_dev_ptr[kMaxDevices] = {nullptr};
std::mutex g_mutex;

// Host staging (static, so that no host heap is used either).
double h_tables[kTableDoubles];
double h_taps[kMaxTaps];
SlabDesc h_desc;
WorkItem h_items[kMaxNodes];

evfdlb_status st_of(cudaError_t e) {
    return e == cudaSuccess ? EVFDLB_OK : (e == cudaErrorMemoryAllocation ? EVFDLB_E_OOM : EVFDLB_E_CUDA);
}

}  // namespace

extern "C" evfdlb_status evfdlb_step_static(const evfdlb_params* p, double* state, int64_t nsteps,
                                            void* cuda_stream) {
    if (!p || !state || nsteps < 0) return EVFDLB_E_INVALID_ARG;
    if (!validate(*p, nullptr)) return EVFDLB_E_INVALID_ARG;
    if (p->precision != EVFDLB_FP64) return EVFDLB_E_UNSUPPORTED;
    if (p->bc == EVFDLB_BC_HALO) return EVFDLB_E_UNSUPPORTED;   // needs a halo exchange between stages
    if (p->nx > kMaxNodes || (long long)p->Q * p->nx > kMaxElems) return EVFDLB_E_INVALID_ARG;
    const int M = force_halfwidth(*p);
    if (M > kMaxHalfWidth) return EVFDLB_E_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)cuda_stream;

    std::lock_guard<std::mutex> lock(g_mutex);
    // an error left pending by earlier, unrelated work of this host thread
    // is reported as it stands (not cleared) before anything is queued, so
    // that it is not mistaken for a failure of this call's launches
    cudaError_t pending = cudaPeekAtLastError();
    if (pending != cudaSuccess) return st_of(pending);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return EVFDLB_E_CUDA;
    int sms = 1;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms < 1) sms = 1;
    const int Z = (int)fmin(fmax(ceil((double)p->nx / sms), 1.0), (double)kZMax);
    if (!g_dev_ptr[dev]) {
        // once per device, with that device current: the device address of
        // the array (host code cannot use the symbol itself)
        void* addr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&addr, g_static_scratch);
        if (e != cudaSuccess || !addr) return EVFDLB_E_CUDA;
        g_dev_ptr[dev] = (double*)addr;
    }
    // the stage kernel's shared-memory limit must cover this call's tile;
    // it is only ever raised, so contexts keep what they configured
    cudaError_t ce = ensure_stage_smem(stage_smem_bytes(p->Q, Z, M));
    if (ce != cudaSuccess) return st_of(ce);
    double* base = g_dev_ptr[dev];
    double* u1 = base + kOffU1;
    double* u2 = base + kOffU2;
    double* mom[3] = {base + kOffMom, base + kOffMom + kNumMoments * (long long)kMaxNodes,
                      base + kOffMom + 2LL * kNumMoments * kMaxNodes};
    double* tables = base + kOffTab;
    double* taps = base + kOffTaps;
    SlabDesc* desc = (SlabDesc*)(base + kOffDesc);
    WorkItem* items = (WorkItem*)(base + kOffItems);
    unsigned* err = (unsigned*)(base + kOffErr);

    // tables, taps, slab descriptor and work list of this call
    double xi[kQMax], w[kQMax];
    if (!velocity_set(p->Q, xi, w)) return EVFDLB_E_INVALID_ARG;
    build_tables(p->Q, xi, w, h_tables);
    int ntaps = fill_taps(*p, h_taps, kMaxTaps);
    if (ntaps < 0) return EVFDLB_E_INVALID_ARG;
    memset(&h_desc, 0, sizeof(h_desc));
    h_desc.nx = p->nx;
    h_desc.Q = p->Q;
    h_desc.bc = p->bc;
    h_desc.relax = p->relax_mode;
    h_desc.M = M;
    h_desc.m = tap_halfwidth(p->sigma, p->dx);
    h_desc.dx = p->dx;
    h_desc.inv_dx = 1.0 / p->dx;
    h_desc.dt = p->dt > 0 ? p->dt : p->cfl * p->dx / fabs(xi[p->Q - 1]);
    h_desc.weno_eps = p->weno_eps;
    h_desc.b = 2.0 * M_PI * p->sigma * p->sigma * p->sigma / 3.0;
    h_desc.eta_coef = M_PI * p->sigma * p->sigma * p->sigma / 6.0;
    h_desc.T_iso = p->T_iso;
    h_desc.mu0_coef = 5.0 / (16.0 * p->sigma * p->sigma * sqrt(M_PI));
    int nitems = 0;
    for (int i0 = 0; i0 < p->nx; i0 += Z) h_items[nitems++] = WorkItem{0, i0, (p->nx - i0) < Z ? p->nx - i0 : Z, 0};
    TableLayout L(p->Q);
    cudaError_t e = cudaMemcpyAsync(tables, h_tables, sizeof(double) * L.total, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(taps, h_taps, sizeof(double) * ntaps, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(desc, &h_desc, sizeof(SlabDesc), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(items, h_items, sizeof(WorkItem) * nitems, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(unsigned), st);   // starts every call at zero
    if (e != cudaSuccess) return st_of(e);

    const long long NF = (long long)p->Q * p->nx, NN = p->nx;
    const size_t smem = stage_smem_bytes(p->Q, Z, M);
    // the moments of the caller's state, then Shu-Osher stages as in evfdlb_step
    launch_sums(nitems, st, desc, items, tables, state, mom[0], NF, NN, err);
    for (int64_t s = 0; s < nsteps; ++s) {
        launch_stage(nitems, smem, st, desc, items, tables, taps, state, nullptr, u1, mom[0], mom[1], NF, NN,
                     0.0, 1.0, 0, Z, err);
        launch_stage(nitems, smem, st, desc, items, tables, taps, u1, state, u2, mom[1], mom[2], NF, NN, 0.75,
                     0.25, 0, Z, err);
        launch_stage(nitems, smem, st, desc, items, tables, taps, u2, state, state, mom[2], mom[0], NF, NN,
                     1.0 / 3.0, 2.0 / 3.0, 0, Z, err);
        if (p->T_iso > 0.0)
            launch_iso_reset_p(EVFDLB_FP64, nitems, smem, st, desc, items, tables, tables, state, mom[0], NF, NN, Z);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return st_of(e);
    unsigned h_err = 0;
    e = cudaMemcpyAsync(&h_err, err, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return st_of(e);
    if (h_err) return (h_err & ERR_NONFINITE) ? EVFDLB_E_NONFINITE : EVFDLB_E_NEGATIVE;
    return EVFDLB_OK;
}
