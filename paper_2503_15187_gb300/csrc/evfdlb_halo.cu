// evfdlb_halo.cu -- halo messages of a z-split slab (EVFDLB_BC_HALO).
//
// The method is an explicit stencil in z: one RK stage of a node reads F and
// G over +-3 nodes (the WENO-5 face fluxes, Sec. III) and the density sums
// over +-M nodes (the Eq. (F1) force and energy taps, the Fischer-Methfessel
// average), and the velocity moments S1, S2, G0 over +-2.  A rank that owns
// the interior nodes [G, nx - G) of its slab therefore needs, before every
// stage, the last 3 F, G columns and the last G moment columns of each
// neighbour.  (The first / last part of a split outflow slab has no ghost
// band at its outer end, which is the slab's boundary: that side sends and
// receives nothing.)  One message per side carries exactly those:
//   [ (d Q + k) 3 + c ]            F (d = 0) and G (d = 1), k < Q, c < 3
//   [ 6 Q + kind G + c ]           moment sums, kind < kNumMoments, c < G
// in FP64 whatever the state precision (an FP32 state widens exactly and
// narrows back exactly).
#include <cuda_runtime.h>

#include "evfdlb_internal.h"

namespace evfdlb {
namespace {

constexpr int kHaloThreads = 256;

// side 0: the left edge (message to the left neighbour / from it), side 1:
// the right edge; lo / hi: ghost nodes below / above the interior (G, or 0
// for an outflow end, whose side is skipped).  pack: interior columns ->
// message; unpack: message -> ghost columns.
template <typename R, bool PACK>
__global__ void __launch_bounds__(kHaloThreads)
halo_kernel(R* state, double* mom, long long NF, long long NN, int nx, int Q, int G, int lo, int hi, double* msg0,
            double* msg1, const double* in0, const double* in1) {
    const int side = blockIdx.y;
    if ((side == 0 ? lo : hi) == 0) return;
    const int nf = 6 * Q, len = nf + kNumMoments * G;
    // first F/G column and first moment column of this side's block
    int cF, cM;
    if (PACK) {
        cF = side == 0 ? lo : nx - hi - 3;
        cM = side == 0 ? lo : nx - hi - G;
    } else {
        cF = side == 0 ? lo - 3 : nx - hi;
        cM = side == 0 ? lo - G : nx - hi;
    }
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < len; e += gridDim.x * blockDim.x) {
        if (e < nf) {
            const int c = e % 3, r = e / 3;   // r = d Q + k
            const int d = r / Q, k = r % Q;
            R* p = state + d * NF + (long long)k * nx + cF + c;
            if (PACK) (side == 0 ? msg0 : msg1)[e] = (double)*p;
            else *p = (R)(side == 0 ? in0 : in1)[e];
        } else {
            const int c = (e - nf) % G, kind = (e - nf) / G;
            double* p = mom + kind * NN + cM + c;
            if (PACK) (side == 0 ? msg0 : msg1)[e] = *p;
            else *p = (side == 0 ? in0 : in1)[e];
        }
    }
}

template <typename R, bool PACK>
void launch_halo_t(cudaStream_t st, void* state, double* mom, long long NF, long long NN, int nx, int Q, int G, int lo,
                   int hi, double* m0, double* m1, const double* i0, const double* i1) {
    const int len = 6 * Q + kNumMoments * G;
    dim3 grid((len + kHaloThreads - 1) / kHaloThreads, 2);
    halo_kernel<R, PACK><<<grid, kHaloThreads, 0, st>>>((R*)state, mom, NF, NN, nx, Q, G, lo, hi, m0, m1, i0, i1);
}

}  // namespace

long long halo_message_len(int Q, int G) { return 6LL * Q + (long long)kNumMoments * G; }

void launch_halo_pack(int prec, cudaStream_t st, const void* state, const double* mom, long long NF, long long NN,
                      int nx, int Q, int G, int lo, int hi, double* to_left, double* to_right) {
    if (prec == EVFDLB_FP32)
        launch_halo_t<float, true>(st, const_cast<void*>(state), const_cast<double*>(mom), NF, NN, nx, Q, G, lo, hi, to_left,
                                   to_right, nullptr, nullptr);
    else
        launch_halo_t<double, true>(st, const_cast<void*>(state), const_cast<double*>(mom), NF, NN, nx, Q, G, lo, hi, to_left,
                                    to_right, nullptr, nullptr);
}

void launch_halo_unpack(int prec, cudaStream_t st, void* state, double* mom, long long NF, long long NN, int nx, int Q,
                        int G, int lo, int hi, const double* from_left, const double* from_right) {
    if (prec == EVFDLB_FP32)
        launch_halo_t<float, false>(st, state, mom, NF, NN, nx, Q, G, lo, hi, nullptr, nullptr, from_left, from_right);
    else
        launch_halo_t<double, false>(st, state, mom, NF, NN, nx, Q, G, lo, hi, nullptr, nullptr, from_left, from_right);
}

}  // namespace evfdlb
