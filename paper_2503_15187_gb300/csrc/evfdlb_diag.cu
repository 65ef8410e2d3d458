// evfdlb_diag.cu -- measurement and self-test entry points of libevfdlb:
// the FP64 fused multiply-add throughput of the device (the denominator of
// the roofline of the FP64 step, which is bound by that pipe), and the
// library's FP64 quotient (div_nr of evfdlb_device.cuh) evaluated on caller
// arrays beside the IEEE quotient, so that its error bound can be tested.
#include <cuda_runtime.h>

#include "evfdlb_device.cuh"

namespace evfdlb {
namespace {

constexpr int kProbeChains = 8;      // independent FMA chains per thread
constexpr int kProbeThreads = 256;

// kProbeChains independent dependency chains a <- a b + c per thread; the
// values stay bounded (|b| < 1) and finite, and the conditional store keeps
// the chains live without writing in practice.
__global__ void __launch_bounds__(kProbeThreads) dfma_probe_kernel(double* sink, int iters, double b, double c) {
    double a[kProbeChains];
#pragma unroll
    for (int j = 0; j < kProbeChains; ++j) a[j] = 1.0 + 1e-3 * (threadIdx.x + j);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < kProbeChains; ++j) a[j] = fma(a[j], b, c);
    }
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < kProbeChains; ++j) s += a[j];
    if (s == -1.0) sink[blockIdx.x] = s;
}

__global__ void divide_kernel(const double* __restrict__ a, const double* __restrict__ b, double* __restrict__ q,
                              double* __restrict__ q_ieee, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        q[i] = div_nr(a[i], b[i]);
        if (q_ieee) q_ieee[i] = a[i] / b[i];
    }
}

evfdlb_status st_of(cudaError_t e) {
    return e == cudaSuccess ? EVFDLB_OK : (e == cudaErrorMemoryAllocation ? EVFDLB_E_OOM : EVFDLB_E_CUDA);
}

}  // namespace
}  // namespace evfdlb

using namespace evfdlb;

extern "C" evfdlb_status evfdlb_probe_fp64_fma(int32_t reps, void* cuda_stream, double* gflops) {
    if (!gflops || reps < 1) return EVFDLB_E_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return st_of(e);
    if (sms < 1) sms = 1;
    const int blocks = sms * 8, iters = 4096;
    // the sink is never written (see the kernel): a null pointer would do,
    // but a kernel argument that is never dereferenced needs no allocation
    double* sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    double best = 0.0;
    for (int r = 0; e == cudaSuccess && r <= reps; ++r) {   // r = 0: warm-up
        e = cudaEventRecord(e0, st);
        dfma_probe_kernel<<<blocks, kProbeThreads, 0, st>>>(sink, iters, 0.9999999, 1e-7);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && r > 0 && ms > 0.f) {
            const double flops = 2.0 * kProbeChains * (double)iters * kProbeThreads * blocks;
            const double g = flops / (ms * 1e-3) / 1e9;
            if (g > best) best = g;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) return st_of(e);
    *gflops = best;
    return EVFDLB_OK;
}

extern "C" evfdlb_status evfdlb_divide_fp64(const double* a, const double* b, double* q, double* q_ieee, int64_t n,
                                            void* cuda_stream) {
    if (n < 0 || (n > 0 && (!a || !b || !q))) return EVFDLB_E_INVALID_ARG;
    if (n == 0) return EVFDLB_OK;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const int blocks = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
    divide_kernel<<<blocks, 256, 0, st>>>(a, b, q, q_ieee, n);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return st_of(e);
}
