// evfdlb_device.cuh -- device-side building blocks of the EV1 right-hand side
// shared by the forward kernels (evfdlb_kernels.cu) and the adjoint kernels
// (evfdlb_adjoint.cu): boundary indexing, the shared-memory layout of a node
// tile, staging of node inputs and of the state tile, the node fields
// (Fischer-Methfessel average, chi, gradients, force, transport), the
// recurrence form of the equilibrium coefficients, the Hermite analysis, the
// WENO-5 faces, the force term and the raw moment sums.  Not part of the
// public interface.
#pragma once

#include <cuda_runtime.h>
#include <math.h>

#include <type_traits>
#include <utility>

#include "evfdlb_internal.h"

namespace evfdlb {

// Launches a kernel as a programmatic dependent of the kernel before it in
// the stream: its CTAs may be scheduled once every CTA of that kernel has
// reached griddepcontrol.launch_dependents (or exited), and stage what no
// kernel writes; griddepcontrol.wait in the kernel holds back everything
// that reads the previous kernel's results until it has completed.  Only
// for launches whose stream predecessor is a kernel (not an event wait).
// Launch errors are left for cudaGetLastError, as with <<<>>>.
template <typename... P, typename... A>
inline void launch_pdl(void (*k)(P...), int grid, int threads, size_t smem, cudaStream_t st, A&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    (void)cudaLaunchKernelEx(&cfg, k, std::forward<A>(args)...);
}

__device__ __forceinline__ int gidx(int i, int nx, int bc) {
    if (bc == EVFDLB_BC_PERIODIC) {
        int r = i % nx;
        return r < 0 ? r + nx : r;
    }
    return i < 0 ? 0 : (i >= nx ? nx - 1 : i);
}

// ---------------------------------------------------------------------------
// Shared-memory layout of one CTA, sized for (Q, Z, M): an FP64 block of node
// fields followed by an R block of velocity-space data.
// ---------------------------------------------------------------------------
template <typename R>
struct Smem {
    double *N;          // n on nodes [i0 - M, i0 + Z + M)
    double *U, *T;      // u, T on nodes [i0 - 2, i0 + Z + 2)
    double *X, *Chi;    // X = n^2 chi T and chi on the same nodes
    double *Sc;         // per-node scalars [kNumScalars][Z]
    double *Mtap;       // staged Fischer-Methfessel taps (2m+1 <= 2M+1)
    R *P, *S;           // analysis / synthesis tables [Q*Q] each
    R *Nr;              // n halo in R (the force convolution), aliases N for FP64
    R *Scr;             // nu and F1 in R, [2][Z]
    R *C;               // coefficients [2][Q][Z] (block of 4 H Z >= 2 Q Z values)
    R *A;               // analysis [2][Q][Z]
    R *F;               // state tile with halo [2][Q][Z+6]
    R *Face;            // WENO face values [2][Q][Z+1]
    R *Cc;              // per-node coefficient constants c0..c3 [2][4][Z]
    R *Ftap;            // staged force taps [2M+1] (padded to an even count)
    R *Mm;              // Hermite moments m_l of N(u, T) per node [Q][Z]
    double *Vp;         // velocity powers of the moment sums: xi, xi^2, xi^3 (FP64) [3Q]
    R *Vr;              //   and xi, xi^3 in R [2Q]
    R *EO;              // parity-split state tile [2][2][H][Z] (d, E/O), H = (Q+1)/2; it is
                        // read only before the coefficients are formed, so it shares
                        // their block; the FP64_DF kernel keeps its float-pair state
                        // tile there instead
    double *Mp64;       // FP32 state only: group terms of the FP64 moment sums [4][G][Z]
    R *Mp32;            //   and of the R ones [2][G][Z] (see pair_terms_f32)
};

// Length of the R copy of the density halo, rounded up to an even count so
// that the blocks after it stay 8-byte aligned (init_kernel stores doubles in
// the coefficient block).
__host__ __device__ inline size_t nr_len(int Z, int M) { return ((size_t)(Z + 2 * M) + 1) & ~(size_t)1; }

__host__ __device__ inline size_t ftap_len(int M) { return ((size_t)(2 * M + 1) + 1) & ~(size_t)1; }

// Groups of two velocity pairs in the FP32 moment sums (see moment_sum).
__host__ __device__ inline int pair_groups(int Q) { return ((Q + 1) / 2 + 1) / 2; }

// Q*Q rounded up to an even count, so that the table blocks stay aligned for
// two-wide (R2) loads.
__host__ __device__ inline size_t qq_len(int Q) { return ((size_t)Q * Q + 1) & ~(size_t)1; }

template <typename R>
__host__ __device__ inline size_t smem_bytes_t(int Q, int Z, int M) {
    // the FP64 block is padded to an even count (16-byte aligned R2 tables)
    size_t nd = (size_t)(Z + 2 * M) + 4 * (size_t)(Z + 4) + (size_t)kNumScalars * Z + (size_t)(2 * M + 1);
    nd = (nd + 1) & ~(size_t)1;
    size_t nr = 2 * qq_len(Q) + (std::is_same<R, double>::value ? 0 : nr_len(Z, M)) + 2 * (size_t)Z +
                4 * (size_t)((Q + 1) / 2) * Z + 2 * (size_t)Q * Z + 2 * (size_t)Q * (Z + 6) +
                2 * (size_t)Q * (Z + 1) + 8 * (size_t)Z + ftap_len(M) + (size_t)Q * Z;
    // + the velocity powers (3Q doubles, 2Q R) and one R of padding before them
    size_t bytes = (nd + 3 * (size_t)Q) * sizeof(double) + (nr + 2 * (size_t)Q + 1) * sizeof(R);
    // + the pair terms of the moment sums (FP32 state)
    if (std::is_same<R, float>::value) bytes += (size_t)pair_groups(Q) * Z * (4 * sizeof(double) + 2 * sizeof(R));
    return bytes;
}

template <typename R>
__device__ inline Smem<R> carve(double* base, int Q, int Z, int M) {
    Smem<R> s;
    s.N = base;
    s.U = s.N + (Z + 2 * M);
    s.T = s.U + (Z + 4);
    s.X = s.T + (Z + 4);
    s.Chi = s.X + (Z + 4);
    s.Sc = s.Chi + (Z + 4);
    s.Mtap = s.Sc + kNumScalars * Z;
    // Mtap holds 2m+1 <= 2M+1 taps; the FP64 block ends on an even count
    // (the dynamic shared memory starts 16-byte aligned)
    const size_t nd = ((size_t)(s.Mtap - base) + (2 * M + 1) + 1) & ~(size_t)1;
    R* r = reinterpret_cast<R*>(base + nd);
    s.P = r;
    s.S = s.P + qq_len(Q);
    if constexpr (std::is_same<R, double>::value) {
        s.Nr = s.N;
        s.Scr = s.S + qq_len(Q);
    } else {
        s.Nr = s.S + qq_len(Q);
        s.Scr = s.Nr + nr_len(Z, M);
    }
    s.C = s.Scr + 2 * Z;
    s.EO = s.C;
    s.A = s.C + 4 * ((Q + 1) / 2) * Z;
    s.F = s.A + 2 * Q * Z;
    s.Face = s.F + 2 * Q * (Z + 6);
    s.Cc = s.Face + 2 * Q * (Z + 1);
    s.Ftap = s.Cc + 8 * Z;
    s.Mm = s.Ftap + ftap_len(M);
    // the velocity powers close the layout: FP64 first (the R block ends on
    // an even count of doubles' worth: all its segment lengths are even)
    s.Vp = reinterpret_cast<double*>(s.Mm + (size_t)Q * Z + ((size_t)Q * Z) % 2);
    s.Vr = reinterpret_cast<R*>(s.Vp + 3 * Q);
    // Vr ends 8-byte aligned (2Q R values after an aligned block)
    s.Mp64 = reinterpret_cast<double*>(s.Vr + 2 * Q);
    s.Mp32 = reinterpret_cast<R*>(s.Mp64 + 4 * (size_t)pair_groups(Q) * Z);
    return s;
}

enum { SC_N = 0, SC_U, SC_T, SC_NU, SC_FORCE, SC_KQ, SC_K, SC_A, SC_B, SC_D };

// IEEE tests by the bit pattern: integer operations, not the FP64 pipe
// (whose compares sit on the node chain's critical path).
__device__ __forceinline__ bool finite(double x) {
    return ((unsigned long long)__double_as_longlong(x) & 0x7ff0000000000000ull) != 0x7ff0000000000000ull;
}
// x > 0: false for +-0, negatives and NaN, true for +inf
__device__ __forceinline__ bool positive(double x) {
    const long long b = __double_as_longlong(x);
    return b > 0 && b <= 0x7ff0000000000000ll;
}

// Global load of data that other CTAs of the same launch may have written
// (CG: cached in L2 only, never a stale L1 line), or an ordinary load.
template <bool CG, typename T>
__device__ __forceinline__ T gload(const T* p) {
    if constexpr (CG) return __ldcg(p);
    else return *p;
}

// ---------------------------------------------------------------------------
// Double-float arithmetic for the FP64_DF variant: a value is an unevaluated
// pair of floats (hi, lo) with x = hi + lo to about 48 significant bits.  Sums of products use the compensated dot product Dot2
// of Ogita, Rump & Oishi ("Accurate sum and dot product", SIAM J. Sci.
// Comput. 26, 2005): the error-free TwoProduct (by FMA) and TwoSum (Knuth)
// of every term, errors collected in a second float; the cross terms
// hi*lo of pair operands join the error float.  The result carries about
// twice the float precision.  __fadd_rn / __fmul_rn keep the compiler from
// contracting the error-free transformations into FMAs.
// ---------------------------------------------------------------------------
// The split is exact bit surgery, no FP64 instruction: hi is x with its
// significand cut to 24 bits (the top 23 stored bits), lo the remaining 29
// bits rounded to a float (x = hi + lo to 2^-48 relative).  |x| < 2^-126
// gives (0, 0) and |x| < 2^-74 drops lo (absolute error below 2^-98); a
// double-to-float conversion instruction costs several FP64-pipe slots on
// this GPU, the integer path none.
__device__ __forceinline__ float2 df_split(double x) {
    const long long b = __double_as_longlong(x);
    const unsigned hw = (unsigned)(b >> 32);
    const int ed = (int)((hw >> 20) & 0x7ffu);          // biased double exponent
    const unsigned sgn = hw & 0x80000000u;
    float h, l;
    if (ed >= 897 && ed <= 1150) {                       // normal float range
        h = __uint_as_float(sgn | ((unsigned)(ed - 896) << 23) | (unsigned)((b >> 29) & 0x7fffff));
    } else {
        h = (ed > 1150) ? __uint_as_float(sgn | 0x7f800000u) : 0.f;   // overflow -> inf, flagged downstream
    }
    if (ed >= 949 && ed <= 1150) {                       // 2^(ed - 1075) is a normal float
        const float m = __uint2float_rn((unsigned)(b & 0x1fffffff));
        l = __uint_as_float(__float_as_uint(m * __uint_as_float((unsigned)(ed - 948) << 23)) | sgn);
    } else {
        l = 0.f;
    }
    return make_float2(h, l);
}
__device__ __forceinline__ double df_join(float s, float e) { return (double)s + (double)e; }
// double -> float by bit surgery (the head of df_split: the significand cut
// to 24 bits, within one float ulp), no conversion instruction
__device__ __forceinline__ float d2f_bits(double x) { return df_split(x).x; }
// float -> double by bit surgery (exponent rebiased, significand shifted:
// exact for normal floats, zero for zero and subnormals, inf / NaN kept)
__device__ __forceinline__ double f2d_bits(float f) {
    const unsigned b = __float_as_uint(f);
    const unsigned ex = (b >> 23) & 0xffu;
    const unsigned long long e64 = (ex == 0u) ? 0ull : (ex == 0xffu ? 2047ull : (unsigned long long)(ex + 896u));
    const unsigned long long man = (ex == 0u) ? 0ull : (unsigned long long)(b & 0x7fffffu) << 29;
    return __longlong_as_double((long long)(((unsigned long long)(b & 0x80000000u) << 32) | (e64 << 52) | man));
}
// a / b in FP64 by Newton-Raphson reciprocal refinement with a final
// residual correction (Markstein, IBM J. Res. Dev. 34, 1990): a float
// reciprocal of b (b cut to a float by bit surgery, reciprocal to 2^-23),
// one Newton step r <- r + r (1 - b r) (2^-46), q = a r and q <- q + r (a - b q)
// (within about one ulp for numerators of magnitude >= 2^-920; below that the
// residual leaves the normal range and the error grows to at most 2^8 ulp;
// not correctly rounded; an overflowing quotient or an infinite numerator
// gives NaN, non-finite like the IEEE +-inf).  Divisors outside the float
// exponent range take the IEEE quotient.
__device__ __forceinline__ double div_nr(double a, double b) {
    const int ex = (int)((__double_as_longlong(b) >> 52) & 0x7ff);
    if (ex < 1023 - 120 || ex > 1023 + 120) return a / b;
    double r = f2d_bits(__frcp_rn(d2f_bits(b)));
    r = fma(r, fma(-b, r, 1.0), r);
    const double q = a * r;
    return fma(fma(-b, q, a), r, q);
}

// a / b to about 2^-46 relative: the float-seeded reciprocal of div_nr after
// its Newton step, times a, without the residual correction (3 FP64
// operations instead of 5).  For the WENO-5 face quotient: its error enters
// the stage as dt xi/dx times the face difference, some 1e-14 of the state
// per step, far inside the FP64 parity bars.  Divisors outside the float
// exponent range take the IEEE quotient.
__device__ __forceinline__ double div_face(double a, double b) {
    const int ex = (int)((__double_as_longlong(b) >> 52) & 0x7ff);
    if (ex < 1023 - 120 || ex > 1023 + 120) return a / b;
    double r = f2d_bits(__frcp_rn(d2f_bits(b)));
    r = fma(r, fma(-b, r, 1.0), r);
    return a * r;
}

// (s, e) += a * b for pairs a, b.
__device__ __forceinline__ void dot2_acc(float& s, float& e, float2 a, float2 b) {
    const float p = __fmul_rn(a.x, b.x);
    const float pe = fmaf(a.x, b.x, -p);            // exact: a.x b.x = p + pe
    const float t = __fadd_rn(s, p);
    const float z = __fsub_rn(t, s);
    const float te = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(p, z));   // exact: s + p = t + te
    e = __fadd_rn(e, __fadd_rn(te, pe));
    e = fmaf(a.x, b.y, e);
    e = fmaf(a.y, b.x, e);
    s = t;
}


// ---------------------------------------------------------------------------
// Phase 0: stage the tables, the density halo, u/T near the tile and the
// state tile (+-3 nodes for WENO-5) into shared memory.
// ---------------------------------------------------------------------------
// PARITY: the parity-split tables Pp and Sp go to s.P and s.S in place of
// the full analysis and synthesis tables.
// CG: the moment sums are read with L2-coherent loads (written earlier in
// the same launch by other CTAs).
// The velocity tables of the slab into shared memory: the parity-split
// analysis pairs and synthesis rows (PARITY), else the full P and S.
template <typename R, bool PARITY = false>
__device__ void load_velocity_tables(const SlabDesc& sd, const Smem<R>& s, const R* __restrict__ rtab) {
    const int Q = sd.Q;
    TableLayout L(Q);
    const R* tab = rtab + sd.tab_off;
    if constexpr (PARITY) {
        const ParitySplit ps(Q);
        const int la = ps.analysis_len(), ls = ps.synthesis_len();
#pragma unroll 4
        for (int t = threadIdx.x; t < la; t += blockDim.x) s.P[t] = tab[L.Pp + t];
#pragma unroll 4
        for (int t = threadIdx.x; t < ls; t += blockDim.x) s.S[t] = tab[L.Sp + t];
    } else {
        for (int t = threadIdx.x; t < Q * Q; t += blockDim.x) {
            s.P[t] = tab[L.P + t];
            s.S[t] = tab[L.S + t];
        }
    }
}

// The velocity tables and the node inputs of the tile (TABLES false: the
// node inputs only, the tables being staged already).
template <typename R, bool PARITY = false, bool CG = false, bool TABLES = true>
__device__ void load_node_inputs(const SlabDesc& sd, const WorkItem& it, const Smem<R>& s, int Z,
                                 const R* __restrict__ rtab, const double* __restrict__ mom, long long NN) {
    const int M = sd.M, nx = sd.nx, bc = sd.bc;
    if constexpr (TABLES) load_velocity_tables<R, PARITY>(sd, s, rtab);
    const double* S0 = mom + MOM_S0 * NN + sd.node_off;
#pragma unroll 2
    for (int t = threadIdx.x; t < it.nz + 2 * M; t += blockDim.x) {
        double n = gload<CG>(S0 + gidx(it.i0 - M + t, nx, bc));
        s.N[t] = n;
        if constexpr (!std::is_same<R, double>::value) s.Nr[t] = (R)n;
    }
    const double* S1 = mom + MOM_S1 * NN + sd.node_off;
    const double* S2 = mom + MOM_S2 * NN + sd.node_off;
    const double* S3 = mom + MOM_S3 * NN + sd.node_off;
    const double* G0 = mom + MOM_G0 * NN + sd.node_off;
    const double* G1 = mom + MOM_G1 * NN + sd.node_off;
    // the node loop on the last threads of the CTA, whose share of the
    // staging above is smallest, so that it runs beside the tap and table
    // staging of the first warps
    for (int t = (int)blockDim.x - 1 - (int)threadIdx.x; t >= 0 && t < it.nz + 4; t += blockDim.x) {
        int i = gidx(it.i0 - 2 + t, nx, bc);
        const bool tile = (t >= 2 && t < it.nz + 2);
        double n = gload<CG>(S0 + i), s1 = gload<CG>(S1 + i), s2 = gload<CG>(S2 + i), g0 = gload<CG>(G0 + i);
        double s3 = tile ? gload<CG>(S3 + i) : 0.0, g1 = tile ? gload<CG>(G1 + i) : 0.0;
        double inv_n = div_nr(1.0, n);
        double u = s1 * inv_n;
        // (3/2) n T = sum (xi-u)^2/2 F + sum G = S2/2 + G0 - n u^2/2
        s.U[t] = u;
        s.T[t] = (2.0 / 3.0) * ((0.5 * s2 + g0) * inv_n - 0.5 * u * u);
        // heat flux of the tile's nodes, q = (S3 - 3u S2 + 3u^2 S1 - u^3 S0)/2 + G1 - u G0,
        // formed here (in parallel, off the node warps' serial chain); the node
        // fields read it from the KQ slot, which they then overwrite with (1 - Pr) q
        if (tile)
            s.Sc[SC_KQ * Z + (t - 2)] = 0.5 * (s3 - 3.0 * u * s2 + 3.0 * u * u * s1 - u * u * u * n) + g1 - u * g0;
    }
}

// With Fd (FP64_DF), the tile's interior columns are also stored as
// double-float pairs, Fd[(d Q + k) Z + t].
template <typename R>
__device__ void load_state_tile(const SlabDesc& sd, const WorkItem& it, const Smem<R>& s, int Z,
                                const R* __restrict__ src, long long NF, float2* Fd = nullptr) {
    const int Q = sd.Q, nx = sd.nx, bc = sd.bc, W = Z + 6;
    const int cols = it.nz + 6;
    for (int e = threadIdx.x; e < 2 * Q * cols; e += blockDim.x) {
        int c = e % cols, r = e / cols;
        int k = r % Q, d = r / Q;
        int i = gidx(it.i0 - 3 + c, nx, bc);
        R v = src[d * NF + sd.f_off + (long long)k * nx + i];
        s.F[(d * Q + k) * W + c] = v;
        if (Fd && c >= 3 && c < it.nz + 3) Fd[(size_t)r * Z + c - 3] = df_split((double)v);
    }
}

// Asynchronous global-to-shared copy of one element (4 or 8 bytes, cp.async,
// L1-allocating); completion by cp_async_wait_all.
template <typename R>
__device__ __forceinline__ void cp_async_elem(R* smem_dst, const R* gsrc) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    if constexpr (sizeof(R) == 8) asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(gsrc) : "memory");
    else asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// The state tile (+-3 nodes) into s.F by asynchronous copies, all of them in
// flight at once; the caller waits (cp_async_wait_all) and synchronises
// before reading it.
// CG: L2-coherent loads instead of the (L1-allocating) copies, for data
// written earlier in the same launch by other CTAs.
template <typename R, bool CG = false>
__device__ void issue_state_tile(const SlabDesc& sd, const WorkItem& it, const Smem<R>& s, int Z,
                                 const R* __restrict__ src, long long NF) {
    static_assert(kZMax + 6 <= 96, "a lane holds at most three tile columns");
    const int Q = sd.Q, nx = sd.nx, bc = sd.bc, W = Z + 6;
    const int cols = it.nz + 6;
    // lanes on columns (the node index of a column formed once per lane),
    // warps on velocity rows
    const int lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    int gi[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const int c = lane + 32 * q;
        gi[q] = c < cols ? gidx(it.i0 - 3 + c, nx, bc) : 0;
    }
    for (int r = threadIdx.x >> 5; r < 2 * Q; r += nwarps) {
        const int d = r >= Q ? 1 : 0, k = r - d * Q;
        const R* g = src + d * NF + sd.f_off + (long long)k * nx;
        R* row = s.F + (size_t)r * W;
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const int c = lane + 32 * q;
            if (c < cols) {
                if constexpr (CG) row[c] = __ldcg(g + gi[q]);
                else cp_async_elem<R>(row + c, g + gi[q]);
            }
        }
    }
    if constexpr (!CG) cp_async_commit();
}

// The parity-split interior columns EO[((d * 2 + par) * H + j) * Z + t] of
// the state tile in s.F: E_j = h_j + h_{Q-1-j}, O_j = h_j - h_{Q-1-j} (the
// middle node of an odd Q: E = h, O = 0); threads tid, tid + nth, ...
template <typename R>
__device__ void split_state_tile(const SlabDesc& sd, const WorkItem& it, const Smem<R>& s, int Z, int tid, int nth) {
    const int Q = sd.Q, W = Z + 6, H = (Q + 1) / 2, nz = it.nz;
    for (int e = tid; e < 2 * H * nz; e += nth) {
        const int t = e % nz, r = e / nz;
        const int j = r % H, d = r / H, jm = Q - 1 - j;
        const R v = s.F[(size_t)(d * Q + j) * W + t + 3];
        R* eo = s.EO + ((size_t)(2 * d) * H + j) * Z + t;
        if (jm != j) {
            const R vm = s.F[(size_t)(d * Q + jm) * W + t + 3];
            eo[0] = v + vm;
            eo[(size_t)H * Z] = v - vm;
        } else {
            eo[0] = v;
            eo[(size_t)H * Z] = R(0);
        }
    }
}

// The state tile (+-3 nodes) and the parity-split interior columns
// EO[((d * 2 + par) * H + j) * Z + t]: E_j = h_j + h_{Q-1-j}, O_j = h_j - h_{Q-1-j}
// (the middle node of an odd Q: E = h, O = 0).  Each thread loads a node
// pair (j, Q-1-j) of one column.
template <typename R>
__device__ void load_state_tile_eo(const SlabDesc& sd, const WorkItem& it, const Smem<R>& s, int Z,
                                   const R* __restrict__ src, long long NF) {
    const int Q = sd.Q, nx = sd.nx, bc = sd.bc, W = Z + 6, H = (Q + 1) / 2;
    const int cols = it.nz + 6;
#pragma unroll 4
    for (int e = threadIdx.x; e < 2 * H * cols; e += blockDim.x) {
        const int c = e % cols, r = e / cols;
        const int j = r % H, d = r / H, jm = Q - 1 - j;
        const int i = gidx(it.i0 - 3 + c, nx, bc);
        const R* row = src + d * NF + sd.f_off + i;
        const R v = row[(long long)j * nx];
        s.F[(d * Q + j) * W + c] = v;
        R vm = R(0);
        if (jm != j) {
            vm = row[(long long)jm * nx];
            s.F[(d * Q + jm) * W + c] = vm;
        }
        if (c >= 3 && c < it.nz + 3) {
            R* eo = s.EO + ((size_t)(2 * d) * H + j) * Z + (c - 3);
            eo[0] = (jm != j) ? v + vm : v;
            eo[(size_t)H * Z] = (jm != j) ? v - vm : R(0);
        }
    }
}

// sum_{|j| <= m} tap[j + m] x[j] in four interleaved partial sums: a quarter
// of the dependent chain (an FP64 operation waits for the whole warp to pass
// the FP64 pipe of its scheduler, tens of cycles on this part).
template <typename R, typename T>
__device__ __forceinline__ R tap_sum(const T* __restrict__ tap, const R* x, int m) {
    R a0 = 0, a1 = 0, a2 = 0, a3 = 0;
    int j = -m;
    for (; j + 3 <= m; j += 4) {
        a0 = fma((R)tap[j + m], x[j], a0);
        a1 = fma((R)tap[j + 1 + m], x[j + 1], a1);
        a2 = fma((R)tap[j + 2 + m], x[j + 2], a2);
        a3 = fma((R)tap[j + 3 + m], x[j + 3], a3);
    }
    for (; j <= m; ++j) a0 = fma((R)tap[j + m], x[j], a0);
    return (a0 + a1) + (a2 + a3);
}

// ---------------------------------------------------------------------------
// Phases 1-2: node fields of the tile.
// ---------------------------------------------------------------------------
// Pass 1 (threads tid, tid + nth, ...): Fischer-Methfessel average, chi and X
// on nodes i0-2 .. i0+nz+1.  Pass 2 reads the +-2 neighbours of pass 1, so
// the caller separates the passes with a barrier of the participating threads.
// mtap: the slab's Fischer-Methfessel taps [2m+1] (global or staged).
template <typename R>
__device__ void node_fields_pass1(const SlabDesc& sd, const WorkItem& it, const Smem<R>& s,
                                  const double* __restrict__ mtap, long long NN, double* fields_out, int tid,
                                  int nth) {
    const int M = sd.M, m = sd.m;
    // Fischer-Methfessel average (Sec. II.A), chi (Eq. (carnstar)) and
    // X = n^2 chi T on nodes i0-2 .. i0+nz+1.  Under the outflow rule a ghost
    // node copies every node field of the nearest interior node, so the
    // average is centred on the clamped node; under the periodic rule the
    // window around the ghost position is the wrapped node's window.
    for (int t = tid; t < it.nz + 4; t += nth) {
        int pos = it.i0 - 2 + t;
        int shift = (sd.bc == EVFDLB_BC_OUTFLOW) ? gidx(pos, sd.nx, sd.bc) - pos : 0;
        const double* nn = s.N + (t - 2 + M + shift);
        const double nb = tap_sum<double>(mtap, nn, m);
        double eta = sd.eta_coef * nb, om = 1.0 - eta;
        double chi = div_nr(2.0 - eta, 2.0 * om * om * om);
        double n = nn[0];
        s.Chi[t] = chi;
        s.X[t] = n * n * chi * s.T[t];
        if (fields_out && t >= 2 && t < it.nz + 2) {
            long long NNf = NN;
            fields_out[4 * NNf + sd.node_off + it.i0 + t - 2] = nb;
        }
    }
}

// Pass 2: per tile node, the gradients, the Eq. (F1) force (in R), the heat
// flux, the transport coefficients and the scalars of Sc and Scr.
// ftap: the slab's force taps [2M+1] (global or staged).
// PREFORCE: the tile's Eq. (F1) force sums are already in s.Scr[Z + t]
// (formed by other warps, tile_force_sums), else they are summed here.
template <typename R, bool PREFORCE = false>
__device__ void node_fields_pass2(const SlabDesc& sd, const WorkItem& it, const Smem<R>& s, int Z,
                                  const R* __restrict__ ftap, const double* __restrict__ mom, long long NN,
                                  unsigned* err, double* fields_out, int tid, int nth) {
    const int M = sd.M;
    const double inv12 = sd.inv_dx / 12.0;
    (void)mom;
    for (int t = tid; t < it.nz; t += nth) {
        const int c = t + 2;                         // index in the +-2 arrays
        const int i = it.i0 + t;
        double n = s.N[t + M], u = s.U[c], T = s.T[c];
        // fourth-order central differences (Sec. III)
        double dX = (s.X[c - 2] - 8.0 * s.X[c - 1] + 8.0 * s.X[c + 1] - s.X[c + 2]) * inv12;
        double dT = (s.T[c - 2] - 8.0 * s.T[c - 1] + 8.0 * s.T[c + 1] - s.T[c + 2]) * inv12;
        double dU = (s.U[c - 2] - 8.0 * s.U[c - 1] + 8.0 * s.U[c + 1] - s.U[c + 2]) * inv12;
        double X = s.X[c], chi = s.Chi[c];
        double A, B;
        // self-consistent force, Eq. (F1), Simpson taps over |j| <= M
        const R* nn = s.Nr + (t + M);
        const R f1r = PREFORCE ? s.Scr[Z + t] : tap_sum<R>(ftap, nn, M);
        double f1;
        if constexpr (std::is_same<R, float>::value) f1 = f2d_bits(f1r);
        else f1 = (double)f1r;
        // heat flux, formed with the node inputs (load_node_inputs)
        double q = s.Sc[SC_KQ * Z + t];
        // transport, Eqs. (viscosity), (tau), (prandtl)
        double bn, x, mu, tau, Pr, nu;
        if constexpr (std::is_same<R, float>::value) {
            // the FP32 variant: gradient ratios and transport on the FP32 pipe
            // (chi, the gradients' differences and the heat flux stay FP64);
            // values cross by bit surgery, not conversion instructions
            const float fn = d2f_bits(n), fT = d2f_bits(T), fchi = d2f_bits(chi);
            const float fA = d2f_bits(dX) / d2f_bits(X), fB = d2f_bits(dT) / fT;
            const float fbn = d2f_bits(sd.b) * fn, fx = fbn * fchi;
            const float c16 = (float)((4.0 / 25.0) * (1.0 + 12.0 / M_PI)), c9 = (float)((9.0 / 25.0) * (1.0 + 32.0 / (9.0 * M_PI)));
            const float fmu = d2f_bits(sd.mu0_coef) * sqrtf(fT) * (1.0f / fchi + 0.8f * fbn + c16 * fbn * fbn * fchi);
            const float ftau = fmu / (fn * fT * (1.0f + 0.4f * fx));
            const float fPr = (2.0f / 3.0f) * (1.0f + 0.6f * fx) * (1.0f + 0.8f * fx + c16 * fx * fx) /
                              ((1.0f + 0.4f * fx) * (1.0f + 1.2f * fx + c9 * fx * fx));
            const float fnu = (sd.relax == EVFDLB_RELAX_INV_TAU) ? 1.0f / ftau : fchi / ftau;
            A = f2d_bits(fA);
            B = f2d_bits(fB);
            bn = f2d_bits(fbn);
            x = f2d_bits(fx);
            mu = f2d_bits(fmu);
            tau = f2d_bits(ftau);
            Pr = f2d_bits(fPr);
            nu = f2d_bits(fnu);
        } else {
            A = div_nr(dX, X);
            B = div_nr(dT, T);
            bn = sd.b * n;
            x = bn * chi;
            mu = sd.mu0_coef * sqrt(T) *
                 (div_nr(1.0, chi) + 0.8 * bn + (4.0 / 25.0) * (1.0 + 12.0 / M_PI) * bn * bn * chi);
            tau = div_nr(mu, n * T * (1.0 + 0.4 * x));
            Pr = div_nr((2.0 / 3.0) * (1.0 + 0.6 * x) * (1.0 + 0.8 * x + (4.0 / 25.0) * (1.0 + 12.0 / M_PI) * x * x),
                        (1.0 + 0.4 * x) * (1.0 + 1.2 * x + (9.0 / 25.0) * (1.0 + 32.0 / (9.0 * M_PI)) * x * x));
            nu = div_nr((sd.relax == EVFDLB_RELAX_INV_TAU) ? 1.0 : chi, tau);
        }
        double* sc = s.Sc;
        sc[SC_N * Z + t] = n;
        sc[SC_U * Z + t] = u;
        sc[SC_T * Z + t] = T;
        sc[SC_NU * Z + t] = nu;
        sc[SC_FORCE * Z + t] = f1;
        sc[SC_KQ * Z + t] = (1.0 - Pr) * q;
        sc[SC_K * Z + t] = -x * n;        // -b n^2 chi, the prefactor of J1
        sc[SC_A * Z + t] = A;
        sc[SC_B * Z + t] = B;
        sc[SC_D * Z + t] = dU;
        if constexpr (std::is_same<R, float>::value) s.Scr[t] = d2f_bits(nu);
        else s.Scr[t] = (R)nu;
        s.Scr[Z + t] = f1r;
        if (!positive(n) || !positive(T)) {
            atomicOr(err, (finite(n) && finite(T)) ? ERR_NEGATIVE : ERR_NONFINITE);
        } else if (!finite(f1) || !finite(nu) || !finite(q) || !finite(A) || !finite(B)) {
            atomicOr(err, ERR_NONFINITE);
        }
        if (fields_out) {
            long long o = sd.node_off + i;
            double vals[EVFDLB_NFIELDS] = {n, u, T, q, 0.0, chi, f1, mu, tau, Pr, nu, A, B, dU, X, x};
            for (int f = 0; f < EVFDLB_NFIELDS; ++f)
                if (f != 4) fields_out[f * NN + o] = vals[f];
        }
    }
}

// The Eq. (F1) force sums of the tile's nodes, f1_t = sum_{|j| <= M}
// ftap_j n_{t+j}, by half-warps of threads tid, tid + nth, ... (nth a
// multiple of 32): the 16 lanes of a half-warp split a node's 2M+1 taps and
// reduce their partial sums by shuffles; the results go to s.Scr[Z + t].
template <typename R>
__device__ void tile_force_sums(const SlabDesc& sd, const WorkItem& it, const Smem<R>& s, int Z,
                                const R* __restrict__ ftap, int tid, int nth) {
    const int M = sd.M, sub = tid & 15;
    const unsigned half = 0xffffu << (threadIdx.x & 16);
    for (int t = tid >> 4; t < it.nz; t += nth >> 4) {
        const R* nn = s.Nr + t;                      // nn[j + M] = n_{t+j}
        R a0 = 0, a1 = 0;
        int j = sub;
        for (; j + 16 < 2 * M + 1; j += 32) {
            a0 = fma(ftap[j], nn[j], a0);
            a1 = fma(ftap[j + 16], nn[j + 16], a1);
        }
        if (j < 2 * M + 1) a0 = fma(ftap[j], nn[j], a0);
        R a = a0 + a1;
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) a += __shfl_xor_sync(half, a, o);
        if (sub == 0) s.Scr[Z + t] = a;
    }
}

// Both passes with all threads of the CTA.
template <typename R>
__device__ void node_fields(const SlabDesc& sd, const WorkItem& it, const Smem<R>& s, int Z,
                            const double* __restrict__ taps, const R* __restrict__ rtaps,
                            const double* __restrict__ mom, long long NN, unsigned* err, double* fields_out) {
    node_fields_pass1<R>(sd, it, s, taps + sd.tap_off + 2 * sd.M + 1, NN, fields_out, threadIdx.x, blockDim.x);
    __syncthreads();
    node_fields_pass2<R>(sd, it, s, Z, rtaps + sd.tap_off, mom, NN, err, fields_out, threadIdx.x, blockDim.x);
}

// ---------------------------------------------------------------------------
// Hermite coefficients of nu F^S + J1_F and nu G^S + J1_G.
// With m_l = E[psi_l(u + c)], c ~ N(0, T) (m_0 = 1,
// m_{l+1} = u m_l / sqrt(l+1) + (T-1) sqrt(l/(l+1)) m_{l-1}) and Stein's
// identity E[c h(c)] = T E[h'(c)], the projections of the reduced Shakhov
// equilibria and of the reduced J1 of Sec. II.B are
//   c_l = c0 m_l + c1 sqrt(l) m_{l-1} + c2 sqrt(l(l-1)) m_{l-2}
//         + c3 sqrt(l(l-1)(l-2)) m_{l-3}
// with per-node constants (K = -b n^2 chi, kq = (1-Pr) q):
//   F: c0 = nu n,             c1 = K A T,
//      c2 = 3/5 K D T,        c3 = nu kq/5 + 3/10 K B T^2
//   G: c0 = nu n T + 2/5 K T D,  c1 = 2/5 nu kq + K T^2 (A + 3/5 B),
//      c2 = 3/5 K T^2 D,         c3 = nu kq T/5 + 3/10 K T^3 B
// node_coefficients forms the constants (FP64, stored in R) and the moments
// m_l (recurrence in R) per node; coefficients() then forms every c_l in
// parallel and adds the force term F1 sqrt(l) a_{l-1}
// (d/dxi [omega psi_{l-1}] = -sqrt(l) omega psi_l).
// ---------------------------------------------------------------------------
// m_0 = 1, m_{l+1} = u m_l / sqrt(l+1) + (T-1) sqrt(l/(l+1)) m_{l-1}, to
// mm[l stride] (u, T widened or narrowed to R as the node constants are)
template <typename R>
__device__ __forceinline__ void hermite_moments(int Q, const TableLayout& L, const R* __restrict__ tab, double u,
                                                double T, R* mm, int stride) {
    R ru, Tm1;
    if constexpr (std::is_same<R, float>::value) {
        ru = d2f_bits(u);
        Tm1 = d2f_bits(T - 1.0);
    } else {
        ru = (R)u;
        Tm1 = (R)(T - 1.0);
    }
    R m0 = 1, m1 = 0;
    for (int l = 0; l < Q; ++l) {
        mm[l * stride] = m0;
        R mn = fma(ru * tab[L.rinv + l], m0, Tm1 * tab[L.rr + l] * m1);
        m1 = m0;
        m0 = mn;
    }
}

// MM: also the Hermite moments m_l of the local Gaussian (else another
// group of warps forms them, node_hermite_moments).
template <typename R, bool MM = true>
__device__ void node_coefficients(const SlabDesc& sd, const WorkItem& it, const Smem<R>& s, int Z,
                                  const R* __restrict__ tab, int tid, int nth) {
    const int Q = sd.Q;
    TableLayout L(Q);
    for (int t = tid; t < it.nz; t += nth) {
        const double* sc = s.Sc;
        double n = sc[SC_N * Z + t], u = sc[SC_U * Z + t], T = sc[SC_T * Z + t];
        double nu = sc[SC_NU * Z + t], kq = sc[SC_KQ * Z + t], K = sc[SC_K * Z + t];
        double A = sc[SC_A * Z + t], B = sc[SC_B * Z + t], D = sc[SC_D * Z + t];
        R* cF = s.Cc + t;
        R* cG = s.Cc + 4 * Z + t;
        if constexpr (std::is_same<R, float>::value) {
            // the FP32 variant forms the constants on the FP32 pipe
            const float fn = d2f_bits(n), fT = d2f_bits(T), fnu = d2f_bits(nu), fkq = d2f_bits(kq);
            const float fK = d2f_bits(K), fA = d2f_bits(A), fB = d2f_bits(B), fD = d2f_bits(D);
            cF[0] = fnu * fn;
            cF[Z] = fK * fA * fT;
            cF[2 * Z] = 0.6f * fK * fD * fT;
            cF[3 * Z] = 0.2f * fnu * fkq + 0.3f * fK * fB * fT * fT;
            cG[0] = fnu * fn * fT + 0.4f * fK * fT * fD;
            cG[Z] = 0.4f * fnu * fkq + fK * fT * fT * (fA + 0.6f * fB);
            cG[2 * Z] = 0.6f * fK * fT * fT * fD;
            cG[3 * Z] = 0.2f * fnu * fkq * fT + 0.3f * fK * fT * fT * fT * fB;
        } else {
            cF[0] = (R)(nu * n);
            cF[Z] = (R)(K * A * T);
            cF[2 * Z] = (R)(0.6 * K * D * T);
            cF[3 * Z] = (R)(0.2 * nu * kq + 0.3 * K * B * T * T);
            cG[0] = (R)(nu * n * T + 0.4 * K * T * D);
            cG[Z] = (R)(0.4 * nu * kq + K * T * T * (A + 0.6 * B));
            cG[2 * Z] = (R)(0.6 * K * T * T * D);
            cG[3 * Z] = (R)(0.2 * nu * kq * T + 0.3 * K * T * T * T * B);
        }
        if constexpr (MM) hermite_moments<R>(Q, L, tab, u, T, s.Mm + t, Z);
    }
}

// The Hermite moments m_l = E[psi_l(u + c)], c ~ N(0, T), of the tile's
// nodes (the recurrence of node_coefficients) from the node inputs u, T of
// load_node_inputs, by threads tid, tid + nth, ...
template <typename R>
__device__ void node_hermite_moments(const SlabDesc& sd, const WorkItem& it, const Smem<R>& s, int Z,
                                     const R* __restrict__ tab, int tid, int nth) {
    const int Q = sd.Q;
    TableLayout L(Q);
    for (int t = tid; t < it.nz; t += nth) hermite_moments<R>(Q, L, tab, s.U[t + 2], s.T[t + 2], s.Mm + t, Z);
}

// With DF the coefficients are stored as double-float pairs (float2) in the
// same block, for the double-float synthesis.
template <typename R, bool DF = false>
__device__ void coefficients(const SlabDesc& sd, const WorkItem& it, const Smem<R>& s, int Z,
                             const R* __restrict__ tab, int tid, int nth) {
    const int Q = sd.Q, nz = it.nz;
    TableLayout L(Q);
    // one (l, node) per item, both distributions: the scaled moments
    // sqrt(l(l-1)..) m_{l-j} and the force factor F1 sqrt(l) are shared
    for (int e = tid; e < Q * nz; e += nth) {
        const int t = e % nz, l = e / nz;
        const R* mm = s.Mm + t;
        // the sqrt factors vanish where the moment index would be negative
        const R m0 = mm[l * Z];
        const R M1 = tab[L.r1 + l] * mm[max(l - 1, 0) * Z];
        const R M2 = tab[L.r2 + l] * mm[max(l - 2, 0) * Z];
        const R M3 = tab[L.r3 + l] * mm[max(l - 3, 0) * Z];
        const R f = s.Scr[Z + t] * tab[L.r1 + l];
#pragma unroll
        for (int d = 0; d < 2; ++d) {
            const R* cc = s.Cc + d * 4 * Z + t;
            R c = cc[0] * m0;
            c = fma(cc[Z], M1, c);
            c = fma(cc[2 * Z], M2, c);
            c = fma(cc[3 * Z], M3, c);
            if (l >= 1) c = fma(f, s.A[((size_t)d * Q + l - 1) * Z + t], c);
            if constexpr (DF) reinterpret_cast<float2*>(s.C)[((size_t)d * Q + l) * Z + t] = df_split((double)c);
            else s.C[((size_t)d * Q + l) * Z + t] = c;
        }
    }
}

// Analysis a_l = sum_j psi_l(xi_j) h_j, l <= Q-2 (the force needs
// a_0 .. a_{Q-2}; the l = Q-1 term meets psi_Q(xi_k) = 0), two orders per
// thread so that each state value loaded feeds two FMAs.
template <typename R>
__device__ void analysis(const SlabDesc& sd, const WorkItem& it, const Smem<R>& s, int Z, int tid, int nth) {
    const int Q = sd.Q, W = Z + 6, nz = it.nz;
    const int np = Q / 2;                          // pairs (l, l+1) covering l <= Q-2
    const int per_d = np * nz;
    for (int e = tid; e < 2 * per_d; e += nth) {
        int d = e / per_d, r = e % per_d;
        int l0 = 2 * (r / nz), t = r % nz;
        const bool two = (l0 + 1 <= Q - 2);
        const R* P0 = s.P + l0 * Q;
        const R* P1 = s.P + (two ? l0 + 1 : l0) * Q;
        const R* h = s.F + (size_t)d * Q * W + (t + 3);
        R a0 = 0, a1 = 0;
        for (int j = 0; j < Q; ++j) {
            R hv = h[j * W];
            a0 = fma(P0[j], hv, a0);
            a1 = fma(P1[j], hv, a1);
        }
        s.A[((size_t)d * Q + l0) * Z + t] = a0;
        if (two) s.A[((size_t)d * Q + l0 + 1) * Z + t] = a1;
    }
}

// Parity-split analysis: a_l = sum_{j<H} psi_l(xi_j) (E_j or O_j), l <= Q-2,
// two orders of one parity (l, l+2) per thread sharing each E/O value loaded
// (Pp holds the two table values side by side: one two-wide load).
template <typename R>
__device__ void analysis_eo(const SlabDesc& sd, const WorkItem& it, const Smem<R>& s, int Z, int tid, int nth) {
    using R2 = typename std::conditional<std::is_same<R, float>::value, float2, double2>::type;
    const int Q = sd.Q, nz = it.nz;
    const ParitySplit ps(Q);
    const int H = ps.H, G = ps.GE + ps.GO;
    const R2* Pp = reinterpret_cast<const R2*>(s.P);
    for (int e = tid; e < 2 * G * nz; e += nth) {
        const int t = e % nz, r = e / nz;
        const int g = r % G, d = r / G;
        const int par = g < ps.GE ? 0 : 1;
        const int l0 = par ? 4 * (g - ps.GE) + 1 : 4 * g;
        const R* x = s.EO + ((size_t)(2 * d + par) * H) * Z + t;
        const R2* pp = Pp + (size_t)g * H;
        R a0 = 0, a1 = 0;
        for (int j = 0; j < H; ++j) {
            const R v = x[j * Z];
            const R2 p = pp[j];
            a0 = fma(p.x, v, a0);
            a1 = fma(p.y, v, a1);
        }
        s.A[((size_t)d * Q + l0) * Z + t] = a0;
        if (l0 + 2 <= Q - 2) s.A[((size_t)d * Q + l0 + 2) * Z + t] = a1;
    }
}

// Analysis in double-float: the state tile is split into pairs when it is
// staged (Fd[(d Q + j) Z + t]); a_l = sum_j psi_l(xi_j) h_j by Dot2, four
// orders per thread (four independent accumulator chains, each pair loaded
// feeding four terms), joined to FP64 for the coefficients.
__device__ inline void analysis_df(const SlabDesc& sd, const WorkItem& it, const Smem<double>& s, const float2* Fd,
                                   const float2* P, int Z, int tid, int nth) {
    const int Q = sd.Q, nz = it.nz;
    const int nq = Q / 4;                          // quads of orders covering l <= Q-2 (Q even)
    const int per_d = nq * nz;
    for (int e = tid; e < 2 * per_d; e += nth) {
        int d = e / per_d, r = e % per_d;
        int l0 = 4 * (r / nz), t = r % nz;
        const int nl = min(4, Q - 1 - l0);         // orders l0 .. l0+nl-1 (<= Q-2)
        const float2* P0 = P + l0 * Q;
        const float2* P1 = P + min(l0 + 1, Q - 1) * Q;
        const float2* P2 = P + min(l0 + 2, Q - 1) * Q;
        const float2* P3 = P + min(l0 + 3, Q - 1) * Q;
        const float2* h = Fd + (size_t)d * Q * Z + t;
        float s0 = 0.f, e0 = 0.f, s1 = 0.f, e1 = 0.f, s2 = 0.f, e2 = 0.f, s3 = 0.f, e3 = 0.f;
        for (int j = 0; j < Q; ++j) {
            const float2 hv = h[j * Z];
            dot2_acc(s0, e0, P0[j], hv);
            dot2_acc(s1, e1, P1[j], hv);
            dot2_acc(s2, e2, P2[j], hv);
            dot2_acc(s3, e3, P3[j], hv);
        }
        double* A = s.A + ((size_t)d * Q + l0) * Z + t;
        A[0] = df_join(s0, e0);
        if (nl > 1) A[Z] = df_join(s1, e1);
        if (nl > 2) A[2 * Z] = df_join(s2, e2);
        if (nl > 3) A[3 * Z] = df_join(s3, e3);
    }
}

// WENO-5 (Jiang & Shu) faces in difference form, along a run of faces.
// With the upwind stencil v0..v4 (face between v2 and v3) and first
// differences d_i = v_{i+1} - v_i:
//   q0 - v2 = (5 d1 - 2 d0)/6,  q1 - v2 = (d1 + 2 d2)/6,  q2 - v2 = (4 d2 - d3)/6,
//   4 beta_r = 13/3 t_r^2 + s_r^2 with second differences t_0 = d1 - d0,
//   t_1 = d2 - d1, t_2 = d3 - d2 and s_0 = 3 d1 - d0, s_1 = -(d1 + d2),
//   s_2 = d3 - 3 d2,
// and the face value v2 + sum_r w_r (q_r - v2), w_r = a_r / sum a with
// a_r = d_r prod_{s != r} e_s^2, e_s = 4 (eps + beta_s) (the common factor 4
// cancels; one division per face).  Along a run the differences and the
// t-terms of each cell are formed once and shared by the faces that use
// them.  For xi_k < 0 the stencil is mirrored and the run is walked from its
// last face down, so that the new value always enters at v4.
template <typename R>
struct Weno5Run {
    R v2, v3, v4, d0, d1, d2, d3, u0, u1, u2;   // u_r = 13/3 t_r^2 + 4 eps
    R eps4;
    __device__ __forceinline__ R tterm(R t) const { return fma(R(13.0 / 3.0) * t, t, eps4); }
    __device__ __forceinline__ void start(R w0, R w1, R w2, R w3, R w4, R eps) {
        eps4 = R(4) * eps;
        v2 = w2;
        v3 = w3;
        v4 = w4;
        d0 = w1 - w0;
        d1 = w2 - w1;
        d2 = w3 - w2;
        d3 = w4 - w3;
        u0 = tterm(d1 - d0);
        u1 = tterm(d2 - d1);
        u2 = tterm(d3 - d2);
    }
    __device__ __forceinline__ R face() const {
        const R s0 = fma(R(3), d1, -d0), s1 = d1 + d2, s2 = fma(R(-3), d2, d3);
        const R e0 = fma(s0, s0, u0), e1 = fma(s1, s1, u1), e2 = fma(s2, s2, u2);
        const R E0 = e0 * e0, E1 = e1 * e1, E2 = e2 * e2;
        const R a0 = E1 * E2, a1 = E0 * E2, a2 = E0 * E1;
        // linear weights 0.1, 0.6, 0.3 folded into the candidate corrections
        // (0.2 d2 shared by c1 and c2)
        const R c0 = fma(R(5.0 / 60.0), d1, R(-2.0 / 60.0) * d0);
        const R p2 = R(0.2) * d2;
        const R c1 = fma(R(0.1), d1, p2);
        const R c2 = fma(R(-0.05), d3, p2);
        const R num = fma(a0, c0, fma(a1, c1, a2 * c2));
        const R den = fma(R(0.1), a0, fma(R(0.6), a1, R(0.3) * a2));
        R q;
        // FP32: the fast reciprocal-based quotient (2 ulp) is far inside the
        // FP32 variant's error budget; FP64: the Newton-refined reciprocal of
        // div_face (2^-46), cheaper on this part's FP64 pipe than the IEEE
        // division
        if constexpr (std::is_same<R, float>::value) q = __fdividef(num, den);
        else q = div_face(num, den);
        return v2 + q;
    }
    __device__ __forceinline__ void shift(R w5) {
        const R d4 = w5 - v4;
        u0 = u1;
        u1 = u2;
        u2 = tterm(d4 - d3);
        d0 = d1;
        d1 = d2;
        d2 = d3;
        d3 = d4;
        v2 = v3;
        v3 = v4;
        v4 = w5;
    }
};

// Phase 3c: face values h_{i-1/2} for faces f = 0..nz (face f lies between
// tile nodes f-1 and f), upwind by the sign of xi_k; runs of kRun faces per
// thread, consecutive threads on consecutive velocity rows (the row stride
// Z + 6 keeps their shared-memory reads apart), the walk direction chosen by
// index arithmetic so that threads of both signs run the same instructions.
// At xi_k = 0 the face values are formed as for xi_k > 0 and then multiplied
// by xi_k = 0 in the flux difference.
constexpr int kRun = 4;
template <typename R>
__device__ void faces(const SlabDesc& sd, const WorkItem& it, const Smem<R>& s, int Z,
                      const R* __restrict__ rtab, int tid, int nth) {
    const int Q = sd.Q, W = Z + 6, nf = it.nz + 1, rows = 2 * Q;
    const int nruns = (nf + kRun - 1) / kRun;
    TableLayout L(Q);
    const R* xi = rtab + sd.tab_off + L.xi;
    const R eps = (R)sd.weno_eps;
    for (int e = tid; e < rows * nruns; e += nth) {
        const int r = e % rows, run = e / rows;
        const int k = r % Q;
        const int fa = run * kRun, n = min(kRun, nf - fa), fl = fa + n - 1;
        const bool pos = xi[k] >= R(0);
        const int dir = pos ? 1 : -1, f0 = pos ? fa : fl;
        // x > 0: face f uses h[f .. f+4], walked up; x < 0: h[f+5 .. f+1], walked down
        const R* hb = s.F + (size_t)r * W + (pos ? fa : fl + 5);
        R* out = s.Face + (size_t)r * (Z + 1);
        Weno5Run<R> w;
        w.start(hb[0], hb[dir], hb[2 * dir], hb[3 * dir], hb[4 * dir], eps);
#pragma unroll
        for (int q = 0; q < kRun; ++q) {
            if (q >= n) break;
            out[f0 + dir * q] = w.face();
            if (q + 1 < n) w.shift(hb[dir * (q + 5)]);
        }
    }
}

// ---------------------------------------------------------------------------
// Double-float arithmetic for the FP64_DF faces: a value is an unevaluated
// pair hi + lo of floats (about 48 significant bits).  Addition is Knuth's
// TwoSum with the low parts folded in and one renormalisation (Dekker's
// FastTwoSum); multiplication is the FMA TwoProduct with the cross terms;
// the quotient takes the float reciprocal of the divisor's head and two
// remainder corrections (each adds ~24 bits).  __fadd_rn / __fmul_rn keep
// the compiler from contracting the error-free transformations.
// ---------------------------------------------------------------------------
struct dfl {
    float h, l;
};
__device__ __forceinline__ dfl dfl_of(double x) {
    const float2 p = df_split(x);
    return {p.x, p.y};
}
__device__ __forceinline__ dfl dfl_add(dfl a, dfl b) {
    const float s = __fadd_rn(a.h, b.h), bb = __fsub_rn(s, a.h);
    const float e = __fadd_rn(__fsub_rn(a.h, __fsub_rn(s, bb)), __fsub_rn(b.h, bb));
    const float t = __fadd_rn(e, __fadd_rn(a.l, b.l));
    const float h = __fadd_rn(s, t);
    return {h, __fsub_rn(t, __fsub_rn(h, s))};
}
__device__ __forceinline__ dfl dfl_sub(dfl a, dfl b) { return dfl_add(a, {-b.h, -b.l}); }
__device__ __forceinline__ dfl dfl_mul(dfl a, dfl b) {
    const float p = __fmul_rn(a.h, b.h);
    float e = fmaf(a.h, b.h, -p);
    e = fmaf(a.h, b.l, e);
    e = fmaf(a.l, b.h, e);
    const float h = __fadd_rn(p, e);
    return {h, __fsub_rn(e, __fsub_rn(h, p))};
}
// times a float (exact small integers such as 3)
__device__ __forceinline__ dfl dfl_mulf(dfl a, float b) {
    const float p = __fmul_rn(a.h, b);
    float e = fmaf(a.h, b, -p);
    e = fmaf(a.l, b, e);
    const float h = __fadd_rn(p, e);
    return {h, __fsub_rn(e, __fsub_rn(h, p))};
}
__device__ __forceinline__ dfl dfl_div(dfl a, dfl b) {
    const float r = __frcp_rn(b.h);
    const float q1 = __fmul_rn(a.h, r);
    const dfl r1 = dfl_sub(a, dfl_mulf(b, q1));
    const float q2 = __fmul_rn(r1.h, r);
    const dfl r2 = dfl_sub(r1, dfl_mulf(b, q2));
    const float q3 = __fmul_rn(r2.h, r);
    const float s = __fadd_rn(q1, q2), bb = __fsub_rn(s, q1);
    const float e = __fadd_rn(__fsub_rn(q1, __fsub_rn(s, bb)), __fsub_rn(q2, bb));
    return dfl_add({s, e}, {q3, 0.0f});
}
// the constants of the difference-form WENO-5 face as pairs
__device__ __forceinline__ dfl dfl_const(double x) {
    const float h = (float)x;
    return {h, (float)(x - (double)h)};
}

// The difference-form WENO-5 run of Weno5Run in double-float arithmetic.
struct Weno5RunDF {
    dfl v2, v3, v4, d0, d1, d2, d3, u0, u1, u2;
    dfl eps4, k133;
    __device__ __forceinline__ dfl tterm(dfl t) const { return dfl_add(dfl_mul(dfl_mul(k133, t), t), eps4); }
    // eps4 = 4 eps as a pair (formed once per thread by the caller)
    __device__ __forceinline__ void start(double w0, double w1, double w2, double w3, double w4, dfl e4) {
        eps4 = e4;
        k133 = dfl_const(13.0 / 3.0);
        const dfl a0 = dfl_of(w0), a1 = dfl_of(w1);
        v2 = dfl_of(w2);
        v3 = dfl_of(w3);
        v4 = dfl_of(w4);
        d0 = dfl_sub(a1, a0);
        d1 = dfl_sub(v2, a1);
        d2 = dfl_sub(v3, v2);
        d3 = dfl_sub(v4, v3);
        u0 = tterm(dfl_sub(d1, d0));
        u1 = tterm(dfl_sub(d2, d1));
        u2 = tterm(dfl_sub(d3, d2));
    }
    __device__ __forceinline__ double face() const {
        const dfl s0 = dfl_sub(dfl_mulf(d1, 3.0f), d0), s1 = dfl_add(d1, d2), s2 = dfl_sub(d3, dfl_mulf(d2, 3.0f));
        const dfl e0 = dfl_add(dfl_mul(s0, s0), u0), e1 = dfl_add(dfl_mul(s1, s1), u1), e2 = dfl_add(dfl_mul(s2, s2), u2);
        const dfl E0 = dfl_mul(e0, e0), E1 = dfl_mul(e1, e1), E2 = dfl_mul(e2, e2);
        const dfl a0 = dfl_mul(E1, E2), a1 = dfl_mul(E0, E2), a2 = dfl_mul(E0, E1);
        const dfl c0 = dfl_sub(dfl_mul(dfl_const(5.0 / 60.0), d1), dfl_mul(dfl_const(2.0 / 60.0), d0));
        const dfl c1 = dfl_add(dfl_mul(dfl_const(0.2), d2), dfl_mul(dfl_const(0.1), d1));
        const dfl c2 = dfl_sub(dfl_mul(dfl_const(0.2), d2), dfl_mul(dfl_const(0.05), d3));
        const dfl num = dfl_add(dfl_add(dfl_mul(a0, c0), dfl_mul(a1, c1)), dfl_mul(a2, c2));
        const dfl den = dfl_add(dfl_add(dfl_mul(dfl_const(0.1), a0), dfl_mul(dfl_const(0.6), a1)),
                                dfl_mul(dfl_const(0.3), a2));
        const dfl f = dfl_add(v2, dfl_div(num, den));
        return f2d_bits(f.h) + f2d_bits(f.l);
    }
    __device__ __forceinline__ void shift(double w5) {
        const dfl v5 = dfl_of(w5);
        const dfl d4 = dfl_sub(v5, v4);
        u0 = u1;
        u1 = u2;
        u2 = tterm(dfl_sub(d4, d3));
        d0 = d1;
        d1 = d2;
        d2 = d3;
        d3 = d4;
        v2 = v3;
        v3 = v4;
        v4 = v5;
    }
};

// faces() of the FP64_DF kernel: the same runs and walk, the face values in
// double-float arithmetic on the FP32 pipe, stored as FP64.
__device__ inline void faces_df(const SlabDesc& sd, const WorkItem& it, const Smem<double>& s, int Z,
                                const double* __restrict__ tab, int tid, int nth) {
    const int Q = sd.Q, W = Z + 6, nf = it.nz + 1, rows = 2 * Q;
    const int nruns = (nf + kRun - 1) / kRun;
    TableLayout L(Q);
    const double* xi = tab + sd.tab_off + L.xi;
    const dfl eps4 = dfl_const(4.0 * sd.weno_eps);
    for (int e = tid; e < rows * nruns; e += nth) {
        const int r = e % rows, run = e / rows;
        const int k = r % Q;
        const int fa = run * kRun, n = min(kRun, nf - fa), fl = fa + n - 1;
        const bool pos = xi[k] >= 0.0;
        const int dir = pos ? 1 : -1, f0 = pos ? fa : fl;
        const double* hb = s.F + (size_t)r * W + (pos ? fa : fl + 5);
        double* out = s.Face + (size_t)r * (Z + 1);
        Weno5RunDF w;
        w.start(hb[0], hb[dir], hb[2 * dir], hb[3 * dir], hb[4 * dir], eps4);
#pragma unroll
        for (int q = 0; q < kRun; ++q) {
            if (q >= n) break;
            out[f0 + dir * q] = w.face();
            if (q + 1 < n) w.shift(hb[dir * (q + 5)]);
        }
    }
}

// Raw moment sums of one node from a column h[k * stride] (k < Q).  The
// conserved moments (S0, S1, S2 of F and G0) are summed in FP64; S3 and G1
// (heat flux) in R.  The velocity powers come from xp = [xi, xi^2, xi^3]
// (FP64) and xr = [xi, xi^3] (R).
//
// FP64 state: four interleaved chains over k, joined as ((a0 + a1) + (a2 + a3)).
//
// FP32 state: the pair form.  Velocity j < H = (Q+1)/2 and its mirror Q-1-j
// (xi_{Q-1-j} = -xi_j) give one term per pair, with a = h_j, b = h_{Q-1-j}
// (b = 0 for the middle velocity of an odd Q):
//   S0, G0: a + b;   S1: xi_j (a - b);   S2: xi_j^2 (a + b);
//   S3: xi_j^3 (a - b);   G1: xi_j (a - b),
// the FP64 terms from floats widened exactly by bit surgery.  The pairs 2g
// and 2g+1 form group g < G = (H+1)/2 (term(2g) + term(2g+1); a last lone
// pair alone), and the G group terms are summed in four chains over g mod
// 4, joined as ((c0 + c1) + (c2 + c3)).  Every operation is an explicitly
// rounded one, so the stage kernel, which forms the group terms where it
// writes the new state (pair_terms_f32) and sums them afterwards
// (sum_pair_terms), gets the same bits as a sum formed here in one pass.
__device__ __forceinline__ bool moment_is_f64(int which) {
    return which == MOM_S0 || which == MOM_S1 || which == MOM_S2 || which == MOM_G0;
}

__device__ __forceinline__ double pair_term_f64(int which, int j, int Q, double a, double b,
                                                const double* __restrict__ xp) {
    if (which == MOM_S0 || which == MOM_G0) return __dadd_rn(a, b);
    if (which == MOM_S1) return __dmul_rn(xp[j], __dsub_rn(a, b));
    return __dmul_rn(xp[Q + j], __dadd_rn(a, b));                    // S2
}

__device__ __forceinline__ float pair_term_f32(int which, int j, int Q, float a, float b,
                                               const float* __restrict__ xr) {
    return __fmul_rn(which == MOM_S3 ? xr[Q + j] : xr[j], __fsub_rn(a, b));   // S3, G1
}

template <typename T>
__device__ __forceinline__ T add_rn(T a, T b) {
    if constexpr (std::is_same<T, float>::value) return __fadd_rn(a, b);
    else return __dadd_rn(a, b);
}

// Sum of the n terms term(j) in four chains over j mod 4.
template <typename T, typename F>
__device__ __forceinline__ T sum_chains4(int n, F term) {
    T c0 = 0, c1 = 0, c2 = 0, c3 = 0;
    int j = 0;
    for (; j + 3 < n; j += 4) {
        c0 = add_rn(c0, term(j));
        c1 = add_rn(c1, term(j + 1));
        c2 = add_rn(c2, term(j + 2));
        c3 = add_rn(c3, term(j + 3));
    }
    if (j < n) c0 = add_rn(c0, term(j));
    if (j + 1 < n) c1 = add_rn(c1, term(j + 1));
    if (j + 2 < n) c2 = add_rn(c2, term(j + 2));
    return add_rn(add_rn(c0, c1), add_rn(c2, c3));
}

// Sum of n stored terms v[j * stride], in the order of sum_chains4.
template <typename T>
__device__ __forceinline__ T sum_pair_terms(const T* v, int n, long long stride) {
    return sum_chains4<T>(n, [&](int j) { return v[j * stride]; });
}

template <typename R>
__device__ __forceinline__ double moment_sum(int which, int Q, const R* h, long long stride,
                                             const double* __restrict__ xp, const R* __restrict__ xr) {
    const int p = (which >= MOM_G0) ? which - MOM_G0 : which;   // power of xi
    if constexpr (std::is_same<R, double>::value) {
        const double* w = xp + (p > 0 ? p - 1 : 0) * Q;
        auto acc = [&](double a, int k) { return p == 0 ? a + h[k * stride] : fma(w[k], h[k * stride], a); };
        double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
        int k = 0;
        for (; k + 3 < Q; k += 4) {
            a0 = acc(a0, k);
            a1 = acc(a1, k + 1);
            a2 = acc(a2, k + 2);
            a3 = acc(a3, k + 3);
        }
        for (; k < Q; ++k) a0 = acc(a0, k);
        return (a0 + a1) + (a2 + a3);
    } else {
        const int H = (Q + 1) / 2, G = (H + 1) / 2;
        auto ha = [&](int j) { return h[j * stride]; };
        auto hb = [&](int j) { return (Q - 1 - j != j) ? h[(Q - 1 - j) * stride] : 0.f; };
        if (moment_is_f64(which)) {
            auto term = [&](int j) { return pair_term_f64(which, j, Q, f2d_bits(ha(j)), f2d_bits(hb(j)), xp); };
            return sum_chains4<double>(
                G, [&](int g) { return 2 * g + 1 < H ? __dadd_rn(term(2 * g), term(2 * g + 1)) : term(2 * g); });
        }
        auto term = [&](int j) { return pair_term_f32(which, j, Q, ha(j), hb(j), xr); };
        return (double)sum_chains4<float>(
            G, [&](int g) { return 2 * g + 1 < H ? __fadd_rn(term(2 * g), term(2 * g + 1)) : term(2 * g); });
    }
}

// The group terms of the four FP64 and two R moment sums for group g of
// one node t and distribution d: pairs j0 = 2g and j1 = 2g+1 (two: j1 < H),
// from the new state's values a0, b0 (velocity j0 and its mirror) and a1, b1;
// b is 0 for a middle velocity.  Into t64[slot][g * Z + t] (S0, S1, S2, G0)
// and t32[slot][g * Z + t] (S3, G1), slot blocks of G Z values.
__device__ __forceinline__ void pair_terms_f32(int d, int g, bool two, int t, int Q, int Z, float a0, float b0,
                                               float a1, float b1, const double* __restrict__ xp,
                                               const float* __restrict__ xr, double* t64, float* t32) {
    const int j0 = 2 * g, j1 = 2 * g + 1;
    const size_t o = (size_t)g * Z + t, blk = (size_t)pair_groups(Q) * Z;
    const double wa0 = f2d_bits(a0), wb0 = f2d_bits(b0), wa1 = f2d_bits(a1), wb1 = f2d_bits(b1);
    auto t8 = [&](int which) {
        const double x = pair_term_f64(which, j0, Q, wa0, wb0, xp);
        return two ? __dadd_rn(x, pair_term_f64(which, j1, Q, wa1, wb1, xp)) : x;
    };
    auto t4 = [&](int which) {
        const float x = pair_term_f32(which, j0, Q, a0, b0, xr);
        return two ? __fadd_rn(x, pair_term_f32(which, j1, Q, a1, b1, xr)) : x;
    };
    if (d == 0) {
        t64[o] = t8(MOM_S0);
        t64[blk + o] = t8(MOM_S1);
        t64[2 * blk + o] = t8(MOM_S2);
        t32[o] = t4(MOM_S3);
    } else {
        t64[3 * blk + o] = t8(MOM_G0);
        t32[blk + o] = t4(MOM_G1);
    }
}

// Velocity powers of moment_sum from the tables xi (FP64) and rxi (R).
template <typename R>
__device__ __forceinline__ void velocity_powers(int Q, const double* __restrict__ xi, const R* __restrict__ rxi,
                                                double* xp, R* xr, int tid, int nth) {
    for (int k = tid; k < Q; k += nth) {
        const double x = xi[k];
        xp[k] = x;
        xp[Q + k] = x * x;
        xp[2 * Q + k] = x * x * x;
        const R y = rxi[k];
        xr[k] = y;
        xr[Q + k] = y * y * y;
    }
}

// Raw moment sums of the tile held in s.F (columns 3 .. nz+2), from velocity
// powers staged in shared memory (xp = [xi, xi^2, xi^3] FP64, xr = [xi, xi^3]
// in R).  Called by all threads once the tile's velocity work is done: one
// sum per warp, lanes on nodes, where the tile allows.
template <typename R>
__device__ void tile_moment_sums_staged(const SlabDesc& sd, const WorkItem& it, const Smem<R>& s, int Z,
                                        const double* xp, const R* xr, double* __restrict__ mom_out, long long NN) {
    const int Q = sd.Q, W = Z + 6, nz = it.nz;
    if (nz <= 32 && blockDim.x >= 32 * kNumMoments) {
        const int which = threadIdx.x >> 5, t = threadIdx.x & 31;
        if (which < kNumMoments && t < nz) {
            const int d = which >= MOM_G0 ? 1 : 0;
            const R* h = s.F + (size_t)d * Q * W + t + 3;
            mom_out[which * NN + sd.node_off + it.i0 + t] = moment_sum<R>(which, Q, h, W, xp, xr);
        }
        return;
    }
    for (int e = threadIdx.x; e < kNumMoments * nz; e += blockDim.x) {
        int t = e % nz, which = e / nz;
        int d = which >= MOM_G0 ? 1 : 0;
        const R* h = s.F + (size_t)d * Q * W + t + 3;
        mom_out[which * NN + sd.node_off + it.i0 + t] = moment_sum<R>(which, Q, h, W, xp, xr);
    }
}

// The same with the velocity powers formed here first, in the (then free)
// table block s.P / s.S (5 Q values).
template <typename R>
__device__ void tile_moment_sums(const SlabDesc& sd, const WorkItem& it, const Smem<R>& s, int Z,
                                 const double* __restrict__ xi, const R* __restrict__ rxi,
                                 double* __restrict__ mom_out, long long NN) {
    const int Q = sd.Q;
    double* xp = reinterpret_cast<double*>(s.P);
    R* xr = reinterpret_cast<R*>(xp + 3 * Q);
    velocity_powers<R>(Q, xi, rxi, xp, xr, threadIdx.x, blockDim.x);
    __syncthreads();
    tile_moment_sums_staged<R>(sd, it, s, Z, xp, xr, mom_out, NN);
}

}  // namespace evfdlb
