// mad_internal.cuh -- device-side definitions shared by the kernels of the
// exact variable-length matrix profile (VALMOD / MAD).
//
// Notation follows the paper: series x[0..n), window length l, n_l = n-l+1
// windows, exclusion half-width E(l). For a window i the kernels keep its
// mean mu_i and centred second moment M2_i = sum_t (x_{i+t} - mu_i)^2
// (= l sigma_i^2, population sigma). The correlation of windows i and j is
// q = C(i,j) / sqrt(M2_i M2_j) with the centred co-moment
// C(i,j) = sum_t (x_{i+t} - mu_i)(x_{j+t} - mu_j), and Eq. DIST gives
// d = sqrt(2 l (1 - q)).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

namespace mad {

constexpr int CH = 32;              // columns per wavefront chunk (one per lane)
constexpr int MAXP = 64;            // largest p (entries kept per row)
constexpr int KMAX = 64;            // largest discord-table rank count

// Geometry of the diagonal band kernel: BAND_NW warps per CTA, RPL rows per
// lane, so a band holds R = 32 * RPL * BAND_NW consecutive rows; R is also
// the re-seed period of every diagonal (each diagonal restarts from a direct
// dot product at the top or left edge of every work unit). RPL is at most 4:
// four rows per lane keep the FP32 kernel within 80 registers, so three CTAs
// (24 warps) share an SM, which hides the recurrence's latency better than
// eight rows per lane at two CTAs. Smaller RPL when the per-row top-p lists
// would not fit in shared memory.
constexpr int BAND_NW = 8;
__host__ __device__ __forceinline__ int band_nbins(int p) { return 2 * p; }
template <typename T> inline int band_rpl(int p)
{
    // shared bytes per row for the top-p list: p * (sizeof(T) + 4) + 4
    const int budget = 96 * 1024;
    const int max_rpl = 4;
    for (int rpl = max_rpl; rpl > 1; rpl /= 2)
        if (32 * rpl * BAND_NW * (p * (int)(sizeof(T) + 4) + 4) <= budget) return rpl;
    return 1;
}

// Per-window data the band kernel reads for column j (and for row j):
//   df = df_{j-1} = (x_{j-1+l} - x_{j-1}) / 2
//   dg = dg_{j-1} = (x_{j-1+l} - mu_j) + (x_{j-1} - mu_{j-1})
//   inv = 1 / sqrt(M2_j)  (0 for a flat window, NaN past the last window)
// with df_{-1} = dg_{-1} = 0 for the virtual window before the first.
// The centred co-moment then obeys, along every diagonal,
//   C(i, j) = C(i-1, j-1) + df_{i-1} dg_{j-1} + df_{j-1} dg_{i-1}.
template <typename T> struct __align__(4 * sizeof(T)) Col { T df, dg, inv, pad; };

// Dynamic shared-memory opt-in of kernel `fn` raised, once per device, to the
// largest the device allows next to the kernel's static shared memory. Set
// per launch instead, a smaller value set by one host thread could meet
// another thread's larger launch (the batch path profiles series from
// several threads).
inline void smem_optin_max(const void *fn, std::once_flag (&once)[64])
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return;
    std::call_once(once[dev], [fn, dev] {
        int mx = 0;
        cudaFuncAttributes fa{};
        if (cudaDeviceGetAttribute(&mx, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
            cudaFuncGetAttributes(&fa, fn) != cudaSuccess)
            return;
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, mx - (int)fa.sharedSizeBytes);
    });
}

// Row flags of the per-length pipeline.
// ROW_SKIP: motif mode, a non-valid row left undefined at this length.
enum : int32_t { ROW_DONE = 0, ROW_RECOMPUTE = 1, ROW_FLAT = 2, ROW_DIRECT = 3, ROW_SKIP = 4 };

// Order-preserving maps from floating point to signed integers (for
// atomicMax on shared or global memory).
__device__ __forceinline__ int f2ord(float f)
{
    int i = __float_as_int(f);
    return i >= 0 ? i : (i ^ 0x7fffffff);
}
__device__ __forceinline__ float ord2f(int i) { return __int_as_float(i >= 0 ? i : (i ^ 0x7fffffff)); }

__host__ __device__ __forceinline__ int64_t excl_zone(int l, int num, int den)
{
    return ((int64_t)l * num + den - 1) / den;
}

__device__ __forceinline__ bool nontrivial(int64_t i, int64_t j, int64_t E)
{
    int64_t d = i - j;
    return d > E || -d > E;
}

// Number of non-trivial partners of window i among n_l windows.
__device__ __forceinline__ int64_t nontrivial_count(int64_t i, int64_t nl, int64_t E)
{
    int64_t lo = i - E < 0 ? 0 : i - E;
    int64_t hi = i + E > nl - 1 ? nl - 1 : i + E;
    return nl - (hi - lo + 1);
}

__device__ __forceinline__ double clamp_q(double q) { return q > 1.0 ? 1.0 : (q < -1.0 ? -1.0 : q); }

// Eq. DIST from the correlation.
__device__ __forceinline__ double dist_from_q(double q, int l) { return sqrt(2.0 * l * (1.0 - clamp_q(q))); }

// Correlation with the flat-window reading: two flat windows correlate 1, a
// flat and a non-flat window 0.
__device__ __forceinline__ double corr(double C, double m2i, double m2j, bool flat_i, bool flat_j)
{
    if (flat_i || flat_j) return (flat_i && flat_j) ? 1.0 : 0.0;
    return clamp_q(C / sqrt(m2i * m2j));
}

}  // namespace mad
