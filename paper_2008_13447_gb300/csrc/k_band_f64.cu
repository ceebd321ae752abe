// k_band_f64.cu -- FP64 instantiation of the seed and band kernels
// (k_band.cuh), with the FP64 seed kernel.
#include "k_band.cuh"

namespace mad {

// FP64 seeds: the centred dot product evaluated directly in FP64.
template <>
__global__ void k_seed<double>(SeedArgs<double> A)
{
    if (A.nbands && *A.nbands == 0) return;
    extern __shared__ double sh_d[];
    const int l = A.l;
    double *arow = sh_d;                  // centred row window (l)
    const int k = A.krows[blockIdx.y];
    const int64_t kr = (int64_t)k * A.R;
    const int64_t a = (k == 0) ? 0 : kr - 1;
    const double mua = A.mu[a];
    for (int t = threadIdx.x; t < l; t += blockDim.x) arow[t] = A.x[a + t] - mua;
    __syncthreads();
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= A.spitch) return;
    int64_t ra, c;
    if (k == 0) { ra = 0; c = j; }
    else if (j == 0) { ra = kr; c = 0; }
    else { ra = kr - 1; c = j - 1; }
    double s = 0.0;
    if (c < A.nl && ra < A.nl) {
        const double muc = A.mu[c];
        if (ra == a) {
            for (int t = 0; t < l; ++t) s = fma(arow[t], A.x[c + t] - muc, s);
        } else {
            const double mur = A.mu[ra];
            for (int t = 0; t < l; ++t) s = fma(A.x[ra + t] - mur, A.x[c + t] - muc, s);
        }
    }
    A.seed[(int64_t)k * A.spitch + j] = s;
}

template <>
void launch_seed<double>(const SeedArgs<double> &a, cudaStream_t s)
{
    const int B = 256;
    dim3 grid((unsigned)((a.spitch + B - 1) / B), (unsigned)a.nk);
    const size_t sm = sizeof(double) * a.l;
    static std::once_flag once[64];
    smem_optin_max((const void *)k_seed<double>, once);
    k_seed<double><<<grid, B, sm, s>>>(a);
}
// Seed rows from length l to l + 1 without recomputing them: the centred
// co-moment of two windows gains one pair of elements (the Welford
// co-moment step), C_{l+1}(a, c) = C_l(a, c) + l/(l+1) (x[a+l] - mu_l[a])
// (x[c+l] - mu_l[c]), applied in FP64 to the master copy in place; entries
// whose windows no longer exist at l + 1 become 0 (as the direct kernel
// writes them). The band kernel's copy in T is written from the master.
// Entry (k, j) of the table: row 0 holds C(0, j); row k >= 1 holds C(kS, 0)
// at j = 0 and C(kS - 1, j - 1) for j >= 1.
// Each thread takes one column j and SEED_ROWS consecutive seed rows, so
// the column's factor (x[j-1+l] - mu[j-1]) is loaded once for them; the
// block's row factors are formed once in shared memory. Away from the first
// row and column the rows go in batches of SEED_BATCH whose loads are all
// issued before the first store (several loads in flight per thread: the
// step is HBM-bound).
constexpr int SEED_ROWS = 16;
constexpr int SEED_BATCH = 4;

__device__ __forceinline__ double seed_entry(const double *x, const double *mu, int64_t nl, int l, int S, int64_t k,
                                             int64_t j, double f, double v)
{
    int64_t ra, c;
    if (k == 0) {
        ra = 0;
        c = j;
    } else if (j == 0) {
        ra = k * S;
        c = 0;
    } else {
        ra = k * S - 1;
        c = j - 1;
    }
    return (ra < nl && c < nl) ? fma(f * (x[ra + l] - mu[ra]), x[c + l] - mu[c], v) : 0.0;
}

template <typename T>
__global__ void __launch_bounds__(128, 16) k_seed_step(const double *__restrict__ x, const double *__restrict__ mu,
                                                       int64_t nl, int l, int S, int64_t K, int64_t spitch,
                                                       double *__restrict__ master, T *__restrict__ seed, int update)
{
    // the block's row factors l/(l+1) (x[kS-1+l] - mu[kS-1]) (the same for
    // every column), and which of its rows still exist at l + 1
    __shared__ double sa[SEED_ROWS];
    __shared__ unsigned svalid;
    const int64_t k0 = (int64_t)blockIdx.y * SEED_ROWS;
    const int64_t k1 = k0 + SEED_ROWS < K ? k0 + SEED_ROWS : K;
    const double f = (double)l / (double)(l + 1);
    if (threadIdx.x < 32) {
        const int64_t k = k0 + threadIdx.x;
        const int64_t ra = k * S - 1;
        const bool ok = threadIdx.x < SEED_ROWS && k >= 1 && k < k1 && ra < nl;
        if (threadIdx.x < SEED_ROWS) sa[threadIdx.x] = ok ? f * (x[ra + l] - mu[ra]) : 0.0;
        const unsigned m = __ballot_sync(0xffffffffu, ok);
        if (threadIdx.x == 0) svalid = m;
    }
    __syncthreads();
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= spitch) return;
    if (k0 == 0 || j == 0) {
        // the first seed row (row 0's windows) and the first column
#pragma unroll 1
        for (int64_t k = k0; k < k1; ++k) {
            const int64_t at = k * spitch + j;
            double v = master[at];
            if (update) {
                v = seed_entry(x, mu, nl, l, S, k, j, f, v);
                master[at] = v;
            }
            seed[at] = (T)v;
        }
        return;
    }
    // rows k >= 1, column j >= 1: C(kS - 1, j - 1) gains the row factor
    // times (x[j-1+l] - mu[j-1])
    const unsigned valid = (j - 1 < nl) ? svalid : 0u;
    const double bj = (j - 1 < nl) ? x[j - 1 + l] - mu[j - 1] : 0.0;
    double *mp = master + k0 * spitch + j;
    T *sp = seed + k0 * spitch + j;
    const int nrow = (int)(k1 - k0);
#pragma unroll 1
    for (int t0 = 0; t0 < nrow; t0 += SEED_BATCH) {
        double v[SEED_BATCH];
#pragma unroll
        for (int t = 0; t < SEED_BATCH; ++t) v[t] = t0 + t < nrow ? mp[(int64_t)t * spitch] : 0.0;
        if (update) {
#pragma unroll
            for (int t = 0; t < SEED_BATCH; ++t) {
                v[t] = (valid >> (t0 + t)) & 1u ? fma(sa[t0 + t], bj, v[t]) : 0.0;
                if (t0 + t < nrow) mp[(int64_t)t * spitch] = v[t];
            }
        }
#pragma unroll
        for (int t = 0; t < SEED_BATCH; ++t)
            if (t0 + t < nrow) sp[(int64_t)t * spitch] = (T)v[t];
        mp += SEED_BATCH * spitch;
        sp += SEED_BATCH * spitch;
    }
}

template <typename T>
void launch_seed_step(const double *x, const double *mu, int64_t nl, int l, int S, int64_t K, int64_t spitch,
                      double *master, T *seed, bool update, cudaStream_t s)
{
    // 128-thread blocks at <= 32 registers: they fit beside the band kernel
    const int B = 128;
    const int64_t gx = (spitch + B - 1) / B;
    const int64_t gy = (K + SEED_ROWS - 1) / SEED_ROWS;
    k_seed_step<T><<<dim3((unsigned)gx, (unsigned)gy), B, 0, s>>>(x, mu, nl, l, S, K, spitch, master, seed,
                                                                    update ? 1 : 0);
}
template void launch_seed_step<float>(const double *, const double *, int64_t, int, int, int64_t, int64_t, double *,
                                      float *, bool, cudaStream_t);
template void launch_seed_step<double>(const double *, const double *, int64_t, int, int, int64_t, int64_t, double *,
                                       double *, bool, cudaStream_t);

template void launch_band<double>(const BandArgs<double> &, bool, int, cudaStream_t);
template int band_occupancy<double>(bool, int, int);
template size_t band_smem<double>(bool, int, int);

}  // namespace mad
