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
// the column's factor (x[j-1+l] - mu[j-1]) is loaded once for them.
constexpr int SEED_ROWS = 16;

template <typename T>
__global__ void __launch_bounds__(128, 16) k_seed_step(const double *x, const double *mu, int64_t nl, int l, int S, int64_t K, int64_t spitch,
                            double *master, T *seed, int update)
{
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= spitch) return;
    const int64_t k0 = (int64_t)blockIdx.y * SEED_ROWS;
    const double f = (double)l / (double)(l + 1);
    const int64_t cj = j - 1;   // the column window of rows k >= 1
    const double bj = (cj >= 0 && cj < nl) ? x[cj + l] - mu[cj] : 0.0;
    for (int64_t k = k0; k < k0 + SEED_ROWS && k < K; ++k) {
        const int64_t at = k * spitch + j;
        double v = master[at];
        if (update) {
            const int64_t kS = k * S;
            int64_t ra, c;
            double b = bj;
            if (k == 0) {
                ra = 0;
                c = j;
                b = (c < nl) ? x[c + l] - mu[c] : 0.0;
            } else if (j == 0) {
                ra = kS;
                c = 0;
                b = x[l] - mu[0];
            } else {
                ra = kS - 1;
                c = cj;
            }
            v = (ra < nl && c < nl) ? fma(f * (x[ra + l] - mu[ra]), b, v) : 0.0;
            master[at] = v;
        }
        seed[at] = (T)v;
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
