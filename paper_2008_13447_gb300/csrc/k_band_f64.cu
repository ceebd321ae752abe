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
template void launch_band<double>(const BandArgs<double> &, bool, int, cudaStream_t);
template int band_occupancy<double>(bool, int, int);
template size_t band_smem<double>(bool, int, int);

}  // namespace mad
