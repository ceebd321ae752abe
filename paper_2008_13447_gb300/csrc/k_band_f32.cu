// k_band_f32.cu -- FP32 instantiation of the seed and band kernels
// (k_band.cuh), with the FP32 seed kernel.
#include "k_band.cuh"

namespace mad {

// FP32 seeds: the row window is centred in FP64 and rounded; the column
// windows are shifted by one constant per block of columns (close to their
// means) and rounded; the dot product runs in FP32 and the shift is removed
// exactly to first order with the FP32 sum of the rounded row window.
template <>
__global__ void k_seed<float>(SeedArgs<float> A)
{
    if (A.nbands && *A.nbands == 0) return;
    extern __shared__ float sh_f[];
    const int l = A.l;
    const int B = blockDim.x;
    float *arow = sh_f;                   // l
    float *ycol = sh_f + l;               // B + l
    __shared__ float s_asum;
    const int k = A.krows[blockIdx.y];
    const int64_t kr = (int64_t)k * A.R;
    const int64_t a = (k == 0) ? 0 : kr - 1;
    const int64_t jb = (int64_t)blockIdx.x * B;
    // first column window of this block and its shift
    const int64_t cb = (k == 0) ? jb : (jb > 0 ? jb - 1 : 0);
    const int64_t cshift = cb < A.nl ? cb : A.nl - 1;
    const double shift = A.mu[cshift];
    const double mua = A.mu[a];
    for (int t = threadIdx.x; t < l; t += B) arow[t] = (float)(A.x[a + t] - mua);
    for (int u = threadIdx.x; u < B + l; u += B) {
        const int64_t idx = cb + u;
        ycol[u] = idx < A.nl + l - 1 ? (float)(A.x[idx] - shift) : 0.0f;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        float s = 0.0f;
        for (int t = threadIdx.x; t < l; t += 32) s += arow[t];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0) s_asum = s;
    }
    __syncthreads();
    const int64_t j = jb + threadIdx.x;
    if (j >= A.spitch) return;
    int64_t ra, c;
    if (k == 0) { ra = 0; c = j; }
    else if (j == 0) { ra = kr; c = 0; }
    else { ra = kr - 1; c = j - 1; }
    float out = 0.0f;
    if (c < A.nl && ra < A.nl) {
        if (ra == a) {
            const float *y = ycol + (c - cb);
            float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
            int t = 0;
            for (; t + 3 < l; t += 4) {
                s0 = fmaf(arow[t], y[t], s0);
                s1 = fmaf(arow[t + 1], y[t + 1], s1);
                s2 = fmaf(arow[t + 2], y[t + 2], s2);
                s3 = fmaf(arow[t + 3], y[t + 3], s3);
            }
            for (; t < l; ++t) s0 = fmaf(arow[t], y[t], s0);
            const double corr = (double)s_asum * (A.mu[c] - shift);
            out = (float)(((double)s0 + (double)s1) + ((double)s2 + (double)s3) - corr);
        } else {
            // the single (kR, 0) entry: direct FP64
            const double mur = A.mu[ra], muc = A.mu[c];
            double s = 0.0;
            for (int t = 0; t < l; ++t) s = fma(A.x[ra + t] - mur, A.x[c + t] - muc, s);
            out = (float)s;
        }
    }
    A.seed[(int64_t)k * A.spitch + j] = out;
}

template void launch_seed<float>(const SeedArgs<float> &, cudaStream_t);
template void launch_band<float>(const BandArgs<float> &, bool, int, cudaStream_t);
template int band_occupancy<float>(bool, int, int);
template size_t band_smem<float>(bool, int, int);

}  // namespace mad
