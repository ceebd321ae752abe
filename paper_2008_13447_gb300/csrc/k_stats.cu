// k_stats.cu -- window statistics (mean, centred second moment) and the
// per-window data of the diagonal recurrence.
//
// Sec. 4.3 computes mu and sigma of every window from running sums (Eq. DIST
// needs them). Running sums of raw values cancel badly on drifting series,
// so here every window's mean and M2 = l sigma^2 are formed once at lmin by
// a two-pass loop over the window and then carried from length l-1 to l by
// one Welford step per window (the window gains x_{i+l-1}); the statistics
// stay FP64.
#include "kernels.cuh"

namespace mad {

// run[i] = number of equal consecutive values starting at x[i], capped at
// cap (a window (i, l) is flat iff run[i] >= l).
__global__ void k_flat_runs(const double *__restrict__ x, int64_t n, int cap, int32_t *__restrict__ run)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int r = 1;
        const double v = x[i];
        while (r < cap && i + r < n && x[i + r] == v) ++r;
        run[i] = r;
    }
}

// Two-pass mean and M2 of every window of length l (i < nl).
__global__ void k_stats_init(const double *__restrict__ x, int64_t nl, int l, double *__restrict__ mu,
                             double *__restrict__ m2)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nl; i += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int t = 0; t < l; ++t) s += x[i + t];
        const double m = s / l;
        double v = 0.0;
        for (int t = 0; t < l; ++t) {
            const double d = x[i + t] - m;
            v = fma(d, d, v);
        }
        mu[i] = m;
        m2[i] = v;
    }
}

// The per-length preparation kernels run on a side stream beside the band
// kernel, whose three CTAs per SM leave 4096 registers of each SM free: in
// blocks of PREP_THREADS threads at no more than 32 registers a block fits
// in that room, so these kernels overlap the band kernel instead of waiting
// for its end.
constexpr int PREP_THREADS = 128;

// Welford step from length l-1 to l for windows i < nl (= n - l + 1):
// mu_new = mu + (x_{i+l-1} - mu) / l ; M2_new = M2 + (x_{i+l-1} - mu)(x_{i+l-1} - mu_new).
// Reads mu_o/m2_o, writes mu_n/m2_n (distinct buffers).
__global__ void __launch_bounds__(PREP_THREADS, 16)
k_stats_step(const double *__restrict__ x, int64_t nl, int l, const double *__restrict__ mu_o,
                             const double *__restrict__ m2_o, double *__restrict__ mu_n, double *__restrict__ m2_n)
{
    const double inv_l = 1.0 / l;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nl; i += (int64_t)gridDim.x * blockDim.x) {
        const double xn = x[i + l - 1];
        const double m = mu_o[i];
        const double d = xn - m;
        const double mn = fma(d, inv_l, m);
        mu_n[i] = mn;
        m2_n[i] = fma(d, xn - mn, m2_o[i]);
    }
}

// Per-window recurrence data Col<T> for j in [0, npad):
//   j <  nl: df_{j-1}, dg_{j-1} (0 for j = 0), inv_j (0 if flat)
//   j >= nl: df = dg = 0, inv = NaN (so no padded column ever passes a test)
template <typename T>
__global__ void __launch_bounds__(PREP_THREADS, 16) k_coldata(const double *__restrict__ x, int64_t nl, int64_t npad, int l,
                          const double *__restrict__ mu, const double *__restrict__ m2,
                          const int32_t *__restrict__ run, Col<T> *__restrict__ col, double *__restrict__ isd)
{
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < npad; j += (int64_t)gridDim.x * blockDim.x) {
        Col<T> c;
        c.pad = T(0);
        if (j < nl) {
            if (j > 0) {
                const double a = x[j - 1 + l], b = x[j - 1];
                c.df = T(0.5 * (a - b));
                c.dg = T((a - mu[j]) + (b - mu[j - 1]));
            } else {
                c.df = T(0);
                c.dg = T(0);
            }
            const double iv = (run[j] >= l) ? 0.0 : 1.0 / sqrt(m2[j]);
            c.inv = T(iv);
            isd[j] = iv;
        } else {
            c.df = T(0);
            c.dg = T(0);
            c.inv = T(__longlong_as_double(0x7ff8000000000000ULL));
        }
        col[j] = c;
    }
}

template <typename T>
void launch_coldata(const double *x, int64_t nl, int64_t npad, int l, const double *mu, const double *m2,
                    const int32_t *run, Col<T> *col, double *isd, cudaStream_t s)
{
    k_coldata<T><<<(unsigned)((npad + PREP_THREADS - 1) / PREP_THREADS), PREP_THREADS, 0, s>>>(x, nl, npad, l, mu, m2,
                                                                                          run, col, isd);
}
template void launch_coldata<float>(const double *, int64_t, int64_t, int, const double *, const double *,
                                    const int32_t *, Col<float> *, double *, cudaStream_t);
template void launch_coldata<double>(const double *, int64_t, int64_t, int, const double *, const double *,
                                     const int32_t *, Col<double> *, double *, cudaStream_t);

__global__ void k_split_x(const double *__restrict__ x, int64_t n, float *__restrict__ xh, float *__restrict__ xl)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const float h = (float)x[k];
        xh[k] = h;
        xl[k] = (float)(x[k] - (double)h);
    }
}

void launch_stats_step(const double *x, int64_t nl, int l, const double *mu_o, const double *m2_o, double *mu_n,
                       double *m2_n, cudaStream_t s)
{
    k_stats_step<<<(unsigned)((nl + PREP_THREADS - 1) / PREP_THREADS), PREP_THREADS, 0, s>>>(x, nl, l, mu_o, m2_o, mu_n,
                                                                                          m2_n);
}

void launch_split_x(const double *x, int64_t n, float *xh, float *xl, cudaStream_t s)
{
    int64_t g = (n + 255) / 256;
    if (g > 4096) g = 4096;
    k_split_x<<<(unsigned)g, 256, 0, s>>>(x, n, xh, xl);
}

// Contrast factor kappa_i (see ErrModel). Along the diagonal chain of a
// cell (i, j) of the band kernel (at most R + 1 windows above-left of it,
// back to its seed), each recurrence step rounds twice relative to the
// running co-moment (|C| <= sqrt(M2_a M2_b) by Cauchy-Schwarz) and once for
// each FP32 input df, dg; per step the total is below
//     2u sqrt(w_a w_b),   w_k = M2_k + 1.5 (df_k^2 + dg_k^2)
// (Cauchy-Schwarz on (sqrt M2, sqrt 1.5 h) vectors, h^2 = df^2 + dg^2), so the
// correlation error of the cell is below u (2R + 4) kappa_i kappa_j with
//     kappa_i = sqrt(max of w over the chain windows of i / M2_i).
// Block maxima of w over 256 windows are taken, then for each window the
// maximum over the blocks covering the R + 2 windows ending at it (a
// superset, so kappa is never underestimated).
__global__ void k_m2_blockmax(const double *__restrict__ x, const double *__restrict__ mu,
                              const double *__restrict__ m2, int64_t nl, int l, double *__restrict__ blkmax)
{
    __shared__ double sh[32];
    const int64_t i = blockIdx.x * (int64_t)256 + threadIdx.x;
    double v = 0.0;
    if (i < nl) {
        v = m2[i];
        if (i + 1 < nl) {
            const double df = 0.5 * (x[i + l] - x[i]);
            const double dg = (x[i + l] - mu[i + 1]) + (x[i] - mu[i]);
            v += 1.5 * (df * df + dg * dg);
        }
    }
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        v = threadIdx.x < 8 ? sh[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
        if (threadIdx.x == 0) blkmax[blockIdx.x] = v;
    }
}

__global__ void k_kappa(const double *__restrict__ m2, const int32_t *__restrict__ run, int64_t nl, int l, int R,
                        const double *__restrict__ blkmax, float *__restrict__ kappa, float *__restrict__ kappa_max)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    float k = 1.0f;
    if (i < nl) {
        const double mi = m2[i];
        if (run[i] < l && mi > 0.0) {
            const int64_t lo = i - R - 1 < 0 ? 0 : i - R - 1;
            double mx = mi;
            for (int64_t b = lo / 256; b <= i / 256; ++b) mx = fmax(mx, blkmax[b]);
            k = (float)sqrt(mx / mi) * 1.0001f;
            if (!(k >= 1.0f)) k = 1.0f;
        }
        kappa[i] = k;
    }
    for (int o = 16; o > 0; o >>= 1) k = fmaxf(k, __shfl_xor_sync(0xffffffffu, k, o));
    if ((threadIdx.x & 31) == 0) atomicMax(reinterpret_cast<int *>(kappa_max), __float_as_int(k));
}

void launch_kappa(const double *x, const double *mu, const double *m2, const int32_t *run, int64_t nl, int l, int R,
                  double *blkmax, float *kappa, float *kappa_max, cudaStream_t s)
{
    const unsigned nb = (unsigned)((nl + 255) / 256);
    k_m2_blockmax<<<nb, 256, 0, s>>>(x, mu, m2, nl, l, blkmax);
    cudaMemsetAsync(kappa_max, 0, sizeof(float), s);
    k_kappa<<<nb, 256, 0, s>>>(m2, run, nl, l, R, blkmax, kappa, kappa_max);
}

__global__ void k_widen_f32(const float *__restrict__ in, int64_t n, double *__restrict__ out)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (double)in[i];
}

}  // namespace mad
