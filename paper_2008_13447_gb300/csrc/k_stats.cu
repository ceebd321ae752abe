// k_stats.cu -- window statistics (mean, centred second moment) and the
// per-window data of the diagonal recurrence.
//
// Sec. 4.2 computes mu and sigma of every window from running sums (Eq. DIST
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

// Welford step from length l-1 to l for windows i < nl (= n - l + 1):
// mu_new = mu + (x_{i+l-1} - mu) / l ; M2_new = M2 + (x_{i+l-1} - mu)(x_{i+l-1} - mu_new).
// Reads mu_o/m2_o, writes mu_n/m2_n (distinct buffers).
__global__ void k_stats_step(const double *__restrict__ x, int64_t nl, int l, const double *__restrict__ mu_o,
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
__global__ void k_coldata(const double *__restrict__ x, int64_t nl, int64_t npad, int l,
                          const double *__restrict__ mu, const double *__restrict__ m2,
                          const int32_t *__restrict__ run, Col<T> *__restrict__ col)
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
            c.inv = (run[j] >= l) ? T(0) : T(1.0 / sqrt(m2[j]));
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
                    const int32_t *run, Col<T> *col, cudaStream_t s)
{
    k_coldata<T><<<(unsigned)((npad + 255) / 256), 256, 0, s>>>(x, nl, npad, l, mu, m2, run, col);
}
template void launch_coldata<float>(const double *, int64_t, int64_t, int, const double *, const double *,
                                    const int32_t *, Col<float> *, cudaStream_t);
template void launch_coldata<double>(const double *, int64_t, int64_t, int, const double *, const double *,
                                     const int32_t *, Col<double> *, cudaStream_t);

__global__ void k_widen_f32(const float *__restrict__ in, int64_t n, double *__restrict__ out)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (double)in[i];
}

}  // namespace mad
