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
// Seed rows at lmin for the FP32 paths, on the FP32 pipe (GB300's FP64 rate
// is 1/64 of its FP32 rate): each seed value C(ra, c) = sum_t a_t (x[c+t] -
// mu_c), a_t = x[ra+t] - mu_ra, as a dot product in FP32 pairs.
//  - a_t (FP64) is split into FP32 pairs (ah + al, within 2^-48 |a_t|);
//    the block's columns use x'_i = x[cb+i] - m (m the mean of the block's
//    middle window), split the same way, and
//    C = sum_t a_t x'_{c+t} - (mu_c - m) sum_t a_t.
//  - each product's high part ah*xh is formed exactly (FMA), its low part
//    from the cross terms; the high parts are summed by TwoSum (exact), the
//    low parts and the TwoSum errors in FP32 over runs of 16 terms, each run
//    added to an FP64 total.
// Error (Sec. "Computing The Matrix Profile", Eq. DIST's co-moment): with
// P = sum_t |a_t x'_{c+t}| <= sqrt(M2_ra (M2_c + l (mu_c - m)^2))
// (Cauchy-Schwarz), |C~ - C| <= eps P, eps = (32 l + 80) 2^-48 (pair
// representations and cross terms <= 2^-44 P; the FP32 runs <= 32 u^2 (l + 2) P).
// A value is taken from this sum only when eps P <= 2^-25 sqrt(M2_ra M2_c),
// i.e. half an FP32 unit of the co-moment scale, which the band kernel's
// error model counts (one unit for the seed); otherwise (near-flat column
// windows, long windows) it is computed directly in FP64.
constexpr int SEEDP_THREADS = 256;

__device__ __forceinline__ float2 split_pair(double v)
{
    const float h = (float)v;
    return make_float2(h, (float)(v - (double)h));
}

__device__ __forceinline__ double seed_fp64(const double *x, const double *mu, int64_t ra, int64_t c, int l)
{
    const double mua = mu[ra], muc = mu[c];
    double s = 0.0;
    for (int t = 0; t < l; ++t) s = fma(x[ra + t] - mua, x[c + t] - muc, s);
    return s;
}

__global__ void __launch_bounds__(SEEDP_THREADS) k_seed_pair(SeedArgs<double> A, const double *m2, int64_t n)
{
    extern __shared__ float2 shp[];          // [l] row pairs, then [SEEDP_THREADS + l] column pairs
    __shared__ double red[SEEDP_THREADS / 32];
    const int l = A.l;
    const int tid = threadIdx.x;
    const int k = A.krows[blockIdx.y];
    const int64_t kr = (int64_t)k * A.R;
    const int64_t ra = (k == 0) ? 0 : kr - 1;
    const int64_t j0 = (int64_t)blockIdx.x * SEEDP_THREADS;
    const int64_t cb = (k == 0) ? j0 : j0 - 1;       // column window of thread 0 (-1 in the first block)
    const bool row_ok = ra < A.nl;
    float2 *ap = shp, *xp = shp + l;
    // the row window as pairs, and the sum of its represented values
    const double mua = row_ok ? A.mu[ra] : 0.0;
    double sa = 0.0;
    for (int t = tid; t < l; t += SEEDP_THREADS) {
        const float2 v = split_pair(row_ok ? A.x[ra + t] - mua : 0.0);
        ap[t] = v;
        sa += (double)v.x + (double)v.y;
    }
    for (int o = 16; o > 0; o >>= 1) sa += __shfl_xor_sync(0xffffffffu, sa, o);
    if ((tid & 31) == 0) red[tid >> 5] = sa;
    // the block's columns relative to the mean of its middle window
    int64_t cm = cb + SEEDP_THREADS / 2;
    cm = cm < 0 ? 0 : (cm >= A.nl ? A.nl - 1 : cm);
    const double m = A.mu[cm];
    for (int i = tid; i < SEEDP_THREADS + l; i += SEEDP_THREADS) {
        const int64_t g = cb + i;
        xp[i] = split_pair((g >= 0 && g < n) ? A.x[g] - m : 0.0);
    }
    __syncthreads();
    sa = 0.0;
    for (int w = 0; w < SEEDP_THREADS / 32; ++w) sa += red[w];
    const int64_t j = j0 + tid;
    if (j >= A.spitch) return;
    const int64_t c = cb + tid;
    double out = 0.0;
    if (k != 0 && j == 0) {
        // C(kS, 0): another row window, one value per seed row
        if (kr < A.nl) out = seed_fp64(A.x, A.mu, kr, 0, l);
    } else if (row_ok && c >= 0 && c < A.nl) {
        const double m2c = m2[c], dm = A.mu[c] - m;
        const double eps = (32.0 * l + 80.0) * 0x1p-48;
        if (m2c > 0.0 && eps * eps * (m2c + (double)l * dm * dm) <= 0x1p-50 * m2c) {
            float sh = 0.0f;
            double lo = 0.0;
            const float2 *xr = xp + tid;
            int t = 0;
            for (; t < l; t += 16) {
                float sl = 0.0f;
                const int te = t + 16 < l ? t + 16 : l;
#pragma unroll 4
                for (int u = t; u < te; ++u) {
                    const float2 a = ap[u], b = xr[u];
                    // (explicit roundings: no contraction into FMAs, which
                    // would break the exactness of TwoProd / TwoSum)
                    const float p = __fmul_rn(a.x, b.x);
                    float e = fmaf(a.x, b.x, -p);
                    e = fmaf(a.x, b.y, e);
                    e = fmaf(a.y, b.x, e);
                    const float sn = __fadd_rn(sh, p);
                    const float v = __fsub_rn(sn, sh);
                    const float er = __fadd_rn(__fsub_rn(sh, __fsub_rn(sn, v)), __fsub_rn(p, v));
                    sh = sn;
                    sl = __fadd_rn(sl, __fadd_rn(er, e));
                }
                lo += (double)sl;
            }
            out = ((double)sh + lo) - dm * sa;
        } else {
            out = seed_fp64(A.x, A.mu, ra, c, l);
        }
    }
    A.seed[(int64_t)k * A.spitch + j] = out;
}

size_t seed_pair_smem(int l) { return (size_t)(2 * l + SEEDP_THREADS) * sizeof(float2); }

void launch_seed_pair(const SeedArgs<double> &a, const double *m2, int64_t n, cudaStream_t s)
{
    dim3 grid((unsigned)((a.spitch + SEEDP_THREADS - 1) / SEEDP_THREADS), (unsigned)a.nk);
    static std::once_flag once[64];
    smem_optin_max((const void *)k_seed_pair, once);
    k_seed_pair<<<grid, SEEDP_THREADS, seed_pair_smem(a.l), s>>>(a, m2, n);
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
// the column's factor (x[j-1+l] - mu[j-1]) is loaded once for them (the
// tables are streamed with evict-first hints: they pass through L2 once per
// length and would otherwise push out the working sets of the kernels that
// run beside this one); the
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
        for (int t = 0; t < SEED_BATCH; ++t) v[t] = t0 + t < nrow ? __ldcs(mp + (int64_t)t * spitch) : 0.0;
        if (update) {
#pragma unroll
            for (int t = 0; t < SEED_BATCH; ++t) {
                v[t] = (valid >> (t0 + t)) & 1u ? fma(sa[t0 + t], bj, v[t]) : 0.0;
                if (t0 + t < nrow) __stcs(mp + (int64_t)t * spitch, v[t]);
            }
        }
#pragma unroll
        for (int t = 0; t < SEED_BATCH; ++t)
            if (t0 + t < nrow) __stcs(sp + (int64_t)t * spitch, (T)v[t]);
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
