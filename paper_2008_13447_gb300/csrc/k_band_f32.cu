// k_band_f32.cu -- FP32 instantiation of the seed and band kernels
// (k_band.cuh), with the FP32 seed kernel.
#include "k_band.cuh"

namespace mad {

// FP32 seeds: the row window is centred in FP64 and rounded; the column
// windows are shifted by one constant per tile of columns (close to their
// means) and rounded; the dot product runs in FP32 (two partial sums, by the
// parity of t, added in FP64) and the shift is removed exactly to first order
// with the FP32 sum of the rounded row window.
//
// Seed row k holds, for j >= 1, C(a_k, j - 1) with a_k = kS - 1 (the
// predecessor of cell (kS, j) on its diagonal), and C(kS, 0) at j = 0; row 0
// holds C(0, j). Register blocking: a block takes SEED_ROWS seed rows and
// SEED_THREADS * SEED_COLS columns; each thread keeps SEED_ROWS x SEED_COLS
// dot products, reading the rows' values at one t as one float4 (layout
// [t][row]) and its columns' shifted values as float4 runs, so shared-memory
// reads stay a small fraction of the FMAs; the next step's operands are
// loaded before the current step's FMAs, and 88 registers let four blocks
// share an SM.
constexpr int SEED_ROWS = 4;
constexpr int SEED_COLS = 4;
constexpr int SEED_THREADS = 128;
constexpr int SEED_TILE = SEED_THREADS * SEED_COLS;

__host__ __device__ inline int seed_l4(int l) { return (l + 3) & ~3; }

__global__ void __launch_bounds__(SEED_THREADS, 4) k_seed_f32(SeedArgs<float> A)
{
    if (A.nbands && *A.nbands == 0) return;
    extern __shared__ __align__(16) float sh_f[];
    const int l = A.l;
    const int l4 = seed_l4(l);
    float4 *arow = reinterpret_cast<float4 *>(sh_f);      // [l4] (one value per seed row)
    float *ycol = sh_f + 4 * l4;                          // [SEED_TILE + l4 + 4]
    __shared__ float s_asum[SEED_ROWS];
    __shared__ int64_t s_a[SEED_ROWS];
    __shared__ int s_k[SEED_ROWS];
    const int64_t cb = (int64_t)blockIdx.x * SEED_TILE;
    if (threadIdx.x < SEED_ROWS) {
        const int q = blockIdx.y * SEED_ROWS + threadIdx.x;
        const int k = q < A.nk ? A.krows[q] : -1;
        int64_t a = k < 0 ? -1 : (k == 0 ? 0 : (int64_t)k * A.R - 1);
        if (a >= A.nl) a = -1;
        s_k[threadIdx.x] = k;
        s_a[threadIdx.x] = a;
    }
    __syncthreads();
    const int64_t cshift = cb < A.nl ? cb : A.nl - 1;
    const double shift = A.mu[cshift];
    for (int t = threadIdx.x; t < l4; t += SEED_THREADS) {
        float v[SEED_ROWS];
#pragma unroll
        for (int r = 0; r < SEED_ROWS; ++r) {
            const int64_t a = s_a[r];
            v[r] = (a >= 0 && t < l) ? (float)(A.x[a + t] - A.mu[a]) : 0.0f;
        }
        arow[t] = make_float4(v[0], v[1], v[2], v[3]);
    }
    for (int u = threadIdx.x; u < SEED_TILE + l4 + 4; u += SEED_THREADS) {
        const int64_t idx = cb + u;
        ycol[u] = idx < A.nl + l - 1 ? (float)(A.x[idx] - shift) : 0.0f;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        float sr[SEED_ROWS] = {0.f, 0.f, 0.f, 0.f};
        for (int t = threadIdx.x; t < l; t += 32) {
            const float4 v = arow[t];
            sr[0] += v.x;
            sr[1] += v.y;
            sr[2] += v.z;
            sr[3] += v.w;
        }
#pragma unroll
        for (int r = 0; r < SEED_ROWS; ++r) {
            for (int o = 16; o > 0; o >>= 1) sr[r] += __shfl_xor_sync(0xffffffffu, sr[r], o);
            if (threadIdx.x == 0) s_asum[r] = sr[r];
        }
    }
    __syncthreads();

    const int c0 = threadIdx.x * SEED_COLS;
    float acc[2][SEED_ROWS][SEED_COLS];
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int r = 0; r < SEED_ROWS; ++r)
#pragma unroll
            for (int c = 0; c < SEED_COLS; ++c) acc[h][r][c] = 0.0f;
    float4 y0n = *reinterpret_cast<const float4 *>(ycol + c0);
    float4 y1n = *reinterpret_cast<const float4 *>(ycol + c0 + 4);
    float4 an[4] = {arow[0], arow[1], arow[2], arow[3]};
    for (int t0 = 0; t0 < l4; t0 += 4) {
        const float4 y0 = y0n, y1 = y1n;
        const float4 ac[4] = {an[0], an[1], an[2], an[3]};
        if (t0 + 4 < l4) {
            y0n = *reinterpret_cast<const float4 *>(ycol + c0 + t0 + 4);
            y1n = *reinterpret_cast<const float4 *>(ycol + c0 + t0 + 8);
#pragma unroll
            for (int h = 0; h < 4; ++h) an[h] = arow[t0 + 4 + h];
        }
        const float yv[8] = {y0.x, y0.y, y0.z, y0.w, y1.x, y1.y, y1.z, y1.w};
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            const float a4[SEED_ROWS] = {ac[h].x, ac[h].y, ac[h].z, ac[h].w};
#pragma unroll
            for (int r = 0; r < SEED_ROWS; ++r)
#pragma unroll
                for (int c = 0; c < SEED_COLS; ++c) acc[h & 1][r][c] = fmaf(a4[r], yv[c + h], acc[h & 1][r][c]);
        }
    }
#pragma unroll
    for (int r = 0; r < SEED_ROWS; ++r) {
        const int k = s_k[r];
        if (k < 0) continue;
        const int64_t a = s_a[r];
        const int64_t o = k == 0 ? 0 : 1;   // output index j = c + o
#pragma unroll
        for (int c = 0; c < SEED_COLS; ++c) {
            const int64_t col = cb + c0 + c;
            const int64_t j = col + o;
            if (j >= A.spitch) continue;
            float out = 0.0f;
            if (a >= 0 && col < A.nl) {
                const double corr = (double)s_asum[r] * (A.mu[col] - shift);
                out = (float)(((double)acc[0][r][c] + (double)acc[1][r][c]) - corr);
            }
            A.seed[(int64_t)k * A.spitch + j] = out;
        }
    }
    // the single (kS, 0) entry of rows k >= 1: direct FP64
    if (blockIdx.x == 0 && threadIdx.x < SEED_ROWS) {
        const int k = s_k[threadIdx.x];
        if (k >= 1) {
            const int64_t ra = (int64_t)k * A.R;
            double sum = 0.0;
            if (ra < A.nl) {
                const double mur = A.mu[ra], muc = A.mu[0];
                for (int t = 0; t < l; ++t) sum = fma(A.x[ra + t] - mur, A.x[t] - muc, sum);
            }
            A.seed[(int64_t)k * A.spitch] = (float)sum;
        }
    }
}

template <>
void launch_seed<float>(const SeedArgs<float> &a, cudaStream_t s)
{
    dim3 grid((unsigned)((a.spitch + SEED_TILE - 1) / SEED_TILE), (unsigned)((a.nk + SEED_ROWS - 1) / SEED_ROWS));
    const int l4 = seed_l4(a.l);
    const size_t sm = sizeof(float) * (4 * (size_t)l4 + SEED_TILE + l4 + 4);
    static std::once_flag once[64];
    smem_optin_max((const void *)k_seed_f32, once);
    k_seed_f32<<<grid, SEED_THREADS, sm, s>>>(a);
}

template void launch_band<float>(const BandArgs<float> &, bool, int, cudaStream_t);
template int band_occupancy<float>(bool, int, int);
template size_t band_smem<float>(bool, int, int);

}  // namespace mad
