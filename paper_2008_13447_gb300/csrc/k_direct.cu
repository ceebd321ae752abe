// k_direct.cu -- recompute of listed rows' full distance profiles from
// direct dot products (Algorithm 4's SlidingDotProduct for the non-valid
// rows, Algorithm 10's recompute loop), for rows that are too few in their
// band for the diagonal band kernel to pay off, and for rows whose lists fell
// short in the band kernel.
//
// For each listed row r and every column j the centred co-moment
//     C(r, j) = sum_t (x_{r+t} - mu_r)(x_{j+t} - mu_j)
// is formed as sum_t a_t (x_{j+t} - s) - (sum_t a_t)(mu_j - s), a_t the
// row's centred window and s a shift close to the column block's values (so
// FP32 values stay small); the key C / sqrt(M2_j) orders the row's partners
// like the correlation. Each block takes DR rows x DCOLS columns; each thread
// keeps its rows' best p keys over its columns, and the block reduces them
// to one list of p per row and column block.
//
// Error bound of a key (in correlation units), written with every kept
// entry: the sum of l products in T has error <= (l + 2) u sum_t |a_t y_t|
// (each FMA rounds once, each input once), with sum_t |a_t y_t| <=
// sqrt(M2_r (M2_j + l (mu_j - s)^2)) by Cauchy-Schwarz; the key's own
// rounding adds u:
//     dq_j = 1.5 ((l + 3) u sqrt(1 + l (mu_j - s)^2 / M2_j) + u).
// A column is a candidate when key + dq_j sqrt(M2_r) beats the row's
// threshold.
#include "kernels.cuh"

namespace mad {

constexpr int DR = 4;          // rows per block
constexpr int DTHREADS = 256;
constexpr int DCPT = 16;       // columns per thread
constexpr int DCOLS = DTHREADS * DCPT;

__device__ __forceinline__ double d_pinf() { return __longlong_as_double(0x7ff0000000000000LL); }

template <typename T>
__device__ __forceinline__ void local_insert(T *K, int32_t *J, float *D, int &cnt, int p, T key, int32_t j, float dq)
{
    if (cnt == p && !(key > K[p - 1] || (key == K[p - 1] && j < J[p - 1]))) return;
    int b = cnt < p ? cnt++ : p - 1;
    while (b > 0 && (K[b - 1] < key || (K[b - 1] == key && J[b - 1] > j))) {
        K[b] = K[b - 1];
        J[b] = J[b - 1];
        D[b] = D[b - 1];
        --b;
    }
    K[b] = key;
    J[b] = j;
    D[b] = dq;
}

template <typename T> struct Unit;
template <> struct Unit<float> { static constexpr double u = 0x1p-24; };
template <> struct Unit<double> { static constexpr double u = 0x1p-53; };

template <typename T>
__global__ void __launch_bounds__(DTHREADS) k_direct(DirectArgs<T> A)
{
    extern __shared__ __align__(16) unsigned char dsm[];
    const int nrows = *A.nrows;
    const int l = A.l;
    T *aw = reinterpret_cast<T *>(dsm);                 // [l][DR] centred row windows
    T *yw = aw + (size_t)l * DR;                        // [DCOLS + l] shifted column values
    __shared__ double asum[DR];
    __shared__ int64_t rr[DR];
    const int64_t items = (int64_t)((nrows + DR - 1) / DR) * A.nblk;
    for (int64_t item = blockIdx.x; item < items; item += gridDim.x) {
    const int g = (int)(item / A.nblk);
    const int by = (int)(item % A.nblk);
    const int64_t cb0 = (int64_t)by * DCOLS;
    if (cb0 >= A.nl) continue;
    __syncthreads();
    const int nr = nrows - g * DR < DR ? nrows - g * DR : DR;
    if (threadIdx.x < DR) rr[threadIdx.x] = threadIdx.x < nr ? A.rows[g * DR + threadIdx.x] : -1;
    __syncthreads();
    const double shift = A.mu[cb0];
    for (int k = 0; k < DR; ++k) {
        const int64_t r = rr[k];
        const double mr = r >= 0 ? A.mu[r] : 0.0;
        for (int t = threadIdx.x; t < l; t += DTHREADS) aw[t * DR + k] = r >= 0 ? T(A.x[r + t] - mr) : T(0);
    }
    const int64_t span = DCOLS + l - 1;
    for (int64_t u = threadIdx.x; u < span; u += DTHREADS) {
        const int64_t idx = cb0 + u;
        yw[u] = idx < A.nl + l - 1 ? T(A.x[idx] - shift) : T(0);
    }
    __syncthreads();
    if (threadIdx.x < DR) {
        double s = 0.0;
        for (int t = 0; t < l; ++t) s += (double)aw[t * DR + threadIdx.x];
        asum[threadIdx.x] = s;
    }
    __syncthreads();

    T K[DR][MAXP];
    int32_t J[DR][MAXP];
    float D[DR][MAXP];
    int cnt[DR];
    T th[DR];
    double sqr[DR];
    for (int k = 0; k < DR; ++k) {
        cnt[k] = 0;
        th[k] = rr[k] >= 0 ? A.thr[rr[k]] : T(d_pinf());
        const double ir = rr[k] >= 0 ? (double)A.col[rr[k]].inv : 0.0;
        sqr[k] = ir > 0.0 ? 1.0001 / ir : 0.0;
    }
    float dqmax = 0.0f;
    for (int u = 0; u < DCPT; ++u) {
        const int64_t jl = threadIdx.x + (int64_t)u * DTHREADS;
        const int64_t j = cb0 + jl;
        if (j >= A.nl) break;
        T acc[DR];
        for (int k = 0; k < DR; ++k) acc[k] = T(0);
        const T *y = yw + jl;
        for (int t = 0; t < l; ++t) {
            const T yv = y[t];
#pragma unroll
            for (int k = 0; k < DR; ++k) acc[k] = fma(aw[t * DR + k], yv, acc[k]);
        }
        const Col<T> cj = A.col[j];
        const double dmu = A.mu[j] - shift;
        const double ij = (double)cj.inv;
        const float dq = (float)(1.5 * ((l + 3.0) * Unit<T>::u * sqrt(1.0 + (double)l * dmu * dmu * ij * ij) +
                                        Unit<T>::u));
        dqmax = fmaxf(dqmax, dq);
        for (int k = 0; k < DR; ++k) {
            const int64_t r = rr[k];
            if (r < 0 || !nontrivial(r, j, A.E)) continue;
            const double c = (double)acc[k] - asum[k] * dmu;
            const T key = T(c * ij);
            if ((double)key + dq * sqr[k] > (double)th[k])
                local_insert<T>(K[k], J[k], D[k], cnt[k], A.p, key, (int32_t)j, dq);
        }
    }
    // block-wide: p rounds of "largest head among the threads" per row
    __shared__ T hk[DTHREADS / 32];
    __shared__ int32_t hj[DTHREADS / 32];
    __shared__ float hd[DTHREADS / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int k = 0; k < DR; ++k) {
        if (rr[k] < 0) break;
        int head = 0;
        const int64_t slot = ((int64_t)(g * DR + k) * A.nblk + by);
        int outc = 0;
        for (int e = 0; e < A.p; ++e) {
            T v = head < cnt[k] ? K[k][head] : T(-d_pinf());
            int32_t jj = head < cnt[k] ? J[k][head] : INT32_MAX;
            float dd = head < cnt[k] ? D[k][head] : 0.0f;
            for (int o = 16; o > 0; o >>= 1) {
                const T v2 = __shfl_xor_sync(0xffffffffu, v, o);
                const int32_t j2 = __shfl_xor_sync(0xffffffffu, jj, o);
                const float d2 = __shfl_xor_sync(0xffffffffu, dd, o);
                if (v2 > v || (v2 == v && j2 < jj)) { v = v2; jj = j2; dd = d2; }
            }
            if (lane == 0) { hk[wid] = v; hj[wid] = jj; hd[wid] = dd; }
            __syncthreads();
            if (wid == 0) {
                v = lane < DTHREADS / 32 ? hk[lane] : T(-d_pinf());
                jj = lane < DTHREADS / 32 ? hj[lane] : INT32_MAX;
                dd = lane < DTHREADS / 32 ? hd[lane] : 0.0f;
                for (int o = 16; o > 0; o >>= 1) {
                    const T v2 = __shfl_xor_sync(0xffffffffu, v, o);
                    const int32_t j2 = __shfl_xor_sync(0xffffffffu, jj, o);
                    const float d2 = __shfl_xor_sync(0xffffffffu, dd, o);
                    if (v2 > v || (v2 == v && j2 < jj)) { v = v2; jj = j2; dd = d2; }
                }
                if (lane == 0) { hk[0] = v; hj[0] = jj; hd[0] = dd; }
            }
            __syncthreads();
            v = hk[0];
            jj = hj[0];
            dd = hd[0];
            __syncthreads();
            if (jj == INT32_MAX) break;
            if (head < cnt[k] && J[k][head] == jj) ++head;
            if (threadIdx.x == 0) {
                A.okey[slot * A.p + e] = v;
                A.oj[slot * A.p + e] = jj;
                A.odq[slot * A.p + e] = dd;
            }
            ++outc;
        }
        if (threadIdx.x == 0) A.ocnt[slot] = outc;
    }
    if (dqmax > 0.0f) atomicMax(reinterpret_cast<int *>(A.dq_max), __float_as_int(dqmax));
    }
}

template <typename T>
void launch_direct(const DirectArgs<T> &a, int grid, cudaStream_t s)
{
    // (the opt-in covers dynamic plus static shared memory above 48 KB)
    const size_t sm = sizeof(T) * ((size_t)a.l * DR + DCOLS + a.l);
    static std::once_flag once[64];
    smem_optin_max((const void *)k_direct<T>, once);
    k_direct<T><<<grid, DTHREADS, sm, s>>>(a);
}
template void launch_direct<float>(const DirectArgs<float> &, int, cudaStream_t);
template void launch_direct<double>(const DirectArgs<double> &, int, cudaStream_t);

int direct_cols_per_block() { return DCOLS; }

}  // namespace mad
