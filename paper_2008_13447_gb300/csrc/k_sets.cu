// k_sets.cu -- variable-length motif sets (Sec. "Finding Motif Sets",
// Algorithm 6), grown on the GPU from the top-k motif pairs.
//
// For a pair (a, b) at length l and radius r = D * d(a, b):
//  - k_set_candidates evaluates, for every window j at l, the FP64
//    z-normalised distances to a and to b (two-pass statistics per window,
//    Eq. DIST from the centred dot products), and keeps j when
//    min(d(a, j), d(b, j)) <= r, j is not a trivial match of a or b, and j
//    is not within max(E(l), E(l_t)) of a member of an earlier set t (the
//    used subsequences leave the search space, so sets never meet);
//  - k_set_greedy grows the set: a and b first, then candidates by
//    (distance, offset) ascending, each accepted unless within E(l) of an
//    accepted member (the merge that removes trivial matches), up to `cap`
//    members.
#include "kernels.cuh"

namespace mad {

constexpr int SET_THREADS = 256;
constexpr int GREEDY_THREADS = 1024;

__device__ __forceinline__ double set_dinf() { return __longlong_as_double(0x7ff0000000000000LL); }

template <int NT>
__device__ double block_sum_d(double v, double *sh)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x < 32) {
        t = threadIdx.x < NT / 32 ? sh[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (threadIdx.x == 0) sh[0] = t;
    }
    __syncthreads();
    t = sh[0];
    __syncthreads();
    return t;
}

__global__ void __launch_bounds__(SET_THREADS) k_set_candidates(SetArgs A)
{
    extern __shared__ double sw[];        // centred windows a, b: [2][l]
    __shared__ double red[32];
    __shared__ double m2s[2];
    __shared__ int flats[2];
    const int l = A.l;
    const int64_t nl = A.n - l + 1;
    double *wa = sw, *wb = sw + l;
    // the pair's centred windows (two-pass) and their M2
    for (int w = 0; w < 2; ++w) {
        const int64_t o = w == 0 ? A.a : A.b;
        double *dst = w == 0 ? wa : wb;
        double s = 0.0;
        int same = 1;
        for (int t = threadIdx.x; t < l; t += SET_THREADS) {
            s += A.x[o + t];
            same &= (A.x[o + t] == A.x[o]);
        }
        const double mu = block_sum_d<SET_THREADS>(s, red) / l;
        const int nsame = __syncthreads_and(same);
        double v = 0.0;
        for (int t = threadIdx.x; t < l; t += SET_THREADS) {
            const double c = A.x[o + t] - mu;
            dst[t] = c;
            v = fma(c, c, v);
        }
        v = block_sum_d<SET_THREADS>(v, red);
        if (threadIdx.x == 0) {
            m2s[w] = v;
            flats[w] = nsame;
        }
    }
    __syncthreads();
    const double m2a = m2s[0], m2b = m2s[1];
    const bool fa = flats[0] != 0, fb = flats[1] != 0;
    for (int64_t j = blockIdx.x * (int64_t)SET_THREADS + threadIdx.x; j < nl; j += (int64_t)gridDim.x * SET_THREADS) {
        const int64_t da = j - A.a, db = j - A.b;
        if ((da <= A.E && -da <= A.E) || (db <= A.E && -db <= A.E)) continue;
        bool blocked = false;
        for (int q = 0; q < A.nprev && !blocked; ++q) {
            const int64_t Em = A.E > A.prev_E[q] ? A.E : A.prev_E[q];
            const int64_t dd = j - A.prev_off[q];
            blocked = dd <= Em && -dd <= Em;
        }
        if (blocked) continue;
        double s = 0.0;
        bool fj = true;
        const double x0 = A.x[j];
        for (int t = 0; t < l; ++t) {
            const double v = A.x[j + t];
            s += v;
            fj &= (v == x0);
        }
        const double mu = s / l;
        double m2 = 0.0, ca = 0.0, cb = 0.0;
        for (int t = 0; t < l; ++t) {
            const double c = A.x[j + t] - mu;
            m2 = fma(c, c, m2);
            ca = fma(c, wa[t], ca);
            cb = fma(c, wb[t], cb);
        }
        // flat windows: two flat windows correlate 1, flat vs non-flat 0
        const double qa = (fa || fj) ? ((fa && fj) ? 1.0 : 0.0) : ca / sqrt(m2a * m2);
        const double qb = (fb || fj) ? ((fb && fj) ? 1.0 : 0.0) : cb / sqrt(m2b * m2);
        const double d = fmin(dist_from_q(qa, l), dist_from_q(qb, l));
        if (d <= A.r) {
            const int pos = atomicAdd(A.ccount, 1);
            if (pos < A.capc) {
                A.ckey[pos] = d;
                A.cj[pos] = (int32_t)j;
            }
        }
    }
}

// One block: a and b first, then the best remaining candidate, with the
// candidates within E of each accepted member struck out (key = +inf).
__global__ void __launch_bounds__(GREEDY_THREADS) k_set_greedy(double *ckey, const int32_t *cj, const int32_t *ccount,
                                                               int64_t capc, int64_t a, int64_t b, int64_t E, int cap,
                                                               int64_t *members, int32_t *mcount)
{
    __shared__ double bk[32];
    __shared__ int32_t bjj[32];
    __shared__ int cnt;
    __shared__ int32_t pick;
    const int64_t c = *ccount < capc ? *ccount : capc;
    if (threadIdx.x == 0) {
        cnt = 0;
        if (cnt < cap) members[cnt++] = a;
        if (cnt < cap) members[cnt++] = b;
    }
    __syncthreads();
    while (cnt < cap) {
        double v = set_dinf();
        int32_t jj = INT32_MAX;
        for (int64_t i = threadIdx.x; i < c; i += GREEDY_THREADS) {
            const double k = ckey[i];
            if (k < v || (k == v && cj[i] < jj)) {
                v = k;
                jj = cj[i];
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const double v2 = __shfl_xor_sync(0xffffffffu, v, o);
            const int32_t j2 = __shfl_xor_sync(0xffffffffu, jj, o);
            if (v2 < v || (v2 == v && j2 < jj)) {
                v = v2;
                jj = j2;
            }
        }
        if ((threadIdx.x & 31) == 0) {
            bk[threadIdx.x >> 5] = v;
            bjj[threadIdx.x >> 5] = jj;
        }
        __syncthreads();
        if (threadIdx.x < 32) {
            v = bk[threadIdx.x];
            jj = bjj[threadIdx.x];
            for (int o = 16; o > 0; o >>= 1) {
                const double v2 = __shfl_xor_sync(0xffffffffu, v, o);
                const int32_t j2 = __shfl_xor_sync(0xffffffffu, jj, o);
                if (v2 < v || (v2 == v && j2 < jj)) {
                    v = v2;
                    jj = j2;
                }
            }
            if (threadIdx.x == 0) {
                pick = (v < set_dinf()) ? jj : -1;
                if (pick >= 0) members[cnt++] = pick;
            }
        }
        __syncthreads();
        if (pick < 0) break;
        for (int64_t i = threadIdx.x; i < c; i += GREEDY_THREADS) {
            const int64_t dd = (int64_t)cj[i] - pick;
            if (dd <= E && -dd <= E) ckey[i] = set_dinf();
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) *mcount = cnt;
}

void launch_motif_set(const SetArgs &a, int cap, int64_t *members, int32_t *mcount, cudaStream_t s)
{
    const int64_t nl = a.n - a.l + 1;
    int64_t g = (nl + SET_THREADS - 1) / SET_THREADS;
    if (g > 65535) g = 65535;
    const size_t sm = sizeof(double) * 2 * (size_t)a.l;
    static std::once_flag once[64];
    smem_optin_max((const void *)k_set_candidates, once);
    k_set_candidates<<<(unsigned)g, SET_THREADS, sm, s>>>(a);
    k_set_greedy<<<1, GREEDY_THREADS, 0, s>>>(a.ckey, a.cj, a.ccount, a.capc, a.a, a.b, a.E, cap, members, mcount);
}

}  // namespace mad
