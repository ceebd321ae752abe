// k_band.cuh -- the matrix-profile kernel: diagonal (QT) recurrence over R x R
// tiles, wavefront across warps, per-row candidate selection.
//
// What it computes (Algorithm 3 ComputeMatrixProfile, restricted to the rows
// of the active bands): for every row r of a band and every column j, the
// centred co-moment C(r, j) by the recurrence along diagonals
//     C(r, j) = C(r-1, j-1) + df_{r-1} dg_{j-1} + df_{j-1} dg_{r-1}
// (the mean-centred form of QT[j] = QT[j-1] - t_{j-1} t_{i-1} + t_{j+l-1} t_{i+l-1}),
// started at every tile's top row and left column from direct dot products
// (the "seed" rows). Instead of a distance it evaluates the row key
// key = C(r, j) / sqrt(M2_j): within a row the key orders columns exactly
// like the correlation q, hence like Eq. DIST and like Eq. LB (the p smallest
// lower bounds of a row are its p largest correlations).
//
// Two modes:
//  - append: every non-trivial cell whose key exceeds the row's threshold is
//    appended to the row's candidate list (the threshold is a proven lower
//    bound on the row's p-th best key, so the list holds the row's top-p);
//    a work unit that fills a row's list publishes its p-th kept key (an
//    atomic max per row) and later units of the row start from it;
//  - bins: per row, the maximum key over the columns of each chunk index
//    modulo p is recorded; the smallest of those p maxima is a lower bound on
//    the row's p-th best key (p distinct columns), used as the first
//    threshold at lmin.
//
// Layout: a band is R = 32 * RPL * NW consecutive rows. Lane t of warp w
// owns rows rfirst(w) + t*RPL + [0, RPL); all lanes of a warp walk the same
// column j at a time, so the row r's predecessor C(r-1, j-1) sits in the
// same lane (previous row, previous column) or in lane t-1 (one shuffle). The
// first row of warp w takes it from the seed row at rfirst(w) when there is
// one (seed rows every A.sp rows, down to one per warp), else from warp w-1
// through shared memory, one chunk of CH columns behind (a wavefront over
// the unseeded warps, synchronised pairwise by mbarriers). Per-column data
// (df, dg, inv) is staged per chunk in shared memory and read as broadcasts.
#pragma once
#include "kernels.cuh"

namespace mad {

// ------------------------------------------------------------------ seeds

template <typename T>
__global__ void k_seed(SeedArgs<T> A);

// ------------------------------------------------------------- band kernel

template <typename T> __device__ __forceinline__ T neg_inf();
template <> __device__ __forceinline__ float neg_inf<float>() { return -__int_as_float(0x7f800000); }
template <> __device__ __forceinline__ double neg_inf<double>() { return -__longlong_as_double(0x7ff0000000000000LL); }

__device__ __forceinline__ float to_float_rd(float v) { return v; }
__device__ __forceinline__ float to_float_rd(double v) { return __double2float_rd(v); }

// IEEE maxNum: a NaN operand (a padded column) is ignored.
__device__ __forceinline__ float fmax_t(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ double fmax_t(double a, double b) { return fmax(a, b); }

// Insert (key, j) into a row's top-p list in shared memory (only the lane
// owning the row touches it). The list keeps the p largest keys seen; among
// equal keys the smaller offset wins (columns arrive in increasing j, and an
// equal key never replaces a kept one). th is the row's current threshold:
// max(lower bound given at launch, smallest kept key once p are kept).
template <typename T>
__device__ __forceinline__ void topp_insert(T *K, int32_t *J, int32_t &cnt, int p, T key, int32_t j, T &th)
{
    if (cnt < p) {
        K[cnt] = key;
        J[cnt] = j;
        ++cnt;
        if (cnt == p) {
            T mn = K[0];
            for (int e = 1; e < p; ++e) mn = K[e] < mn ? K[e] : mn;
            th = mn > th ? mn : th;
        }
        return;
    }
    int m = 0;
    for (int e = 1; e < p; ++e)
        if (K[e] < K[m] || (K[e] == K[m] && J[e] > J[m])) m = e;
    K[m] = key;
    J[m] = j;
    T mn = K[0];
    for (int e = 1; e < p; ++e) mn = K[e] < mn ? K[e] : mn;
    th = mn > th ? mn : th;
}

template <int RPL>
__device__ __forceinline__ bool any_positive(const float (&C)[RPL], float inv, const float (&th)[RPL])
{
    unsigned acc = 0xffffffffu;
#pragma unroll
    for (int a = 0; a < RPL; ++a) acc &= __float_as_uint(fmaf(C[a], inv, -th[a]));
    return (int)acc >= 0;
}

template <int RPL>
__device__ __forceinline__ bool any_positive(const double (&C)[RPL], double inv, const double (&th)[RPL])
{
    unsigned acc = 0xffffffffu;
#pragma unroll
    for (int a = 0; a < RPL; ++a) acc &= (unsigned)(__double_as_longlong(fma(C[a], inv, -th[a])) >> 32);
    return (int)acc >= 0;
}

// any key - th > 0 over two columns' co-moments (AND of the sign bits of all
// 2 RPL values; +0 and NaN count as hits and are re-tested)
template <int RPL>
__device__ __forceinline__ bool any_positive_pair(const float (&C0)[RPL], float inv0, const float (&C1)[RPL], float inv1,
                                                  const float (&th)[RPL])
{
    unsigned acc = 0xffffffffu;
#pragma unroll
    for (int a = 0; a < RPL; ++a)
        acc &= __float_as_uint(fmaf(C0[a], inv0, -th[a])) & __float_as_uint(fmaf(C1[a], inv1, -th[a]));
    return (int)acc >= 0;
}

template <int RPL>
__device__ __forceinline__ bool any_positive_pair(const double (&C0)[RPL], double inv0, const double (&C1)[RPL],
                                                  double inv1, const double (&th)[RPL])
{
    unsigned acc = 0xffffffffu;
#pragma unroll
    for (int a = 0; a < RPL; ++a)
        acc &= (unsigned)(__double_as_longlong(fma(C0[a], inv0, -th[a])) >> 32) &
               (unsigned)(__double_as_longlong(fma(C1[a], inv1, -th[a])) >> 32);
    return (int)acc >= 0;
}

template <int RPL>
__device__ __forceinline__ bool any_positive2(const float (&C)[RPL], float inv, const float (&th)[RPL],
                                              const float (&invr)[RPL], float thc)
{
    unsigned acc = 0xffffffffu;
#pragma unroll
    for (int a = 0; a < RPL; ++a)
        acc &= __float_as_uint(fmaf(C[a], inv, -th[a])) & __float_as_uint(fmaf(C[a], invr[a], -thc));
    return (int)acc >= 0;
}

template <int RPL>
__device__ __forceinline__ bool any_positive2(const double (&C)[RPL], double inv, const double (&th)[RPL],
                                              const double (&invr)[RPL], double thc)
{
    unsigned acc = 0xffffffffu;
#pragma unroll
    for (int a = 0; a < RPL; ++a)
        acc &= (unsigned)(__double_as_longlong(fma(C[a], inv, -th[a])) >> 32) &
               (unsigned)(__double_as_longlong(fma(C[a], invr[a], -thc)) >> 32);
    return (int)acc >= 0;
}

enum { MODE_TOPP = 0, MODE_BINS = 1, MODE_SYM = 2 };
constexpr bool BAND_PAIR = true;   // two columns per hit test in the common case

// One chunk of CH columns for the lane's RPL rows.
//  MODE_TOPP: every column; row keys against the row thresholds.
//  MODE_BINS: every column; running maxima of the row keys.
//  MODE_SYM : cells above the exclusion zone only (j - r > E); each cell is
//             tested for its row (key C / sqrt(M2_j) against th_r, into the
//             row's list) and for its column (key C / sqrt(M2_r) against the
//             column's threshold, staged in cd.pad, appended to row j's
//             candidate list in global memory).
template <typename T, int RPL, int NW, int MODE, bool DIAG>
__device__ __forceinline__ void band_chunk(const BandArgs<T> &A, const Col<T> *cbuf, T tp, T *bout, int lane,
                                           bool feeds,
                                           int64_t cs, int64_t rbase, int rl0, T (&C)[RPL], const T (&dfr)[RPL],
                                           const T (&dgr)[RPL], T (&th)[RPL], const T (&invr)[RPL],
                                           T (&runmax)[RPL], T *lkey, int32_t *lj, int32_t *lcnt, unsigned &ninsert)
{
#pragma unroll
    for (int c = 0; c < CH; ++c) {
        const Col<T> cd = cbuf[c];
        T v = __shfl_up_sync(0xffffffffu, C[RPL - 1], 1);
        const T vt = __shfl_sync(0xffffffffu, tp, c);
        if (lane == 0) v = vt;
#pragma unroll
        for (int a = RPL - 1; a >= 1; --a) C[a] = fma(dfr[a], cd.dg, fma(cd.df, dgr[a], C[a - 1]));
        C[0] = fma(dfr[0], cd.dg, fma(cd.df, dgr[0], v));
        if (feeds && lane == 31) bout[c] = C[RPL - 1];
        if (MODE == MODE_BINS) {
#pragma unroll
            for (int a = 0; a < RPL; ++a) {
                T key = C[a] * cd.inv;
                if (DIAG && !nontrivial(rbase + a, cs + c, A.E)) key = neg_inf<T>();
                runmax[a] = fmax_t(runmax[a], key);   // NaN keys (padding) are ignored
            }
            continue;
        }
        bool hit = false;
        if (MODE == MODE_TOPP) {
            if (DIAG) {
#pragma unroll
                for (int a = 0; a < RPL; ++a)
                    hit |= (C[a] * cd.inv > th[a]) && nontrivial(rbase + a, cs + c, A.E);
            } else {
                // any key - th > 0 ? (AND of the sign bits of key - th over the
                // rows; +0 and NaN count as hits and are re-tested below)
                hit = any_positive(C, cd.inv, th);
            }
        } else {
            if (DIAG) {
#pragma unroll
                for (int a = 0; a < RPL; ++a)
                    hit |= ((cs + c) - (rbase + a) > A.E) && ((C[a] * cd.inv > th[a]) || (C[a] * invr[a] > cd.pad));
            } else {
                hit = any_positive2(C, cd.inv, th, invr, cd.pad);
            }
        }
        // warp-uniform branch: the common no-hit path costs one vote and
        // no reconvergence bookkeeping; lanes without a hit idle inside
        if (__any_sync(0xffffffffu, hit) && hit) {
            const int32_t j = (int32_t)(cs + c);
#pragma unroll
            for (int a = 0; a < RPL; ++a) {
                const int64_t r = rbase + a;
                const bool valid = MODE == MODE_SYM ? (j - r > A.E) : nontrivial(r, j, A.E);
                if (!valid) continue;
                const T key = C[a] * cd.inv;
                if (key > th[a]) {
                    const int rl = rl0 + a;
                    int32_t cnt = lcnt[rl];
                    topp_insert<T>(lkey + rl * A.p, lj + rl * A.p, cnt, A.p, key, j, th[a]);
                    lcnt[rl] = cnt;
                    ++ninsert;
                }
                if (MODE == MODE_SYM) {
                    const T kc = C[a] * invr[a];
                    if (kc > cd.pad) {
                        const int slot = atomicAdd(&A.ccnt[j], 1);
                        if (slot < A.cap) {
                            A.ckey[(int64_t)j * A.cap + slot] = kc;
                            A.cj[(int64_t)j * A.cap + slot] = (int32_t)r;
                        }
                        ninsert += 1u << 16;
                    }
                }
            }
        }
    }
}

// The common case of the full-rows form (MODE_TOPP away from the exclusion
// zone) two columns at a time: both columns' co-moments are formed first and
// one warp vote covers both threshold tests, which halves the branches and
// gives the scheduler two columns of independent arithmetic per block.
// Column c's co-moments stay in C0 until its hits are handled; a hit in
// column c may raise th before column c+1 is handled, which the per-row test
// re-checks. The chunks of this form lie outside the exclusion zone of every
// row of the warp, so every cell is non-trivial. (An out-of-line insertion
// call measured slower: the registers it saves cost the unrolled chunk.)
template <typename T, int RPL>
__device__ __forceinline__ void topp_hits(const BandArgs<T> &A, const T (&Cc)[RPL], T inv, int32_t j, int rl0,
                                          T (&th)[RPL], T *lkey, int32_t *lj, int32_t *lcnt, unsigned &ninsert)
{
#pragma unroll
    for (int a = 0; a < RPL; ++a) {
        const T key = Cc[a] * inv;
        if (key > th[a]) {
            const int rl = rl0 + a;
            int32_t cnt = lcnt[rl];
            topp_insert<T>(lkey + rl * A.p, lj + rl * A.p, cnt, A.p, key, j, th[a]);
            lcnt[rl] = cnt;
            ++ninsert;
        }
    }
}

// Two consecutive boundary values in one 8- or 16-byte store (c is even and
// the ring slots are 16-byte aligned).
__device__ __forceinline__ void store_pair(float *p, float a, float b)
{
    *reinterpret_cast<float2 *>(p) = make_float2(a, b);
}
__device__ __forceinline__ void store_pair(double *p, double a, double b)
{
    *reinterpret_cast<double2 *>(p) = make_double2(a, b);
}

template <typename T, int RPL, int NW>
__device__ __forceinline__ void band_chunk_pair(const BandArgs<T> &A, const Col<T> *cbuf, T *bout, int lane,
                                                bool feeds, int64_t cs, int rl0, T (&C)[RPL], const T (&dfr)[RPL],
                                                const T (&dgr)[RPL], T (&th)[RPL], T *lkey, int32_t *lj,
                                                int32_t *lcnt, unsigned &ninsert)
{
    const bool send = feeds && lane == 31;
#pragma unroll
    for (int c = 0; c < CH; c += 2) {
        // (the spare field of a column holds the top edge of its chunk: the
        // predecessor of the warp's first row in that column)
        const Col<T> cd0 = cbuf[c];
        const Col<T> cd1 = cbuf[c + 1];
        T C0[RPL];
        T v = __shfl_up_sync(0xffffffffu, C[RPL - 1], 1);
        if (lane == 0) v = cd0.pad;
#pragma unroll
        for (int a = RPL - 1; a >= 1; --a) C0[a] = fma(dfr[a], cd0.dg, fma(cd0.df, dgr[a], C[a - 1]));
        C0[0] = fma(dfr[0], cd0.dg, fma(cd0.df, dgr[0], v));
        v = __shfl_up_sync(0xffffffffu, C0[RPL - 1], 1);
        if (lane == 0) v = cd1.pad;
#pragma unroll
        for (int a = RPL - 1; a >= 1; --a) C[a] = fma(dfr[a], cd1.dg, fma(cd1.df, dgr[a], C0[a - 1]));
        C[0] = fma(dfr[0], cd1.dg, fma(cd1.df, dgr[0], v));
        if (send) store_pair(bout + c, C0[RPL - 1], C[RPL - 1]);
        // one sign test over both columns' keys; the rare hits re-test per column
        if (__any_sync(0xffffffffu, any_positive_pair(C0, cd0.inv, C, cd1.inv, th))) {
            if (any_positive(C0, cd0.inv, th))
                topp_hits<T, RPL>(A, C0, cd0.inv, (int32_t)(cs + c), rl0, th, lkey, lj, lcnt, ninsert);
            if (any_positive(C, cd1.inv, th))
                topp_hits<T, RPL>(A, C, cd1.inv, (int32_t)(cs + c + 1), rl0, th, lkey, lj, lcnt, ninsert);
        }
    }
}

// Pairwise synchronisation of the warp wavefront: warp w (producer) hands
// the last row of its rows to warp w+1 (consumer) one chunk of CH columns at
// a time through a ring of NSLOT buffers guarded by shared-memory mbarriers:
// full[w+1][slot] (producer arrives after writing) and empty[w+1][slot]
// (consumer arrives after reading). Chunks are counted across the CTA's work
// units so slot and phase parity stay consistent. Every wait is bounded: when
// the bound runs out the kernel records an error (reported as MAD_ETIMEOUT)
// and carries on without blocking.
constexpr int NSLOT = 4;
constexpr int WAIT_LIMIT = 1 << 20;

__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t *b, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *b)
{
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_u32(b))
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *b, unsigned parity)
{
    unsigned ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok)
                 : "r"(smem_u32(b)), "r"(parity)
                 : "memory");
    return ok != 0;
}
__device__ __forceinline__ void mbar_wait(uint64_t *b, unsigned parity, int *err, int limit = WAIT_LIMIT)
{
    for (int it = 0; it < limit; ++it)
        if (mbar_try_wait(b, parity)) return;
    atomicExch(err, 1);
}

// FP32 with up to four rows per lane fits three CTAs per SM (80 registers);
// otherwise two.
template <typename T, int RPL> constexpr int band_min_blocks() { return (sizeof(T) == 4 && RPL <= 4) ? 3 : 2; }

template <typename T, int RPL, int NW, int MODE>
__global__ void __launch_bounds__(NW * 32, band_min_blocks<T, RPL>()) k_band(const BandArgs<T> A)
{
    constexpr bool BINS = MODE == MODE_BINS;
    constexpr bool SYM = MODE == MODE_SYM;
    constexpr int R = 32 * RPL * NW;
    extern __shared__ __align__(32) unsigned char smem_raw[];
    uint64_t *mfull = reinterpret_cast<uint64_t *>(smem_raw);       // [NW][NSLOT]
    uint64_t *mempty = mfull + NW * NSLOT;                         // [NW][NSLOT]
    Col<T> *colbuf = reinterpret_cast<Col<T> *>(mempty + NW * NSLOT);  // [NW][CH]
    T *bbuf = reinterpret_cast<T *>(colbuf + NW * CH);             // [NW][NSLOT][CH]
    unsigned char *tail = reinterpret_cast<unsigned char *>(bbuf + NW * NSLOT * CH);
    // bins mode: int [R][nbins];  top-p mode: T [R][p], int32 [R][p], int32 [R]
    int *sbins = reinterpret_cast<int *>(tail);
    T *lkey = reinterpret_cast<T *>(tail);
    int32_t *lj = reinterpret_cast<int32_t *>(lkey + R * A.p);
    int32_t *lcnt = lj + R * A.p;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    // Seed rows sit every A.sp rows (a multiple of the rows per warp): a warp
    // whose first row is one starts every chain from it; a warp below a
    // warp that is not seeded takes its top edge from that warp. So every
    // chain is at most A.sp steps long.
    const bool seeded = ((int64_t)w * 32 * RPL) % A.sp == 0;
    const bool feeds = w < NW - 1 && ((int64_t)(w + 1) * 32 * RPL) % A.sp != 0;
    const int nb_active = *A.nbands;
    // The symmetric form walks all bands and only the upper triangle; it is
    // used when at least half of the rows need recomputing.
    const bool sym_on = sym_rule(A.allow_sym, *A.nflagged, A.nl);
    if (MODE == MODE_SYM && !sym_on) return;
    if (MODE == MODE_TOPP && sym_on) return;
    const int nb = SYM ? A.kb_total : nb_active;
    const int64_t total = (int64_t)nb * A.ngroups;
    const int NEG_ORD = f2ord(-__int_as_float(0x7f800000));
    const int nbins = A.nbins;

    if (BINS)
        for (int t = threadIdx.x; t < R * nbins; t += blockDim.x) sbins[t] = NEG_ORD;
    // unit queue: warp 0 takes the next work unit from the global counter and
    // hands its index to every warp through uq[] (full: 1 arrival from warp
    // 0; empty: one arrival per warp), so warps flow from one unit into the
    // next without a CTA-wide barrier and units are balanced dynamically.
    __shared__ int uq[NSLOT];
    __shared__ __align__(8) uint64_t ufull[NSLOT], uempty[NSLOT];
    if (threadIdx.x < NW * NSLOT) {
        mbar_init(&mfull[threadIdx.x], 1);
        mbar_init(&mempty[threadIdx.x], 1);
    }
    if (threadIdx.x < NSLOT) {
        mbar_init(&ufull[threadIdx.x], 1);
        mbar_init(&uempty[threadIdx.x], NW);
    }
    __syncthreads();
    unsigned qg = 0;    // chunks processed by this CTA so far (same for every warp)
    unsigned ninsert = 0;

    for (unsigned useq = 0;; ++useq) {
        const int us = (int)(useq % NSLOT);
        const unsigned upar = (useq / NSLOT) & 1u;
        if (w == 0) {
            mbar_wait(&uempty[us], upar ^ 1u, A.err);
            if (lane == 0) {
                uq[us] = atomicAdd(A.unit_ctr, 1);
                mbar_arrive(&ufull[us]);
            }
        }
        mbar_wait(&ufull[us], upar, A.err);
        const int64_t u = uq[us];
        __syncwarp();
        if (lane == 0) mbar_arrive(&uempty[us]);
        if (u >= total) break;
        {
        const int band = SYM ? (int)(u % nb) : A.bands[u % nb];
        int g = (int)(u / nb);
        if (!SYM) {
            // each band's diagonal group first, then to the right (wrapping)
            const int gd = (int)(((int64_t)band * R) / A.group_w);
            g += gd;
            if (g >= A.ngroups) g -= A.ngroups;
        }
        const int64_t i0 = (int64_t)band * R;
        const int64_t c0 = (int64_t)g * A.group_w;
        if (c0 >= A.nl) continue;
        if (SYM && c0 + A.group_w <= i0) continue;   // entirely below the diagonal
        const int64_t c1 = c0 + A.group_w < A.nl ? c0 + A.group_w : A.nl;
        if (threadIdx.x == 0 && A.stats) atomicAdd(&A.stats[5], 1ull);
        const int nchunk = (int)((c1 - c0 + CH - 1) / CH);
        const int64_t rfirst = i0 + (int64_t)w * 32 * RPL;
        const int64_t rbase = rfirst + lane * RPL;
        const int rl0 = w * 32 * RPL + lane * RPL;
        const T *sleft = A.seed + (c0 / A.sp) * A.spitch;
        // a warp whose first row is a seed row starts from it (like the
        // band's first warp); the others take their top edge from the warp
        // above through the ring
        const T *stop = A.seed + (rfirst / A.sp) * A.spitch;

        T C[RPL], dfr[RPL], dgr[RPL], th[RPL], runmax[RPL], invr[RPL];
#pragma unroll
        for (int a = 0; a < RPL; ++a) {
            const int64_t r = rbase + a;
            const Col<T> cr = A.col[r];
            dfr[a] = cr.df;
            dgr[a] = cr.dg;
            invr[a] = cr.inv;
            th[a] = A.thr[r];
            // the best threshold another unit of this row has established
            if (MODE == MODE_TOPP && A.rowbest) {
                const T tb = (T)ord2f(A.rowbest[r]);
                th[a] = tb > th[a] ? tb : th[a];
            }
            C[a] = sleft[r + 1];
            runmax[a] = neg_inf<T>();
            if (!BINS) lcnt[rl0 + a] = 0;
        }
        // (top-p form) a warp none of whose rows is wanted (threshold +inf:
        // certified, flat or past the end), and that neither takes its top
        // edge from the warp above nor hands one to the warp below, skips
        // the unit: none of its cells could enter a list
        if (MODE == MODE_TOPP && seeded && !feeds) {
            bool want = false;
#pragma unroll
            for (int a = 0; a < RPL; ++a) want |= th[a] < T(INFINITY);
            if (!__any_sync(0xffffffffu, want)) {
#pragma unroll
                for (int a = 0; a < RPL; ++a)
                    if (rbase + a < A.nl) A.scnt[(rbase + a) * A.ngroups + g] = 0;
                qg += nchunk;
                continue;
            }
        }
        if (lane == 0 && A.stats) atomicAdd(&A.stats[6], (unsigned long long)(32 * RPL) * (unsigned long long)(c1 - c0));
        T carry = sleft[rfirst];
        // prefetched column data / top edge of the next chunk (the symmetric
        // form carries the column's threshold in the spare field)
        Col<T> ncol = A.col[c0 + lane];
        if (SYM) ncol.pad = A.thr[c0 + lane];
        T ntop = seeded ? stop[c0 + lane] : T(0);

        for (int q = 0; q < nchunk; ++q, ++qg) {
            const int slot = (int)(qg % NSLOT);
            const unsigned par = (qg / NSLOT) & 1u;
            const int64_t cs = c0 + (int64_t)q * CH;
            Col<T> *cbuf = colbuf + w * CH;
            Col<T> cw = ncol;
            T tp;
            if (q + 1 < nchunk) {
                ncol = A.col[cs + CH + lane];
                if (SYM) ncol.pad = A.thr[cs + CH + lane];
            }
            if (seeded) {
                tp = ntop;
                if (q + 1 < nchunk) ntop = stop[cs + CH + lane];
            } else {
                mbar_wait(&mfull[w * NSLOT + slot], par, A.err, A.wave_limit);   // chunk q from warp w-1
                const T *bb = bbuf + (w * NSLOT + slot) * CH;
                const T prev = bb[lane == 0 ? 0 : lane - 1];
                tp = lane == 0 ? carry : prev;
                carry = bb[CH - 1];
                __syncwarp();
                if (lane == 0) mbar_arrive(&mempty[w * NSLOT + slot]);   // slot free again
            }
            // the top edge rides in the column's spare field in the append
            // form (the symmetric form keeps the column threshold there)
            if (MODE == MODE_TOPP) cw.pad = tp;
            cbuf[lane] = cw;
            if (feeds) mbar_wait(&mempty[(w + 1) * NSLOT + slot], par ^ 1u, A.err, A.wave_limit);  // slot free
            __syncwarp();
            T *bout = bbuf + ((w + 1 < NW ? w + 1 : 0) * NSLOT + slot) * CH;
            // does this warp's row range meet the exclusion zone in this chunk?
            const int64_t rlo = rfirst, rhi = rfirst + 32 * RPL - 1;
            // (symmetric form: everything not wholly above the zone is tested cell by cell)
            const bool diag = SYM ? !(cs > rhi + A.E) : (cs <= rhi + A.E) && (cs + CH - 1 >= rlo - A.E);
            if (diag)
                band_chunk<T, RPL, NW, MODE, true>(A, cbuf, tp, bout, lane, feeds, cs, rbase, rl0, C, dfr, dgr, th,
                                                   invr, runmax, lkey, lj, lcnt, ninsert);
            else if (MODE == MODE_TOPP && BAND_PAIR)
                band_chunk_pair<T, RPL, NW>(A, cbuf, bout, lane, feeds, cs, rl0, C, dfr, dgr, th, lkey, lj, lcnt,
                                            ninsert);
            else
                band_chunk<T, RPL, NW, MODE, false>(A, cbuf, tp, bout, lane, feeds, cs, rbase, rl0, C, dfr, dgr, th,
                                                    invr, runmax, lkey, lj, lcnt, ninsert);
            if (feeds && lane == 31) mbar_arrive(&mfull[(w + 1) * NSLOT + slot]);   // chunk q written
            if (BINS) {
                const int bin = (int)((cs / CH) % nbins);
#pragma unroll
                for (int a = 0; a < RPL; ++a) {
                    atomicMax(&sbins[(rl0 + a) * nbins + bin], f2ord(to_float_rd(runmax[a])));
                    runmax[a] = neg_inf<T>();
                }
            }
            __syncwarp();
        }
        if (BINS) {
            __syncthreads();
            for (int t = threadIdx.x; t < R * nbins; t += blockDim.x) {
                const int64_t r = i0 + t / nbins;
                if (r < A.nl && sbins[t] != NEG_ORD) atomicMax(&A.bins[r * nbins + (t % nbins)], sbins[t]);
                sbins[t] = NEG_ORD;
            }
            __syncthreads();
        } else {
            // this unit's per-row lists -> the row's slot for column group g
#pragma unroll
            for (int a = 0; a < RPL; ++a) {
                const int64_t r = rbase + a;
                if (r >= A.nl) continue;
                const int rl = rl0 + a;
                const int32_t cnt = lcnt[rl];
                const int64_t slot = r * A.ngroups + g;
                A.scnt[slot] = cnt;
                // a full list's p-th kept key bounds the row's p-th best key
                // from below: later units of the row start from it
                if (MODE == MODE_TOPP && A.rowbest && cnt == A.p)
                    atomicMax(&A.rowbest[r], f2ord(to_float_rd(th[a])));
                for (int e = 0; e < cnt; ++e) {
                    A.skey[slot * A.p + e] = lkey[rl * A.p + e];
                    A.sj[slot * A.p + e] = lj[rl * A.p + e];
                }
            }
        }
        }
    }
    if (!BINS) {
        // low 16 bits: row-list insertions, high 16 bits: column-side appends
        unsigned long long rowi = ninsert & 0xffffu, coli = ninsert >> 16;
        for (int o = 16; o > 0; o >>= 1) {
            rowi += __shfl_xor_sync(0xffffffffu, rowi, o);
            coli += __shfl_xor_sync(0xffffffffu, coli, o);
        }
        if (lane == 0 && rowi) atomicAdd(A.ninsert, rowi);
        if (lane == 0 && coli && A.stats) atomicAdd(&A.stats[7], coli);
    }
}

template <typename T>
size_t band_smem(bool bins_mode, int p, int rpl)
{
    constexpr int NW = BAND_NW;
    const int R = 32 * rpl * NW;
    size_t s = (size_t)2 * NW * NSLOT * sizeof(uint64_t) + (size_t)NW * CH * sizeof(Col<T>) +
               (size_t)NW * NSLOT * CH * sizeof(T);
    if (bins_mode) s += (size_t)R * band_nbins(p) * sizeof(int);
    else s += (size_t)R * p * (sizeof(T) + sizeof(int32_t)) + (size_t)R * sizeof(int32_t);
    return s;
}

template <typename T, int RPL>
static const void *band_fn_rpl(int mode)
{
    switch (mode) {
    case MODE_BINS: return (const void *)k_band<T, RPL, BAND_NW, MODE_BINS>;
    case MODE_SYM: return (const void *)k_band<T, RPL, BAND_NW, MODE_SYM>;
    default: return (const void *)k_band<T, RPL, BAND_NW, MODE_TOPP>;
    }
}

template <typename T>
static const void *band_fn(int mode, int rpl)
{
    switch (rpl) {
    case 4: return band_fn_rpl<T, 4>(mode);
    case 2: return band_fn_rpl<T, 2>(mode);
    default: return band_fn_rpl<T, 1>(mode);
    }
}

// Shared-memory opt-in of each band kernel variant, once per device.
template <typename T>
static void band_optin(int mode, int rpl)
{
    static std::once_flag once[3][3][64];
    const int ri = rpl == 4 ? 0 : (rpl == 2 ? 1 : 2);
    smem_optin_max(band_fn<T>(mode, rpl), once[mode][ri]);
}

template <typename T>
int band_occupancy(bool bins_mode, int p, int rpl)
{
    int worst = 1 << 30;
    for (int mode : {bins_mode ? (int)MODE_BINS : (int)MODE_TOPP, bins_mode ? (int)MODE_BINS : (int)MODE_SYM}) {
        const void *fn = band_fn<T>(mode, rpl);
        const size_t sm = band_smem<T>(bins_mode, p, rpl);
        band_optin<T>(mode, rpl);
        int blocks = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, fn, BAND_NW * 32, sm) != cudaSuccess) return 0;
        worst = blocks < worst ? blocks : worst;
    }
    return worst;
}

template <typename T>
static void launch_mode(const BandArgs<T> &a, int mode, bool bins_mode, int grid, cudaStream_t s)
{
    const size_t sm = band_smem<T>(bins_mode, a.p, a.rpl);
    const void *fn = band_fn<T>(mode, a.rpl);
    band_optin<T>(mode, a.rpl);
    void *args[] = {const_cast<BandArgs<T> *>(&a)};
    cudaLaunchKernel(fn, dim3(grid), dim3(BAND_NW * 32), args, sm, s);
}

// bins mode: one launch. Otherwise two launches, of which exactly one works:
// the symmetric form when at least half of the bands are active (and
// allowed), the full-square form on the active bands otherwise.
template <typename T>
void launch_band(const BandArgs<T> &a, bool bins_mode, int grid, cudaStream_t s)
{
    if (bins_mode) {
        launch_mode<T>(a, MODE_BINS, true, grid, s);
        return;
    }
    launch_mode<T>(a, MODE_TOPP, false, grid, s);
    if (a.allow_sym) launch_mode<T>(a, MODE_SYM, false, grid, s);
}


}  // namespace mad
