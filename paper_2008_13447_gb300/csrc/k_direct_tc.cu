// k_direct_tc.cu -- recompute of listed rows' full distance profiles on the
// 5th-generation tensor cores (tcgen05): Algorithm 4's SlidingDotProduct for
// the non-valid rows and Algorithm 10's recompute loop, for rows that are too
// few in their band for the diagonal band kernel to pay off.
//
// A block of co-moments is a dense product of two Hankel-shaped matrices:
//     acc(r, j) = sum_t A_r[t] B_j[t],
//     A_r[t] = S_a (x[r+t] - mu_r) / sqrt(M2_r)          (row r, centred, unit norm)
//     B_j[t] = S_b (x[j+t] - s)                          (column j, one shift s per tile)
// so that C(r, j) sqrt(...) follows from acc by a rank-one correction:
//     q(r, j) = (acc - S_b (mu_j - s) sum_t A_r[t]) / sqrt(M2_j) / (S_a S_b),
// the correlation of Eq. DIST. Both operands are split into FP16 pairs
// (hi + lo, about 22 significant bits) and the product is taken as
// hi*hi + hi*lo + lo*hi, accumulated in FP32 in tensor memory (TMEM).
//
// Per work item (128 listed rows x one block of 4096 columns): for each tile
// of 256 columns and each chunk of 64 lags, the row operand is copied into
// shared memory by the bulk-copy engine (cp.async.bulk, from an image the
// prep kernel wrote in the swizzled layout), the column operand is expanded
// from the series by the block's threads, and one thread issues 4 x 3 MMAs
// (M = 128, N = 256, K = 16) into one TMEM accumulator. Then the warps read
// the accumulator back (tcgen05.ld: warp w reads TMEM lanes 32 (w mod 4) ..,
// one row per thread; with p <= 32 the eight warps split the 256 columns in
// two halves), form the correlation and its error bound, and keep each
// row's p best keys over the column block (the halves' lists merged at the
// end of the block).
//
// Error bound of a kept correlation (in q units), from the arithmetic above:
// the pair representation (|a - hi - lo| <= 2^-22 |a| per operand, the
// omitted lo*lo term <= 2^-22 |a b|), the FP32 accumulation of 3K products
// (<= 3K 2^-24 sum|A B|, K the padded lag count), and the FP32 correction and
// scaling, with sum_t |A_r[t] B_j[t]| <= S_a S_b sqrt(M2_j + l (mu_j - s)^2)
// (Cauchy-Schwarz):
//     dq_j = 1.5 ((3 2^-22 + (3K + 4) 2^-24) f_j + 2^-23),
//     f_j  = sqrt(1 + l (mu_j - s)^2 / M2_j)
// (the pipelined form forms x - s in FP32 from the series' FP32 pairs, one
// more rounding of 2^-23 relative to the column operand: 4 2^-22 there).
// A candidate is kept when q + dq_j could beat the row's threshold, and
// carries dq_j to the merge.
#include <cstring>
#include <cuda.h>
#include <cuda_fp16.h>
#include <cudaTypedefs.h>

#include "kernels.cuh"

namespace mad {
namespace {

constexpr int TC_M = 128;          // rows per tile (TMEM lanes)
constexpr int TC_N = 256;          // columns per MMA tile (TMEM columns of the accumulator)
constexpr int TC_KC = 64;          // lags per chunk (one 128-byte swizzle atom of FP16)
constexpr int TC_THREADS = 256;
constexpr int TC_COLS = 4096;      // columns per work item (same blocks as the direct kernel)
constexpr float TC_SA = 256.0f;    // scale of the row operand (|A| <= 256)
constexpr int TC_WAIT = 1 << 22;   // tries of a bounded mbarrier wait
constexpr int A_TILE_BYTES = TC_M * TC_KC * 2;   // 16 KB, one of hi / lo
constexpr int B_TILE_BYTES = TC_N * TC_KC * 2;   // 32 KB
constexpr int SHIFT_LEN = 312;     // halves per shifted copy of the column values

__device__ __forceinline__ unsigned su32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

// Byte offset of element (row m, lag k) in a K-major 128-byte-swizzled tile
// (rows of 64 FP16 at 128 B, the 16-byte chunk index XOR-ed with m mod 8).
__host__ __device__ __forceinline__ int swz(int m, int k)
{
    return m * 128 + ((((k >> 3) ^ (m & 7)) & 7) << 4) + (k & 7) * 2;
}

// Shared-memory matrix descriptor (tcgen05): start address, stride between
// 8-row groups (1024 B), descriptor version 1, 128-byte swizzle.
__device__ __forceinline__ uint64_t sdesc(unsigned addr)
{
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFF) >> 4);
    d |= (uint64_t)1 << 16;                 // leading byte offset (unused with this swizzle)
    d |= (uint64_t)(1024 >> 4) << 32;       // stride byte offset
    d |= (uint64_t)1 << 46;                 // version
    d |= (uint64_t)2 << 61;                 // 128-byte swizzle
    return d;
}

// Instruction descriptor of kind::f16: FP16 A and B, FP32 D, both K-major,
// N = 256, M = 128.
constexpr uint32_t IDESC = (1u << 4) | (0u << 7) | (0u << 10) | ((uint32_t)(TC_N >> 3) << 17) |
                           ((uint32_t)(TC_M >> 4) << 24);

__device__ __forceinline__ void mbar_init(uint64_t *b, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *b, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t *b, unsigned parity)
{
    unsigned ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok)
                 : "r"(su32(b)), "r"(parity)
                 : "memory");
    return ok != 0;
}
// Bounded wait; false (and the error word set) if the phase never completed.
__device__ __forceinline__ bool mbar_wait_b(uint64_t *b, unsigned parity, int *err)
{
    for (int it = 0; it < TC_WAIT; ++it)
        if (mbar_try(b, parity)) return true;
    atomicExch(err, 2);
    return false;
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     su32(dst)),
                 "l"(src), "r"(bytes), "r"(su32(bar))
                 : "memory");
}
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tc_mma(uint32_t dtmem, uint64_t a, uint64_t b, uint32_t accumulate)
{
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
                 "l"(a), "l"(b), "r"(IDESC), "r"(accumulate)
                 : "memory");
}
__device__ __forceinline__ void tc_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar))
                 : "memory");
}

// 32 consecutive accumulator columns of this thread's TMEM lane.
__device__ __forceinline__ void tc_ld32(uint32_t taddr, float (&v)[32])
{
    uint32_t r[32];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
                 "%13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, "
                 "[%32];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                   "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
                   "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
                   "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                 : "r"(taddr)
                 : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int c = 0; c < 32; ++c) v[c] = __uint_as_float(r[c]);
}

__device__ __forceinline__ void split_half(float v, __half &hi, __half &lo)
{
    hi = __float2half_rn(v);
    lo = __float2half_rn(v - __half2float(hi));
}

// Row operand images of the listed rows at length l, in the layout the MMA
// reads: [row tile][lag chunk][hi, lo][128 rows x 64 lags, swizzled], zero
// past the row's length and past the last listed row; plus per row the sum
// of its represented values (for the rank-one correction) and sqrt(M2).
__global__ void k_tc_rows(TcArgs A)
{
    const int nrows = *A.nrows;
    const int l = A.l;
    const int nkc = A.nkc;
    const int64_t ntile = (nrows + TC_M - 1) / TC_M;
    __shared__ float red[TC_THREADS / 32];
    for (int64_t pos = blockIdx.x; pos < ntile * TC_M; pos += gridDim.x) {
        const int rt = (int)(pos / TC_M), m = (int)(pos % TC_M);
        const bool live = pos < nrows;
        const int64_t r = live ? A.rows[pos] : 0;
        const double mu = live ? A.mu[r] : 0.0;
        const double isd = live ? A.isd[r] : 0.0;
        float part = 0.0f;
        for (int k = threadIdx.x; k < nkc * TC_KC; k += blockDim.x) {
            float v = 0.0f;
            if (live && k < l) v = (float)((A.x[r + k] - mu) * isd) * TC_SA;
            __half hi, lo;
            split_half(v, hi, lo);
            part += __half2float(hi) + __half2float(lo);
            const int kc = k / TC_KC, kk = k % TC_KC;
            unsigned char *base = A.aimg + ((size_t)(rt * nkc + kc) * 2) * A_TILE_BYTES;
            *reinterpret_cast<__half *>(base + swz(m, kk)) = hi;
            *reinterpret_cast<__half *>(base + A_TILE_BYTES + swz(m, kk)) = lo;
        }
        for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
        __syncthreads();
        if (threadIdx.x == 0) {
            float s = 0.0f;
            for (int w = 0; w < TC_THREADS / 32; ++w) s += red[w];
            A.asum[pos] = s;
            A.sqm2[pos] = (live && isd > 0.0) ? (float)(1.0 / isd) : 0.0f;
        }
        __syncthreads();
    }
}

// Insert (key, j, dq) into a row's list (keys descending, at most p). The
// callers test key > kmin first, kmin = the p-th kept key once p are kept
// (else -inf): the same test this insert makes, held in a register so that
// the columns that cannot enter skip the call.
template <typename T>
__device__ __forceinline__ void list_insert(T *K, int32_t *J, float *D, int &cnt, int p, T key, int32_t j, float dq)
{
    if (cnt == p && !(key > K[p - 1])) return;
    int b = cnt < p ? cnt++ : p - 1;
    while (b > 0 && K[b - 1] < key) {
        K[b] = K[b - 1];
        J[b] = J[b - 1];
        D[b] = D[b - 1];
        --b;
    }
    K[b] = key;
    J[b] = j;
    D[b] = dq;
}

struct __align__(16) ColC { float c, g, dq, pad; };

__global__ void __launch_bounds__(TC_THREADS, 1) k_direct_tc(TcArgs A)
{
    const int nrows = *A.nrows;
    if (nrows <= 0) return;
    const int l = A.l;
    const int nkc = A.nkc;
    const int p = A.p;
    const int rtiles = (nrows + TC_M - 1) / TC_M;
    const int64_t items = (int64_t)rtiles * A.nblk;
    if (blockIdx.x >= items) return;

    extern __shared__ __align__(1024) unsigned char sm_raw[];
    // 1024-byte aligned tiles first: A hi/lo (16 KB each), B hi/lo (32 KB each)
    unsigned char *sm = reinterpret_cast<unsigned char *>(((uintptr_t)sm_raw + 1023) & ~(uintptr_t)1023);
    unsigned char *sa = sm;                              // [2][A_TILE_BYTES]
    unsigned char *sb = sa + 2 * A_TILE_BYTES;           // [2][B_TILE_BYTES]
    __half *shift = reinterpret_cast<__half *>(sb + 2 * B_TILE_BYTES);   // [2][8][SHIFT_LEN]
    ColC *cc = reinterpret_cast<ColC *>(shift + 2 * 8 * SHIFT_LEN);      // [TC_N]
    // column halves of the epilogue (threads per row) and each thread's list
    const int H = p <= 32 ? 2 : 1;
    float *lk = reinterpret_cast<float *>(cc + TC_N);                   // [H][TC_M][p]
    int32_t *lj = reinterpret_cast<int32_t *>(lk + H * TC_M * p);
    float *ld = reinterpret_cast<float *>(lj + H * TC_M * p);
    __shared__ __align__(8) uint64_t bar_a, bar_mma;
    __shared__ uint32_t tmem_base;
    __shared__ float red[TC_THREADS / 32];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) {
        mbar_init(&bar_a, 1);
        mbar_init(&bar_mma, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tmem_base)),
                     "r"(TC_N)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;
    unsigned pa = 0, pm = 0;           // mbarrier phases
    bool ok = true;
    float dqmax = 0.0f;

    for (int64_t item = blockIdx.x; item < items && ok; item += gridDim.x) {
        const int rt = (int)(item / A.nblk);
        const int cb = (int)(item % A.nblk);
        const int64_t cb0 = (int64_t)cb * TC_COLS;
        // this thread's row (TMEM lane m = tid mod 128) and column half h
        const int m = tid & (TC_M - 1), h = tid / TC_M;
        const bool ethread = h < H;
        const int64_t pos = (int64_t)rt * TC_M + m;
        const bool erow = ethread && pos < nrows;
        const int64_t r = erow ? A.rows[pos] : -1;
        const float asum = erow ? A.asum[pos] : 0.0f;
        const float sq = erow ? A.sqm2[pos] : 0.0f;
        // threshold in correlation units (listed rows are not flat: sq > 0)
        const float thq = erow ? (float)A.thr[r] / sq : 0.0f;
        const int64_t exlo = r - A.E, exhi = r + A.E;   // trivial matches of the row
        float *mk = lk + (h * TC_M + m) * p;
        int32_t *mj = lj + (h * TC_M + m) * p;
        float *md = ld + (h * TC_M + m) * p;
        int cnt = 0;
        float kmin = -INFINITY;   // the p-th kept key once p are kept
        for (int st0 = 0; st0 < TC_COLS / TC_N && ok; ++st0) {
            const int64_t j0 = cb0 + (int64_t)st0 * TC_N;
            if (j0 >= A.nl) break;
            // ---- column constants of this tile: shift s, scale S_b, correction,
            // normaliser and error bound per column
            const int64_t jm = j0 + TC_N / 2 < A.nl ? j0 + TC_N / 2 : A.nl - 1;
            const double s = A.mu[jm];
            float spread = 0.0f;
            {
                const int64_t j = j0 + tid;
                if (j < A.nl) {
                    const double m2 = A.m2[j];
                    spread = (float)(sqrt(m2 > 0.0 ? m2 : 0.0) + fabs(A.mu[j] - s));
                }
                for (int o = 16; o > 0; o >>= 1) spread = fmaxf(spread, __shfl_xor_sync(0xffffffffu, spread, o));
                if (lane == 0) red[warp] = spread;
            }
            __syncthreads();
            float mx = 0.0f;
            for (int w = 0; w < TC_THREADS / 32; ++w) mx = fmaxf(mx, red[w]);
            // S_b: a power of two with max |B| <= 256
            const float Sb = mx > 0.0f ? exp2f(floorf(log2f(255.0f / mx))) : 1.0f;
            {
                const int64_t j = j0 + tid;
                ColC c{0.0f, 0.0f, 0.0f, 0.0f};
                if (j < A.nl) {
                    const double isd = A.isd[j];
                    const double dm = A.mu[j] - s;
                    c.c = (float)(Sb * dm);
                    c.g = (float)(isd / ((double)TC_SA * Sb));
                    const double f = sqrt(1.0 + (double)l * dm * dm * isd * isd);
                    const double K = (double)nkc * TC_KC;
                    c.dq = (float)(1.5 * ((3.0 * 0x1p-22 + (3.0 * K + 4.0) * 0x1p-24) * f + 0x1p-23));
                    dqmax = fmaxf(dqmax, c.dq);
                }
                cc[tid] = c;
            }
            // ---- lag chunks: stage A, build B, 12 MMAs
            for (int kc = 0; kc < nkc; ++kc) {
                if (tid == 0) {
                    mbar_expect_tx(&bar_a, 2 * A_TILE_BYTES);
                    const unsigned char *src = A.aimg + ((size_t)(rt * nkc + kc) * 2) * A_TILE_BYTES;
                    bulk_g2s(sa, src, A_TILE_BYTES, &bar_a);
                    bulk_g2s(sa + A_TILE_BYTES, src + A_TILE_BYTES, A_TILE_BYTES, &bar_a);
                }
                // column values v[i] = S_b (x[g0 + i] - s), i in [0, 320), as FP16
                // pairs in eight copies shifted by 0..7 (every row of the tile is
                // then an aligned 16-byte copy)
                const int64_t g0 = j0 + (int64_t)kc * TC_KC;
                for (int e = tid; e < 8 * SHIFT_LEN; e += TC_THREADS) {
                    const int sft = e / SHIFT_LEN, i = e % SHIFT_LEN;
                    const int64_t g = g0 + i + sft;
                    const float v = g < A.n ? (float)(A.x[g] - s) * Sb : 0.0f;
                    __half hi, lo;
                    split_half(v, hi, lo);
                    shift[sft * SHIFT_LEN + i] = hi;
                    shift[(8 + sft) * SHIFT_LEN + i] = lo;
                }
                __syncthreads();
                for (int e = tid; e < 2 * TC_N * 8; e += TC_THREADS) {
                    const int hl = e / (TC_N * 8), rem = e % (TC_N * 8);
                    const int nn = rem / 8, c = rem % 8;
                    const int sft = nn & 7;
                    const uint4 v = *reinterpret_cast<const uint4 *>(shift + (hl * 8 + sft) * SHIFT_LEN +
                                                                     (nn - sft) + 8 * c);
                    *reinterpret_cast<uint4 *>(sb + hl * B_TILE_BYTES + swz(nn, 8 * c)) = v;
                }
                fence_async_smem();
                tc_fence_before();
                __syncthreads();
                if (tid == TC_M) {
                    tc_fence_after();
                    if (!mbar_wait_b(&bar_a, pa, A.err)) ok = false;
                    if (ok) {
                        const unsigned a0 = su32(sa), b0 = su32(sb);
#pragma unroll
                        for (int ks = 0; ks < TC_KC / 16; ++ks) {
                            const uint64_t ah = sdesc(a0 + ks * 32), al = sdesc(a0 + A_TILE_BYTES + ks * 32);
                            const uint64_t bh = sdesc(b0 + ks * 32), bl = sdesc(b0 + B_TILE_BYTES + ks * 32);
                            tc_mma(tmem, ah, bh, (kc > 0 || ks > 0) ? 1u : 0u);
                            tc_mma(tmem, ah, bl, 1u);
                            tc_mma(tmem, al, bh, 1u);
                        }
                    }
                    tc_commit(&bar_mma);
                }
                pa ^= 1u;
                // the MMAs have read the tiles (and written the accumulator)
                // before anything is overwritten
                if (!mbar_wait_b(&bar_mma, pm, A.err)) ok = false;
                pm ^= 1u;
                tc_fence_after();
                ok = __syncthreads_and(ok);
                if (!ok) break;
            }
            if (!ok) break;
            // ---- epilogue: one row per thread, the thread's column half, 32
            // columns per TMEM load; candidates where q + dq_j beats the
            // threshold, then the validity checks
            if (ethread) {
                const int cw = TC_N / H;
                for (int c0 = h * cw; c0 < (h + 1) * cw; c0 += 32) {
                    float v[32];
                    __syncwarp();
                    tc_ld32(tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)c0, v);
                    if (!erow) continue;
                    unsigned hits = 0;
#pragma unroll
                    for (int c = 0; c < 32; ++c) {
                        const ColC k = cc[c0 + c];
                        const float t = fmaf(-k.c, asum, v[c]);
                        hits |= (unsigned)(fmaf(t, k.g, k.dq) > thq && t * k.g * sq > kmin) << c;
                    }
                    if (hits) {
#pragma unroll
                        for (int c = 0; c < 32; ++c) {
                            if (!((hits >> c) & 1u)) continue;
                            const ColC k = cc[c0 + c];
                            const float key = fmaf(-k.c, asum, v[c]) * k.g * sq;
                            const int64_t j = j0 + c0 + c;
                            if (key > kmin && j < A.nl && (j < exlo || j > exhi)) {
                                list_insert<float>(mk, mj, md, cnt, p, key, (int32_t)j, k.dq);
                                if (cnt == p) kmin = mk[p - 1];
                            }
                        }
                    }
                }
            }
            tc_fence_before();
            __syncthreads();
            tc_fence_after();
        }
        // ---- this item's per-row lists: the halves merged by (key desc,
        // offset asc), the p best written
        __shared__ int hcnt[TC_M];
        if (h == 1) hcnt[m] = cnt;
        __syncthreads();
        if (erow && h == 0 && ok) {
            const int64_t slot = pos * A.nblk + cb;
            const float *bk = lk + (TC_M + m) * p;
            const int32_t *bj = lj + (TC_M + m) * p;
            const float *bd = ld + (TC_M + m) * p;
            const int nb = H > 1 ? hcnt[m] : 0;
            int ia = 0, ib = 0, e = 0;
            for (; e < p && (ia < cnt || ib < nb); ++e) {
                bool takea = ib >= nb;
                if (!takea && ia < cnt) takea = mk[ia] > bk[ib] || (mk[ia] == bk[ib] && mj[ia] < bj[ib]);
                if (takea) {
                    A.okey[slot * p + e] = mk[ia];
                    A.oj[slot * p + e] = mj[ia];
                    A.odq[slot * p + e] = md[ia];
                    ++ia;
                } else {
                    A.okey[slot * p + e] = bk[ib];
                    A.oj[slot * p + e] = bj[ib];
                    A.odq[slot * p + e] = bd[ib];
                    ++ib;
                }
            }
            A.ocnt[slot] = e;
        }
        __syncthreads();
    }
    if (dqmax > 0.0f) atomicMax(reinterpret_cast<int *>(A.dq_max), __float_as_int(dqmax));
    // after a wait that ran out, give the MMAs in flight one more bounded
    // wait before the accumulator is freed
    if (!ok && tid == TC_M) mbar_wait_b(&bar_mma, pm ^ 1u, A.err);
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_N) : "memory");
    }
}

// ------------------------------------------------------------------
// Pipelined form (p <= TC2_MAXP): the same products and epilogue, with the
// steps overlapped by warp roles and mbarriers instead of run one after the
// other:
//   warps 0..7  (producers): per 64-lag chunk, wait until the chunk's
//               shared-memory stage is free, start the row operand's bulk
//               copy, build the column tile, arrive on the stage's "full"
//               barrier; per 256-column tile, the column constants;
//   warp 12     (MMA): per chunk, wait for "full", issue the 12 MMAs into the
//               tile's accumulator, commit to the stage's "free" barrier
//               (and after the tile's last chunk to the accumulator's "full");
//   warps 8..11 (epilogue): per tile, wait for the accumulator, read it back
//               (TMEM lanes 32 (w mod 4) .., one row per thread), keep the
//               rows' best p keys, arrive on the accumulator's "free".
// Two stages (row and column operands) and two accumulators (512 TMEM
// columns): the column tile of chunk c + 1 is built while the MMAs of chunk c
// run, and the epilogue of tile t runs while the MMAs of tile t + 1 run.
// Every role walks the same (item, tile, chunk) sequence, so the barriers'
// phases follow from the counters. Every wait is bounded; after the first
// one that runs out (error word set) every later wait returns at once, and
// all threads still walk the whole sequence, so that the producers' named
// barriers (which cannot time out) are always met by all of them.
constexpr int TC2_THREADS = 416;   // 8 producer warps, 4 epilogue warps, 1 MMA warp
constexpr int TC2_PROD = 256;
constexpr int TC2_EPI0 = 256;      // first epilogue thread (warp 8)
constexpr int TC2_MMA = 384;       // MMA warp (warp 12)
constexpr int TC2_MAXP = 10;
constexpr int TC2_STAGE = 2 * A_TILE_BYTES + 2 * B_TILE_BYTES;   // 96 KB
static_assert(TC2_PROD == TC_N, "one producer thread per tile row");

__device__ __forceinline__ void mbar_arrive1(uint64_t *b)
{
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(su32(b)) : "memory");
}
__device__ __forceinline__ void prod_sync() { asm volatile("bar.sync 1, 256;" ::: "memory"); }

struct Tc2Bars {
    uint64_t full[2], freeb[2], accfull[2], accfree[2], ccready[2], fin;
};

__global__ void __launch_bounds__(TC2_THREADS, 1) k_direct_tc2(TcArgs A)
{
    const int nrows = *A.nrows;
    if (nrows <= 0) return;
    const int l = A.l;
    const int nkc = A.nkc;
    const int p = A.p;
    const int rtiles = (nrows + TC_M - 1) / TC_M;
    const int64_t items = (int64_t)rtiles * A.nblk;
    if (blockIdx.x >= items) return;

    extern __shared__ __align__(1024) unsigned char sm_raw[];
    unsigned char *sm = reinterpret_cast<unsigned char *>(((uintptr_t)sm_raw + 1023) & ~(uintptr_t)1023);
    // stage g: A hi, A lo (16 KB each), B hi, B lo (32 KB each)
    __half *shift = reinterpret_cast<__half *>(sm + 2 * TC2_STAGE);          // [hi, lo][8][SHIFT_LEN]
    ColC *cc = reinterpret_cast<ColC *>(shift + 2 * 8 * SHIFT_LEN);          // [2][TC_N]
    float *lk = reinterpret_cast<float *>(cc + 2 * TC_N);                    // [TC_M][p]
    int32_t *lj = reinterpret_cast<int32_t *>(lk + TC_M * p);
    float *ld = reinterpret_cast<float *>(lj + TC_M * p);
    __shared__ __align__(8) Tc2Bars bars;
    __shared__ uint32_t tmem_base;
    __shared__ float red[TC2_PROD / 32];
    __shared__ int abort_flag;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) {
        for (int g = 0; g < 2; ++g) {
            mbar_init(&bars.full[g], TC2_PROD + 1);    // producers + the copy's expect-tx
            mbar_init(&bars.freeb[g], 1);              // MMA commit
            mbar_init(&bars.accfull[g], 1);            // MMA commit
            mbar_init(&bars.accfree[g], TC_M);         // epilogue threads
            mbar_init(&bars.ccready[g], TC2_PROD);     // producers
        }
        mbar_init(&bars.fin, 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == TC2_MMA / 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tmem_base)),
                     "r"(2 * TC_N)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;
    volatile int *abortv = &abort_flag;
    auto wait = [&](uint64_t *b, unsigned par) {
        if (*abortv) return false;
        if (mbar_wait_b(b, par, A.err)) return true;
        *abortv = 1;
        return false;
    };

    if (tid < TC2_PROD) {
        // ------------------------------------------------------ producers
        unsigned t = 0, c = 0;
        float dqmax = 0.0f;
        for (int64_t item = blockIdx.x; item < items; item += gridDim.x) {
            const int rt = (int)(item / A.nblk);
            const int64_t cb0 = (int64_t)(item % A.nblk) * TC_COLS;
            for (int st0 = 0; st0 < TC_COLS / TC_N; ++st0, ++t) {
                const int64_t j0 = cb0 + (int64_t)st0 * TC_N;
                if (j0 >= A.nl) break;
                const int a = t & 1;
                if (t >= 2) wait(&bars.accfree[a], ((t >> 1) - 1) & 1);
                // tile shift s, scale S_b, per-column constants (one column per thread)
                const int64_t jm = j0 + TC_N / 2 < A.nl ? j0 + TC_N / 2 : A.nl - 1;
                const double sft = A.mu[jm];
                const int64_t jc = j0 + tid;
                float spread = 0.0f;
                if (jc < A.nl) {
                    const double m2 = A.m2[jc];
                    spread = (float)(sqrt(m2 > 0.0 ? m2 : 0.0) + fabs(A.mu[jc] - sft));
                }
                for (int o = 16; o > 0; o >>= 1) spread = fmaxf(spread, __shfl_xor_sync(0xffffffffu, spread, o));
                if (lane == 0) red[warp] = spread;
                prod_sync();
                float mx = 0.0f;
                for (int w = 0; w < TC2_PROD / 32; ++w) mx = fmaxf(mx, red[w]);
                const float Sb = mx > 0.0f ? exp2f(floorf(log2f(255.0f / mx))) : 1.0f;
                {
                    ColC cv{0.0f, 0.0f, 0.0f, 0.0f};
                    if (jc < A.nl) {
                        const double isd = A.isd[jc];
                        const double dm = A.mu[jc] - sft;
                        cv.c = (float)(Sb * dm);
                        cv.g = (float)(isd / ((double)TC_SA * Sb));
                        const double f = sqrt(1.0 + (double)l * dm * dm * isd * isd);
                        const double K = (double)nkc * TC_KC;
                        cv.dq = (float)(1.5 * ((4.0 * 0x1p-22 + (3.0 * K + 4.0) * 0x1p-24) * f + 0x1p-23));
                        dqmax = fmaxf(dqmax, cv.dq);
                    }
                    cc[a * TC_N + tid] = cv;
                }
                mbar_arrive1(&bars.ccready[a]);
                // x - s in FP32 from the series' FP32 pairs (GB300's FP64 rate
                // is 1/64 of FP32): relative error below 2^-23
                const float s_hi = (float)sft, s_lo = (float)(sft - (double)s_hi);
                // the chunk's values v[i], i = tid and tid + 256 (< SHIFT_LEN + 7),
                // loaded one chunk ahead so their latency overlaps the tile build
                float xa_h = 0.0f, xa_l = 0.0f, xb_h = 0.0f, xb_l = 0.0f;
                {
                    const int64_t gx = j0 + tid, gy = gx + TC2_PROD;
                    if (gx < A.n) { xa_h = A.xh[gx]; xa_l = A.xl[gx]; }
                    if (tid + TC2_PROD < SHIFT_LEN + 7 && gy < A.n) { xb_h = A.xh[gy]; xb_l = A.xl[gy]; }
                }
                for (int kc = 0; kc < nkc; ++kc, ++c) {
                    const int g = c & 1;
                    unsigned char *sa = sm + g * TC2_STAGE;
                    unsigned char *sb = sa + 2 * A_TILE_BYTES;
                    if (c >= 2) wait(&bars.freeb[g], ((c >> 1) - 1) & 1);
                    if (tid == 0) {
                        mbar_expect_tx(&bars.full[g], 2 * A_TILE_BYTES);
                        const unsigned char *src = A.aimg + ((size_t)(rt * nkc + kc) * 2) * A_TILE_BYTES;
                        bulk_g2s(sa, src, A_TILE_BYTES, &bars.full[g]);
                        bulk_g2s(sa + A_TILE_BYTES, src + A_TILE_BYTES, A_TILE_BYTES, &bars.full[g]);
                    }
                    // column values in eight copies shifted by 0..7, then the
                    // swizzled tile rows (the previous chunk's rows are built
                    // from the copies before they are overwritten)
                    if (kc > 0) prod_sync();
                    __half *sh = shift;
                    const int64_t gb = j0 + (int64_t)kc * TC_KC;
                    // each value v[i] (i < SHIFT_LEN + 7) once, stored to the
                    // eight copies at i - sf (copy sf holds v[i' + sf] at i')
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int i = tid + h * TC2_PROD;
                        if (i >= SHIFT_LEN + 7) break;
                        const float xh = h ? xb_h : xa_h, xl = h ? xb_l : xa_l;
                        const float v = gb + i < A.n ? ((xh - s_hi) + (xl - s_lo)) * Sb : 0.0f;
                        __half hi, lo;
                        split_half(v, hi, lo);
#pragma unroll
                        for (int sf = 0; sf < 8; ++sf) {
                            const int ip = i - sf;
                            if (ip >= 0 && ip < SHIFT_LEN) {
                                sh[sf * SHIFT_LEN + ip] = hi;
                                sh[(8 + sf) * SHIFT_LEN + ip] = lo;
                            }
                        }
                    }
                    // the next chunk's values
                    if (kc + 1 < nkc) {
                        const int64_t gx = gb + TC_KC + tid, gy = gx + TC2_PROD;
                        xa_h = xa_l = xb_h = xb_l = 0.0f;
                        if (gx < A.n) { xa_h = A.xh[gx]; xa_l = A.xl[gx]; }
                        if (tid + TC2_PROD < SHIFT_LEN + 7 && gy < A.n) { xb_h = A.xh[gy]; xb_l = A.xl[gy]; }
                    }
                    prod_sync();
                    // tile row nn (hi and lo): eight aligned 16-byte copies from
                    // the copy shifted by nn mod 8
                    {
                        const int nn = tid, sf = nn & 7;
#pragma unroll
                        for (int hl = 0; hl < 2; ++hl) {
                            const __half *src = sh + (hl * 8 + sf) * SHIFT_LEN + (nn - sf);
                            unsigned char *dst = sb + hl * B_TILE_BYTES + nn * 128;
#pragma unroll
                            for (int q = 0; q < 8; ++q)
                                *reinterpret_cast<uint4 *>(dst + (((q ^ sf) & 7) << 4)) =
                                    *reinterpret_cast<const uint4 *>(src + 8 * q);
                        }
                    }
                    fence_async_smem();
                    mbar_arrive1(&bars.full[g]);
                }
            }
        }
        if (dqmax > 0.0f) atomicMax(reinterpret_cast<int *>(A.dq_max), __float_as_int(dqmax));
    } else if (tid == TC2_MMA) {
        // ----------------------------------------------------------- MMA
        unsigned t = 0, c = 0;
        for (int64_t item = blockIdx.x; item < items; item += gridDim.x) {
            const int64_t cb0 = (int64_t)(item % A.nblk) * TC_COLS;
            for (int st0 = 0; st0 < TC_COLS / TC_N; ++st0, ++t) {
                if (cb0 + (int64_t)st0 * TC_N >= A.nl) break;
                const int a = t & 1;
                if (t >= 2) wait(&bars.accfree[a], ((t >> 1) - 1) & 1);
                tc_fence_after();
                const uint32_t dacc = tmem + (uint32_t)(a * TC_N);
                for (int kc = 0; kc < nkc; ++kc, ++c) {
                    const int g = c & 1;
                    wait(&bars.full[g], (c >> 1) & 1);
                    tc_fence_after();
                    if (!*abortv) {
                        const unsigned a0 = su32(sm + g * TC2_STAGE), b0 = a0 + 2 * A_TILE_BYTES;
#pragma unroll
                        for (int ks = 0; ks < TC_KC / 16; ++ks) {
                            const uint64_t ah = sdesc(a0 + ks * 32), al = sdesc(a0 + A_TILE_BYTES + ks * 32);
                            const uint64_t bh = sdesc(b0 + ks * 32), bl = sdesc(b0 + B_TILE_BYTES + ks * 32);
                            tc_mma(dacc, ah, bh, (kc > 0 || ks > 0) ? 1u : 0u);
                            tc_mma(dacc, ah, bl, 1u);
                            tc_mma(dacc, al, bh, 1u);
                        }
                    }
                    tc_commit(&bars.freeb[g]);                 // the stage may be refilled
                    if (kc == nkc - 1) tc_commit(&bars.accfull[a]);   // the tile's accumulator is complete
                }
            }
        }
        // every MMA issued has completed before the accumulators are freed
        tc_commit(&bars.fin);
        mbar_wait_b(&bars.fin, 0, A.err);
    } else if (tid >= TC2_EPI0 && tid < TC2_MMA) {
        // ------------------------------------------------------ epilogue
        const int m = tid - TC2_EPI0;      // TMEM lane (warps 8..11 read quarters 0..3)
        float *mk = lk + m * p;
        int32_t *mj = lj + m * p;
        float *md = ld + m * p;
        unsigned t = 0;
        for (int64_t item = blockIdx.x; item < items; item += gridDim.x) {
            const int rt = (int)(item / A.nblk);
            const int cb = (int)(item % A.nblk);
            const int64_t cb0 = (int64_t)cb * TC_COLS;
            const int64_t pos = (int64_t)rt * TC_M + m;
            const bool erow = pos < nrows;
            const int64_t r = erow ? A.rows[pos] : -1;
            const float asum = erow ? A.asum[pos] : 0.0f;
            const float sq = erow ? A.sqm2[pos] : 0.0f;
            const float thq = erow ? (float)A.thr[r] / sq : 0.0f;
            const int64_t exlo = r - A.E, exhi = r + A.E;
            int cnt = 0;
            float kmin = -INFINITY;   // the p-th kept key once p are kept
            for (int st0 = 0; st0 < TC_COLS / TC_N; ++st0, ++t) {
                const int64_t j0 = cb0 + (int64_t)st0 * TC_N;
                if (j0 >= A.nl) break;
                const int a = t & 1;
                wait(&bars.accfull[a], (t >> 1) & 1);
                wait(&bars.ccready[a], (t >> 1) & 1);
                tc_fence_after();
                const ColC *ca = cc + a * TC_N;
                for (int c0 = 0; c0 < TC_N; c0 += 32) {
                    float v[32];
                    __syncwarp();
                    tc_ld32(tmem + ((uint32_t)(m & ~31) << 16) + (uint32_t)(a * TC_N + c0), v);
                    if (!erow || *abortv) continue;
                    // the 32 columns' tests first (independent, no branches),
                    // then the rare candidates in column order
                    unsigned hits = 0;
#pragma unroll
                    for (int q = 0; q < 32; ++q) {
                        const ColC k = ca[c0 + q];
                        const float tt = fmaf(-k.c, asum, v[q]);
                        hits |= (unsigned)(fmaf(tt, k.g, k.dq) > thq && tt * k.g * sq > kmin) << q;
                    }
                    if (hits) {
#pragma unroll
                        for (int q = 0; q < 32; ++q) {
                            if (!((hits >> q) & 1u)) continue;
                            const ColC k = ca[c0 + q];
                            const float key = fmaf(-k.c, asum, v[q]) * k.g * sq;
                            const int64_t j = j0 + c0 + q;
                            if (key > kmin && j < A.nl && (j < exlo || j > exhi)) {
                                list_insert<float>(mk, mj, md, cnt, p, key, (int32_t)j, k.dq);
                                if (cnt == p) kmin = mk[p - 1];
                            }
                        }
                    }
                }
                tc_fence_before();
                mbar_arrive1(&bars.accfree[a]);   // accumulator and column constants released
            }
            if (erow && !*abortv) {
                const int64_t slot = pos * A.nblk + cb;
                for (int e = 0; e < cnt; ++e) {
                    A.okey[slot * p + e] = mk[e];
                    A.oj[slot * p + e] = mj[e];
                    A.odq[slot * p + e] = md[e];
                }
                A.ocnt[slot] = cnt;
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == TC2_MMA / 32) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * TC_N) : "memory");
    }
}

// ------------------------------------------------------------------
// Column tiles by TMA (p <= TC3_MAXP): the same products and error bounds,
// without building the column operand in shared memory. The column operand
// of a 256-column tile is a Hankel matrix: for chunk kc its row for column
// j holds V[j - j0 + 64 kc + k], k < 64, with V = S_b (x - s) the tile's
// scaled values. k_tc_cols writes, once per length and tile, V as FP16
// pairs in eight copies shifted by 0..7 values (copy sf holds V[i + sf] at
// i); the column j = j0 + 8 r + sf then starts at copy sf, offset
// 8 r + 64 kc: 16-byte aligned rows 16 bytes apart, so one 5-D TMA box
// {64 lags, 32 rows, 8 copies, tile, hi | lo} lands the 256 x 64 tile in
// the 128-byte-swizzled K-major layout the MMA reads, its row n' = 32 sf + r
// holding column j0 + 8 (n' mod 32) + n' / 32 (so do the accumulator's
// columns and the column constants).
//   warp 0 (loader): per tile the column constants (bulk copy), per chunk
//          the row operand (two bulk copies) and the column operand (two
//          TMA loads), each into a stage freed by the MMA's commit;
//   warp 1 (MMA):    as in k_direct_tc2;
//   warps 2..9 (epilogue): warp w reads TMEM lanes 32 (w mod 4) .. and the
//          column half (w - 2) / 4 of each tile; each thread keeps its row's
//          best p keys of its half in registers; the halves are merged at
//          the end of each work item.
// Every wait is bounded; after the first one that runs out no further copy
// is issued, every later wait returns at once, and before the block ends
// the loader waits (bounded) for the copies it issued.
constexpr int TC3_THREADS = 320;
constexpr int TC3_EPI0 = 64;          // first epilogue thread (warp 2)
constexpr int TC3_MAXP = 16;
constexpr int TC3_STAGE = 2 * A_TILE_BYTES + 2 * B_TILE_BYTES;   // 96 KB
constexpr int TC3_CC_BYTES = TC_N * 16;                          // column constants of a tile

struct Tc3Params {
    TcArgs a;
    CUtensorMap bmap;     // the shifted copies, dims {lc, 32, 8, tiles, 2}
};

struct Tc3Bars {
    uint64_t full[2], freeb[2], accfull[2], accfree[2], ccfull[2], fin;
};

__device__ __forceinline__ void tma_load_5d(void *dst, const CUtensorMap *map, int c0, int c1, int c2, int c3,
                                            int c4, uint64_t *bar)
{
    asm volatile("cp.async.bulk.tensor.5d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, "
                 "%4, %5, %6}], [%7];" ::"r"(su32(dst)),
                 "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(su32(bar))
                 : "memory");
}

// A row's best p (key, column, bound) in registers, sorted by (key
// descending, column ascending); empty slots hold (-inf, INT32_MAX).
__device__ __forceinline__ void top_clear(float (&k)[TC3_MAXP], int32_t (&j)[TC3_MAXP], float (&d)[TC3_MAXP])
{
#pragma unroll
    for (int t = 0; t < TC3_MAXP; ++t) {
        k[t] = -INFINITY;
        j[t] = INT32_MAX;
        d[t] = 0.0f;
    }
}
// one compare-and-swap pass over the p slots (static indices)
__device__ __forceinline__ void top_insert(float (&k)[TC3_MAXP], int32_t (&j)[TC3_MAXP], float (&d)[TC3_MAXP],
                                           float key, int32_t jj, float dq, int p)
{
#pragma unroll
    for (int t = 0; t < TC3_MAXP; ++t) {
        const bool b = t < p && (key > k[t] || (key == k[t] && jj < j[t]));
        const float tk = k[t], td = d[t];
        const int32_t tj = j[t];
        k[t] = b ? key : tk;
        j[t] = b ? jj : tj;
        d[t] = b ? dq : td;
        key = b ? tk : key;
        jj = b ? tj : jj;
        dq = b ? td : dq;
    }
}
// the p-th kept key (-inf until p are kept)
__device__ __forceinline__ float top_last(const float (&k)[TC3_MAXP], int p)
{
    float v = -INFINITY;
#pragma unroll
    for (int t = 0; t < TC3_MAXP; ++t) v = (t == p - 1) ? k[t] : v;
    return v;
}

// Per 256-column tile: shift s, scale S_b, the column constants in
// accumulator order, and the eight shifted copies of the tile's values as
// FP16 pairs (lags up to 64 nkc). One block per tile.
__global__ void __launch_bounds__(TC_N) k_tc_cols(TcArgs A)
{
    if (*A.nrows <= 0) return;
    extern __shared__ __half vsh[];          // [2][lc + 8]: the tile's values, hi and lo
    __shared__ float red[TC_N / 32];
    const int tid = threadIdx.x;
    const int64_t t = blockIdx.x;
    const int64_t j0 = t * TC_N;
    const int l = A.l;
    const int64_t jm = j0 + TC_N / 2 < A.nl ? j0 + TC_N / 2 : A.nl - 1;
    const double sft = A.mu[jm];
    const int64_t jc = j0 + tid;
    float spread = 0.0f;
    if (jc < A.nl) {
        const double m2 = A.m2[jc];
        spread = (float)(sqrt(m2 > 0.0 ? m2 : 0.0) + fabs(A.mu[jc] - sft));
    }
    for (int o = 16; o > 0; o >>= 1) spread = fmaxf(spread, __shfl_xor_sync(0xffffffffu, spread, o));
    if ((tid & 31) == 0) red[tid >> 5] = spread;
    __syncthreads();
    float mx = 0.0f;
    for (int w = 0; w < TC_N / 32; ++w) mx = fmaxf(mx, red[w]);
    const float Sb = mx > 0.0f ? exp2f(floorf(log2f(255.0f / mx))) : 1.0f;
    {
        ColC cv{0.0f, 0.0f, 0.0f, 0.0f};
        float dqm = 0.0f;
        if (jc < A.nl) {
            const double isd = A.isd[jc];
            const double dm = A.mu[jc] - sft;
            cv.c = (float)(Sb * dm);
            cv.g = (float)(isd / ((double)TC_SA * Sb));
            const double f = sqrt(1.0 + (double)l * dm * dm * isd * isd);
            const double K = (double)A.nkc * TC_KC;
            cv.dq = (float)(1.5 * ((4.0 * 0x1p-22 + (3.0 * K + 4.0) * 0x1p-24) * f + 0x1p-23));
            dqm = cv.dq;
        }
        // accumulator column n' = 32 (tid mod 8) + tid / 8
        reinterpret_cast<ColC *>(A.gcc)[t * TC_N + 32 * (tid & 7) + (tid >> 3)] = cv;
        for (int o = 16; o > 0; o >>= 1) dqm = fmaxf(dqm, __shfl_xor_sync(0xffffffffu, dqm, o));
        if ((tid & 31) == 0 && dqm > 0.0f) atomicMax(reinterpret_cast<int *>(A.dq_max), __float_as_int(dqm));
    }
    // the tile's values V[i] = S_b (x[j0 + i] - s), i < need + 7, as FP16 pairs
    const int need = 248 + TC_KC * A.nkc;    // copy length read at this length
    const int lc = A.lc;
    __half *vh = vsh, *vl = vsh + lc + 8;
    const float s_hi = (float)sft, s_lo = (float)(sft - (double)s_hi);
    for (int i = tid; i < need + 7; i += TC_N) {
        const int64_t gx = j0 + i;
        const float v = gx < A.n ? ((A.xh[gx] - s_hi) + (A.xl[gx] - s_lo)) * Sb : 0.0f;
        __half hi, lo;
        split_half(v, hi, lo);
        vh[i] = hi;
        vl[i] = lo;
    }
    __syncthreads();
    // copy sf of half hl at ((hl * tiles + t) * 8 + sf) * lc
    __half *dst = reinterpret_cast<__half *>(A.bcopy);
    for (int e = tid; e < 16 * need; e += TC_N) {
        const int row = e / need, i = e - row * need;      // row = hl * 8 + sf
        const int hl = row >> 3, sf = row & 7;
        dst[((size_t)(hl * A.tiles_ws + t) * 8 + sf) * lc + i] = (hl ? vl : vh)[i + sf];
    }
}

__global__ void __launch_bounds__(TC3_THREADS, 1) k_direct_tc3(const __grid_constant__ Tc3Params P)
{
    const TcArgs &A = P.a;
    const int nrows = *A.nrows;
    if (nrows <= 0) return;
    const int nkc = A.nkc;
    const int p = A.p;
    const int rtiles = (nrows + TC_M - 1) / TC_M;
    const int64_t items = (int64_t)rtiles * A.nblk;
    if (blockIdx.x >= items) return;

    extern __shared__ __align__(1024) unsigned char sm_raw[];
    unsigned char *sm = reinterpret_cast<unsigned char *>(((uintptr_t)sm_raw + 1023) & ~(uintptr_t)1023);
    // stage g: A hi, A lo (16 KB each), B hi, B lo (32 KB each)
    ColC *cc = reinterpret_cast<ColC *>(sm + 2 * TC3_STAGE);                 // [2][TC_N]
    float *xk = reinterpret_cast<float *>(cc + 2 * TC_N);                    // [TC_M][TC3_MAXP] half 1's lists
    int32_t *xj = reinterpret_cast<int32_t *>(xk + TC_M * TC3_MAXP);
    float *xd = reinterpret_cast<float *>(xj + TC_M * TC3_MAXP);
    __shared__ __align__(8) Tc3Bars bars;
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;
    __shared__ int xcnt[TC_M];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) {
        for (int g = 0; g < 2; ++g) {
            mbar_init(&bars.full[g], 1);               // the loader's expect-tx
            mbar_init(&bars.freeb[g], 1);              // MMA commit
            mbar_init(&bars.accfull[g], 1);            // MMA commit
            mbar_init(&bars.accfree[g], 2 * TC_M);     // epilogue threads
            mbar_init(&bars.ccfull[g], 1);             // the loader's expect-tx
        }
        mbar_init(&bars.fin, 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&P.bmap)) : "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tmem_base)),
                     "r"(2 * TC_N)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;
    volatile int *abortv = &abort_flag;
    auto wait = [&](uint64_t *b, unsigned par) {
        if (*abortv) return false;
        if (mbar_wait_b(b, par, A.err)) return true;
        *abortv = 1;
        return false;
    };

    if (tid == 0) {
        // ------------------------------------------------------- loader
        unsigned t = 0, c = 0;
        int lastc0 = -1, lastc1 = -1, lastt0 = -1, lastt1 = -1;   // last copies issued per buffer
        for (int64_t item = blockIdx.x; item < items; item += gridDim.x) {
            const int rt = (int)(item / A.nblk);
            const int64_t cb0 = (int64_t)(item % A.nblk) * TC_COLS;
            for (int st0 = 0; st0 < TC_COLS / TC_N; ++st0, ++t) {
                const int64_t j0 = cb0 + (int64_t)st0 * TC_N;
                if (j0 >= A.nl) break;
                const int a = t & 1;
                const int tile = (int)(j0 / TC_N);
                if (t >= 2) wait(&bars.accfree[a], ((t >> 1) - 1) & 1);
                if (!*abortv) {
                    mbar_expect_tx(&bars.ccfull[a], TC3_CC_BYTES);
                    bulk_g2s(cc + a * TC_N, reinterpret_cast<const ColC *>(A.gcc) + (size_t)tile * TC_N,
                             TC3_CC_BYTES, &bars.ccfull[a]);
                    if (a) lastt1 = (int)t; else lastt0 = (int)t;
                }
                for (int kc = 0; kc < nkc; ++kc, ++c) {
                    const int g = c & 1;
                    unsigned char *sa = sm + g * TC3_STAGE;
                    unsigned char *sb = sa + 2 * A_TILE_BYTES;
                    if (c >= 2) wait(&bars.freeb[g], ((c >> 1) - 1) & 1);
                    if (*abortv) continue;
                    mbar_expect_tx(&bars.full[g], TC3_STAGE);
                    const unsigned char *src = A.aimg + ((size_t)(rt * nkc + kc) * 2) * A_TILE_BYTES;
                    bulk_g2s(sa, src, A_TILE_BYTES, &bars.full[g]);
                    bulk_g2s(sa + A_TILE_BYTES, src + A_TILE_BYTES, A_TILE_BYTES, &bars.full[g]);
                    tma_load_5d(sb, &P.bmap, kc * TC_KC, 0, 0, tile, 0, &bars.full[g]);
                    tma_load_5d(sb + B_TILE_BYTES, &P.bmap, kc * TC_KC, 0, 0, tile, 1, &bars.full[g]);
                    if (g) lastc1 = (int)c; else lastc0 = (int)c;
                }
            }
        }
        // the copies issued have landed before the block ends
        if (lastc0 >= 0) mbar_wait_b(&bars.full[0], ((unsigned)lastc0 >> 1) & 1, A.err);
        if (lastc1 >= 0) mbar_wait_b(&bars.full[1], ((unsigned)lastc1 >> 1) & 1, A.err);
        if (lastt0 >= 0) mbar_wait_b(&bars.ccfull[0], ((unsigned)lastt0 >> 1) & 1, A.err);
        if (lastt1 >= 0) mbar_wait_b(&bars.ccfull[1], ((unsigned)lastt1 >> 1) & 1, A.err);
    } else if (tid == 32) {
        // ----------------------------------------------------------- MMA
        unsigned t = 0, c = 0;
        for (int64_t item = blockIdx.x; item < items; item += gridDim.x) {
            const int64_t cb0 = (int64_t)(item % A.nblk) * TC_COLS;
            for (int st0 = 0; st0 < TC_COLS / TC_N; ++st0, ++t) {
                if (cb0 + (int64_t)st0 * TC_N >= A.nl) break;
                const int a = t & 1;
                if (t >= 2) wait(&bars.accfree[a], ((t >> 1) - 1) & 1);
                tc_fence_after();
                const uint32_t dacc = tmem + (uint32_t)(a * TC_N);
                for (int kc = 0; kc < nkc; ++kc, ++c) {
                    const int g = c & 1;
                    wait(&bars.full[g], (c >> 1) & 1);
                    tc_fence_after();
                    if (!*abortv) {
                        const unsigned a0 = su32(sm + g * TC3_STAGE), b0 = a0 + 2 * A_TILE_BYTES;
#pragma unroll
                        for (int ks = 0; ks < TC_KC / 16; ++ks) {
                            const uint64_t ah = sdesc(a0 + ks * 32), al = sdesc(a0 + A_TILE_BYTES + ks * 32);
                            const uint64_t bh = sdesc(b0 + ks * 32), bl = sdesc(b0 + B_TILE_BYTES + ks * 32);
                            tc_mma(dacc, ah, bh, (kc > 0 || ks > 0) ? 1u : 0u);
                            tc_mma(dacc, ah, bl, 1u);
                            tc_mma(dacc, al, bh, 1u);
                        }
                    }
                    tc_commit(&bars.freeb[g]);                 // the stage may be refilled
                    if (kc == nkc - 1) tc_commit(&bars.accfull[a]);   // the tile's accumulator is complete
                }
            }
        }
        // every MMA issued has completed before the accumulators are freed
        tc_commit(&bars.fin);
        mbar_wait_b(&bars.fin, 0, A.err);
    } else if (tid >= TC3_EPI0) {
        // ------------------------------------------------------ epilogue
        const int q = warp & 3;                     // TMEM lane quarter of this warp
        const int h = (warp - 2) >> 2;              // column half of each tile
        const int m = 32 * q + lane;                // row of the tile (TMEM lane)
        unsigned t = 0;
        float Lk[TC3_MAXP], Ld[TC3_MAXP];
        int32_t Lj[TC3_MAXP];
        for (int64_t item = blockIdx.x; item < items; item += gridDim.x) {
            const int rt = (int)(item / A.nblk);
            const int cb = (int)(item % A.nblk);
            const int64_t cb0 = (int64_t)cb * TC_COLS;
            const int64_t pos = (int64_t)rt * TC_M + m;
            const bool erow = pos < nrows;
            const int64_t r = erow ? A.rows[pos] : -1;
            const float asum = erow ? A.asum[pos] : 0.0f;
            const float sq = erow ? A.sqm2[pos] : 0.0f;
            const float thq = erow ? (float)A.thr[r] / sq : 0.0f;
            const int64_t exlo = r - A.E, exhi = r + A.E;
            top_clear(Lk, Lj, Ld);
            int cnt = 0;
            float kmin = -INFINITY;   // the p-th kept key once p are kept
            for (int st0 = 0; st0 < TC_COLS / TC_N; ++st0, ++t) {
                const int64_t j0 = cb0 + (int64_t)st0 * TC_N;
                if (j0 >= A.nl) break;
                const int a = t & 1;
                wait(&bars.accfull[a], (t >> 1) & 1);
                wait(&bars.ccfull[a], (t >> 1) & 1);
                tc_fence_after();
                const ColC *ca = cc + a * TC_N;
#pragma unroll 1
                for (int c0 = h * (TC_N / 2); c0 < (h + 1) * (TC_N / 2); c0 += 32) {
                    const int sf = c0 >> 5;             // accumulator columns 32 sf + r: series column j0 + 8 r + sf
                    float v[32];
                    __syncwarp();
                    tc_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(a * TC_N + c0), v);
                    if (!erow || *abortv) continue;
                    // the 32 columns' tests first (independent, no branches),
                    // then the rare candidates
                    unsigned hits = 0;
#pragma unroll
                    for (int rr = 0; rr < 32; ++rr) {
                        const ColC k = ca[c0 + rr];
                        const float tt = fmaf(-k.c, asum, v[rr]);
                        hits |= (unsigned)(fmaf(tt, k.g, k.dq) > thq && tt * k.g * sq >= kmin) << rr;
                    }
                    if (hits) {
#pragma unroll
                        for (int rr = 0; rr < 32; ++rr) {
                            if (!((hits >> rr) & 1u)) continue;
                            const ColC k = ca[c0 + rr];
                            const float key = fmaf(-k.c, asum, v[rr]) * k.g * sq;
                            const int64_t j = j0 + 8 * rr + sf;
                            if (key >= kmin && j < A.nl && (j < exlo || j > exhi)) {
                                top_insert(Lk, Lj, Ld, key, (int32_t)j, k.dq, p);
                                cnt = cnt < p ? cnt + 1 : p;
                                kmin = top_last(Lk, p);
                            }
                        }
                    }
                }
                tc_fence_before();
                mbar_arrive1(&bars.accfree[a]);   // accumulator and column constants released
            }
            // the halves' lists merged: half 1 hands its list over
            if (h == 1) {
#pragma unroll
                for (int e = 0; e < TC3_MAXP; ++e) {
                    xk[m * TC3_MAXP + e] = Lk[e];
                    xj[m * TC3_MAXP + e] = Lj[e];
                    xd[m * TC3_MAXP + e] = Ld[e];
                }
                xcnt[m] = cnt;
            }
            asm volatile("bar.sync 2, 256;" ::: "memory");
            if (h == 0 && erow && !*abortv) {
                const int nb = xcnt[m];
                for (int e = 0; e < nb; ++e) {
                    top_insert(Lk, Lj, Ld, xk[m * TC3_MAXP + e], xj[m * TC3_MAXP + e], xd[m * TC3_MAXP + e], p);
                    cnt = cnt < p ? cnt + 1 : p;
                }
                const int64_t slot = pos * A.nblk + cb;
#pragma unroll
                for (int e = 0; e < TC3_MAXP; ++e) {
                    if (e < cnt) {
                        A.okey[slot * p + e] = Lk[e];
                        A.oj[slot * p + e] = Lj[e];
                        A.odq[slot * p + e] = Ld[e];
                    }
                }
                A.ocnt[slot] = cnt;
            }
            asm volatile("bar.sync 2, 256;" ::: "memory");
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * TC_N) : "memory");
    }
}
}  // namespace

size_t tc_smem_bytes(int p)
{
    const int H = p <= 32 ? 2 : 1;
    return 1024 + 2 * (size_t)A_TILE_BYTES + 2 * (size_t)B_TILE_BYTES + 2 * 8 * SHIFT_LEN * sizeof(__half) +
           TC_N * sizeof(ColC) + (size_t)H * TC_M * p * (sizeof(float) + sizeof(int32_t) + sizeof(float));
}

size_t tc_aimg_bytes(int64_t max_rows, int lmax)
{
    const int64_t tiles = (max_rows + TC_M - 1) / TC_M;
    const int64_t nkc = (lmax + TC_KC - 1) / TC_KC;
    return (size_t)tiles * nkc * 2 * A_TILE_BYTES;
}

int tc_chunks(int l) { return (l + TC_KC - 1) / TC_KC; }

size_t tc2_smem_bytes(int p)
{
    return 1024 + 2 * (size_t)TC2_STAGE + 2 * 8 * SHIFT_LEN * sizeof(__half) + 2 * TC_N * sizeof(ColC) +
           (size_t)TC_M * p * (sizeof(float) + sizeof(int32_t) + sizeof(float));
}

int tc_copy_len(int lmax) { return 248 + TC_KC * tc_chunks(lmax); }

// (+1 KB: the descriptor's last rows reach 494 bytes past the last copy
// for lags the kernel never asks for)
size_t tc_bcopy_bytes(int64_t ntiles, int lmax)
{
    return (size_t)2 * ntiles * 8 * tc_copy_len(lmax) * sizeof(__half) + 1024;
}

size_t tc_gcc_bytes(int64_t ntiles) { return (size_t)ntiles * TC_N * sizeof(ColC); }

int64_t tc_col_tiles(int64_t nl) { return (nl + TC_N - 1) / TC_N; }

size_t tc3_smem_bytes() { return 1024 + 2 * (size_t)TC3_STAGE + 2 * TC3_CC_BYTES + (size_t)TC_M * TC3_MAXP * 12; }

bool tc_encode_bmap(void *map, void *gaddr, int64_t ntiles, int lc)
{
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    });
    if (!encode || !map || !gaddr || ntiles <= 0 || lc % 8 != 0) return false;
    // dims {lag i, row r (16 B apart: rows overlap, the Hankel form), copy sf, tile, hi|lo}
    const cuuint64_t dims[5] = {(cuuint64_t)lc, 32, 8, (cuuint64_t)ntiles, 2};
    const cuuint64_t strides[4] = {16, (cuuint64_t)lc * 2, (cuuint64_t)lc * 16, (cuuint64_t)lc * 16 * ntiles};
    const cuuint32_t box[5] = {TC_KC, 32, 8, 1, 1};
    const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
    const CUresult r = encode(reinterpret_cast<CUtensorMap *>(map), CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 5, gaddr, dims,
                              strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

void launch_direct_tc(const TcArgs &a, int num_sms, cudaStream_t s)
{
    k_tc_rows<<<num_sms * 8, TC_THREADS, 0, s>>>(a);
    if (a.bmap && a.p <= TC3_MAXP && a.ntiles > 0) {
        k_tc_cols<<<(unsigned)a.ntiles, TC_N, (size_t)2 * (a.lc + 8) * sizeof(__half), s>>>(a);
        Tc3Params P;
        P.a = a;
        memcpy(&P.bmap, a.bmap, sizeof(CUtensorMap));
        static std::once_flag once3[64];
        smem_optin_max((const void *)k_direct_tc3, once3);
        k_direct_tc3<<<num_sms, TC3_THREADS, tc3_smem_bytes(), s>>>(P);
        return;
    }
    if (a.p <= TC2_MAXP) {
        static std::once_flag once2[64];
        smem_optin_max((const void *)k_direct_tc2, once2);
        k_direct_tc2<<<num_sms, TC2_THREADS, tc2_smem_bytes(a.p), s>>>(a);
    } else {
        static std::once_flag once[64];
        smem_optin_max((const void *)k_direct_tc, once);
        k_direct_tc<<<num_sms, TC_THREADS, tc_smem_bytes(a.p), s>>>(a);
    }
}

}  // namespace mad
