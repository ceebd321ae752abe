// k_readout.cu -- discord table per length (Sec. 6: dkm_l and its merge into
// dkm_{lmin,lmax}, Algorithms 8 and 9), top-k motif pairs from VALMP
// (Sec. 3 length normalisation, Algorithm 5's best pairs), and FP64 re-checks
// of the reported distances.
#include "kernels.cuh"

namespace mad {

__device__ __forceinline__ double ninf() { return -__longlong_as_double(0x7ff0000000000000LL); }
__device__ __forceinline__ double dinf() { return __longlong_as_double(0x7ff0000000000000LL); }

// (v, i) ordering for discords: larger v first, then smaller i.
__device__ __forceinline__ bool better_desc(double v, int32_t i, double w, int32_t j)
{
    return v > w || (v == w && i >= 0 && (j < 0 || i < j));
}
// (v, i) ordering for motifs: smaller v first, then smaller i.
__device__ __forceinline__ bool better_asc(double v, int32_t i, double w, int32_t j)
{
    return v < w || (v == w && i >= 0 && (j < 0 || i < j));
}

template <bool DESC>
__device__ void block_best(double &v, int32_t &i)
{
    __shared__ double sv[32];
    __shared__ int32_t si[32];
    for (int o = 16; o > 0; o >>= 1) {
        const double w = __shfl_xor_sync(0xffffffffu, v, o);
        const int32_t j = __shfl_xor_sync(0xffffffffu, i, o);
        if (DESC ? better_desc(w, j, v, i) : better_asc(w, j, v, i)) { v = w; i = j; }
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    __syncthreads();
    if (lane == 0) { sv[wid] = v; si[wid] = i; }
    __syncthreads();
    if (wid == 0) {
        v = lane < nw ? sv[lane] : (DESC ? ninf() : dinf());
        i = lane < nw ? si[lane] : -1;
        for (int o = 16; o > 0; o >>= 1) {
            const double w = __shfl_xor_sync(0xffffffffu, v, o);
            const int32_t j = __shfl_xor_sync(0xffffffffu, i, o);
            if (DESC ? better_desc(w, j, v, i) : better_asc(w, j, v, i)) { v = w; i = j; }
        }
        if (lane == 0) { sv[0] = v; si[0] = i; }
    }
    __syncthreads();
    v = sv[0];
    i = si[0];
    __syncthreads();
}

// ------------------------------------------------------------- discords

constexpr int DBLK = 256;
static_assert(GDISC_TILE == DBLK, "host tile count must match the kernels' tile");

// Per block of DBLK offsets and column m: the best (score desc, offset asc)
// m-th best-match distance. Offsets without an m-th best match are skipped.
__global__ void k_disc_blockmax(const double *nnd, int64_t n0, int64_t nl, int nblk, double *bval, int32_t *bidx)
{
    const int m = blockIdx.y, b = blockIdx.x;
    const int64_t i = (int64_t)b * DBLK + threadIdx.x;
    double v = ninf();
    int32_t ix = -1;
    if (i < nl) {
        const double s = nnd[m * n0 + i];
        if (isfinite(s)) { v = s; ix = (int32_t)i; }
    }
    block_best<true>(v, ix);
    if (threadIdx.x == 0) {
        bval[m * nblk + b] = v;
        bidx[m * nblk + b] = ix;
    }
}

// Column m of dkm_l by greedy selection: repeatedly take the best remaining
// offset and exclude every offset within E(l) of it (the picks of a length
// must not be trivial matches of one another); then merge rank by rank into
// dkm_{lmin,lmax}, keeping the largest dist / sqrt(l) and letting a later
// (longer) length win ties (Algorithm 9's ">=").
__global__ void k_disc_greedy(const double *nnd, const int32_t *nnj, int64_t n0, int64_t nl, int l, int64_t E,
                              int k_max, int m_max, const double *bval, const int32_t *bidx, int nblk, DiscTable tab)
{
    extern __shared__ unsigned char sm_raw[];
    double *bv = reinterpret_cast<double *>(sm_raw);
    int32_t *bi = reinterpret_cast<int32_t *>(bv + nblk);
    __shared__ int32_t picks[KMAX];
    const int m = blockIdx.x;
    const double *score = nnd + (int64_t)m * n0;
    for (int t = threadIdx.x; t < nblk; t += blockDim.x) {
        bv[t] = bval[m * nblk + t];
        bi[t] = bidx[m * nblk + t];
    }
    __syncthreads();
    const double f = sqrt((double)l);
    for (int r = 0; r < k_max; ++r) {
        double v = ninf();
        int32_t g = -1;
        for (int t = threadIdx.x; t < nblk; t += blockDim.x)
            if (better_desc(bv[t], bi[t], v, g)) { v = bv[t]; g = bi[t]; }
        block_best<true>(v, g);
        if (g < 0) break;
        if (threadIdx.x == 0) {
            picks[r] = g;
            const int cell = r * m_max + m;
            const double d = score[g];
            const double nd = d / f;
            if (tab.len[cell] == 0 || nd >= tab.norm[cell]) {
                tab.norm[cell] = nd;
                tab.dist[cell] = d;
                tab.off[cell] = g;
                tab.len[cell] = l;
                tab.nn[cell] = nnj[(int64_t)m * n0 + g];
            }
        }
        __syncthreads();
        // refresh the blocks that meet [g - E, g + E]
        const int64_t lo = g - E < 0 ? 0 : g - E;
        const int64_t hi = g + E >= nl ? nl - 1 : g + E;
        for (int64_t blk = lo / DBLK; blk <= hi / DBLK; ++blk) {
            double w = ninf();
            int32_t wi = -1;
            if (threadIdx.x < DBLK) {
                const int64_t e = blk * DBLK + threadIdx.x;
                if (e < nl) {
                    bool free = true;
                    for (int q = 0; q <= r; ++q) {
                        const int64_t d = e - picks[q];
                        free &= (d > E || -d > E);
                    }
                    const double s = score[e];
                    if (free && isfinite(s)) { w = s; wi = (int32_t)e; }
                }
            }
            block_best<true>(w, wi);
            if (threadIdx.x == 0) { bv[blk] = w; bi[blk] = wi; }
            __syncthreads();
        }
    }
}

void launch_discords_length(const double *nnd, const int32_t *nnj, int64_t n0, int64_t nl, int l, int64_t E,
                            int k_max, int m_max, double *bval, int32_t *bidx, DiscTable tab, cudaStream_t s)
{
    const int nblk = (int)((nl + DBLK - 1) / DBLK);
    k_disc_blockmax<<<dim3(nblk, m_max), DBLK, 0, s>>>(nnd, n0, nl, nblk, bval, bidx);
    const size_t sm = (size_t)nblk * (sizeof(double) + sizeof(int32_t));
    static std::once_flag once[64];
    smem_optin_max((const void *)k_disc_greedy, once);
    k_disc_greedy<<<m_max, 1024, sm, s>>>(nnd, nnj, n0, nl, l, E, k_max, m_max, bval, bidx, nblk, tab);
}

// ------------------------------------------------ global-greedy discords

// Variable-length m-th discords ranked over every (offset, length) at once:
// candidates by score NN_l^m[i] / sqrt(l) descending, then longer length, then
// smaller offset, each accepted unless within max(E(l), E(l')) of an accepted
// (i', l'). A candidate's key (nL - 1 - li) * n0 + i orders the ties. The
// kept profiles are cut into tiles of DBLK offsets of one length; a tile's
// best free candidate is kept in (tv, tk), and after each pick only the tiles
// that meet its zone are re-scanned.
__device__ __forceinline__ bool better_key(double v, int64_t a, double w, int64_t b)
{
    return v > w || (v == w && a >= 0 && (b < 0 || a < b));
}

__device__ __forceinline__ void warp_best_key(double &v, int64_t &k)
{
    for (int o = 16; o > 0; o >>= 1) {
        const double w = __shfl_xor_sync(0xffffffffu, v, o);
        const int64_t b = __shfl_xor_sync(0xffffffffu, k, o);
        if (better_key(w, b, v, k)) { v = w; k = b; }
    }
}

// One warp re-scans tile (li, blk) of column c, skipping the np picks' zones.
__device__ void gdisc_tile(const GDiscArgs &A, int c, int li, int blk, const int64_t *po, const int64_t *pe, int np)
{
    const int lane = threadIdx.x & 31;
    const int l = A.lmin + li;
    const int64_t nl = A.n - l + 1;
    const int64_t E = excl_zone(l, A.num, A.den);
    const double f = sqrt((double)l);
    const double *sc = A.nnd + ((int64_t)li * A.m_max + c) * A.n0;
    double v = ninf();
    int64_t key = -1;
    for (int t = lane; t < DBLK; t += 32) {
        const int64_t e = (int64_t)blk * DBLK + t;
        if (e >= nl) break;
        const double d = sc[e];
        if (!isfinite(d)) continue;
        bool ok = true;
        for (int q = 0; q < np && ok; ++q) {
            const int64_t Em = E > pe[q] ? E : pe[q];
            const int64_t dd = e - po[q];
            ok = dd > Em || -dd > Em;
        }
        if (!ok) continue;
        const double s = d / f;
        const int64_t kk = (int64_t)(A.nL - 1 - li) * A.n0 + e;
        if (better_key(s, kk, v, key)) { v = s; key = kk; }
    }
    warp_best_key(v, key);
    if (lane == 0) {
        const int64_t t = (int64_t)c * A.nL * A.nblk + (int64_t)li * A.nblk + blk;
        A.tv[t] = v;
        A.tk[t] = key;
    }
}

__global__ void k_gdisc_tiles(GDiscArgs A)
{
    const int c = blockIdx.y;
    const int64_t t = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (t >= (int64_t)A.nL * A.nblk) return;
    gdisc_tile(A, c, (int)(t / A.nblk), (int)(t % A.nblk), nullptr, nullptr, 0);
}

// One block per column: k rounds of argmax over the tile table, then the
// re-scan of the tiles within max(E(l), E(l_pick)) of the pick, per length.
__global__ void __launch_bounds__(1024) k_gdisc_greedy(GDiscArgs A)
{
    __shared__ int64_t po[KMAX], pe[KMAX];
    __shared__ double rv[32];
    __shared__ int64_t rk[32];
    const int c = blockIdx.x;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int64_t nt = (int64_t)A.nL * A.nblk;
    const double *tv = A.tv + c * nt;
    const int64_t *tk = A.tk + c * nt;
    for (int r = 0; r < A.k; ++r) {
        double v = ninf();
        int64_t key = -1;
        for (int64_t t = threadIdx.x; t < nt; t += blockDim.x)
            if (better_key(tv[t], tk[t], v, key)) { v = tv[t]; key = tk[t]; }
        warp_best_key(v, key);
        if (lane == 0) { rv[wid] = v; rk[wid] = key; }
        __syncthreads();
        if (wid == 0) {
            v = lane < nw ? rv[lane] : ninf();
            key = lane < nw ? rk[lane] : -1;
            warp_best_key(v, key);
            if (lane == 0) { rv[0] = v; rk[0] = key; }
        }
        __syncthreads();
        v = rv[0];
        key = rk[0];
        if (key < 0) break;
        const int li = A.nL - 1 - (int)(key / A.n0);
        const int64_t i = key % A.n0;
        const int l = A.lmin + li;
        if (threadIdx.x == 0) {
            po[r] = i;
            pe[r] = excl_zone(l, A.num, A.den);
            const int cell = r * A.mcols + c;
            const int64_t at = ((int64_t)li * A.m_max + c) * A.n0 + i;
            A.out.norm[cell] = v;
            A.out.dist[cell] = A.nnd[at];
            A.out.off[cell] = (int32_t)i;
            A.out.len[cell] = l;
            A.out.nn[cell] = A.nnj[at];
        }
        __syncthreads();
        for (int l2i = wid; l2i < A.nL; l2i += nw) {
            const int l2 = A.lmin + l2i;
            const int64_t nl2 = A.n - l2 + 1;
            const int64_t E2 = excl_zone(l2, A.num, A.den), Em = E2 > pe[r] ? E2 : pe[r];
            const int64_t lo = i - Em < 0 ? 0 : i - Em;
            const int64_t hi = i + Em >= nl2 ? nl2 - 1 : i + Em;
            for (int64_t blk = lo / DBLK; lo <= hi && blk <= hi / DBLK; ++blk)
                gdisc_tile(A, c, l2i, (int)blk, po, pe, r + 1);
        }
        __syncthreads();
    }
}

void launch_discords_global(const GDiscArgs &a, cudaStream_t s)
{
    const int64_t nt = (int64_t)a.nL * a.nblk;
    k_gdisc_tiles<<<dim3((unsigned)((nt + 7) / 8), a.mcols), 256, 0, s>>>(a);
    k_gdisc_greedy<<<a.mcols, 1024, 0, s>>>(a);
}

// ------------------------------------------------------ streamed dkm_l

// dkm_l as Algorithms 7 and 8 print it, one warp per length: windows in
// offset order; one with a trivial match among the offsets present anywhere
// in the matrix is skipped; else columns m..1 are tried and the window
// enters the first column where it beats an entry, at the first rank it
// beats, the rest of the column moving down one rank. A column's last entry
// (its minimum, -inf while not full) only grows, so a batch of 32 windows is
// screened against it first and only the windows above some column's minimum
// run the exact steps, one at a time in offset order.
constexpr int STREAM_WARPS = 4;

// One warp: has window ii a trivial match among the offsets present in the
// k x m matrix (cells entries of O)?
__device__ __forceinline__ bool dkm_trivial_warp(const int32_t *O, int cells, int64_t ii, int64_t E, int lane)
{
    bool triv = false;
    for (int c = lane; c < cells; c += 32) {
        const int64_t o = O[c];
        triv |= o >= 0 && ii - o <= E && o - ii <= E;
    }
    return __any_sync(0xffffffffu, triv);
}

// One warp: Algorithm 8 for window ii, whose c-th best-match distance and
// neighbour are v[c * vs] and vj[c * vs]; cmin[c] mirrors the last entry of
// column c. Every lane takes the same path. Returns the column entered (-1:
// none) and in *dropped the offset that left it (-1: none).
__device__ int dkm_insert_warp(double *D, int32_t *O, int32_t *N, double *cmin, int k, int m, int64_t ii,
                               const double *v, const int32_t *vj, int64_t vs, int lane, int32_t *dropped)
{
    *dropped = -1;
    for (int j = m - 1; j >= 0; --j) {
        const double vv = v[(int64_t)j * vs];
        if (!isfinite(vv) || !(vv > cmin[j])) continue;
        // first rank r0 with vv > D[r0][j] (exists: vv beats the last entry)
        const unsigned lo = __ballot_sync(0xffffffffu, lane < k && vv > D[lane * m + j]);
        const unsigned hi = __ballot_sync(0xffffffffu, lane + 32 < k && vv > D[(lane + 32) * m + j]);
        if (!lo && !hi) return -1;   // cannot happen while cmin[j] mirrors the last entry
        const int r0 = lo ? __ffs(lo) - 1 : 32 + __ffs(hi) - 1;
        *dropped = O[(k - 1) * m + j];
        double sd[2];
        int32_t so[2], sn[2];
        for (int h = 0; h < 2; ++h) {
            const int rr = lane + 32 * h;
            if (rr >= r0 && rr < k - 1) {
                sd[h] = D[rr * m + j];
                so[h] = O[rr * m + j];
                sn[h] = N[rr * m + j];
            }
        }
        __syncwarp();
        for (int h = 0; h < 2; ++h) {
            const int rr = lane + 32 * h;
            if (rr >= r0 && rr < k - 1) {
                D[(rr + 1) * m + j] = sd[h];
                O[(rr + 1) * m + j] = so[h];
                N[(rr + 1) * m + j] = sn[h];
            }
        }
        __syncwarp();
        if (lane == 0) {
            D[r0 * m + j] = vv;
            O[r0 * m + j] = (int32_t)ii;
            N[r0 * m + j] = vj[(int64_t)j * vs];
        }
        __syncwarp();
        if (lane == 0) cmin[j] = D[(k - 1) * m + j];
        __syncwarp();
        return j;
    }
    return -1;
}

__global__ void __launch_bounds__(STREAM_WARPS * 32) k_dkm_streamed(StreamArgs A)
{
    __shared__ double cmin_all[STREAM_WARPS][KMAX];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int li = blockIdx.x * STREAM_WARPS + wid;
    if (li >= A.nL) return;
    double *cmin = cmin_all[wid];
    const int l = A.lmin + li, k = A.k, m = A.m;
    const int64_t nl = A.n - l + 1;
    const int64_t E = excl_zone(l, A.num, A.den);
    const int cells = k * m;
    double *D = A.d + (int64_t)li * cells;
    int32_t *O = A.o + (int64_t)li * cells;
    int32_t *N = A.nn + (int64_t)li * cells;
    const double *sc = A.nnd + (int64_t)li * A.m_max * A.n0;      // column c at sc + c * n0
    const int32_t *sj = A.nnj + (int64_t)li * A.m_max * A.n0;
    for (int c = lane; c < cells; c += 32) {
        D[c] = ninf();
        O[c] = -1;
        N[c] = -1;
    }
    for (int c = lane; c < m; c += 32) cmin[c] = ninf();
    __syncwarp();
    for (int64_t base = 0; base < nl; base += 32) {
        const int64_t i = base + lane;
        bool cand = false;
        if (i < nl)
            for (int c = 0; c < m && !cand; ++c) {
                const double v = sc[(int64_t)c * A.n0 + i];
                cand = isfinite(v) && v > cmin[c];
            }
        unsigned mask = __ballot_sync(0xffffffffu, cand);
        while (mask) {
            const int t = __ffs(mask) - 1;
            mask &= mask - 1;
            const int64_t ii = base + t;
            if (dkm_trivial_warp(O, cells, ii, E, lane)) continue;
            int32_t dropped;
            dkm_insert_warp(D, O, N, cmin, k, m, ii, sc + ii, sj + ii, A.n0, lane, &dropped);
        }
    }
}

// ------------------------------------- discord mode (Algorithms 7 and 10)
//
// Only the windows that change dkm_l need to be visited one at a time: a
// window enters by Algorithm 8 only if one of its distances beats its
// column's last entry, and non-valid rows never change dkm_l in the first
// pass. So each pass is
//  - a sequential kernel (one block): chunks of DP_CHUNK windows are
//    screened in parallel against the column minima as they stand, the
//    windows that might enter are compacted in order, and warp 0 takes them
//    one by one (trivial-match test, Algorithm 8), logging every entry and
//    every exit: ins[o] = l for a window that entered at this length,
//    drop[o] = the window whose entry pushed it out (INT32_MAX: never);
//  - a parallel kernel that decides every other window from the log: the
//    offsets present when window i is visited are those that entered before
//    i (so within [i - E, i - 1] for a trivial match) and left after it.
// First pass: valid rows (exact 1st..m-th distances; every row at lmin) in
// offset order; non-valid rows without a trivial match are listed. Only the
// listed rows whose upper values still beat a column's last entry after the
// first pass can be recomputed by the second pass (the last entries only
// grow): they are kept (ROW_RECOMPUTE / ROW_FLAT), the rest are left
// undefined (ROW_SKIP, NaN distances). Second pass over the kept rows in
// offset order: a row enters with its exact distances only if one beats its
// column's last entry (its upper value then does too); the rows it would
// have recomputed are those without a trivial match whose upper value beats
// the last entry as it stood at their visit (kept in the log of the column
// minima); the other kept rows take back their row state.
constexpr int DP_THREADS = 1024;
constexpr int DP_RPT = 4;                       // consecutive windows per thread
constexpr int DP_CHUNK = DP_THREADS * DP_RPT;
constexpr int DP_STAGE = 2;                     // columns staged in shared memory (m <= DP_STAGE)

// Ordered compaction within the block: thread t contributes c (its flagged
// windows, in order); returns its first output position; *total = sum.
__device__ int block_excl_scan(int c, int *wsum, int *total)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int x = c;
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    if (w == 0) {
        const int v = wsum[lane];
        int z = v;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, z, o);
            if (lane >= o) z += y;
        }
        wsum[lane] = z - v;                 // exclusive offsets of the warps
        if (lane == 31) wsum[32] = z;
    }
    __syncthreads();
    const int pos = wsum[w] + x - c;
    *total = wsum[32];
    __syncthreads();
    return pos;
}

struct DpSmem {
    double *D, *cmin;
    int32_t *O, *N, *cand;
    double *cv;             // the candidates' distances [DP_CHUNK][DP_STAGE]
    int *wsum;
};

__device__ DpSmem dp_smem(unsigned char *raw, int cells, int m)
{
    DpSmem s;
    s.D = reinterpret_cast<double *>(raw);
    s.cmin = s.D + cells;
    s.O = reinterpret_cast<int32_t *>(s.cmin + m);
    s.N = s.O + cells;
    s.cand = s.N + cells;
    s.cv = reinterpret_cast<double *>(s.cand + DP_CHUNK);
    s.wsum = reinterpret_cast<int *>(s.cv + DP_CHUNK * DP_STAGE);
    return s;
}

size_t dp_smem_bytes(int k, int m)
{
    const size_t cells = (size_t)k * m;
    return cells * sizeof(double) + m * sizeof(double) + 2 * cells * sizeof(int32_t) + DP_CHUNK * sizeof(int32_t) +
           (size_t)DP_CHUNK * DP_STAGE * sizeof(double) + 33 * sizeof(int);
}

// pass = 1: first pass (screen: valid rows); pass = 2: second pass (screen:
// kept rows, exact distances). Entries / exits are logged in ins/drop of the
// pass; the second pass also logs the column minima after each entry.
template <int PASS>
__global__ void __launch_bounds__(DP_THREADS) k_dp_seq(DiscPassArgs A)
{
    extern __shared__ __align__(16) unsigned char dp_raw[];
    const int k = A.k, m = A.m, cells = k * m;
    DpSmem sm = dp_smem(dp_raw, cells, m);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int32_t *ins = PASS == 1 ? A.ins1 : A.ins2;
    int32_t *drop = PASS == 1 ? A.drop1 : A.drop2;
    if (PASS == 1) {
        for (int c = threadIdx.x; c < cells; c += DP_THREADS) {
            sm.D[c] = ninf();
            sm.O[c] = -1;
            sm.N[c] = -1;
        }
    } else {
        for (int c = threadIdx.x; c < cells; c += DP_THREADS) {
            sm.D[c] = A.D[c];
            sm.O[c] = A.O[c];
            sm.N[c] = A.N[c];
            if (sm.O[c] >= 0) drop[sm.O[c]] = INT32_MAX;   // present at the start of the pass
        }
    }
    __syncthreads();
    for (int c = threadIdx.x; c < m; c += DP_THREADS) sm.cmin[c] = sm.D[(k - 1) * m + c];
    int nev = 0;
    __syncthreads();
    for (int64_t base = 0; base < A.nl; base += DP_CHUNK) {
        // screen this thread's windows against the column minima as they
        // stand (every load issued before the tests)
        const int64_t i0 = base + (int64_t)threadIdx.x * DP_RPT;
        const bool stage = m <= DP_STAGE;
        bool okr[DP_RPT];
#pragma unroll
        for (int r = 0; r < DP_RPT; ++r) {
            const int64_t i = i0 + r;
            okr[r] = i < A.nl && (PASS == 1 ? (A.all_valid || A.flag[i] == ROW_DONE) : A.kept[i] != 0);
        }
        double vr[DP_RPT][DP_STAGE];
        unsigned flags = 0;
#pragma unroll
        for (int r = 0; r < DP_RPT; ++r) {
            bool cand = false;
            if (okr[r]) {
                if (stage) {
#pragma unroll
                    for (int c = 0; c < DP_STAGE; ++c) vr[r][c] = c < m ? A.nnd[(int64_t)c * A.n0 + i0 + r] : ninf();
#pragma unroll
                    for (int c = 0; c < DP_STAGE; ++c) cand |= c < m && isfinite(vr[r][c]) && vr[r][c] > sm.cmin[c];
                } else {
                    for (int c = 0; c < m && !cand; ++c) {
                        const double v = A.nnd[(int64_t)c * A.n0 + i0 + r];
                        cand = isfinite(v) && v > sm.cmin[c];
                    }
                }
            }
            if (cand) flags |= 1u << r;
        }
        int total;
        int pos = block_excl_scan(__popc(flags), sm.wsum, &total);
#pragma unroll
        for (int r = 0; r < DP_RPT; ++r)
            if ((flags >> r) & 1u) {
                sm.cand[pos] = (int32_t)(i0 + r);
                if (stage)
#pragma unroll
                    for (int c = 0; c < DP_STAGE; ++c) sm.cv[pos * DP_STAGE + c] = vr[r][c];
                ++pos;
            }
        __syncthreads();
        if (w == 0) {
            // 32 candidates at a time: every lane re-tests its own against
            // the minima as they stand, and the first that still beats one
            // is taken (those before it cannot change dkm_l)
            for (int t0 = 0; t0 < total; t0 += 32) {
                const int64_t ci = t0 + lane < total ? sm.cand[t0 + lane] : -1;
                int after = -1;
                // (with a small matrix each lane also tests its own window for
                // a trivial match, so a round takes the first window that enters)
                const bool own_triv = cells <= 64;
                while (true) {
                    bool beat = false;
                    if (ci >= 0 && lane > after)
                        for (int c = 0; c < m && !beat; ++c) {
                            const double v = stage ? sm.cv[(t0 + lane) * DP_STAGE + c] : A.nnd[(int64_t)c * A.n0 + ci];
                            beat = isfinite(v) && v > sm.cmin[c];
                        }
                    if (beat && own_triv)
                        for (int c = 0; c < cells && beat; ++c) {
                            const int64_t o = sm.O[c];
                            beat = !(o >= 0 && ci - o <= A.E && o - ci <= A.E);
                        }
                    const unsigned bm = __ballot_sync(0xffffffffu, beat);
                    if (!bm) break;
                    after = __ffs(bm) - 1;
                    const int64_t ii = __shfl_sync(0xffffffffu, ci, after);
                    if (!own_triv && dkm_trivial_warp(sm.O, cells, ii, A.E, lane)) continue;
                    int32_t dropped;
                    const int j = dkm_insert_warp(sm.D, sm.O, sm.N, sm.cmin, k, m, ii, A.nnd + ii, A.nnj + ii, A.n0,
                                                  lane, &dropped);
                    if (j >= 0 && lane == 0) {
                        ins[ii] = A.l;
                        drop[ii] = INT32_MAX;
                        if (dropped >= 0) drop[dropped] = (int32_t)ii;
                        if (PASS == 2) {
                            A.ev_t[nev] = (int32_t)ii;
                            A.ev_j[nev] = j;
                            A.ev_v[nev] = sm.cmin[j];
                        }
                    }
                    if (j >= 0) ++nev;
                    __syncwarp();
                }
            }
        }
        __syncthreads();
    }
    for (int c = threadIdx.x; c < cells; c += DP_THREADS) {
        A.D[c] = sm.D[c];
        A.O[c] = sm.O[c];
        A.N[c] = sm.N[c];
        if (PASS == 1) A.O1[c] = sm.O[c];
    }
    if (PASS == 1)
        for (int c = threadIdx.x; c < m; c += DP_THREADS) A.cmin1[c] = sm.cmin[c];
    if (PASS == 2) {
        if (threadIdx.x == 0) *A.nev = nev;
        // Algorithm 9: fold dkm_l into dkm_{lmin,lmax}
        const double f = sqrt((double)A.l);
        for (int c = threadIdx.x; c < cells; c += DP_THREADS) {
            if (sm.O[c] < 0) continue;
            const double v = sm.D[c] / f;
            if (A.tab.len[c] == 0 || v >= A.tab.norm[c]) {
                A.tab.norm[c] = v;
                A.tab.dist[c] = sm.D[c];
                A.tab.off[c] = sm.O[c];
                A.tab.len[c] = A.l;
                A.tab.nn[c] = sm.N[c];
            }
        }
    }
}

// First-pass decisions of the non-valid rows: listed unless an offset that
// entered before it and had not left is within E; kept if listed and an
// upper value beats its column's last entry after the first pass.
__global__ void k_dp1_list(DiscPassArgs A)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    bool skip = false;
    if (i < A.nl) {
        const int32_t fl = A.flag[i];
        if (fl == ROW_RECOMPUTE || fl == ROW_FLAT) {
            bool blocked = false;
            for (int64_t o = i - A.E < 0 ? 0 : i - A.E; o < i && !blocked; ++o)
                blocked = A.ins1[o] == A.l && A.drop1[o] > i;
            bool keep = false;
            if (!blocked)
                for (int c = 0; c < A.m && !keep; ++c) keep = A.nnd[(int64_t)c * A.n0 + i] > A.cmin1[c];
            if (keep) {
                A.kept[i] = 1;
                for (int c = 0; c < A.m; ++c) A.lub[(int64_t)c * A.n0 + i] = A.nnd[(int64_t)c * A.n0 + i];
            } else {
                skip = true;
                A.flag[i] = ROW_SKIP;
                if (A.thr32) A.thr32[i] = __int_as_float(0x7f800000);
                else A.thr64[i] = dinf();
                for (int c = 0; c < A.m; ++c) {
                    A.nnd[(int64_t)c * A.n0 + i] = __longlong_as_double(0x7ff8000000000000LL);
                    A.nnj[(int64_t)c * A.n0 + i] = -1;
                }
            }
        }
    }
    const int c = __syncthreads_count(skip);
    if (threadIdx.x == 0 && c) atomicAdd(&A.stats[10], (unsigned long long)c);
}

// Second-pass decisions of the kept rows: recomputed by the second pass iff
// no offset present at its visit is within E (the first pass's entries that
// had not left, and the second pass's earlier entries that had not) and an
// upper value beats the column's last entry at its visit. The others take
// back their row state from before the recomputes.
__global__ void k_dp2_used(DiscPassArgs A)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= A.nl || !A.kept[i]) return;
    A.kept[i] = 0;
    bool blocked = false;
    for (int c = 0; c < A.k * A.m && !blocked; ++c) {
        const int64_t o = A.O1[c];
        blocked = o >= 0 && i - o <= A.E && o - i <= A.E && A.drop2[o] > i;
    }
    for (int64_t o = i - A.E < 0 ? 0 : i - A.E; o < i && !blocked; ++o)
        blocked = A.ins2[o] == A.l && A.drop2[o] > i;
    bool used = false;
    if (!blocked) {
        // events before visit i: ev_t is increasing
        int lo = 0, hi = *A.nev;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (A.ev_t[mid] < i) lo = mid + 1;
            else hi = mid;
        }
        for (int c = 0; c < A.m && !used; ++c) {
            double cm = A.cmin1[c];
            for (int e = lo - 1; e >= 0; --e)
                if (A.ev_j[e] == c) {
                    cm = A.ev_v[e];
                    break;
                }
            used = A.lub[(int64_t)c * A.n0 + i] > cm;
        }
    }
    if (!used) {
        // the recompute's top-p stay on as threshold hints
        for (int e = 0; e < A.p; ++e) {
            const int64_t at = (int64_t)e * A.n0 + i;
            A.hint_j[at] = A.st.ent_j[at];
            A.hint_c[at] = A.st.ent_c[at];
            A.hint_dq[at] = A.st.ent_dq[at];
        }
        for (int e = 0; e < A.p; ++e) {
            const int64_t at = (int64_t)e * A.n0 + i;
            A.st.ent_j[at] = A.saved.ent_j[at];
            A.st.ent_c[at] = A.saved.ent_c[at];
            A.st.ent_qb[at] = A.saved.ent_qb[at];
            A.st.ent_dq[at] = A.saved.ent_dq[at];
        }
        A.st.sigb[i] = A.saved.sigb[i];
        A.st.base[i] = A.saved.base[i];
        A.st.bnum[i] = A.saved.bnum[i];
    } else {
        for (int e = 0; e < A.p; ++e) A.hint_j[(int64_t)e * A.n0 + i] = -1;   // the entries are new
    }
}

template <int PASS>
static void launch_dp_seq(const DiscPassArgs &a, cudaStream_t s)
{
    static std::once_flag once[64];
    smem_optin_max((const void *)k_dp_seq<PASS>, once);
    k_dp_seq<PASS><<<1, DP_THREADS, dp_smem_bytes(a.k, a.m), s>>>(a);
}
void launch_discord_pass1(const DiscPassArgs &a, cudaStream_t s) { launch_dp_seq<1>(a, s); }
void launch_discord_mark(const DiscPassArgs &a, cudaStream_t s)
{
    k_dp1_list<<<(unsigned)((a.nl + 255) / 256), 256, 0, s>>>(a);
}
void launch_discord_pass2(const DiscPassArgs &a, cudaStream_t s) { launch_dp_seq<2>(a, s); }
void launch_discord_restore(const DiscPassArgs &a, cudaStream_t s)
{
    k_dp2_used<<<(unsigned)((a.nl + 255) / 256), 256, 0, s>>>(a);
}

// Algorithm 9 over the streamed tables: per cell the largest d / sqrt(l),
// ties to the later length.
__global__ void k_dkm_streamed_merge(StreamArgs A)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int cells = A.k * A.m;
    if (c >= cells) return;
    double best = ninf(), bd = 0.0;
    int32_t bo = -1, bl = 0, bn = -1;
    for (int li = 0; li < A.nL; ++li) {
        const int64_t at = (int64_t)li * cells + c;
        if (A.o[at] < 0) continue;
        const int l = A.lmin + li;
        const double v = A.d[at] / sqrt((double)l);
        if (bl == 0 || v >= best) {
            best = v;
            bd = A.d[at];
            bo = A.o[at];
            bl = l;
            bn = A.nn[at];
        }
    }
    A.out.norm[c] = best;
    A.out.dist[c] = bd;
    A.out.off[c] = bo;
    A.out.len[c] = bl;
    A.out.nn[c] = bn;
}

void launch_discords_streamed(const StreamArgs &a, cudaStream_t s)
{
    k_dkm_streamed<<<(a.nL + STREAM_WARPS - 1) / STREAM_WARPS, STREAM_WARPS * 32, 0, s>>>(a);
    const int cells = a.k * a.m;
    k_dkm_streamed_merge<<<(cells + 255) / 256, 256, 0, s>>>(a);
}

// --------------------------------------------------------------- motifs

// One greedy round over VALMP: the best (normalised distance asc, offset asc)
// entry whose pair {i, nn_i} does not come within max(E(len), E(len')) of an
// accepted pair. acc holds (a, b, len) of the r accepted pairs.
__global__ void k_motif_blockmin(Valmp vm, int64_t n0, int num, int den, const int32_t *acc, int r, double *bval,
                                 int32_t *bidx)
{
    const int64_t i = (int64_t)blockIdx.x * DBLK + threadIdx.x;
    double v = dinf();
    int32_t ix = -1;
    if (i < n0 && vm.len[i] > 0 && vm.nn[i] >= 0 && isfinite(vm.norm[i])) {
        const int64_t a = i, b = vm.nn[i];
        const int L = vm.len[i];
        bool ok = true;
        for (int q = 0; q < r && ok; ++q) {
            const int64_t a2 = acc[3 * q], b2 = acc[3 * q + 1];
            int64_t E = excl_zone(L, num, den), E2 = excl_zone(acc[3 * q + 2], num, den);
            if (E2 > E) E = E2;
            ok = llabs(a - a2) > E && llabs(a - b2) > E && llabs(b - a2) > E && llabs(b - b2) > E;
        }
        if (ok) { v = vm.norm[i]; ix = (int32_t)i; }
    }
    block_best<false>(v, ix);
    if (threadIdx.x == 0) {
        bval[blockIdx.x] = v;
        bidx[blockIdx.x] = ix;
    }
}

__global__ void k_motif_pick(Valmp vm, const double *bval, const int32_t *bidx, int nblk, int32_t *acc, int r,
                             int32_t *picked)
{
    double v = dinf();
    int32_t g = -1;
    for (int t = threadIdx.x; t < nblk; t += blockDim.x)
        if (better_asc(bval[t], bidx[t], v, g)) { v = bval[t]; g = bidx[t]; }
    block_best<false>(v, g);
    if (threadIdx.x == 0) {
        picked[r] = g;
        if (g >= 0) {
            const int32_t nn = vm.nn[g];
            acc[3 * r] = g < nn ? g : nn;
            acc[3 * r + 1] = g < nn ? nn : g;
            acc[3 * r + 2] = vm.len[g];
        }
    }
}

void launch_motif_round(const Valmp &vm, int64_t n0, int num, int den, int32_t *acc, int r, double *bval,
                        int32_t *bidx, int32_t *picked, cudaStream_t s)
{
    const int nblk = (int)((n0 + DBLK - 1) / DBLK);
    k_motif_blockmin<<<nblk, DBLK, 0, s>>>(vm, n0, num, den, acc, r, bval, bidx);
    k_motif_pick<<<1, 1024, 0, s>>>(vm, bval, bidx, nblk, acc, r, picked);
}

// --------------------------------------------------------------- re-checks

__device__ double block_sum(double v)
{
    __shared__ double sh[32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    v = 0.0;
    if (wid == 0) {
        v = lane < nw ? sh[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) sh[0] = v;
    }
    __syncthreads();
    v = sh[0];
    __syncthreads();
    return v;
}

__device__ bool window_flat(const double *x, int64_t i, int l)
{
    int diff = 0;
    for (int t = threadIdx.x + 1; t < l; t += blockDim.x) diff |= (x[i + t] != x[i]);
    return !__syncthreads_or(diff);
}

// Eq. DIST for windows a, b at length L straight from two-pass statistics and
// the centred dot product, in FP64 (one block per pair).
__device__ double direct_dist(const double *x, int64_t a, int64_t b, int L)
{
    const bool fa = window_flat(x, a, L), fb = window_flat(x, b, L);
    if (fa || fb) return (fa && fb) ? 0.0 : sqrt(2.0 * L);
    double sa = 0.0, sb = 0.0;
    for (int t = threadIdx.x; t < L; t += blockDim.x) { sa += x[a + t]; sb += x[b + t]; }
    const double ma = block_sum(sa) / L, mb = block_sum(sb) / L;
    double va = 0.0, vb = 0.0, cab = 0.0;
    for (int t = threadIdx.x; t < L; t += blockDim.x) {
        const double da = x[a + t] - ma, db = x[b + t] - mb;
        va = fma(da, da, va);
        vb = fma(db, db, vb);
        cab = fma(da, db, cab);
    }
    va = block_sum(va);
    vb = block_sum(vb);
    cab = block_sum(cab);
    double q = cab / sqrt(va * vb);
    q = q > 1.0 ? 1.0 : (q < -1.0 ? -1.0 : q);
    return sqrt(2.0 * L * (1.0 - q));
}

__global__ void k_recheck_pairs(const double *x, const int32_t *pairs, double *out)
{
    const int64_t a = pairs[3 * blockIdx.x], b = pairs[3 * blockIdx.x + 1];
    const int L = pairs[3 * blockIdx.x + 2];
    const double d = direct_dist(x, a, b, L);
    if (threadIdx.x == 0) out[blockIdx.x] = d;
}

void launch_recheck_pairs(const double *x, int64_t n, const int32_t *pairs, int npairs, double *out, cudaStream_t s)
{
    (void)n;
    if (npairs > 0) k_recheck_pairs<<<npairs, 256, 0, s>>>(x, pairs, out);
}

// m-th best-match distance of window `off` at length L from a full FP64
// distance profile (two-pass statistics for every window). Each cell's
// columns are split over RSLICES blocks; each block keeps its m smallest
// (distance, offset) pairs (per thread, then extracted block-wide one at a
// time); a second kernel merges the slices of a cell.
constexpr int RSLICES = 64;

__global__ void k_recheck_slices(const double *x, int64_t n, const int32_t *cells, int num, int den, double *sd,
                                 int32_t *sj, int mcap)
{
    const int cell = blockIdx.x / RSLICES, slice = blockIdx.x % RSLICES;
    const int64_t off = cells[3 * cell];
    const int L = cells[3 * cell + 1];
    const int m = cells[3 * cell + 2];
    const int64_t nl = n - L + 1;
    const int64_t E = excl_zone(L, num, den);
    const bool fo = window_flat(x, off, L);
    double so = 0.0;
    for (int t = threadIdx.x; t < L; t += blockDim.x) so += x[off + t];
    const double mo = block_sum(so) / L;
    double vo = 0.0;
    for (int t = threadIdx.x; t < L; t += blockDim.x) { const double d = x[off + t] - mo; vo = fma(d, d, vo); }
    vo = block_sum(vo);
    const int64_t per = (nl + RSLICES - 1) / RSLICES;
    const int64_t j0 = (int64_t)slice * per, j1 = j0 + per < nl ? j0 + per : nl;
    double best[MAXP];
    int32_t bj[MAXP];
    int nb = 0;
    for (int64_t j = j0 + threadIdx.x; j < j1; j += blockDim.x) {
        const int64_t dd = j - off;
        if (!(dd > E || -dd > E)) continue;
        double s = 0.0;
        bool fj = true;
        for (int t = 0; t < L; ++t) { s += x[j + t]; fj &= (x[j + t] == x[j]); }
        double d;
        if (fo || fj) {
            d = (fo && fj) ? 0.0 : sqrt(2.0 * L);
        } else {
            const double mj = s / L;
            double vj = 0.0, c = 0.0;
            for (int t = 0; t < L; ++t) {
                const double a = x[j + t] - mj;
                vj = fma(a, a, vj);
                c = fma(x[off + t] - mo, a, c);
            }
            double q = c / sqrt(vo * vj);
            q = q > 1.0 ? 1.0 : (q < -1.0 ? -1.0 : q);
            d = sqrt(2.0 * L * (1.0 - q));
        }
        if (nb < m || d < best[m - 1] || (d == best[m - 1] && (int32_t)j < bj[m - 1])) {
            int b = nb < m ? nb++ : m - 1;
            while (b > 0 && (best[b - 1] > d || (best[b - 1] == d && bj[b - 1] > (int32_t)j))) {
                best[b] = best[b - 1];
                bj[b] = bj[b - 1];
                --b;
            }
            best[b] = d;
            bj[b] = (int32_t)j;
        }
    }
    int head = 0;
    for (int r = 0; r < m; ++r) {
        double v = head < nb ? best[head] : dinf();
        int32_t ix = head < nb ? bj[head] : -1;
        block_best<false>(v, ix);
        if (head < nb && bj[head] == ix && ix >= 0) ++head;
        if (threadIdx.x == 0) {
            sd[((int64_t)cell * RSLICES + slice) * mcap + r] = v;
            sj[((int64_t)cell * RSLICES + slice) * mcap + r] = ix;
        }
    }
}

__global__ void k_recheck_merge(const int32_t *cells, const double *sd, const int32_t *sj, int mcap, double *out)
{
    const int cell = blockIdx.x;
    const int m = cells[3 * cell + 2];
    // m rounds of block-wide minimum over the slices' sorted lists
    __shared__ int head[RSLICES];
    if (threadIdx.x < RSLICES) head[threadIdx.x] = 0;
    __syncthreads();
    double res = dinf();
    for (int r = 0; r < m; ++r) {
        double v = dinf();
        int32_t ix = -1;
        if (threadIdx.x < RSLICES && head[threadIdx.x] < m) {
            const int64_t k = ((int64_t)cell * RSLICES + threadIdx.x) * mcap + head[threadIdx.x];
            v = sd[k];
            ix = sj[k];
        }
        block_best<false>(v, ix);
        if (threadIdx.x < RSLICES && head[threadIdx.x] < m && ix >= 0 &&
            sj[((int64_t)cell * RSLICES + threadIdx.x) * mcap + head[threadIdx.x]] == ix)
            ++head[threadIdx.x];
        __syncthreads();
        res = v;
    }
    if (threadIdx.x == 0) out[cell] = res;
}

void launch_recheck_discords(const double *x, int64_t n, const int32_t *cells, int ncells, int num, int den,
                             double *out, double *sd, int32_t *sj, int mcap, cudaStream_t s)
{
    if (ncells <= 0) return;
    k_recheck_slices<<<ncells * RSLICES, 256, 0, s>>>(x, n, cells, num, den, sd, sj, mcap);
    k_recheck_merge<<<ncells, 64, 0, s>>>(cells, sd, sj, mcap, out);
}

size_t recheck_scratch(int ncells, int mcap) { return (size_t)ncells * RSLICES * mcap; }

}  // namespace mad
