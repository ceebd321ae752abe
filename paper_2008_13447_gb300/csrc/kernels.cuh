// kernels.cuh -- argument structs and declarations of the device kernels.
#pragma once
#include "mad_internal.cuh"

namespace mad {

// ---------------------------------------------------------------- k_stats.cu
__global__ void k_flat_runs(const double *x, int64_t n, int cap, int32_t *run);
__global__ void k_stats_init(const double *x, int64_t nl, int l, double *mu, double *m2);
void launch_stats_step(const double *x, int64_t nl, int l, const double *mu_o, const double *m2_o, double *mu_n,
                       double *m2_n, cudaStream_t s);
// Column data of the band kernel, and isd[j] = 1 / sqrt(M2_j) in FP64 (0 for
// a flat window) for the per-row kernels.
template <typename T>
void launch_coldata(const double *x, int64_t nl, int64_t npad, int l, const double *mu, const double *m2,
                    const int32_t *run, Col<T> *col, double *isd, cudaStream_t s);
// x split into FP32 pairs, x[k] = xh[k] + xl[k] to about 48 bits.
void launch_split_x(const double *x, int64_t n, float *xh, float *xl, cudaStream_t s);
__global__ void k_widen_f32(const float *in, int64_t n, double *out);

// ------------------------------------------- k_band.cuh (k_band_f32.cu, k_band_f64.cu)
// Seed rows of the diagonal recurrence. Seed row k (row kS, S the seed
// spacing) holds, for every column j, the value that precedes cell (kS, j)
// on its diagonal:
//   S_k[j] = C(kS - 1, j - 1)            for k >= 1, j >= 1
//   S_k[j] = C(kS, j)                    for k == 0 or j == 0
// (the second line makes the recurrence start exactly at the first row /
// column, whose virtual predecessors carry df = dg = 0). By symmetry of C,
// S_k[r] is also the value preceding cell (r, kS): the left edge of a column
// group starting at kS. Bands start at multiples of R = 2S. Entries whose
// column is past the last window are 0.
template <typename T> struct SeedArgs {
    const double *x;
    const double *mu;       // window means at l
    int64_t nl;
    int l;
    int R;                  // seed spacing S
    const int32_t *krows;   // seed rows to compute
    int nk;
    int64_t spitch;         // elements per seed row
    T *seed;
    const int32_t *nbands;  // nothing to do when the device count is 0
};
template <typename T> void launch_seed(const SeedArgs<T> &a, cudaStream_t s);
template <> void launch_seed<double>(const SeedArgs<double> &a, cudaStream_t s);
// Seed rows stepped from length l to l + 1 (update) or only copied to T:
// mu = window means at l, nl = windows at l + 1, master = FP64 seed rows
// (updated in place), seed = the band kernel's copy.
template <typename T>
void launch_seed_step(const double *x, const double *mu, int64_t nl, int l, int S, int64_t K, int64_t spitch,
                      double *master, T *seed, bool update, cudaStream_t s);

template <typename T> struct BandArgs {
    const Col<T> *col;      // per-window recurrence data, rows and columns
    const T *seed;          // seed rows (pitch spitch)
    int64_t spitch;
    const T *thr;           // per-row key threshold (+inf: row not wanted)
    const int32_t *bands;   // active band ids
    const int32_t *nbands;  // number of active bands (device)
    int32_t *unit_ctr;      // work counter, zero before launch
    int64_t nl;
    int l;
    int64_t E;
    int rpl;                // rows per lane (band height R = 32 * rpl * BAND_NW)
    int64_t sp;             // seed-row spacing (divides R): seed row k sits at row k * sp
    int64_t group_w;        // columns per work unit (multiple of sp)
    int ngroups;
    int p;
    // top-p mode: per row and column group, up to p (key, offset) pairs
    T *skey;                // [row][group][p]
    int32_t *sj;            // [row][group][p]
    int32_t *scnt;          // [row][group]
    // bins mode: per row, the maximum key of each class of column chunks
    int *bins;              // [row][nbins] order-preserving ints
    int nbins;
    int *rowbest;           // per row: the best p-th kept key of finished units (order-preserving
                            // int of a float, rounded down; reset before each launch)
    int *err;               // set to 1 if a bounded wait ran out
    int wave_limit;         // tries of each wavefront wait (the hand-over between warps) before it
                            // gives up; the unit-queue waits always use the full limit
    unsigned long long *ninsert;  // top-p list insertions (diagnostic counter)
    unsigned long long *stats;    // this length's counters ([5] units, [6] cells)
    // symmetric form
    int kb_total;           // number of bands covering n_l rows
    int allow_sym;
    const unsigned long long *nflagged;   // rows to recompute at this length
    T *ckey;                // [row][cap] column-side candidates (key, partner)
    int32_t *cj;
    int32_t *ccnt;          // [row]
    int cap;
};
template <typename T> void launch_band(const BandArgs<T> &a, bool bins_mode, int grid, cudaStream_t s);
template <typename T> int band_occupancy(bool bins_mode, int p, int rpl);
template <typename T> size_t band_smem(bool bins_mode, int p, int rpl);

// ------------------------------------------------------------- error model
// Rounding of the band kernel's recurrence accumulates along a diagonal
// chain of at most R + 1 steps from its seed. With kappa_i = sqrt(max over
// the chain windows of w_k / M2_i), w_k = M2_k + 1.5 (df_k^2 + dg_k^2) (see
// launch_kappa), the correlation of a band key for cell (i, j) is within
//     dq0 kappa_i kappa_j,   dq0 = u (2R + 4)
// of the exact one (u the unit roundoff of the recurrence's type; the FP64
// path adds the error of its seeds, stepped in FP64 from length to length).
// The direct path (k_direct) and the tensor-core path (k_direct_tc) write
// their own per-entry bounds, and the largest of them per length. A distance
// whose resulting error could exceed half its tolerance is re-evaluated
// (compensated FP32 or FP64).
struct ErrModel {
    const float *kappa;     // per window
    const float *kappa_max; // max over windows at this length (device scalar)
    double dq0;
    double rel_tol;         // distance tolerance = rel_tol * d + abs_coef * sqrt(l)
    double abs_coef;
    int audit;              // test hook: re-evaluate every stored entry that carries a bound, in
                            // FP64, so that the observed error over its bound is recorded
};
void launch_kappa(const double *x, const double *mu, const double *m2, const int32_t *run, int64_t nl, int l, int R,
                  double *blkmax, float *kappa, float *kappa_max, cudaStream_t s);

// ----------------------------------------------------------------- k_rows.cu
// Per-row state kept across lengths (structure of arrays, n0 = n - lmin + 1):
//   ent_j[e * n0 + i], ent_c[e * n0 + i] : the p stored entries of row i
//       (partner offset, -1 if empty; centred co-moment at the current length)
//   base[i]  : length l_b at which the entries were selected
//   bnum[i]  : bound numerator  sqrt(l_b (1 - max(q_p, 0)^2)) * sigma_i(l_b)
//              (+inf when every non-trivial partner is stored); the bound at
//              length l is bnum[i] / sigma_i(l) (Eq. LB, rank preservation)
struct RowState {
    int32_t *ent_j;
    double *ent_c;
    double *ent_qb;         // correlation of each entry at the row's base length
    double *sigb;           // sigma_i(l_b)
    float *ent_dq;          // correlation error bound of each entry (0 once re-evaluated in FP64)
    int32_t *base;
    double *bnum;
    int32_t *flag;
};

struct Valmp {
    double *dist;
    double *norm;
    int32_t *len;
    int32_t *nn;
};

struct LenOut {
    double *nnd;            // [m][n0] m-th best-match distance at the current length
    int32_t *nnj;           // [m][n0] its offset
    unsigned long long *stats;  // this length's counters: [1] certified, [2] recomputed,
                                //   [3] largest |q_band - q_FP64| seen on re-evaluated entries (bits),
                                //   [12] largest such error over the entry's own bound (bits)
};

template <typename T> struct ExtArgs {
    const double *x;
    // motif mode (NULL otherwise): per-row bound of non-valid rows, and the
    // smallest certified distance / non-valid bound (bits of non-negative
    // doubles, reduced with atomicMin)
    double *lbmax;
    unsigned long long *min_dist_abs, *min_lb_abs;
    // observation at one length (NULL otherwise): maxLB - minED, mean LB / ED
    double *obs_gap, *obs_tlb;
    // discord mode: non-valid rows write their 1st..m-th smallest pessimistic
    // stored distances (+inf past the stored count; flat rows +inf) to out.nnd
    int ub_out;
    // discord mode (NULL otherwise): per row, p hint partners (the top-p of a
    // recompute whose state was given back), extended like the entries and
    // used only to tighten the band kernel's threshold
    int32_t *hint_j;
    double *hint_c;
    float *hint_dq;
    const float *xh, *xl;   // x as FP32 pairs (compensated re-evaluation)
    const double *isd;      // 1 / sqrt(M2) at l (0: flat)
    int64_t n0, nl;
    int l;
    int64_t E;
    int p, m_max;
    const double *mu_prev;  // means at l-1
    const double *mu;       // means at l
    const double *m2;       // M2 at l
    const int32_t *run;
    RowState st;
    Valmp vm;
    LenOut out;
    T *thr;
    ErrModel em;
};
template <typename T> void launch_extend(const ExtArgs<T> &a, cudaStream_t s);

// Motif mode, after the extension of a length (Algorithm 4's decision):
// bBestM = minDistAbs < minLbAbs -> every non-valid row left undefined;
// else with fewer than `limit` non-valid rows -> those with lbMax <
// minDistAbs recomputed, the others undefined; else the full profile (every
// row recomputed). Undefined rows get ROW_SKIP and NaN / -1 as their value.
template <typename T> struct SubmpArgs {
    int64_t nl;
    int32_t *flag;
    T *thr;
    const double *lbmax;
    const unsigned long long *min_dist_abs, *min_lb_abs;
    const unsigned long long *nonvalid;   // rows flagged by the extension
    double limit;                         // n log(p) / log(n)
    double *nnd;                          // m = 1 row of the current length
    int32_t *nnj;
    unsigned long long *stats;            // [10] undefined rows, [11] full profile
};
template <typename T> void launch_submp_mark(const SubmpArgs<T> &a, cudaStream_t s);

// ----------------------------------------------------------------- k_sets.cu
// One motif set grown from the pair (a, b) at length l with radius r.
struct SetArgs {
    const double *x;
    int64_t n;
    int l;
    int64_t E;                 // E(l)
    int64_t a, b;
    double r;
    const int64_t *prev_off;   // members of earlier sets ...
    const int64_t *prev_E;     // ... and E of their lengths
    int nprev;
    double *ckey;              // candidate list (distance, offset), capacity capc
    int32_t *cj;
    int32_t *ccount;
    int64_t capc;
};
void launch_motif_set(const SetArgs &a, int cap, int64_t *members, int32_t *mcount, cudaStream_t s);

template <typename T> struct MergeArgs {
    const double *x;
    const float *xh, *xl;
    const double *isd;
    int64_t n0, nl;
    int l;
    int64_t E;
    int p, m_max;
    const double *mu;
    const double *m2;
    const int32_t *run;
    const Col<T> *col;
    const T *skey;
    const int32_t *sj;
    const int32_t *scnt;
    int ngroups;
    int64_t group_w;        // columns per group; groups starting at or past n_l are empty
    T *thr;
    RowState st;
    Valmp vm;
    LenOut out;
    ErrModel em;
    unsigned long long *overflow;   // rows that need a second pass
    // symmetric form (same rule as the band kernel)
    const unsigned long long *nflagged;
    int allow_sym;
    int R;
    // direct path
    const int32_t *dindex;
    const T *dkey;
    const int32_t *dj;
    const int32_t *dcnt;
    const float *ddq;       // per-entry error bounds of the direct paths
    const float *ddq_max;   // their largest at this length
    int dnblk;
    const T *ckey;
    const int32_t *cj;
    int32_t *ccnt;
    int cap;
};
template <typename T> void launch_merge(const MergeArgs<T> &a, cudaStream_t s);

template <typename T>
void launch_theta_bins(const int *bins, int nbins, int64_t nl, int p, const double *m2, ErrModel em, T *thr,
                       cudaStream_t s);

struct FlatArgs {
    int64_t n0, nl;
    int l;
    int64_t E;
    int p, m_max;
    const int32_t *run;
    RowState st;
    Valmp vm;
    LenOut out;
    int *left_over;         // set when a row is still waiting for a recompute
};
void launch_flat_rows(const FlatArgs &a, cudaStream_t s);

__global__ void k_init_flags(const int32_t *run, int64_t n0, int l, int32_t *flag, unsigned long long *stats);
template <typename T> void launch_mask_thr(const int32_t *flag, int64_t n0, T *thr, cudaStream_t s);

void launch_compact_bands(const int32_t *flag, int64_t nl, int R, int32_t *bands, int32_t *nbands,
                          cudaStream_t s);

// Rows to recompute, split between the band kernel and the direct path: a
// band whose rows to recompute number at most `lim` hands them to the direct
// path (flag ROW_DIRECT, listed in drows with dindex[row] = position, while
// the list has room), other bands go to the band list. When the symmetric
// band form is on (at least half of the rows to recompute, read from
// *nflagged) nothing goes direct unless force_direct.
struct SplitArgs {
    int32_t *flag;
    int64_t nl;
    int R;
    int lim;
    int force_direct;
    int allow_sym;
    const unsigned long long *nflagged;
    int32_t *bands;
    int32_t *nbands;
    int32_t *drows;
    int32_t *ndirect;       // [0] rows listed, [1] positions reserved (k_split's counter)
    int32_t *dindex;
    int max_direct;
    unsigned long long *stat_direct;   // rows routed to the direct path (counter)
};
void launch_split(const SplitArgs &a, cudaStream_t s);
__host__ __device__ __forceinline__ bool sym_rule(int allow_sym, unsigned long long nflagged, int64_t nl)
{
    return allow_sym && 2 * (int64_t)nflagged >= nl;
}

// Direct recompute of listed rows (k_direct.cu).
template <typename T> struct DirectArgs {
    const double *x;
    const double *mu;
    const Col<T> *col;
    int64_t nl;
    int l;
    int64_t E;
    int p;
    const int32_t *rows;
    const int32_t *nrows;
    const T *thr;
    T *okey;                // [list position][nblk][p]
    int32_t *oj;
    int32_t *ocnt;          // [list position][nblk]
    int nblk;
    float *odq;             // [list position][nblk][p] error bound of each key (correlation units)
    float *dq_max;          // largest bound of any column at this length (device scalar, max-reduced)
};
template <typename T> void launch_direct(const DirectArgs<T> &a, int grid, cudaStream_t s);
int direct_cols_per_block();

// The same recompute on the tensor cores (k_direct_tc.cu): FP16 hi + lo split
// products of the rows' normalised windows and the shifted series, FP32
// accumulation in TMEM; same outputs as the direct kernel.
struct TcArgs {
    const double *x;
    const float *xh, *xl;   // x as FP32 pairs (x = xh + xl to about 48 bits)
    int64_t n, nl;
    int l;
    int64_t E;
    int p;
    const double *mu;       // window means at l
    const double *m2;       // M2 at l
    const double *isd;      // 1 / sqrt(M2) (0: flat)
    const int32_t *rows;    // listed rows
    const int32_t *nrows;   // their count (device)
    const float *thr;       // per-row key threshold
    int nkc;                // lag chunks of 64 covering l
    unsigned char *aimg;    // row operand images [row tile][chunk][hi, lo][16 KB]
    float *asum;            // [list position] sum of the represented row operand
    float *sqm2;            // [list position] sqrt(M2) of the row
    float *okey;            // outputs as DirectArgs
    int32_t *oj;
    int32_t *ocnt;
    float *odq;
    float *dq_max;
    int nblk;
    int *err;               // set if a bounded wait ran out
    // column tiles written per length and loaded by TMA (p <= 16): the
    // tiles' shifted copies [hi, lo][tile][8][lc] (FP16), their column
    // constants [tile][256] (16 B each), and the TMA descriptor of the
    // copies (host memory; nullptr: the kernel builds the tiles itself)
    void *bcopy;
    void *gcc;
    int64_t ntiles;         // column tiles at this length
    int64_t tiles_ws;       // column tiles of the workspace layout (the largest length's count)
    int lc;
    const void *bmap;
};
void launch_direct_tc(const TcArgs &a, int num_sms, cudaStream_t s);
size_t tc_aimg_bytes(int64_t max_rows, int lmax);
// Column tiles by TMA: copy length, byte sizes, and the descriptor of
// [2][tiles][8][lc] FP16 at gaddr written into map (128 bytes, 64-byte
// aligned); false if the driver refuses it (the kernel then builds the
// tiles itself).
int tc_copy_len(int lmax);
size_t tc_bcopy_bytes(int64_t ntiles, int lmax);
size_t tc_gcc_bytes(int64_t ntiles);
int64_t tc_col_tiles(int64_t nl);
bool tc_encode_bmap(void *map, void *gaddr, int64_t ntiles, int lc);
int tc_chunks(int l);

template <typename T>
void launch_fill(T *p, int64_t n, T v, cudaStream_t s);

// ------------------------------------------------------------- k_readout.cu
struct DiscTable {          // k_max x m_max cells, rank-major
    double *norm;
    double *dist;
    int32_t *off;
    int32_t *len;
    int32_t *nn;
};
struct GDiscArgs {          // global-greedy discords over the kept profiles
    const double *nnd;      // [nL][m_max][n0] m-th best-match distances
    const int32_t *nnj;
    int64_t n, n0;
    int lmin, nL, m_max, num, den;
    int nblk;               // tiles of DBLK offsets per length
    int k, mcols;           // ranks, columns 1..mcols
    double *tv;             // [mcols][nL][nblk] best free score per tile
    int64_t *tk;            // its key
    DiscTable out;          // k x mcols cells, rank-major
};
struct StreamArgs {         // dkm_l streamed (Algorithms 7 and 8) and merged (Algorithm 9)
    const double *nnd;      // kept profiles [nL][m_max][n0]
    const int32_t *nnj;
    int64_t n, n0;
    int lmin, nL, m_max, num, den;
    int k, m;               // ranks and columns 1..m
    double *d;              // [nL][k][m] per-length tables
    int32_t *o, *nn;
    DiscTable out;          // k x m cells, rank-major
};
void launch_discords_streamed(const StreamArgs &a, cudaStream_t s);
struct DiscPassArgs {       // discord mode: Algorithm 10's two passes at one length
    int64_t n0, nl;
    int l;
    int64_t E;
    int k, m;               // k_max, m_max
    int all_valid;          // lmin: every row's distances are exact
    int32_t *flag;          // row state after the extension
    float *thr32;           // the row thresholds (one of the two, by precision)
    double *thr64;
    double *nnd;            // [m][n0] exact (valid / recomputed rows) or upper values (non-valid)
    int32_t *nnj;
    double *D;              // dkm_l [k][m] (between the passes)
    int32_t *O, *N;
    int32_t *O1;            // dkm_l's offsets after the first pass
    double *cmin1;          // its column minima [m]
    int32_t *ins1, *drop1;  // first-pass log [n0]: ins = l if entered at l; drop = who pushed it out
    int32_t *ins2, *drop2;  // second-pass log [n0]
    int32_t *ev_t, *ev_j;   // second-pass entries: window, column, the column's new minimum
    double *ev_v;
    int32_t *nev;
    double *lub;            // [m][n0] upper values of the kept rows
    int32_t *kept;          // [n0] 1: kept for the second pass
    DiscTable tab;          // dkm_{lmin,lmax}
    unsigned long long *stats;
    RowState st, saved;     // row state and its copy from before the recomputes
    int p;
    int32_t *hint_j;        // [p][n0] threshold hints (see ExtArgs)
    double *hint_c;
    float *hint_dq;
};
void launch_discord_pass1(const DiscPassArgs &a, cudaStream_t s);
void launch_discord_mark(const DiscPassArgs &a, cudaStream_t s);
void launch_discord_pass2(const DiscPassArgs &a, cudaStream_t s);
void launch_discord_restore(const DiscPassArgs &a, cudaStream_t s);
constexpr int GDISC_TILE = 256;
void launch_discords_global(const GDiscArgs &a, cudaStream_t s);
void launch_discords_length(const double *nnd, const int32_t *nnj, int64_t n0, int64_t nl, int l, int64_t E,
                            int k_max, int m_max, double *bval, int32_t *bidx, DiscTable tab, cudaStream_t s);

void launch_motif_round(const Valmp &vm, int64_t n0, int num, int den, int32_t *acc /* 3 ints per pick */,
                        int r, double *bval, int32_t *bidx, int32_t *picked, cudaStream_t s);

void launch_recheck_pairs(const double *x, int64_t n, const int32_t *pairs /* a,b,len */, int npairs,
                          double *out, cudaStream_t s);
void launch_recheck_discords(const double *x, int64_t n, const int32_t *cells /* off,len,m */, int ncells,
                             int num, int den, double *out, double *sd, int32_t *sj, int mcap, cudaStream_t s);
size_t recheck_scratch(int ncells, int mcap);   // entries of sd / sj

}  // namespace mad
