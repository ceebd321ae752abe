/*
 * mad.h -- C ABI of the GB300 (sm_103a) exact variable-length matrix profile.
 *
 * The library computes, on one GPU, what the VALMOD / MAD method of
 * "Matrix Profile Goes MAD" computes:
 *   - the z-normalised matrix profile of a data series at every length of a
 *     range [lmin, lmax] (Problem 1, variable-length motif pair discovery),
 *     using the paper's lower bound (Eq. LB) to skip rows whose p stored
 *     entries already certify the result (Algorithms 1, 3, 4, 10);
 *   - the variable-length matrix profile VALMP (Algorithm 2) and its top-k
 *     length-normalised motif pairs (Sec. 3, Algorithm 5);
 *   - the variable-length Top-k m-th discord table dkm_{lmin,lmax}
 *     (Problem 3, Algorithms 7-9).
 *
 * Conventions (all calls):
 *   - Offsets are 0-based. A window (subsequence) of length l starting at i
 *     covers x[i .. i+l-1]; n_l = n - l + 1 windows exist at length l.
 *   - A pair (i, j) is a trivial match at length l iff |i - j| <= E(l),
 *     E(l) = ceil(l * excl_num / excl_den) (Sec. 2 "exclusion zone"; the paper
 *     uses l/2, the default here is l/4).
 *   - Distances are z-normalised Euclidean distances (Eq. DIST), with the
 *     population standard deviation. A window whose values are all equal is
 *     "flat": two flat windows are at distance 0, a flat and a non-flat
 *     window at sqrt(2 l).
 *   - Every call returns a mad_status; no C++ exception crosses the ABI.
 *     After an error, mad_last_error(ctx) describes it (ctx may be NULL for
 *     errors of mad_create*; then a thread-local message is returned).
 *   - Host pointers are caller-owned and only read/written during the call.
 *     Device pointers passed to mad_create_device stay caller-owned and must
 *     remain valid until mad_destroy.
 *   - Every call is synchronous with respect to the host: when it returns,
 *     all GPU work it issued on the context's stream has completed.
 *   - A context is not thread-safe; use one context per host thread.
 */
#ifndef MAD_H
#define MAD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define MAD_API __attribute__((visibility("default")))
#else
#define MAD_API
#endif

typedef struct mad_ctx mad_ctx;

typedef enum {
    MAD_OK = 0,
    MAD_EINVAL = 1,     /* invalid argument (sizes, ranges, NULL pointers) */
    MAD_ENOMEM = 2,     /* device or host allocation failed */
    MAD_ECUDA = 3,      /* a CUDA runtime call failed */
    MAD_ESTATE = 4,     /* call out of order (e.g. read-out before profile) */
    MAD_ETIMEOUT = 5,   /* a bounded device-side wait ran out */
    MAD_EINTERNAL = 6   /* an internal consistency check failed */
} mad_status;

/* Arithmetic of the matrix-profile kernels.
 *   MAD_FP64: FP64 everywhere (the plain reference path on the GPU).
 *   MAD_FP32: the O(n^2) diagonal (QT) recurrence in FP32 on centred
 *             co-moments, re-seeded from FP64 dot products every band of
 *             rows; rows recomputed on their own (the direct path) use FP32
 *             dot products. Window statistics, the per-row stored entries,
 *             the length extension, the bound test and the reported
 *             distances stay FP64 (or compensated FP32, within the error the
 *             library bounds). Every kept correlation carries a proven error
 *             bound; distances agree with FP64 within 1e-4 * sqrt(l).
 *   MAD_SPLIT_TC: as MAD_FP32, but the direct path runs on the tensor cores
 *             (tcgen05): each block of co-moments is a dense product of the
 *             rows' normalised windows and the shifted series (Hankel form),
 *             both split into FP16 hi + lo pairs (hi*hi + hi*lo + lo*hi),
 *             accumulated in FP32; more of the rows to recompute take that
 *             path. Same guarantees as MAD_FP32. */
typedef enum { MAD_FP64 = 0, MAD_FP32 = 1, MAD_SPLIT_TC = 2 } mad_precision;

typedef struct mad_options {
    int32_t excl_num;       /* exclusion zone numerator   (0 with excl_den 0: 1/4) */
    int32_t excl_den;       /* exclusion zone denominator */
    int32_t precision;      /* mad_precision, default MAD_FP64 */
    int32_t k_max;          /* discord table rows (ranks) kept, default 10, <= 64 */
    int32_t m_max;          /* discord table columns (m-th best match), default 1; must be <= p */
    int32_t keep_profiles;  /* nonzero: keep every per-length matrix profile and m-th best
                               match table for mad_matrix_profile (|L| * n_lmin * (1 + m_max)
                               doubles and offsets; meant for small inputs) */
    int32_t mode;           /* 0 (exact rows): every row the bound cannot certify is recomputed,
                               so every per-length result is exact for every offset;
                               1 (motif mode, Algorithm 1 with ComputeSubMP, Algorithm 4): per
                               length only the motif is guaranteed. Rows whose bound is not
                               below the best certified distance are left undefined (NaN in the
                               kept profiles, no VALMP update); when that test fails and too many
                               rows are non-valid (n log p / log n or more) the full profile is
                               computed. The best length-normalised VALMP entry (the top-1
                               variable-length motif) is exact. Needs m_max = 1; no discord
                               table (mad_discords returns MAD_ESTATE);
                               2 (discord mode, Algorithm 7 driving Algorithm 10): per length,
                               windows in offset order; one with a trivial match in dkm_l is
                               skipped, a valid row (stored entries certify its 1st..m_max-th best
                               matches) enters dkm_l by Algorithm 8, a non-valid row is listed;
                               then each listed row whose upper values can still beat a column's
                               k_max-th entry (m_max down to 1) is recomputed and entered; dkm_l
                               is merged by Algorithm 9. mad_discords returns that table; rows
                               neither valid nor recomputed are undefined at that length (NaN in
                               the kept profiles, no VALMP update). */
    int32_t band_form;      /* matrix-profile kernel form: 0 = full rows (each row band walks every
                               column; the faster form on GB300), 1 = symmetric (upper triangle only,
                               each pair computed once and fed to both windows, used for the lengths
                               where at least half of the row bands need recomputing) */
    int32_t observe_len;    /* 0 = off; else a length in (lmin, lmax] at which mad_profile records,
                               per row, maxLB - minED and the mean tightness of the lower bound
                               (read with mad_observe) */
    void *stream;           /* cudaStream_t to issue work on; NULL = the legacy default stream */
} mad_options;

/* One motif pair: windows a < b of length len. */
typedef struct {
    int64_t a, b;
    int32_t len;
    int32_t reserved;
    double dist;            /* z-normalised Euclidean distance at len */
    double norm_dist;       /* dist * sqrt(1 / len) (Sec. 3) */
    double dist_recheck;    /* the same distance recomputed directly in FP64 (two-pass
                               statistics, centred dot product) on the GPU */
} mad_motif;

/* One cell <d*, o*, l*> of dkm_{lmin,lmax}: the Top-rank m-th discord. */
typedef struct {
    int64_t off;            /* o*: window offset (-1 if the cell is empty) */
    int64_t nn;             /* offset of its m-th best match at len */
    int32_t len;            /* l* (0 if the cell is empty) */
    int32_t rank;           /* 1-based rank k */
    int32_t m;              /* 1-based column m */
    int32_t reserved;
    double dist;            /* its m-th best-match distance at len */
    double norm_dist;       /* d* = dist / sqrt(len) */
    double dist_recheck;    /* the m-th best-match distance recomputed on the GPU from a
                               full FP64 distance profile (two-pass statistics per window) */
} mad_discord;

/* Pruning counters of one length (Sec. 7.2 "valid / non-valid / recomputed"). */
typedef struct {
    int32_t len;
    int32_t reserved;
    int64_t rows;           /* windows alive at len (n_len) */
    int64_t certified;      /* rows whose stored entries certified the result */
    int64_t recomputed;     /* rows whose full distance profile was recomputed */
    int64_t tiles;          /* band x column-range units the recompute kernel ran */
    int64_t passes;         /* recompute kernel passes (1 + candidate-list refills) */
    int64_t band_cells;     /* cells the matrix-profile (band) kernel evaluated at this length:
                               rows of its active bands x columns, summed over passes */
    int64_t launches;       /* GPU kernel launches issued for this length */
    int64_t inserts;        /* insertions into the band kernel's per-row top-p lists (cells that
                               beat their row's running p-th best key) */
    int64_t col_appends;    /* symmetric band form: cells appended to their column row's
                               candidate list */
    int64_t second_pass_rows; /* rows whose lists fell short and were redone in full */
    int64_t direct_rows;    /* rows recomputed by direct dot products instead of the band kernel */
    double band_ms;         /* device time of those band-kernel launches (CUDA events recorded
                               on the context's stream around each launch) */
    double fp32_dq_max;     /* MAD_FP32: largest |q_FP32 - q_FP64| among stored entries that were
                               re-evaluated in FP64 at this length (0 when none / MAD_FP64) */
    int64_t skipped;        /* motif mode: non-valid rows left undefined at this length */
    int32_t full_profile;   /* motif mode: 1 if the full profile was computed at this length */
    int32_t reserved2;
    double dq_ratio_max;    /* largest observed error of a re-evaluated stored entry's correlation
                               divided by the error bound the library kept for it (the bound holds
                               while this is <= 1; against a compensated re-evaluation the
                               observation is an upper estimate); 0 when nothing was re-evaluated */
    double direct_ms;       /* device time of the direct-path recompute launches at this length */
    double rows_ms;         /* device time of the per-row launches (extension, bound test, merge of
                               the recomputed rows' candidates) at this length */
    int32_t graph;          /* 1 if this profile ran as a replayed CUDA graph (a repeat of the
                               previous profile's shape, see mad_profile) */
    int32_t band_rows;      /* rows per band of the matrix-profile kernel in this profile (chosen
                               by the autotuner, see mad_set_autotune) */
} mad_length_stats;

/* Create a context for one series copied from host memory (FP64, n values).
 * Needs n >= 4. On success *out owns all device memory it allocates. */
MAD_API mad_status mad_create(const double *host_series, int64_t n, const mad_options *opt,
                              mad_ctx **out);

/* Same, for a series already in device memory: dtype 0 = FP64, 1 = FP32
 * (widened to FP64 on the device). The caller keeps ownership of
 * dev_series; it must stay valid until mad_destroy. */
MAD_API mad_status mad_create_device(const void *dev_series, int32_t dtype, int64_t n,
                                     const mad_options *opt, mad_ctx **out);

/* Create one context over `count` independent host series (series[s] has
 * n[s] values), profiled together by mad_profile_batch. */
MAD_API mad_status mad_create_batch(const double *const *series, const int64_t *n, int32_t count,
                                    const mad_options *opt, mad_ctx **out);

/* Compute the exact variable-length matrix profile over [lmin, lmax] keeping
 * p entries per row (Algorithm 1 VALMOD with the Top-k m-th discord table
 * of Algorithm 7). Requires 2 <= lmin <= lmax, 1 <= p <= 64, m_max <= p, and
 * n - lmax + 1 > 2 E(lmax) + 2 (every window keeps a non-trivial neighbour).
 * A context may be profiled again (results are replaced). Device memory: the
 * first profile allocates the workspace; a profile with the same lmin, lmax,
 * p and options reuses it (no allocation), and from the second such profile
 * on the whole launch sequence is captured once into a CUDA graph and
 * replayed (mad_set_graphs(0) turns that off). The series' device data is
 * read at every profile, so new values written to a caller-owned series
 * between profiles are used. */
MAD_API mad_status mad_profile(mad_ctx *ctx, int32_t lmin, int32_t lmax, int32_t p);

/* Batched form: lmin[s], lmax[s] per series of a mad_create_batch context.
 * Series are started on eight streams without waiting on the host; a repeat
 * with the same ranges reuses every series' workspace (launched eagerly, not
 * replayed as graphs: with many series in flight that measured faster). */
MAD_API mad_status mad_profile_batch(mad_ctx *ctx, const int32_t *lmin, const int32_t *lmax,
                                     int32_t p);

/* Top-k length-normalised motif pairs of series `series` from VALMP: offsets
 * visited by (norm_dist, offset) ascending, a pair accepted unless one of its
 * offsets lies within max(E(len), E(len')) of an offset of an accepted pair.
 * Writes up to k entries to out (caller array of k) and their count to
 * *n_out (fewer than k is not an error). MAD_ESTATE before mad_profile. */
MAD_API mad_status mad_motifs(mad_ctx *ctx, int32_t series, int32_t k, mad_motif *out,
                              int32_t *n_out);

/* Variable-length motif sets (Sec. "Finding Motif Sets", Algorithm 6) grown
 * from the top-k motif pairs of mad_motifs: set s starts from pair s
 * (offsets a < b at length len) with radius = D * the pair's FP64 distance;
 * it adds, by (distance, offset) ascending, windows j at len whose FP64
 * distance to a or to b is at most the radius, that are not trivial matches
 * of a, b or an accepted member (|j - m| <= E(len)), and that do not lie
 * within max(E(len), E(len')) of a member of an earlier set (sets never
 * meet), up to cap members (a and b first).
 *   sets     host, k entries; sets[s].count members written
 *   members  host, k x cap offsets, row s for set s
 *   *n_out   the number of sets (the number of motif pairs found, <= k).
 * Requires 2 <= cap <= 256, D >= 0, k in [1, 64]. */
typedef struct {
    int64_t a, b;           /* the motif pair */
    int32_t len;            /* its length */
    int32_t count;          /* members written */
    double radius;          /* D times the pair's FP64 distance */
} mad_motif_set;

MAD_API mad_status mad_motif_sets(mad_ctx *ctx, int32_t series, int32_t k, double D, int32_t cap,
                                  mad_motif_set *sets, int64_t *members, int32_t *n_out);

/* The k x m block (ranks 1..k, columns 1..m) of dkm_{lmin,lmax}: per length
 * and column, offsets ranked by m-th best-match distance descending (ties:
 * smaller offset) with pairwise non-trivial picks; across lengths each cell
 * keeps the largest dist / sqrt(len), ties to the longer length (Alg. 9).
 * out must hold k * m entries, written rank-major (out[(r-1)*m + (c-1)]);
 * *n_out = k * m. Requires k <= k_max, m <= m_max. */
MAD_API mad_status mad_discords(mad_ctx *ctx, int32_t series, int32_t k, int32_t m,
                                mad_discord *out, int32_t *n_out);

/* Global-greedy variable-length m-th discords (a variant of Sec. 6's
 * Top-k m-th discords with the per-rank merge of Algorithm 9 replaced by one
 * ranking over all lengths): for each column c in 1..m, every (offset i,
 * length l) with a c-th best match is a candidate of score
 * NN_l^c[i] / sqrt(l); candidates are taken by score descending, then longer
 * length, then smaller offset, each accepted unless |i - i'| <=
 * max(E(l), E(l')) for an accepted (i', l'), until k are accepted. Unlike
 * mad_discords, two picks never overlap by more than the exclusion zone,
 * whatever their lengths. Needs a mode-0 profile made with keep_profiles.
 * out must hold k * m entries, rank-major as for mad_discords (cells without
 * a candidate have off = -1, len = 0, NaN distances); dist_recheck is the
 * FP64 re-check. Requires 1 <= k <= 64, 1 <= m <= m_max. Errors: MAD_EINVAL
 * for bad arguments or a profile without keep_profiles, MAD_ESTATE before
 * mad_profile or in mode 1 or 2, MAD_ENOMEM when the scratch
 * (16 B per (column, length, 256 offsets) tile) cannot be allocated. */
MAD_API mad_status mad_discords_global(mad_ctx *ctx, int32_t series, int32_t k, int32_t m,
                                       mad_discord *out, int32_t *n_out);

/* dkm_{lmin,lmax} built the way Algorithms 7 and 8 print it (the
 * "streamed" form), then merged across lengths by Algorithm 9: per length,
 * windows are visited by offset ascending; a window with a trivial match
 * (|i - o| <= E(l)) among the offsets present anywhere in the k x m matrix is
 * skipped; otherwise columns m down to 1 are tried with its j-th best-match
 * distance, and it enters the first column where it is larger than some
 * entry, at the first such rank (the entries below move down one rank, the
 * last leaves), so a window holds at most one cell. The result depends on
 * the visiting order and on m; mad_discords ranks each column on its own
 * instead. Needs a mode-0 profile made with keep_profiles. out: k * m
 * entries, rank-major as for mad_discords (an empty cell has off = -1,
 * len = 0); dist_recheck is the FP64 re-check. Requires 1 <= k <= 64,
 * 1 <= m <= m_max. Errors: MAD_EINVAL for bad arguments or a profile without
 * keep_profiles, MAD_ESTATE before mad_profile or in mode 1 or 2, MAD_ENOMEM
 * when the per-length tables (16 B per cell and length) cannot be
 * allocated. */
MAD_API mad_status mad_discords_streamed(mad_ctx *ctx, int32_t series, int32_t k, int32_t m,
                                         mad_discord *out, int32_t *n_out);

/* Copy VALMP of series `series` to host arrays of n - lmin + 1 entries:
 * raw distance, normalised distance, length, nearest-neighbour offset. */
MAD_API mad_status mad_valmp(mad_ctx *ctx, int32_t series, double *dist, double *norm,
                             int32_t *len, int64_t *nn);

/* Copy the matrix profile of series `series` at one length len in
 * [lmin, lmax] (needs keep_profiles): mp/ip have n_len entries, nnd/nnj
 * n_len * m_max (row-major, m fastest). Any output pointer may be NULL. */
MAD_API mad_status mad_matrix_profile(mad_ctx *ctx, int32_t series, int32_t len, double *mp,
                                      int64_t *ip, double *nnd, int64_t *nnj);

/* Per-length pruning counters of series `series`: writes min(cap, |L|)
 * entries and |L| to *n_out. */
MAD_API mad_status mad_stats(mad_ctx *ctx, int32_t series, mad_length_stats *out, int32_t cap,
                             int32_t *n_out);

/* Largest ncells * m_max of one mad_mth_nn_dist_noalloc call: the number of
 * (cell, rank) slots in its fixed scratch (1024 slots, about 0.8 MB of
 * device memory per device, linked into the library). */
#define MAD_NOALLOC_MAX_SLOTS 1024

/* The m-th best-match distance of listed windows, recomputed directly in
 * FP64 from a full distance profile (Eq. DIST with two-pass window
 * statistics; Def. "m-th best match"), i.e. the computation
 * behind mad_discords' dist_recheck, without allocating any memory. The
 * paper has no counterpart of this function: it serves callers that cannot
 * allocate device memory during the call (memory held in a caching
 * allocator's pools, latency-bound code that cannot afford cudaFree's
 * device-wide wait, or a fixed footprint known up front).
 *   x      device, n doubles: the series (current device's memory).
 *   cells  host, ncells x 3 int32, row-major (off, len, m): window
 *          [off, off + len) and the rank m of the best match wanted.
 *   m_max  the largest m among the cells, in [1, 64]; ncells * m_max must
 *          not exceed MAD_NOALLOC_MAX_SLOTS (else MAD_EINVAL, nothing run).
 *   excl_num / excl_den  exclusion zone E(len) = ceil(len * num / den).
 *   out    device, ncells doubles: the distances (+inf when the window has
 *          fewer than m non-trivial partners).
 *   stream the CUDA stream to use (NULL: legacy default stream).
 * Errors: MAD_EINVAL for a bad argument or cell (checked on the host before
 * any GPU work, or x / out not device memory of the current device),
 * MAD_ECUDA for a failed CUDA call; mad_last_error(NULL) gives the text.
 * n must not exceed 2^31 (offsets are 32-bit in the kernels; else MAD_EINVAL).
 * The call makes no cudaMalloc / cudaFree or other allocating call. Its
 * scratch is one statically sized device array per device; every call looks
 * up the array's address in the calling context (so a cudaDeviceReset in
 * between is harmless), and the first call in a context loads the library's
 * device code there, which is set-up work: make that first call before any
 * stream capture begins. The scratch needs no zero initialisation. All calls on a device
 * share the one scratch, so calls that overlap in time (other streams or
 * host threads) race: order them. Synchronous with respect to the host. */
MAD_API mad_status mad_mth_nn_dist_noalloc(const double *x, int64_t n, const int32_t *cells,
                                           int32_t ncells, int32_t m_max, int32_t excl_num,
                                           int32_t excl_den, double *out, void *stream);

/* Pruning observation at options.observe_len (Sec. 7.2 diagnostics), for
 * the n - observe_len + 1 rows at that length, host arrays:
 *   gap[i] = maxLB - minED: the row's bound (Eq. LB from its p-th stored
 *            entry) minus its smallest stored distance; > 0 exactly when
 *            the stored entries certify the row's nearest neighbour;
 *   tlb[i] = mean over its stored entries of LB / ED (Eq. LB with the
 *            entry's correlation at the row's base length over the entry's
 *            distance at observe_len), the tightness of the lower bound;
 * NaN for flat rows and rows without stored entries. Needs a profile whose
 * range contains observe_len with lmin < observe_len (MAD_ESTATE otherwise).
 * Either pointer may be NULL. */
MAD_API mad_status mad_observe(mad_ctx *ctx, int32_t series, double *gap, double *tlb);

/* Test hook for the failure path (no counterpart in the paper). Sets, for
 * the whole process, how many times each wavefront wait of the
 * matrix-profile kernel (the hand-over of boundary values between the warps
 * of a block) tries before it gives up; a negative value restores the
 * kernel's own limit (the default, about 10^6 tries). With 0 every such wait
 * gives up at once: the kernel still keeps every access in bounds and runs
 * to its end, the results of that profile are meaningless, and mad_profile
 * returns MAD_ETIMEOUT. The waits that hand out work units keep their own
 * limit. Meant for tests; takes effect at the next mad_profile. */
MAD_API void mad_debug_wavefront_wait_limit(int32_t tries);

/* Test hook for the error model (no counterpart in the paper). When on (for
 * the whole process, from the next mad_profile), every stored entry whose
 * correlation carries an error bound -- the FP32 recurrence's, or the direct
 * path's -- is re-evaluated in FP64 as soon as it is selected, so that
 * mad_length_stats.dq_ratio_max records the largest observed error over
 * its bound for all of them, not only for the reported entries near
 * distance 0. Results stay exact; the profile is slower. */
MAD_API void mad_debug_audit_error_bounds(int32_t on);

/* Process-wide switch for the CUDA-graph replay of repeated profiles
 * (default on). Off: every profile launches its kernels one by one (the
 * workspace is still reused). Takes effect at the next mad_profile. */
MAD_API void mad_set_graphs(int32_t on);

/* Process-wide switch of how the tensor-core path (MAD_SPLIT_TC) forms its
 * column operand. 0 (default): producer warps of the tensor-core kernel
 * build each 256 x 64 column tile in shared memory from the series. 1 (p <=
 * 16): a prep kernel writes each 256-column tile's values once per length
 * as eight shifted FP16-pair copies, and the tensor-core kernel loads each
 * chunk's tile by one TMA tensor load (Hankel rows 16 bytes apart), with
 * eight epilogue warps. Results are the same bit for bit (the same FP16
 * pairs and products; ties between equal keys go to the smaller column
 * either way). Form 1 is faster for an isolated launch (3.2 against 4.2 ms
 * on a 262,144-point series) but slower inside the profile pipeline, where
 * its 64 KB of column tile per row tile and chunk compete for L2 with the
 * seed rows streamed beside it. Takes effect at the next mad_profile; form
 * 1 falls back to form 0 when the driver refuses the TMA descriptor.
 * Sec. "Computing The Matrix Profile" (the recomputed rows' sliding dot
 * products). */
MAD_API void mad_debug_tc_tma(int32_t on);

/* Process-wide switch of the launch autotuner (default on). On: the first
 * profile of a series of at most 32768 windows in a new size bucket (log2 of
 * the window count, log2 of lmin, p, precision, mode) times a short trial
 * profile for each candidate band height (1024, 512, 256 rows) and, on the
 * tensor-core path, each direct-path routing threshold, and keeps the
 * fastest for that bucket for the rest of the process. Off: the defaults
 * (the tallest band that fits, the default routing). Results do not depend
 * on the choice beyond FP32 rounding within the stated bounds. */
MAD_API void mad_set_autotune(int32_t on);

/* Human-readable description of the last error on ctx (or of the calling
 * thread's last mad_create* or mad_mth_nn_dist_noalloc error when ctx is
 * NULL). Never NULL. */
MAD_API const char *mad_last_error(const mad_ctx *ctx);

/* Release the context and its device memory. NULL-safe. */
MAD_API void mad_destroy(mad_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* MAD_H */
