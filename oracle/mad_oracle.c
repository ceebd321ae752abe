/*
 * mad_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, FP64 CPU restatement of what the exact variable-length
 * matrix profile (VALMOD / MAD, "Matrix Profile Goes MAD") computes. Only the
 * test suite, the smoke check and the benchmark's CPU-baseline leg may load
 * this library. It shares no code, header, table or helper with the CUDA
 * path and must never be used as a fallback for it.
 *
 * Every result with a plain definition is that definition written out:
 *   - window mean / population standard deviation by a two-pass loop
 *     (Sec. 4.3, the mu and sigma used by the distance formula);
 *   - the z-normalised Euclidean distance through the Pearson correlation
 *     (Eq. DIST), and directly from z-normalised windows (Def. of a motif
 *     pair, "z-normalized Euclidean distance");
 *   - distance profiles with the trivial-match exclusion zone (Def. distance
 *     profile, Sec. 2 "exclusion zone");
 *   - matrix profile / index and m-th best match per window (Def. matrix
 *     profile, Def. m-th best match);
 *   - the variable-length matrix profile VALMP (Algorithm 2 updateVALMP);
 *   - the lower bound of Eq. LB and the pruned VALMOD iteration that uses it
 *     (Algorithms 1, 3, 4 and 10), restated in the reading documented below;
 *   - the top-k motif and Top-k m-th discord read-outs (Sec. 5-6, Algorithms
 *     5, 8 and 9, in the deterministic reading documented below);
 *   - the paper-literal pruned iterations: motif mode (Algorithm 1 with
 *     ComputeSubMP, Algorithm 4) and the discords with Algorithm 10's
 *     pruning (driven by Algorithm 7);
 *   - motif sets (Algorithm 6), the pruning observation (Sec. 7.2), and the
 *     discord ranking variants (a global greedy over every offset and length,
 *     and dkm_l streamed as Algorithms 7 and 8 print it).
 *
 * Conventions: offsets are 0-based; a window of length l starts at i and
 * covers x[i .. i+l-1]; n_l = n - l + 1 windows exist. A pair (i, j) is a
 * trivial match iff |i - j| <= E(l) with E(l) = ceil(l * num / den).
 * Arithmetic is IEEE FP64, built without FMA contraction so that x86 and Arm
 * give identical bits.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <omp.h>

typedef int64_t i64;

/* ---------------------------------------------------------------- basics */

/* Exclusion half-width E(l) = ceil(l * num / den) (Sec. 2: the paper sets the
 * zone heuristically to l/2; the workloads here use l/4). */
i64 orc_excl(int l, int num, int den)
{
    return ((i64)l * num + den - 1) / den;
}

/* Mean and population standard deviation of x[i .. i+l-1], two passes
 * (mu = s / l and sigma = sqrt(ss / l - mu^2) in Sec. 4.3, computed here
 * without running sums). */
void orc_window_stats(const double *x, i64 n, int l, i64 i, double *mu, double *sigma)
{
    (void)n;
    double s = 0.0;
    for (int t = 0; t < l; ++t) s += x[i + t];
    double m = s / l;
    double v = 0.0;
    for (int t = 0; t < l; ++t) {
        double d = x[i + t] - m;
        v += d * d;
    }
    *mu = m;
    *sigma = sqrt(v / l);
}

/* A window is flat iff all of its values are equal. The paper does not
 * treat flat windows; the reading used throughout: two flat windows have
 * correlation 1, a flat and a non-flat window have correlation 0. */
int orc_is_flat(const double *x, i64 n, int l, i64 i)
{
    (void)n;
    for (int t = 1; t < l; ++t)
        if (x[i + t] != x[i]) return 0;
    return 1;
}

/* Pearson correlation q of the windows at i and j (the quantity inside
 * Eq. DIST: (QT - l mu_i mu_j) / (l sigma_i sigma_j)), evaluated as the
 * centred dot product divided by l sigma_i sigma_j, clamped to [-1, 1]. */
double orc_pearson(const double *x, i64 n, int l, i64 i, i64 j)
{
    int fi = orc_is_flat(x, n, l, i), fj = orc_is_flat(x, n, l, j);
    if (fi && fj) return 1.0;
    if (fi || fj) return 0.0;
    double mi, si, mj, sj;
    orc_window_stats(x, n, l, i, &mi, &si);
    orc_window_stats(x, n, l, j, &mj, &sj);
    double c = 0.0;
    for (int t = 0; t < l; ++t) c += (x[i + t] - mi) * (x[j + t] - mj);
    double q = c / ((double)l * (si * sj));
    if (q > 1.0) q = 1.0;
    if (q < -1.0) q = -1.0;
    return q;
}

/* Eq. DIST: d = sqrt(2 l (1 - q)). */
double orc_dist(const double *x, i64 n, int l, i64 i, i64 j)
{
    double q = orc_pearson(x, n, l, i, j);
    return sqrt(2.0 * l * (1.0 - q));
}

/* The same distance straight from its definition: the Euclidean norm of the
 * difference of the two z-normalised windows (Def. motif pair). Flat windows
 * z-normalise to all-zero vectors here, which is NOT the reading above; the
 * brute-force tier only calls it on non-flat windows. */
double orc_dist_direct(const double *x, i64 n, int l, i64 i, i64 j)
{
    double mi, si, mj, sj;
    orc_window_stats(x, n, l, i, &mi, &si);
    orc_window_stats(x, n, l, j, &mj, &sj);
    double s = 0.0;
    for (int t = 0; t < l; ++t) {
        double a = (x[i + t] - mi) / si;
        double b = (x[j + t] - mj) / sj;
        s += (a - b) * (a - b);
    }
    (void)n;
    return sqrt(s);
}

/* Eq. LB: lower bound on the distance at length l_new >= l_b between the
 * window whose profile is kept (the row, statistics sigma_row at both
 * lengths) and another window, given their correlation q at length l_b.
 *   LB = sqrt(l_b)          * sigma_row(l_b) / sigma_row(l_new)   if q <= 0
 *   LB = sqrt(l_b (1-q^2))  * sigma_row(l_b) / sigma_row(l_new)   otherwise */
double orc_lower_bound(int l_b, double q, double sigma_row_lb, double sigma_row_lnew)
{
    double base = (q <= 0.0) ? sqrt((double)l_b) : sqrt((double)l_b * (1.0 - q * q));
    return base * sigma_row_lb / sigma_row_lnew;
}

/* --------------------------------------------------------- profiles / MP */

/* Distance profile of window i at length l (Def. distance profile): out[j]
 * for j in [0, n_l), +inf for trivial matches |i - j| <= E(l). */
void orc_distance_profile(const double *x, i64 n, int l, int num, int den, i64 i, double *out)
{
    i64 nl = n - l + 1, E = orc_excl(l, num, den);
    for (i64 j = 0; j < nl; ++j) {
        i64 dd = i > j ? i - j : j - i;
        out[j] = (dd <= E) ? INFINITY : orc_dist(x, n, l, i, j);
    }
}

typedef struct { double d; i64 j; } dj_t;

static int cmp_dj(const void *a, const void *b)
{
    const dj_t *u = (const dj_t *)a, *v = (const dj_t *)b;
    if (u->d < v->d) return -1;
    if (u->d > v->d) return 1;
    return (u->j < v->j) ? -1 : (u->j > v->j);
}

/* Sort a profile's non-trivial entries by (distance, offset) ascending and
 * return how many there are. */
static i64 sorted_profile(const double *prof, i64 nl, dj_t *buf)
{
    i64 c = 0;
    for (i64 j = 0; j < nl; ++j)
        if (isfinite(prof[j])) { buf[c].d = prof[j]; buf[c].j = j; ++c; }
    qsort(buf, (size_t)c, sizeof(dj_t), cmp_dj);
    return c;
}

/* Matrix profile at length l (Def. matrix profile) plus the m-th best match
 * for m = 1..m_max (Def. m-th best match): for every window i,
 *   mp[i]   = min_j d(i, j) over non-trivial j,   ip[i] = the smallest such j,
 *   nnd[i*m_max + m-1] = m-th smallest non-trivial distance (ties: smaller j),
 *   nnj[i*m_max + m-1] = its offset;  +inf / -1 when i has fewer than m
 *   non-trivial neighbours. */
void orc_matrix_profile(const double *x, i64 n, int l, int num, int den, int m_max,
                        double *mp, i64 *ip, double *nnd, i64 *nnj)
{
    i64 nl = n - l + 1;
#pragma omp parallel
    {
        double *prof = (double *)malloc(sizeof(double) * (size_t)nl);
        dj_t *buf = (dj_t *)malloc(sizeof(dj_t) * (size_t)nl);
#pragma omp for schedule(dynamic, 4)
        for (i64 i = 0; i < nl; ++i) {
            orc_distance_profile(x, n, l, num, den, i, prof);
            i64 c = sorted_profile(prof, nl, buf);
            mp[i] = c > 0 ? buf[0].d : INFINITY;
            ip[i] = c > 0 ? buf[0].j : -1;
            for (int m = 0; m < m_max; ++m) {
                if (nnd) nnd[i * m_max + m] = (m < c) ? buf[m].d : INFINITY;
                if (nnj) nnj[i * m_max + m] = (m < c) ? buf[m].j : -1;
            }
        }
        free(prof);
        free(buf);
    }
}

/* Matrix-profile quantities of one window only (the same definitions as
 * orc_matrix_profile, for sampled checks on large inputs). */
void orc_row(const double *x, i64 n, int l, int num, int den, int m_max, i64 i,
             double *mp, i64 *ip, double *nnd, i64 *nnj)
{
    i64 nl = n - l + 1;
    double *prof = (double *)malloc(sizeof(double) * (size_t)nl);
    dj_t *buf = (dj_t *)malloc(sizeof(dj_t) * (size_t)nl);
    orc_distance_profile(x, n, l, num, den, i, prof);
    i64 c = sorted_profile(prof, nl, buf);
    *mp = c > 0 ? buf[0].d : INFINITY;
    *ip = c > 0 ? buf[0].j : -1;
    for (int m = 0; m < m_max; ++m) {
        nnd[m] = (m < c) ? buf[m].d : INFINITY;
        nnj[m] = (m < c) ? buf[m].j : -1;
    }
    free(prof);
    free(buf);
}

/* orc_row for a list of windows at one length, in parallel over windows
 * (same definitions; used to time the oracle on a sample of a workload). */
void orc_rows(const double *x, i64 n, int l, int num, int den, const i64 *rows, i64 nrows, double *mp, i64 *ip)
{
    i64 nl = n - l + 1;
#pragma omp parallel
    {
        double *prof = (double *)malloc(sizeof(double) * (size_t)nl);
        dj_t *buf = (dj_t *)malloc(sizeof(dj_t) * (size_t)nl);
#pragma omp for schedule(dynamic, 1)
        for (i64 r = 0; r < nrows; ++r) {
            orc_distance_profile(x, n, l, num, den, rows[r], prof);
            i64 c = sorted_profile(prof, nl, buf);
            mp[r] = c > 0 ? buf[0].d : INFINITY;
            ip[r] = c > 0 ? buf[0].j : -1;
        }
        free(prof);
        free(buf);
    }
}

int orc_num_threads(void)
{
    int t = 1;
#pragma omp parallel
    {
#pragma omp single
        t = omp_get_num_threads();
    }
    return t;
}

/* Algorithm 2 (updateVALMP) applied to one length: for i < n_l, if
 * MP[i]/sqrt(l) is strictly smaller than the stored normalised distance (or
 * none is stored yet) store the raw distance, the normalised one, l and the
 * nearest-neighbour offset. (The listing compares the raw distances field
 * against the normalised value and tests a non-existent VALMP.MP field; both
 * are read as the normalised-distance field.) */
void orc_valmp_update(i64 nl, int l, const double *mp, const i64 *ip,
                      double *dist, double *norm, int32_t *len, i64 *nn)
{
    double f = sqrt(1.0 / l);
    for (i64 i = 0; i < nl; ++i) {
        double nd = mp[i] * f;
        if (len[i] == 0 || nd < norm[i]) {
            dist[i] = mp[i];
            norm[i] = nd;
            len[i] = l;
            nn[i] = ip[i];
        }
    }
}

/* VALMP over [lmin, lmax] from independent per-length matrix profiles
 * (the plain definition the pruned method must reproduce). Outputs have
 * n_lmin entries; len[] must be zero-initialised by the caller. Optionally
 * stores every per-length m-th-NN table (for the discord read-out):
 * nnd_all[(l-lmin) * n_lmin * m_max + i * m_max + m-1]. */
void orc_valmp_plain(const double *x, i64 n, int lmin, int lmax, int num, int den, int m_max,
                     double *dist, double *norm, int32_t *len, i64 *nn,
                     double *nnd_all, i64 *nnj_all)
{
    i64 n0 = n - lmin + 1;
    double *mp = (double *)malloc(sizeof(double) * (size_t)n0);
    i64 *ip = (i64 *)malloc(sizeof(i64) * (size_t)n0);
    for (int l = lmin; l <= lmax; ++l) {
        i64 nl = n - l + 1;
        double *nd = nnd_all ? nnd_all + (i64)(l - lmin) * n0 * m_max : NULL;
        i64 *nj = nnj_all ? nnj_all + (i64)(l - lmin) * n0 * m_max : NULL;
        orc_matrix_profile(x, n, l, num, den, m_max, mp, ip, nd, nj);
        if (nd)
            for (i64 i = nl; i < n0; ++i)
                for (int m = 0; m < m_max; ++m) { nd[i * m_max + m] = NAN; nj[i * m_max + m] = -1; }
        orc_valmp_update(nl, l, mp, ip, dist, norm, len, nn);
    }
    free(mp);
    free(ip);
}

/* ------------------------------------------------------ pruned VALMOD */

/*
 * The pruned iteration (Algorithm 1 VALMOD with Algorithm 3
 * ComputeMatrixProfile, Algorithm 4 ComputeSubMP and Algorithm 10
 * Topkm_nextLength), in the "exact rows" reading:
 *
 *  - At lmin (and whenever a row is recomputed at length l) the row's full
 *    distance profile is evaluated. The row keeps the p non-trivial entries
 *    with the smallest Eq. LB; since the factor sigma_row(l_b)/sigma_row(l')
 *    is common to a row, that is the p entries of largest correlation q
 *    (ties: smaller offset), and the bound base is the p-th entry's
 *    sqrt(l_b (1 - max(q_p, 0)^2)). If the row has at most p non-trivial
 *    columns, every column is stored and the bound is +inf.
 *  - For each longer length l' the stored entries are re-evaluated exactly
 *    (updateDistAndLB); entries that became trivial (|i-j| <= E(l')) or fell
 *    off the end (j >= n_l') leave the minimum but not the bound.
 *  - The row's bound is B = base * sigma_row(l_b) / sigma_row(l')
 *    (rank preservation, Sec. 4.1). The row is valid ("certified") iff it has
 *    at least m_max remaining entries and the m_max-th smallest remaining
 *    distance is strictly below B (the minDist < maxLB test of Algorithm 4 and
 *    the mDist < maxLB test of Algorithm 10; "popMax" is read as a peek).
 *  - Every non-valid row is recomputed at l' (its base moves to l'); a flat
 *    row at l' is always recomputed. The paper instead recomputes only the
 *    rows that could hold the global motif (or enter the discord table) and
 *    falls back to a full matrix profile above n log p / log n of them; the
 *    exact-rows reading makes MP_l, the m-th best matches and VALMP exact
 *    for every offset.
 * Results equal orc_valmp_plain / orc_matrix_profile exactly (same distance
 * function), which is what the tests check. stats[(l-lmin)*3 + {0,1,2}] =
 * {rows alive at l, valid rows, recomputed rows}.
 */
/* Row validity test of Algorithms 4 and 10: with the row's remaining stored
 * distances sorted ascending (d_sorted[0..count)), the row is valid for the
 * m-th best match iff it has at least m of them and the m-th is strictly
 * below the row's bound (minDist < maxLB for m = 1, mDist < maxLB in
 * Algorithm 10). The listing's strict "<" is kept; the prose says "<=". */
int orc_row_valid(const double *d_sorted, int count, int m, double bound)
{
    return count >= m && d_sorted[m - 1] < bound;
}

typedef struct { double q; i64 j; } qj_t;

static int cmp_qj(const void *a, const void *b)
{
    const qj_t *u = (const qj_t *)a, *v = (const qj_t *)b;
    if (u->q > v->q) return -1;
    if (u->q < v->q) return 1;
    return (u->j < v->j) ? -1 : (u->j > v->j);
}

typedef struct {
    int base;          /* l_b */
    double sig_b;      /* sigma_row(l_b) */
    double bound_base; /* sqrt(l_b (1 - max(q_p,0)^2)), or +inf */
    int cnt;           /* stored entries */
    i64 *j;            /* p offsets */
} row_state;

/* Algorithm 3 restricted to one row at length l: full profile, MP, m-th
 * best matches, and the p smallest-LB entries. */
static void recompute_row(const double *x, i64 n, int l, int num, int den, int p, int m_max, i64 i,
                          row_state *st, double *mp, i64 *ip, double *nnd, i64 *nnj,
                          double *prof, dj_t *dbuf, qj_t *qbuf)
{
    i64 nl = n - l + 1, E = orc_excl(l, num, den);
    orc_distance_profile(x, n, l, num, den, i, prof);
    i64 c = sorted_profile(prof, nl, dbuf);
    mp[i] = c > 0 ? dbuf[0].d : INFINITY;
    ip[i] = c > 0 ? dbuf[0].j : -1;
    for (int m = 0; m < m_max; ++m) {
        nnd[i * m_max + m] = m < c ? dbuf[m].d : INFINITY;
        nnj[i * m_max + m] = m < c ? dbuf[m].j : -1;
    }
    i64 qc = 0;
    for (i64 j = 0; j < nl; ++j) {
        i64 dd = i > j ? i - j : j - i;
        if (dd <= E) continue;
        qbuf[qc].q = orc_pearson(x, n, l, i, j);
        qbuf[qc].j = j;
        ++qc;
    }
    qsort(qbuf, (size_t)qc, sizeof(qj_t), cmp_qj);
    st->cnt = (int)(qc < p ? qc : p);
    for (int e = 0; e < st->cnt; ++e) st->j[e] = qbuf[e].j;
    st->base = l;
    double mu;
    orc_window_stats(x, n, l, i, &mu, &st->sig_b);
    if (qc <= p) {
        st->bound_base = INFINITY;
    } else {
        double qp = qbuf[p - 1].q;
        if (qp < 0.0) qp = 0.0;
        st->bound_base = sqrt((double)l * (1.0 - qp * qp));
    }
}

/* Observation at one length obs_len (> lmin, optional; the paper's
 * pruning diagnostics, Sec. 7.2): for every row with stored entries, before
 * its recompute decision, obs_gap[i] = maxLB - minED = B - (smallest stored
 * distance) (> 0 exactly when the row is certified for its motif) and
 * obs_tlb[i] = mean over its stored entries of LB / ED, the tightness of
 * the lower bound, LB from Eq. LB with the entry's correlation at the row's
 * base length; NaN for flat rows and rows without entries. */
void orc_valmod_pruned(const double *x, i64 n, int lmin, int lmax, int num, int den, int p, int m_max,
                       double *dist, double *norm, int32_t *len, i64 *nn,
                       double *nnd_all, i64 *nnj_all, i64 *stats,
                       int obs_len, double *obs_gap, double *obs_tlb)
{
    i64 n0 = n - lmin + 1;
    row_state *st = (row_state *)calloc((size_t)n0, sizeof(row_state));
    i64 *jstore = (i64 *)malloc(sizeof(i64) * (size_t)(n0 * p));
    for (i64 i = 0; i < n0; ++i) st[i].j = jstore + i * p;
    double *mp = (double *)malloc(sizeof(double) * (size_t)n0);
    i64 *ip = (i64 *)malloc(sizeof(i64) * (size_t)n0);
    double *nnd = (double *)malloc(sizeof(double) * (size_t)(n0 * m_max));
    i64 *nnj = (i64 *)malloc(sizeof(i64) * (size_t)(n0 * m_max));

    for (int l = lmin; l <= lmax; ++l) {
        i64 nl = n - l + 1, E = orc_excl(l, num, den);
        i64 nvalid = 0, nrecomp = 0;
#pragma omp parallel reduction(+ : nvalid, nrecomp)
        {
            double *prof = (double *)malloc(sizeof(double) * (size_t)n0);
            dj_t *dbuf = (dj_t *)malloc(sizeof(dj_t) * (size_t)n0);
            qj_t *qbuf = (qj_t *)malloc(sizeof(qj_t) * (size_t)n0);
#pragma omp for schedule(dynamic, 8)
            for (i64 i = 0; i < nl; ++i) {
                int valid = 0;
                if (l == obs_len && obs_gap) {
                    obs_gap[i] = NAN;
                    obs_tlb[i] = NAN;
                }
                if (l > lmin && !orc_is_flat(x, n, l, i)) {
                    /* Algorithm 4 / 10 row loop: re-evaluate stored entries */
                    dj_t cand[64];
                    int c = 0;
                    for (int e = 0; e < st[i].cnt; ++e) {
                        i64 j = st[i].j[e];
                        i64 dd = i > j ? i - j : j - i;
                        if (j >= nl || dd <= E) continue;
                        cand[c].d = orc_dist(x, n, l, i, j);
                        cand[c].j = j;
                        ++c;
                    }
                    qsort(cand, (size_t)c, sizeof(dj_t), cmp_dj);
                    double mu, sig;
                    orc_window_stats(x, n, l, i, &mu, &sig);
                    double B = st[i].bound_base * st[i].sig_b / sig;
                    double dsort[64];
                    for (int e = 0; e < c; ++e) dsort[e] = cand[e].d;
                    if (l == obs_len && obs_gap && c > 0) {
                        obs_gap[i] = B - cand[0].d;
                        double tsum = 0.0;
                        int tc = 0;
                        for (int e = 0; e < c; ++e) {
                            if (!(cand[e].d > 0.0)) continue;
                            double qb = orc_pearson(x, n, st[i].base, i, cand[e].j);
                            tsum += orc_lower_bound(st[i].base, qb, st[i].sig_b, sig) / cand[e].d;
                            ++tc;
                        }
                        obs_tlb[i] = tc > 0 ? tsum / tc : NAN;
                    }
                    if (orc_row_valid(dsort, c, m_max, B)) {
                        valid = 1;
                        mp[i] = cand[0].d;
                        ip[i] = cand[0].j;
                        for (int m = 0; m < m_max; ++m) {
                            nnd[i * m_max + m] = cand[m].d;
                            nnj[i * m_max + m] = cand[m].j;
                        }
                    }
                }
                if (valid) {
                    ++nvalid;
                } else {
                    recompute_row(x, n, l, num, den, p, m_max, i, &st[i], mp, ip, nnd, nnj,
                                  prof, dbuf, qbuf);
                    ++nrecomp;
                }
            }
            free(prof);
            free(dbuf);
            free(qbuf);
        }
        orc_valmp_update(nl, l, mp, ip, dist, norm, len, nn);
        if (nnd_all) {
            double *nd = nnd_all + (i64)(l - lmin) * n0 * m_max;
            i64 *nj = nnj_all + (i64)(l - lmin) * n0 * m_max;
            for (i64 i = 0; i < n0; ++i)
                for (int m = 0; m < m_max; ++m) {
                    nd[i * m_max + m] = i < nl ? nnd[i * m_max + m] : NAN;
                    nj[i * m_max + m] = i < nl ? nnj[i * m_max + m] : -1;
                }
        }
        if (stats) {
            stats[(l - lmin) * 3 + 0] = nl;
            stats[(l - lmin) * 3 + 1] = nvalid;
            stats[(l - lmin) * 3 + 2] = nrecomp;
        }
    }
    free(st);
    free(jstore);
    free(mp);
    free(ip);
    free(nnd);
    free(nnj);
}

static i64 iabs64(i64 v) { return v < 0 ? -v : v; }

/* The paper-literal pruned iteration (Algorithm 1 with ComputeSubMP,
 * Algorithm 4), whose guarantee is the motif of every length, not every
 * row: at lmin the full matrix profile (Algorithm 3); at every longer length
 *  - each row's stored entries are re-evaluated (trivial / out-of-range ones
 *    skipped); a row is valid iff its smallest stored distance is strictly
 *    below its bound B = bound_base * sigma_b / sigma_l (Eq. LB with rank
 *    preservation); valid rows give SubMP[i] exactly and minDistAbs is the
 *    smallest of them; the others are non-valid with lbMax = B (a flat row
 *    has no usable bound: non-valid with lbMax = 0);
 *  - bBestM = minDistAbs < min over non-valid rows of lbMax;
 *  - if not, and fewer than n log(p) / log(n) rows are non-valid (n = |T|,
 *    natural logarithms; the ratio does not depend on the base), every
 *    non-valid row with lbMax < minDistAbs is recomputed in full (its
 *    profile minimum, new stored entries and bound), and bBestM holds;
 *  - if bBestM still fails, the full matrix profile at l is computed
 *    (Algorithm 1's ComputeMatrixProfile branch: every row recomputed);
 *  - VALMP is updated with the defined SubMP values only.
 * Rows that stay undefined keep their (extended) stored entries. Outputs:
 * VALMP (len[] zero-initialised by the caller); optionally SubMP per length
 * submp_all[(l-lmin)*n_lmin + i] (NaN where undefined) and stats
 * [(l-lmin)*5 + {0..4}] = rows, valid, non-valid, recomputed, full (0/1). */
void orc_valmod_motif(const double *x, i64 n, int lmin, int lmax, int num, int den, int p,
                      double *dist, double *norm, int32_t *len, i64 *nn, double *submp_all, i64 *stats)
{
    i64 n0 = n - lmin + 1;
    row_state *st = (row_state *)calloc((size_t)n0, sizeof(row_state));
    i64 *jstore = (i64 *)malloc(sizeof(i64) * (size_t)(n0 * p));
    for (i64 i = 0; i < n0; ++i) st[i].j = jstore + i * p;
    double *mp = (double *)malloc(sizeof(double) * (size_t)n0);
    i64 *ip = (i64 *)malloc(sizeof(i64) * (size_t)n0);
    double *nnd = (double *)malloc(sizeof(double) * (size_t)n0);
    i64 *nnj = (i64 *)malloc(sizeof(i64) * (size_t)n0);
    double *lbmax = (double *)malloc(sizeof(double) * (size_t)n0);
    signed char *state = (signed char *)malloc((size_t)n0);   /* 1 valid, 0 non-valid */
    const double limit = (double)n * log((double)p) / log((double)n);

    for (int l = lmin; l <= lmax; ++l) {
        i64 nl = n - l + 1, E = orc_excl(l, num, den);
        i64 nvalid = 0, nnon = 0, nrecomp = 0;
        int full = (l == lmin);
        double min_dist_abs = INFINITY, min_lb_abs = INFINITY;
        if (!full) {
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : nvalid, nnon) reduction(min : min_dist_abs, min_lb_abs)
            for (i64 i = 0; i < nl; ++i) {
                mp[i] = INFINITY;
                ip[i] = -1;
                if (orc_is_flat(x, n, l, i)) {
                    state[i] = 0;
                    lbmax[i] = 0.0;
                    ++nnon;
                    min_lb_abs = fmin(min_lb_abs, 0.0);
                    continue;
                }
                double best = INFINITY;
                i64 bj = -1;
                for (int e = 0; e < st[i].cnt; ++e) {
                    i64 j = st[i].j[e];
                    i64 dd = i > j ? i - j : j - i;
                    if (j >= nl || dd <= E) continue;
                    double d = orc_dist(x, n, l, i, j);
                    if (d < best || (d == best && j < bj)) { best = d; bj = j; }
                }
                double mu, sig;
                orc_window_stats(x, n, l, i, &mu, &sig);
                double B = st[i].bound_base * st[i].sig_b / sig;
                if (bj >= 0 && best < B) {
                    state[i] = 1;
                    mp[i] = best;
                    ip[i] = bj;
                    ++nvalid;
                    min_dist_abs = fmin(min_dist_abs, best);
                } else {
                    state[i] = 0;
                    lbmax[i] = B;
                    ++nnon;
                    min_lb_abs = fmin(min_lb_abs, B);
                }
            }
            int best_m = min_dist_abs < min_lb_abs;
            if (!best_m && (double)nnon < limit) {
#pragma omp parallel reduction(+ : nrecomp)
                {
                    double *prof = (double *)malloc(sizeof(double) * (size_t)n0);
                    dj_t *dbuf = (dj_t *)malloc(sizeof(dj_t) * (size_t)n0);
                    qj_t *qbuf = (qj_t *)malloc(sizeof(qj_t) * (size_t)n0);
#pragma omp for schedule(dynamic, 1)
                    for (i64 i = 0; i < nl; ++i) {
                        if (state[i] != 0 || !(lbmax[i] < min_dist_abs)) continue;
                        recompute_row(x, n, l, num, den, p, 1, i, &st[i], mp, ip, nnd, nnj, prof, dbuf, qbuf);
                        ++nrecomp;
                    }
                    free(prof);
                    free(dbuf);
                    free(qbuf);
                }
                best_m = 1;
            }
            if (!best_m) full = 1;
        }
        if (full) {
            nrecomp = 0;
#pragma omp parallel reduction(+ : nrecomp)
            {
                double *prof = (double *)malloc(sizeof(double) * (size_t)n0);
                dj_t *dbuf = (dj_t *)malloc(sizeof(dj_t) * (size_t)n0);
                qj_t *qbuf = (qj_t *)malloc(sizeof(qj_t) * (size_t)n0);
#pragma omp for schedule(dynamic, 8)
                for (i64 i = 0; i < nl; ++i) {
                    recompute_row(x, n, l, num, den, p, 1, i, &st[i], mp, ip, nnd, nnj, prof, dbuf, qbuf);
                    ++nrecomp;
                }
                free(prof);
                free(dbuf);
                free(qbuf);
            }
        }
        /* VALMP with the defined values only */
        double f = sqrt(1.0 / l);
        for (i64 i = 0; i < nl; ++i) {
            if (!isfinite(mp[i]) || ip[i] < 0) continue;
            double nd = mp[i] * f;
            if (len[i] == 0 || nd < norm[i]) {
                dist[i] = mp[i];
                norm[i] = nd;
                len[i] = l;
                nn[i] = ip[i];
            }
        }
        if (submp_all) {
            double *o = submp_all + (i64)(l - lmin) * n0;
            for (i64 i = 0; i < n0; ++i) o[i] = (i < nl && ip[i] >= 0) ? mp[i] : NAN;
        }
        if (stats) {
            i64 *s5 = stats + (i64)(l - lmin) * 5;
            s5[0] = nl;
            s5[1] = full && l == lmin ? 0 : nvalid;
            s5[2] = full && l == lmin ? nl : nnon;
            s5[3] = nrecomp;
            s5[4] = full;
        }
    }
    free(st);
    free(jstore);
    free(mp);
    free(ip);
    free(nnd);
    free(nnj);
    free(lbmax);
    free(state);
}

/* Variable-length motif sets (Sec. "Finding Motif Sets", Algorithm 6): for
 * each motif pair s (offsets a_s, b_s at length l_s with distance d_s, in
 * the order given) and radius r_s = D * d_s, the set is grown from the pair:
 *  - candidates: windows j at l_s with min(d(a_s, j), d(b_s, j)) <= r_s that
 *    are not trivial matches of a_s or b_s (|j - a_s|, |j - b_s| > E(l_s)),
 *    and do not lie within max(E(l_s), E(l_t)) of a member of an earlier set
 *    t (the used subsequences leave the search space, so sets never meet);
 *  - a_s and b_s are members first; then candidates by (min distance,
 *    offset) ascending, each accepted unless within E(l_s) of an accepted
 *    member (the merge that removes trivial matches), until cap members.
 * Writes members[s * cap + 0..counts[s]) (a_s, b_s, then in acceptance
 * order). Distances are the FP64 distance profiles by definition. */
void orc_motif_sets(const double *x, i64 n, int k, const i64 *a, const i64 *b, const int32_t *len,
                    const double *dist, double D, int num, int den, int cap, i64 *members, int32_t *counts)
{
    i64 nmax = n;
    double *pa = (double *)malloc(sizeof(double) * (size_t)nmax);
    double *pb = (double *)malloc(sizeof(double) * (size_t)nmax);
    dj_t *cand = (dj_t *)malloc(sizeof(dj_t) * (size_t)nmax);
    for (int s = 0; s < k; ++s) {
        int l = len[s];
        i64 nl = n - l + 1, E = orc_excl(l, num, den);
        double r = D * dist[s];
        orc_distance_profile(x, n, l, num, den, a[s], pa);
        orc_distance_profile(x, n, l, num, den, b[s], pb);
        i64 c = 0;
        for (i64 j = 0; j < nl; ++j) {
            if (iabs64(j - a[s]) <= E || iabs64(j - b[s]) <= E) continue;
            double d = fmin(pa[j], pb[j]);
            if (!(d <= r)) continue;
            int used = 0;
            for (int t = 0; t < s && !used; ++t) {
                i64 Et = orc_excl(len[t], num, den);
                i64 Em = E > Et ? E : Et;
                for (int u = 0; u < counts[t] && !used; ++u)
                    if (iabs64(j - members[(i64)t * cap + u]) <= Em) used = 1;
            }
            if (used) continue;
            cand[c].d = d;
            cand[c].j = j;
            ++c;
        }
        qsort(cand, (size_t)c, sizeof(dj_t), cmp_dj);
        i64 *m = members + (i64)s * cap;
        int cnt = 0;
        if (cnt < cap) m[cnt++] = a[s];
        if (cnt < cap) m[cnt++] = b[s];
        for (i64 t = 0; t < c && cnt < cap; ++t) {
            int ok = 1;
            for (int u = 0; u < cnt && ok; ++u)
                if (iabs64(cand[t].j - m[u]) <= E) ok = 0;
            if (ok) m[cnt++] = cand[t].j;
        }
        counts[s] = cnt;
    }
    free(pa);
    free(pb);
    free(cand);
}

/* ------------------------------------------------------------ read-outs */

typedef struct { double key; i64 i; } ki_t;

static int cmp_key_asc(const void *a, const void *b)
{
    const ki_t *u = (const ki_t *)a, *v = (const ki_t *)b;
    if (u->key < v->key) return -1;
    if (u->key > v->key) return 1;
    return (u->i < v->i) ? -1 : (u->i > v->i);
}

static int cmp_key_desc(const void *a, const void *b)
{
    const ki_t *u = (const ki_t *)a, *v = (const ki_t *)b;
    if (u->key > v->key) return -1;
    if (u->key < v->key) return 1;
    return (u->i < v->i) ? -1 : (u->i > v->i);
}


/* Top-k length-normalised motif pairs from VALMP (the ranking kept by
 * Algorithm 5's heap of best pairs, with the trivial-match removal of the
 * top-k unfolding in Sec. 7): visit offsets by (normalised distance, offset)
 * ascending; accept the pair {i, nn[i]} of length len[i] unless one of its
 * two offsets lies within max(E(len), E(len')) of an offset of an already
 * accepted pair of length len'. Writes a = min(i, nn), b = max, length, raw
 * and normalised distance; returns the number accepted (<= k). */
int orc_topk_motifs(i64 n0, const double *dist, const double *norm, const int32_t *len, const i64 *nn,
                    int num, int den, int k,
                    i64 *out_a, i64 *out_b, int32_t *out_len, double *out_d, double *out_nd)
{
    ki_t *ord = (ki_t *)malloc(sizeof(ki_t) * (size_t)n0);
    i64 c = 0;
    for (i64 i = 0; i < n0; ++i)
        if (len[i] > 0 && nn[i] >= 0 && isfinite(norm[i])) { ord[c].key = norm[i]; ord[c].i = i; ++c; }
    qsort(ord, (size_t)c, sizeof(ki_t), cmp_key_asc);
    int got = 0;
    for (i64 t = 0; t < c && got < k; ++t) {
        i64 i = ord[t].i, a = i, b = nn[i];
        int L = len[i];
        int ok = 1;
        for (int g = 0; g < got && ok; ++g) {
            i64 E = orc_excl(L, num, den), E2 = orc_excl(out_len[g], num, den);
            if (E2 > E) E = E2;
            if (iabs64(a - out_a[g]) <= E || iabs64(a - out_b[g]) <= E ||
                iabs64(b - out_a[g]) <= E || iabs64(b - out_b[g]) <= E)
                ok = 0;
        }
        if (!ok) continue;
        out_a[got] = a < b ? a : b;
        out_b[got] = a < b ? b : a;
        out_len[got] = L;
        out_d[got] = dist[i];
        out_nd[got] = norm[i];
        ++got;
    }
    free(ord);
    return got;
}

/* Column m of dkm_l (Sec. 6.1): the Top-k m-th discords of one length.
 * score(i) = m-th best-match distance of window i; offsets with no m-th best
 * match (score not finite) are skipped. Visit by (score desc, offset asc) and
 * accept i unless |i - i'| <= E(l) for an accepted i' (the pairwise
 * non-trivial requirement on dkm_l). Each column is computed on its own
 * (the listing's streaming insert of Algorithm 8 depends on visiting order,
 * so the columns are read as independent rankings). Returns the count. */
int orc_discords_one_length(i64 nl, const double *score, const i64 *nbr, int l, int num, int den, int k,
                            i64 *out_off, double *out_d, i64 *out_nn)
{
    ki_t *ord = (ki_t *)malloc(sizeof(ki_t) * (size_t)(nl > 0 ? nl : 1));
    i64 c = 0;
    for (i64 i = 0; i < nl; ++i)
        if (isfinite(score[i])) { ord[c].key = score[i]; ord[c].i = i; ++c; }
    qsort(ord, (size_t)c, sizeof(ki_t), cmp_key_desc);
    i64 E = orc_excl(l, num, den);
    int got = 0;
    for (i64 t = 0; t < c && got < k; ++t) {
        i64 i = ord[t].i;
        int ok = 1;
        for (int g = 0; g < got; ++g)
            if (iabs64(i - out_off[g]) <= E) { ok = 0; break; }
        if (!ok) continue;
        out_off[got] = i;
        out_d[got] = score[i];
        out_nn[got] = nbr ? nbr[i] : -1;
        ++got;
    }
    free(ord);
    return got;
}

/* Global-greedy variable-length m-th discords (the variant of Algorithm 9's
 * per-rank merge): for column m, every (i, l) with an m-th best match is a
 * candidate with score NN_l^m[i] / sqrt(l); candidates are visited by score
 * descending, then length descending (the ">=" of Algorithm 9), then offset
 * ascending, and accepted unless within max(E(l), E(l')) of an accepted
 * (i', l'); the first k accepted. nnd_all / nnj_all as for orc_discords.
 * Outputs k entries: off, len, raw d, normalised d, neighbour; returns the
 * number accepted. */
typedef struct { double s; int l; i64 i; } sli_t;

static int cmp_sli(const void *a, const void *b)
{
    const sli_t *u = (const sli_t *)a, *v = (const sli_t *)b;
    if (u->s > v->s) return -1;
    if (u->s < v->s) return 1;
    if (u->l > v->l) return -1;
    if (u->l < v->l) return 1;
    return (u->i < v->i) ? -1 : (u->i > v->i);
}

int orc_discords_global(i64 n, int lmin, int lmax, int num, int den, int k, int m_max, int m,
                        const double *nnd_all, const i64 *nnj_all,
                        i64 *out_off, int32_t *out_len, double *out_d, double *out_nd, i64 *out_nn)
{
    i64 n0 = n - lmin + 1;
    i64 cap = n0 * (i64)(lmax - lmin + 1);
    sli_t *c = (sli_t *)malloc(sizeof(sli_t) * (size_t)cap);
    i64 cnt = 0;
    for (int l = lmin; l <= lmax; ++l) {
        i64 nl = n - l + 1;
        const double *nd = nnd_all + (i64)(l - lmin) * n0 * m_max;
        for (i64 i = 0; i < nl; ++i) {
            double d = nd[i * m_max + m - 1];
            if (!isfinite(d)) continue;
            c[cnt].s = d / sqrt((double)l);
            c[cnt].l = l;
            c[cnt].i = i;
            ++cnt;
        }
    }
    qsort(c, (size_t)cnt, sizeof(sli_t), cmp_sli);
    int got = 0;
    for (i64 t = 0; t < cnt && got < k; ++t) {
        int ok = 1;
        i64 E = orc_excl(c[t].l, num, den);
        for (int g = 0; g < got && ok; ++g) {
            i64 Eg = orc_excl(out_len[g], num, den);
            i64 Em = E > Eg ? E : Eg;
            if (iabs64(c[t].i - out_off[g]) <= Em) ok = 0;
        }
        if (!ok) continue;
        i64 at = (i64)(c[t].l - lmin) * n0 * m_max + c[t].i * m_max + m - 1;
        out_off[got] = c[t].i;
        out_len[got] = c[t].l;
        out_d[got] = nnd_all[at];
        out_nd[got] = c[t].s;
        out_nn[got] = nnj_all[at];
        ++got;
    }
    free(c);
    return got;
}

/* dkm_l built as Algorithms 7 and 8 print it (the "streamed" form): windows
 * visited by offset ascending; a window with a trivial match (|i - o| <= E(l))
 * among the offsets currently anywhere in the matrix is skipped; otherwise
 * columns are tried from m down to 1 with the window's j-th best-match
 * distance, and it enters the first column where it is larger than some
 * entry, at the first such rank, the entries below moving down one rank (the
 * last one leaves). A window enters at most one cell. Empty cells hold -inf;
 * a column value that is not finite is not tried. nd / nq: n_l x m_max
 * (row-major) best-match distances and neighbours; outputs k x m (rank-major):
 * off (-1 = empty), d, nn. */
static void dkm_clear(int k, int m, i64 *off, double *d, i64 *nn)
{
    for (int c = 0; c < k * m; ++c) {
        off[c] = -1;
        d[c] = -INFINITY;
        nn[c] = -1;
    }
}

/* Has window i a trivial match among the offsets present in the matrix? */
static int dkm_trivial(int k, int m, const i64 *off, i64 i, i64 E)
{
    for (int c = 0; c < k * m; ++c)
        if (off[c] >= 0 && iabs64(i - off[c]) <= E) return 1;
    return 0;
}

/* Algorithm 8 for window i with j-th best-match distances v[0..m) and
 * neighbours vj[0..m): columns m..1, the first column and rank where it is
 * larger, the rest of the column moving down. */
static void dkm_insert(int k, int m, i64 *off, double *d, i64 *nn, i64 i, const double *v, const i64 *vj)
{
    for (int j = m - 1; j >= 0; --j) {
        if (!isfinite(v[j])) continue;
        for (int r = 0; r < k; ++r) {
            if (!(v[j] > d[r * m + j])) continue;
            for (int q = k - 1; q > r; --q) {
                off[q * m + j] = off[(q - 1) * m + j];
                d[q * m + j] = d[(q - 1) * m + j];
                nn[q * m + j] = nn[(q - 1) * m + j];
            }
            off[r * m + j] = i;
            d[r * m + j] = v[j];
            nn[r * m + j] = vj[j];
            return;
        }
    }
}

void orc_dkm_streamed(i64 nl, const double *nd, const i64 *nq, int m_max, int l, int num, int den, int k, int m,
                      i64 *out_off, double *out_d, i64 *out_nn)
{
    i64 E = orc_excl(l, num, den);
    dkm_clear(k, m, out_off, out_d, out_nn);
    for (i64 i = 0; i < nl; ++i) {
        if (dkm_trivial(k, m, out_off, i, E)) continue;
        dkm_insert(k, m, out_off, out_d, out_nn, i, nd + i * m_max, nq + i * m_max);
    }
}

/* Algorithm 9: cell by cell, the largest d / sqrt(l), ties to the later
 * length. */
static void dkm_merge(int k, int m, int l, const i64 *off, const double *d, const i64 *nn, i64 *out_off,
                      int32_t *out_len, double *out_d, double *out_nd, i64 *out_nn)
{
    double f = sqrt((double)l);
    for (int c = 0; c < k * m; ++c) {
        if (off[c] < 0) continue;
        double v = d[c] / f;
        if (out_len[c] == 0 || v >= out_nd[c]) {
            out_nd[c] = v;
            out_d[c] = d[c];
            out_off[c] = off[c];
            out_len[c] = l;
            out_nn[c] = nn[c];
        }
    }
}

/* Top-k m-th discords with the paper's pruning (Algorithm 7 driving
 * Algorithm 10, each dkm_l merged by Algorithm 9):
 *  - lmin: every row's full profile (Algorithm 3), then windows in offset
 *    order, each without a trivial match in dkm_lmin inserted by
 *    Algorithm 8 with its exact 1st..m-th best-match distances;
 *  - every longer length, first pass in offset order: each row's stored
 *    entries are re-evaluated (trivial / out-of-range ones skipped) and
 *    sorted; s_j is the j-th smallest (+inf when fewer than j); a window
 *    with a trivial match in dkm_l is skipped; otherwise it is valid iff
 *    s_m < B (its bound, Eq. LB; a flat row is never valid) and then
 *    inserted with s_1..s_m (exact, as the bound certifies them), else it
 *    joins the non-valid list with its s_1..s_m;
 *  - second pass over the list in order: a window with a trivial match in
 *    dkm_l is skipped; otherwise, for j = m down to 1, the first s_j larger
 *    than the k-th entry of column j triggers the row's full profile
 *    (stored entries, bound base and base length renewed) and its insertion
 *    with the exact distances;
 *  - rows neither valid nor recomputed keep their extended stored entries.
 * Outputs: the merged k x m table (as orc_discords), optionally every
 * dkm_l (dkm_off / dkm_d [(l - lmin) * k * m + cell]), per-length stats
 * [(l - lmin) * 4 + {0..3}] = rows, valid, listed, recomputed, and which rows
 * had their full profile computed (recomp[(l - lmin) * n0 + i] = 1, else 0). */
void orc_valmod_discord(const double *x, i64 n, int lmin, int lmax, int num, int den, int p, int k, int m,
                        i64 *out_off, int32_t *out_len, double *out_d, double *out_nd, i64 *out_nn,
                        i64 *dkm_off, double *dkm_d, i64 *stats, signed char *recomp)
{
    i64 n0 = n - lmin + 1;
    row_state *st = (row_state *)calloc((size_t)n0, sizeof(row_state));
    i64 *jstore = (i64 *)malloc(sizeof(i64) * (size_t)(n0 * p));
    for (i64 i = 0; i < n0; ++i) st[i].j = jstore + i * p;
    double *mp = (double *)malloc(sizeof(double) * (size_t)n0);
    i64 *ip = (i64 *)malloc(sizeof(i64) * (size_t)n0);
    double *nnd = (double *)malloc(sizeof(double) * (size_t)(n0 * m));
    i64 *nnj = (i64 *)malloc(sizeof(i64) * (size_t)(n0 * m));
    double *sv = (double *)malloc(sizeof(double) * (size_t)(n0 * m));   /* s_1..s_m per row */
    i64 *svj = (i64 *)malloc(sizeof(i64) * (size_t)(n0 * m));
    signed char *valid = (signed char *)malloc((size_t)n0);
    i64 *list = (i64 *)malloc(sizeof(i64) * (size_t)n0);
    i64 *off = (i64 *)malloc(sizeof(i64) * (size_t)(k * m));
    double *dd = (double *)malloc(sizeof(double) * (size_t)(k * m));
    i64 *nj = (i64 *)malloc(sizeof(i64) * (size_t)(k * m));
    double *prof = (double *)malloc(sizeof(double) * (size_t)n0);
    dj_t *dbuf = (dj_t *)malloc(sizeof(dj_t) * (size_t)n0);
    qj_t *qbuf = (qj_t *)malloc(sizeof(qj_t) * (size_t)n0);
    for (int c = 0; c < k * m; ++c) {
        out_len[c] = 0;
        out_off[c] = -1;
        out_nn[c] = -1;
        out_d[c] = -INFINITY;
        out_nd[c] = -INFINITY;
    }
    for (int l = lmin; l <= lmax; ++l) {
        i64 nl = n - l + 1, E = orc_excl(l, num, den);
        i64 nvalid = 0, nlist = 0, nrecomp = 0;
        signed char *rc = recomp ? recomp + (i64)(l - lmin) * n0 : NULL;
        if (rc) memset(rc, 0, (size_t)n0);
        dkm_clear(k, m, off, dd, nj);
        if (l == lmin) {
#pragma omp parallel
            {
                double *pr = (double *)malloc(sizeof(double) * (size_t)n0);
                dj_t *db = (dj_t *)malloc(sizeof(dj_t) * (size_t)n0);
                qj_t *qb = (qj_t *)malloc(sizeof(qj_t) * (size_t)n0);
#pragma omp for schedule(dynamic, 8)
                for (i64 i = 0; i < nl; ++i)
                    recompute_row(x, n, l, num, den, p, m, i, &st[i], mp, ip, nnd, nnj, pr, db, qb);
                free(pr);
                free(db);
                free(qb);
            }
            nrecomp = nl;
            if (rc) memset(rc, 1, (size_t)nl);
            for (i64 i = 0; i < nl; ++i) {
                if (dkm_trivial(k, m, off, i, E)) continue;
                dkm_insert(k, m, off, dd, nj, i, nnd + i * m, nnj + i * m);
            }
        } else {
            /* re-evaluate every row's stored entries (independent of dkm) */
#pragma omp parallel for schedule(dynamic, 16)
            for (i64 i = 0; i < nl; ++i) {
                dj_t e[64];
                int c = 0;
                for (int a = 0; a < st[i].cnt; ++a) {
                    i64 j = st[i].j[a];
                    if (j >= nl || iabs64(i - j) <= E) continue;
                    e[c].d = orc_dist(x, n, l, i, j);
                    e[c].j = j;
                    ++c;
                }
                qsort(e, (size_t)c, sizeof(dj_t), cmp_dj);
                for (int j = 0; j < m; ++j) {
                    sv[i * m + j] = j < c ? e[j].d : INFINITY;
                    svj[i * m + j] = j < c ? e[j].j : -1;
                }
                valid[i] = 0;
                if (!orc_is_flat(x, n, l, i) && c >= m) {
                    double mu, sig;
                    orc_window_stats(x, n, l, i, &mu, &sig);
                    double B = st[i].bound_base * st[i].sig_b / sig;
                    valid[i] = sv[i * m + m - 1] < B;
                }
            }
            for (i64 i = 0; i < nl; ++i) {
                if (dkm_trivial(k, m, off, i, E)) continue;
                if (valid[i]) {
                    ++nvalid;
                    dkm_insert(k, m, off, dd, nj, i, sv + i * m, svj + i * m);
                } else {
                    list[nlist++] = i;
                }
            }
            for (i64 t = 0; t < nlist; ++t) {
                i64 i = list[t];
                if (dkm_trivial(k, m, off, i, E)) continue;
                for (int j = m - 1; j >= 0; --j) {
                    if (!(sv[i * m + j] > dd[(k - 1) * m + j])) continue;
                    recompute_row(x, n, l, num, den, p, m, i, &st[i], mp, ip, nnd, nnj, prof, dbuf, qbuf);
                    ++nrecomp;
                    if (rc) rc[i] = 1;
                    dkm_insert(k, m, off, dd, nj, i, nnd + i * m, nnj + i * m);
                    break;
                }
            }
        }
        dkm_merge(k, m, l, off, dd, nj, out_off, out_len, out_d, out_nd, out_nn);
        if (dkm_off) {
            for (int c = 0; c < k * m; ++c) {
                dkm_off[(i64)(l - lmin) * k * m + c] = off[c];
                dkm_d[(i64)(l - lmin) * k * m + c] = dd[c];
            }
        }
        if (stats) {
            i64 *s4 = stats + (i64)(l - lmin) * 4;
            s4[0] = nl;
            s4[1] = nvalid;
            s4[2] = nlist;
            s4[3] = nrecomp;
        }
    }
    free(st);
    free(jstore);
    free(mp);
    free(ip);
    free(nnd);
    free(nnj);
    free(sv);
    free(svj);
    free(valid);
    free(list);
    free(off);
    free(dd);
    free(nj);
    free(prof);
    free(dbuf);
    free(qbuf);
}

/* dkm_{lmin,lmax} from the streamed dkm_l of every length, merged cell by
 * cell as Algorithm 9 does (largest d / sqrt(l), ties to the later length).
 * nnd_all / nnj_all as for orc_discords; outputs k x m as orc_discords. */
void orc_discords_streamed(i64 n, int lmin, int lmax, int num, int den, int k, int m_max, int m,
                           const double *nnd_all, const i64 *nnj_all,
                           i64 *out_off, int32_t *out_len, double *out_d, double *out_nd, i64 *out_nn)
{
    i64 n0 = n - lmin + 1;
    i64 *off = (i64 *)malloc(sizeof(i64) * (size_t)(k * m));
    double *dd = (double *)malloc(sizeof(double) * (size_t)(k * m));
    i64 *nj = (i64 *)malloc(sizeof(i64) * (size_t)(k * m));
    for (int c = 0; c < k * m; ++c) {
        out_len[c] = 0;
        out_off[c] = -1;
        out_nn[c] = -1;
        out_d[c] = -INFINITY;
        out_nd[c] = -INFINITY;
    }
    for (int l = lmin; l <= lmax; ++l) {
        const double *nd = nnd_all + (i64)(l - lmin) * n0 * m_max;
        const i64 *nq = nnj_all + (i64)(l - lmin) * n0 * m_max;
        orc_dkm_streamed(n - l + 1, nd, nq, m_max, l, num, den, k, m, off, dd, nj);
        dkm_merge(k, m, l, off, dd, nj, out_off, out_len, out_d, out_nd, out_nn);
    }
    free(off);
    free(dd);
    free(nj);
}

/* Variable-length Top-k m-th discords dkm_{lmin,lmax} (Algorithm 7 driving
 * Algorithm 9): for every length, every column m = 1..m_max and every rank
 * r = 1..k, keep the entry with the largest d / sqrt(l); ties go to the later
 * length (the ">=" of Algorithm 9; the text's "dividing by the discord
 * length" is read as sqrt(l), as in the formula for d*).
 * nnd_all / nnj_all: per-length m-th-NN tables as written by
 * orc_valmp_plain (stride n_lmin * m_max per length, NaN past n_l).
 * Outputs are k x m_max, row-major by rank: off, len (0 = empty), raw d,
 * normalised d, neighbour offset. */
void orc_discords(i64 n, int lmin, int lmax, int num, int den, int k, int m_max,
                  const double *nnd_all, const i64 *nnj_all,
                  i64 *out_off, int32_t *out_len, double *out_d, double *out_nd, i64 *out_nn)
{
    i64 n0 = n - lmin + 1;
    double *score = (double *)malloc(sizeof(double) * (size_t)n0);
    i64 *nbr = (i64 *)malloc(sizeof(i64) * (size_t)n0);
    i64 *off = (i64 *)malloc(sizeof(i64) * (size_t)k);
    double *dd = (double *)malloc(sizeof(double) * (size_t)k);
    i64 *nj = (i64 *)malloc(sizeof(i64) * (size_t)k);
    for (int r = 0; r < k * m_max; ++r) {
        out_len[r] = 0;
        out_off[r] = -1;
        out_nn[r] = -1;
        out_d[r] = -INFINITY;
        out_nd[r] = -INFINITY;
    }
    for (int l = lmin; l <= lmax; ++l) {
        i64 nl = n - l + 1;
        const double *nd = nnd_all + (i64)(l - lmin) * n0 * m_max;
        const i64 *nq = nnj_all + (i64)(l - lmin) * n0 * m_max;
        for (int m = 0; m < m_max; ++m) {
            for (i64 i = 0; i < nl; ++i) {
                score[i] = nd[i * m_max + m];
                nbr[i] = nq[i * m_max + m];
            }
            int got = orc_discords_one_length(nl, score, nbr, l, num, den, k, off, dd, nj);
            double f = sqrt((double)l);
            for (int r = 0; r < got; ++r) {
                int cell = r * m_max + m;
                double v = dd[r] / f;
                if (out_len[cell] == 0 || v >= out_nd[cell]) {
                    out_nd[cell] = v;
                    out_d[cell] = dd[r];
                    out_off[cell] = off[r];
                    out_len[cell] = l;
                    out_nn[cell] = nj[r];
                }
            }
        }
    }
    free(score);
    free(nbr);
    free(off);
    free(dd);
    free(nj);
}
