// k_rows.cu -- per-row work of each length: extension of the stored entries
// and the bound test (Algorithm 4 / Algorithm 10 row loops), selection of the
// new top-p after a recompute (Algorithm 3's heap of p smallest lower
// bounds), the flat-window rows, and the compaction of rows to recompute.
//
// All per-row arithmetic is FP64; one thread handles one row (rows are
// independent, the per-row state is stored structure-of-arrays so that a
// warp's accesses are coalesced).
#include "kernels.cuh"

namespace mad {

__device__ __forceinline__ double pinf() { return __longlong_as_double(0x7ff0000000000000LL); }
__device__ __forceinline__ int direct_cols_per_block_dev() { return 4096; }   // k_direct.cu: DCOLS

// Insert (q, j) into arrays sorted by q descending, j ascending; n entries.
__device__ __forceinline__ void ins_qj(double *qs, int32_t *js, int n, double q, int32_t j)
{
    int t = n;
    while (t > 0 && (qs[t - 1] < q || (qs[t - 1] == q && js[t - 1] > j))) {
        qs[t] = qs[t - 1];
        js[t] = js[t - 1];
        --t;
    }
    qs[t] = q;
    js[t] = j;
}

// Algorithm 2 (updateVALMP) for one row: strict improvement of the
// length-normalised distance; lengths ascend, so ties keep the shorter one.
__device__ __forceinline__ void valmp_update(const Valmp &vm, int64_t i, double d, int32_t j, int l)
{
    const double nd = d * sqrt(1.0 / l);
    if (vm.len[i] == 0 || nd < vm.norm[i]) {
        vm.dist[i] = d;
        vm.norm[i] = nd;
        vm.len[i] = l;
        vm.nn[i] = j;
    }
}

// Write the row's m-th best matches (entries sorted by distance ascending).
__device__ __forceinline__ void write_nn(const LenOut &o, int64_t n0, int64_t i, int m_max, const double *d,
                                         const int32_t *j, int cnt)
{
    for (int m = 0; m < m_max; ++m) {
        o.nnd[m * n0 + i] = m < cnt ? d[m] : pinf();
        o.nnj[m * n0 + i] = m < cnt ? j[m] : -1;
    }
}


// Exact FP64 centred co-moment of windows i and j at length l.
__device__ double comoment(const double *x, int64_t i, int64_t j, int l, double mui, double muj)
{
    double s = 0.0;
    for (int t = 0; t < l; ++t) s = fma(x[i + t] - mui, x[j + t] - muj, s);
    return s;
}

// Error of d = sqrt(2 l (1 - q)) caused by an error dq of q (d^2 moves by
// 2 l dq at most).
__device__ __forceinline__ double dist_err(double d, double dq, int l)
{
    const double t = 2.0 * l * dq;
    return t / (d + sqrt(d * d + t));
}
__device__ __forceinline__ bool needs_refine(const ErrModel &em, double d, double dq, int l)
{
    if (!(dq > 0.0)) return false;
    const double tol = em.rel_tol * d + em.abs_coef * sqrt((double)l);
    return dist_err(d, dq, l) > 0.5 * tol;
}
__device__ __forceinline__ double dq_pair(const ErrModel &em, int64_t i, int64_t j)
{
    return em.dq0 * (double)em.kappa[i] * (double)em.kappa[j];
}
__device__ __forceinline__ double dq_row(const ErrModel &em, int64_t i)
{
    return em.dq0 * (double)em.kappa[i] * (double)(*em.kappa_max);
}

// A row's stored entries during one length: correlation q (estimated),
// its error bound dq, partner j and storage slot e, kept sorted by
// (q desc, j asc).
struct Ent {
    double q;
    float dq;
    int32_t j;
    int32_t e;
};

__device__ __forceinline__ void ins_ent(Ent *v, int n, Ent x)
{
    int t = n;
    while (t > 0 && (v[t - 1].q < x.q || (v[t - 1].q == x.q && v[t - 1].j > x.j))) {
        v[t] = v[t - 1];
        --t;
    }
    v[t] = x;
}

// Re-evaluate in FP64 every entry among the first m (in correlation order)
// whose distance error could exceed half the tolerance; repeat until the
// first m are all accurate (re-evaluation can reorder entries).
__device__ void refine_reported(const double *x, int64_t i, int l, double mui, double m2i, const double *mu,
                                const double *m2, const ErrModel &em, RowState st, int64_t n0, Ent *v, int cnt, int m,
                                unsigned long long *stat_dq)
{
    double dqmax = 0.0;
    for (int pass = 0; pass <= cnt; ++pass) {
        int hit = -1;
        for (int a = 0; a < m && a < cnt; ++a)
            if (needs_refine(em, dist_from_q(v[a].q, l), v[a].dq, l)) { hit = a; break; }
        if (hit < 0) break;
        Ent t = v[hit];
        const double c = comoment(x, i, t.j, l, mui, mu[t.j]);
        const double q = clamp_q(c / sqrt(m2i * m2[t.j]));
        dqmax = fmax(dqmax, fabs(q - t.q));
        st.ent_c[(int64_t)t.e * n0 + i] = c;
        st.ent_dq[(int64_t)t.e * n0 + i] = 0.0f;
        t.q = q;
        t.dq = 0.0f;
        for (int a = hit; a + 1 < cnt; ++a) v[a] = v[a + 1];
        ins_ent(v, cnt - 1, t);
    }
    if (dqmax > 0.0 && stat_dq) atomicMax(stat_dq, (unsigned long long)__double_as_longlong(dqmax));
}

// ------------------------------------------------------------ extension
//
// For one length l > lmin and every row i < n_l:
//  - each stored entry (j, C) is extended by one Welford co-moment step
//    C += (l-1)/l (x_{i+l-1} - mu_i(l-1)) (x_{j+l-1} - mu_j(l-1))
//    (updateDistAndLB); entries that became trivial matches or fell off the
//    end are dropped for good (they can only stay trivial / out of range);
//  - the row's bound is B = bnum_i / sigma_i(l) (Eq. LB with the factor
//    sigma_i(l_b) / sigma_i(l) common to the row, rank preservation);
//  - the row is certified iff at least m_max entries remain and the m_max-th
//    smallest distance, evaluated pessimistically (correlation lowered by
//    the entries' error bound), is strictly below B;
//  - certified rows write their matrix profile, m-th best matches and VALMP;
//    the others are flagged for recompute with the threshold
//    key > (theta_q - dq_band) sqrt(M2_i), theta_q being a proven lower bound
//    on the row's p-th best correlation at l (the p-th best of p distinct
//    exactly evaluated partners).
template <typename T>
__device__ __forceinline__ int extend_row(const ExtArgs<T> &A, int64_t i)
{
    const int l = A.l;
    const int64_t n0 = A.n0, E = A.E;
    if (A.run[i] >= l) {                 // flat at l: handled by k_flat_rows
        A.st.flag[i] = ROW_FLAT;
        A.thr[i] = T(pinf());
        return 2;
    }
    const double m2i = A.m2[i];
    const double xi = A.x[i + l - 1] - A.mu_prev[i];
    const double wgt = (l - 1.0) / l;

    Ent v[MAXP];
    int cnt = 0;
    for (int e = 0; e < A.p; ++e) {
        const int32_t j = A.st.ent_j[e * n0 + i];
        if (j < 0) continue;
        if (j >= A.nl || !nontrivial(i, j, E)) {
            A.st.ent_j[e * n0 + i] = -1;
            continue;
        }
        const double c = fma(wgt * xi, A.x[j + l - 1] - A.mu_prev[j], A.st.ent_c[e * n0 + i]);
        A.st.ent_c[e * n0 + i] = c;
        const bool flat_j = A.run[j] >= l;
        Ent t{corr(c, m2i, A.m2[j], false, flat_j), flat_j ? 0.0f : A.st.ent_dq[e * n0 + i], j, e};
        ins_ent(v, cnt, t);
        ++cnt;
    }
    const double sig = sqrt(m2i / l);
    const double B = A.st.bnum[i] / sig;
    const int m = A.m_max;
    // the m-th smallest true distance is at most the m-th smallest pessimistic one
    bool ok = false;
    if (cnt >= m) {
        double dp[MAXP];
        for (int a = 0; a < cnt; ++a) {
            const double d = dist_from_q(v[a].q - v[a].dq, l);
            int b = a;
            while (b > 0 && dp[b - 1] > d) { dp[b] = dp[b - 1]; --b; }
            dp[b] = d;
        }
        ok = dp[m - 1] < B;
    }
    if (ok) {
        refine_reported(A.x, i, l, A.mu[i], m2i, A.mu, A.m2, A.em, A.st, n0, v, cnt, m, &A.out.stats[3]);
        double ds[MAXP];
        int32_t js[MAXP];
        for (int a = 0; a < cnt; ++a) {
            ds[a] = dist_from_q(v[a].q, l);
            js[a] = v[a].j;
        }
        write_nn(A.out, n0, i, m, ds, js, cnt);
        valmp_update(A.vm, i, ds[0], js[0], l);
        A.st.flag[i] = ROW_DONE;
        A.thr[i] = T(pinf());
        return 1;
    }
    // theta_q: p-th best among p distinct partners with known lower bounds
    // on their correlation (the remaining entries lowered by their error
    // bound, then partners next to the exclusion zone evaluated in FP64)
    double qlow[MAXP];
    int nlow = 0;
    for (int a = 0; a < cnt; ++a) qlow[nlow++] = v[a].q - v[a].dq;
    const int64_t ntc = nontrivial_count(i, A.nl, E);
    double theta = -pinf();
    if (ntc > A.p) {
        const double mui = A.mu[i];
        for (int64_t t = 1; nlow < A.p && t <= A.nl; ++t) {
            for (int side = 0; side < 2 && nlow < A.p; ++side) {
                const int64_t j = side == 0 ? i + E + t : i - E - t;
                if (j < 0 || j >= A.nl) continue;
                bool have = false;
                for (int a = 0; a < cnt; ++a) have |= (v[a].j == j);
                if (have) continue;
                const bool flat_j = A.run[j] >= l;
                const double c = flat_j ? 0.0 : comoment(A.x, i, j, l, mui, A.mu[j]);
                qlow[nlow++] = corr(c, m2i, A.m2[j], false, flat_j);
            }
        }
        if (nlow >= A.p) {
            for (int a = 1; a < nlow; ++a) {
                const double val = qlow[a];
                int b = a;
                while (b > 0 && qlow[b - 1] < val) { qlow[b] = qlow[b - 1]; --b; }
                qlow[b] = val;
            }
            theta = qlow[A.p - 1] - dq_row(A.em, i);
        }
    }
    A.st.flag[i] = ROW_RECOMPUTE;
    if (theta == -pinf()) {
        A.thr[i] = T(-pinf());
    } else {
        // key units: key = q sqrt(M2_i); never round the threshold upwards
        const double tk = theta * sqrt(m2i);
        T tt = T(tk);
        if ((double)tt > tk) tt = T(tk - fabs(tk) * 1e-6);
        A.thr[i] = tt;
    }
    return 2;
}

template <typename T>
__global__ void k_extend(ExtArgs<T> A)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int cat = 0;
    if (i < A.n0) {
        if (i >= A.nl) {
            A.st.flag[i] = ROW_DONE;
            A.thr[i] = T(pinf());
        } else {
            cat = extend_row(A, i);
        }
    }
    const unsigned mask = __activemask();
    const unsigned b1 = __ballot_sync(mask, cat == 1), b2 = __ballot_sync(mask, cat == 2);
    if ((threadIdx.x & 31) == __ffs(mask) - 1) {
        if (b1) atomicAdd(&A.out.stats[1], (unsigned long long)__popc(b1));
        if (b2) atomicAdd(&A.out.stats[2], (unsigned long long)__popc(b2));
    }
}

template <typename T>
void launch_extend(const ExtArgs<T> &a, cudaStream_t s)
{
    const int B = 128;
    k_extend<T><<<(unsigned)((a.n0 + B - 1) / B), B, 0, s>>>(a);
}
template void launch_extend<float>(const ExtArgs<float> &, cudaStream_t);
template void launch_extend<double>(const ExtArgs<double> &, cudaStream_t);

// ---------------------------------------------------------------- merge
//
// After the band kernel: for every row flagged for recompute, select the p
// largest keys (ties: smaller offset) among the per-group lists the band
// kernel kept. They are the row's new stored entries at base length l (the
// p smallest Eq. LB values, Algorithm 3 filling listDP); the row's matrix
// profile value and m-th best matches at l come from them; the bound
// numerator is sqrt(l (1 - max(q_p + dq_band, 0)^2)) * sigma_i(l) (+inf when
// the row has at most p non-trivial partners, all of them stored).
// A row whose lists hold fewer than min(p, partners) keys had a threshold
// above its p-th best key; it is flagged for another pass without one.
template <typename T>
__global__ void k_merge(MergeArgs<T> A)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= A.nl) return;
    const int32_t fl = A.st.flag[i];
    if (fl != ROW_RECOMPUTE && fl != ROW_DIRECT) return;
    const int l = A.l;
    const int64_t n0 = A.n0, E = A.E;
    const int p = A.p;
    const int64_t ntc = nontrivial_count(i, A.nl, E);
    const int need = (int)(ntc < p ? ntc : p);

    // top-p by key desc, offset asc over the row's lists. The symmetric form
    // wrote row-side lists for the column groups from the row's band
    // diagonal on, and appended the column-side candidates (cells (i', i),
    // i' < i) to the row's candidate list.
    const bool sym_on = sym_rule(A.allow_sym, *A.nflagged, A.nl) && fl == ROW_RECOMPUTE;
    T bk[MAXP];
    int32_t bj[MAXP];
    int nb = 0;
    auto offer = [&](T v, int32_t j) {
        if (nb == p && !(v > bk[p - 1] || (v == bk[p - 1] && j < bj[p - 1]))) return;
        int b = nb < p ? nb++ : p - 1;
        while (b > 0 && (bk[b - 1] < v || (bk[b - 1] == v && bj[b - 1] > j))) {
            bk[b] = bk[b - 1];
            bj[b] = bj[b - 1];
            --b;
        }
        bk[b] = v;
        bj[b] = j;
    };
    if (fl == ROW_DIRECT) {
        const int64_t d = A.dindex[i];
        for (int g = 0; g < A.dnblk; ++g) {
            const int64_t slot = d * A.dnblk + g;
            if ((int64_t)g * direct_cols_per_block_dev() >= A.nl) break;
            const int cnt = A.dcnt[slot];
            for (int c = 0; c < cnt; ++c) offer(A.dkey[slot * p + c], A.dj[slot * p + c]);
        }
    } else {
        const int g0 = sym_on ? (int)(((i / A.R) * (int64_t)A.R) / A.group_w) : 0;
        for (int g = g0; g < A.ngroups && (int64_t)g * A.group_w < A.nl; ++g) {
            const int64_t slot = i * A.ngroups + g;
            const int cnt = A.scnt[slot];
            for (int c = 0; c < cnt; ++c) offer(A.skey[slot * p + c], A.sj[slot * p + c]);
        }
    }
    if (A.allow_sym && fl == ROW_DIRECT) A.ccnt[i] = 0;
    if (sym_on) {
        const int cc = A.ccnt[i];
        A.ccnt[i] = 0;
        if (cc > A.cap) {
            // more column-side candidates than kept: redo the row in full
            // (its threshold stays valid)
            A.st.flag[i] = ROW_RECOMPUTE;
            atomicAdd(A.overflow, 1ull);
            return;
        }
        for (int c = 0; c < cc; ++c) offer(A.ckey[i * A.cap + c], A.cj[i * A.cap + c]);
    }
    if (nb < need) {
        A.thr[i] = T(-pinf());
        A.st.flag[i] = ROW_RECOMPUTE;
        atomicAdd(A.overflow, 1ull);
        atomicAdd(A.overflow + 8, 1ull);
        return;
    }
    const double m2i = A.m2[i];
    const double sqm2i = sqrt(m2i);
    Ent v[MAXP];
    int nq = 0;
    for (int e = 0; e < p; ++e) {
        if (e < nb) {
            const int32_t j = bj[e];
            const double inv = (double)A.col[j].inv;
            const bool flat_j = A.run[j] >= l;
            const double c = (flat_j || inv == 0.0) ? 0.0 : (double)bk[e] / inv;
            const float dq = flat_j ? 0.0f : (float)dq_pair(A.em, i, j);
            A.st.ent_j[e * n0 + i] = j;
            A.st.ent_c[e * n0 + i] = c;
            A.st.ent_dq[e * n0 + i] = dq;
            Ent t{corr(c, m2i, A.m2[j], false, flat_j), dq, j, e};
            ins_ent(v, nq, t);
            ++nq;
        } else {
            A.st.ent_j[e * n0 + i] = -1;
            A.st.ent_c[e * n0 + i] = 0.0;
            A.st.ent_dq[e * n0 + i] = 0.0f;
        }
    }
    refine_reported(A.x, i, l, A.mu[i], m2i, A.mu, A.m2, A.em, A.st, n0, v, nq, A.m_max, &A.out.stats[3]);
    double ds[MAXP];
    int32_t js[MAXP];
    for (int e = 0; e < nq; ++e) {
        ds[e] = dist_from_q(v[e].q, l);
        js[e] = v[e].j;
    }
    write_nn(A.out, n0, i, A.m_max, ds, js, nq);
    if (nq > 0) valmp_update(A.vm, i, ds[0], js[0], l);
    A.st.base[i] = l;
    const double sig = sqm2i / sqrt((double)l);
    if (ntc <= p) {
        A.st.bnum[i] = pinf();
    } else {
        // unstored partners have band keys <= the p-th kept key
        double qp = (double)bk[p - 1] / sqm2i + dq_row(A.em, i);
        qp = qp > 1.0 ? 1.0 : (qp < 0.0 ? 0.0 : qp);
        A.st.bnum[i] = sqrt((double)l * (1.0 - qp * qp)) * sig;
    }
    A.st.flag[i] = ROW_DONE;
    A.thr[i] = T(pinf());
}

template <typename T>
void launch_merge(const MergeArgs<T> &a, cudaStream_t s)
{
    const int B = 128;
    k_merge<T><<<(unsigned)((a.nl + B - 1) / B), B, 0, s>>>(a);
}
template void launch_merge<float>(const MergeArgs<float> &, cudaStream_t);
template void launch_merge<double>(const MergeArgs<double> &, cudaStream_t);

// First threshold at lmin from the interleaved maxima: bin b holds the
// largest key over the column chunks of index = b (mod nbins); the p-th
// largest of those maxima comes from p distinct columns, so it lower-bounds
// the row's p-th best key. Rows with fewer than p non-empty bins get none.
template <typename T>
__global__ void k_theta_bins(const int *bins, int nbins, int64_t nl, int p, const double *m2, ErrModel em, T *thr)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= nl) return;
    float top[2 * MAXP];
    int nt = 0;
    for (int b = 0; b < nbins; ++b) {
        const float v = ord2f(bins[i * nbins + b]);
        if (!(v > -__int_as_float(0x7f800000))) continue;
        int t = nt++;
        while (t > 0 && top[t - 1] < v) { top[t] = top[t - 1]; --t; }
        top[t] = v;
    }
    if (nt < p) {
        thr[i] = T(-pinf());
        return;
    }
    double th = (double)top[p - 1];
    // bins hold keys rounded down; widen by the key error and one FP32 step
    th -= dq_row(em, i) * sqrt(m2[i]) + fabs(th) * 1e-6;
    thr[i] = T(th);
}

template <typename T>
void launch_theta_bins(const int *bins, int nbins, int64_t nl, int p, const double *m2, ErrModel em, T *thr,
                       cudaStream_t s)
{
    const int B = 256;
    k_theta_bins<T><<<(unsigned)((nl + B - 1) / B), B, 0, s>>>(bins, nbins, nl, p, m2, em, thr);
}
template void launch_theta_bins<float>(const int *, int, int64_t, int, const double *, ErrModel, float *, cudaStream_t);
template void launch_theta_bins<double>(const int *, int, int64_t, int, const double *, ErrModel, double *,
                                        cudaStream_t);

// ----------------------------------------------------------- flat rows
//
// A flat row correlates 1 with every other flat window and 0 with the rest:
// its p entries are the first flat non-trivial partners, then the first
// non-flat ones; its co-moments are exactly 0 and its bound is 0 (recomputed
// at every length while it stays flat). One warp per row.
__global__ void k_flat_rows(FlatArgs A)
{
    const int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= A.nl) return;
    const int32_t fl = A.st.flag[i];
    if ((fl == ROW_RECOMPUTE || fl == ROW_DIRECT) && lane == 0) atomicExch(A.left_over, 1);
    if (fl != ROW_FLAT) return;
    const int l = A.l;
    const int64_t n0 = A.n0, E = A.E;
    const int p = A.p;
    int32_t js[MAXP];
    double qs[MAXP];
    int nf = 0;
    for (int pass = 0; pass < 2 && nf < p; ++pass) {
        const bool want_flat = pass == 0;
        for (int64_t base = 0; base < A.nl && nf < p; base += 32) {
            const int64_t j = base + lane;
            const bool ok = j < A.nl && nontrivial(i, j, E) && ((A.run[j] >= l) == want_flat);
            unsigned b = __ballot_sync(0xffffffffu, ok);
            while (b && nf < p) {
                const int t = __ffs(b) - 1;
                b &= b - 1;
                js[nf] = (int32_t)(base + t);
                qs[nf] = want_flat ? 1.0 : 0.0;
                ++nf;
            }
        }
    }
    if (lane != 0) return;
    double ds[MAXP];
    for (int e = 0; e < p; ++e) {
        A.st.ent_j[e * n0 + i] = e < nf ? js[e] : -1;
        A.st.ent_c[e * n0 + i] = 0.0;
        A.st.ent_dq[e * n0 + i] = 0.0f;
    }
    for (int e = 0; e < nf; ++e) ds[e] = dist_from_q(qs[e], l);
    write_nn(A.out, n0, i, A.m_max, ds, js, nf);
    if (nf > 0) valmp_update(A.vm, i, ds[0], js[0], l);
    A.st.base[i] = l;
    A.st.bnum[i] = 0.0;
    A.st.flag[i] = ROW_DONE;
}

void launch_flat_rows(const FlatArgs &a, cudaStream_t s)
{
    const int B = 256;
    const int64_t thr = a.nl * 32;
    k_flat_rows<<<(unsigned)((thr + B - 1) / B), B, 0, s>>>(a);
}

// lmin: every row is recomputed; flat rows go to k_flat_rows.
__global__ void k_init_flags(const int32_t *run, int64_t n0, int l, int32_t *flag, unsigned long long *stats)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n0) return;
    flag[i] = run[i] >= l ? ROW_FLAT : ROW_RECOMPUTE;
    const unsigned mask = __activemask();
    if ((threadIdx.x & 31) == __ffs(mask) - 1) atomicAdd(&stats[2], (unsigned long long)__popc(mask));
}

// Rows not flagged for recompute take no candidates.
template <typename T>
__global__ void k_mask_thr_t(const int32_t *flag, int64_t n0, T *thr)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n0 && flag[i] != ROW_RECOMPUTE) thr[i] = T(pinf());
}
template <typename T>
void launch_mask_thr(const int32_t *flag, int64_t n0, T *thr, cudaStream_t s)
{
    k_mask_thr_t<T><<<(unsigned)((n0 + 255) / 256), 256, 0, s>>>(flag, n0, thr);
}
template void launch_mask_thr<float>(const int32_t *, int64_t, float *, cudaStream_t);
template void launch_mask_thr<double>(const int32_t *, int64_t, double *, cudaStream_t);

// ------------------------------------------------------------ compaction
// Bands (R consecutive rows) holding at least one row to recompute.
__global__ void k_compact_bands(const int32_t *flag, int64_t nl, int R, int32_t *bands, int32_t *nbands)
{
    const int64_t b = blockIdx.x;
    const int64_t r0 = b * R;
    int any = 0;
    for (int64_t r = r0 + threadIdx.x; r < r0 + R && r < nl; r += blockDim.x) any |= (flag[r] == ROW_RECOMPUTE);
    any = __syncthreads_or(any);
    if (threadIdx.x == 0 && any) {
        const int slot = atomicAdd(nbands, 1);
        bands[slot] = (int32_t)b;
    }
}

void launch_compact_bands(const int32_t *flag, int64_t nl, int R, int32_t *bands, int32_t *nbands, cudaStream_t s)
{
    const int64_t nb = (nl + R - 1) / R;
    cudaMemsetAsync(nbands, 0, sizeof(int32_t), s);
    k_compact_bands<<<(unsigned)nb, 256, 0, s>>>(flag, nl, R, bands, nbands);
}

// One block per band: count the band's rows to recompute; route them to the
// direct path (few rows, room left in the list, symmetric form off) or list
// the band for the band kernel.
__global__ void k_split(SplitArgs A)
{
    const int64_t b = blockIdx.x;
    const int64_t r0 = b * A.R;
    __shared__ int total;
    __shared__ int base;
    if (threadIdx.x == 0) total = 0;
    __syncthreads();
    int mine = 0;
    for (int64_t r = r0 + threadIdx.x; r < r0 + A.R && r < A.nl; r += blockDim.x) mine += (A.flag[r] == ROW_RECOMPUTE);
    for (int o = 16; o > 0; o >>= 1) mine += __shfl_xor_sync(0xffffffffu, mine, o);
    if ((threadIdx.x & 31) == 0 && mine) atomicAdd(&total, mine);
    __syncthreads();
    const int cnt = total;
    if (cnt == 0) return;
    const bool sym_on = sym_rule(A.allow_sym, *A.nflagged, A.nl);
    bool direct = A.force_direct || (!sym_on && cnt <= A.lim);
    if (direct) {
        if (threadIdx.x == 0) {
            base = atomicAdd(A.ndirect, cnt);
            if (base + cnt > A.max_direct) {
                atomicSub(A.ndirect, cnt);
                base = -1;
            } else if (A.stat_direct) {
                atomicAdd(A.stat_direct, (unsigned long long)cnt);
            }
        }
        __syncthreads();
        direct = base >= 0;
    }
    if (!direct) {
        if (threadIdx.x == 0) {
            const int slot = atomicAdd(A.nbands, 1);
            A.bands[slot] = (int32_t)b;
        }
        return;
    }
    // positions within the list: block-wide ballot prefix per pass of rows
    __shared__ int run;
    __shared__ int wsum[32];
    if (threadIdx.x == 0) run = base;
    __syncthreads();
    for (int64_t r0w = r0; r0w < r0 + A.R && r0w < A.nl; r0w += blockDim.x) {
        const int64_t r = r0w + threadIdx.x;
        const bool f = r < r0 + A.R && r < A.nl && A.flag[r] == ROW_RECOMPUTE;
        const unsigned bal = __ballot_sync(0xffffffffu, f);
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        if (lane == 0) wsum[wid] = __popc(bal);
        __syncthreads();
        int before = 0;
        for (int q = 0; q < wid; ++q) before += wsum[q];
        if (f) {
            const int pos = run + before + __popc(bal & ((1u << lane) - 1u));
            A.drows[pos] = (int32_t)r;
            A.dindex[r] = pos;
            A.flag[r] = ROW_DIRECT;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int tot = 0;
            for (int q = 0; q < (int)(blockDim.x >> 5); ++q) tot += wsum[q];
            run += tot;
        }
        __syncthreads();
    }
}

void launch_split(const SplitArgs &a, cudaStream_t s)
{
    const int64_t nb = (a.nl + a.R - 1) / a.R;
    cudaMemsetAsync(a.nbands, 0, sizeof(int32_t), s);
    cudaMemsetAsync(a.ndirect, 0, sizeof(int32_t), s);
    k_split<<<(unsigned)nb, 256, 0, s>>>(a);
}

template <typename T>
__global__ void k_fill(T *p, int64_t n, T v)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) p[i] = v;
}

template <typename T>
void launch_fill(T *p, int64_t n, T v, cudaStream_t s)
{
    if (n <= 0) return;
    const int B = 256;
    int64_t g = (n + B - 1) / B;
    if (g > 65536) g = 65536;
    k_fill<T><<<(unsigned)g, B, 0, s>>>(p, n, v);
}
template void launch_fill<float>(float *, int64_t, float, cudaStream_t);
template void launch_fill<double>(double *, int64_t, double, cudaStream_t);
template void launch_fill<int32_t>(int32_t *, int64_t, int32_t, cudaStream_t);

}  // namespace mad
