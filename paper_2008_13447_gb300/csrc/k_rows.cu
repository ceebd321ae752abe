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


// Exact FP64 centred co-moment of windows i and j at length l (four
// partial sums, so consecutive products do not wait on each other).
__device__ double comoment(const double *x, int64_t i, int64_t j, int l, double mui, double muj)
{
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    int t = 0;
    for (; t + 3 < l; t += 4) {
        s0 = fma(x[i + t] - mui, x[j + t] - muj, s0);
        s1 = fma(x[i + t + 1] - mui, x[j + t + 1] - muj, s1);
        s2 = fma(x[i + t + 2] - mui, x[j + t + 2] - muj, s2);
        s3 = fma(x[i + t + 3] - mui, x[j + t + 3] - muj, s3);
    }
    for (; t < l; ++t) s0 = fma(x[i + t] - mui, x[j + t] - muj, s0);
    return (s0 + s1) + (s2 + s3);
}

// The same co-moment from x split into FP32 pairs (x = xh + xl), in FP32
// with error-free transformations: each centred value is formed as
// (xh - muh) + (xl - mul) (relative error about 2u, u = 2^-24), each product
// is split exactly into p + e by an FMA (TwoProd) and each partial sum into
// s + e by TwoSum (Knuth), the errors accumulating separately. The result is
// within about 4u sum_t |a_t b_t| <= 4u sqrt(M2_i M2_j) (Cauchy-Schwarz) of
// the exact co-moment, i.e. its correlation within DQ_COMP.
constexpr double DQ_COMP = 3e-7;

__device__ double comoment_comp(const float *__restrict__ xh, const float *__restrict__ xl, int64_t i, int64_t j,
                                int l, double mui, double muj)
{
    const float mih = (float)mui, mil = (float)(mui - (double)mih);
    const float mjh = (float)muj, mjl = (float)(muj - (double)mjh);
    float S = 0.0f, Er = 0.0f;
    for (int t = 0; t < l; ++t) {
        const float a = (xh[i + t] - mih) + (xl[i + t] - mil);
        const float b = (xh[j + t] - mjh) + (xl[j + t] - mjl);
        // (explicit roundings: a contraction of S + a*b into an FMA would
        // break the exactness of TwoProd / TwoSum)
        const float pr = __fmul_rn(a, b);
        const float pe = fmaf(a, b, -pr);
        const float sn = __fadd_rn(S, pr);
        const float bv = __fsub_rn(sn, S);
        const float se = __fadd_rn(__fsub_rn(S, __fsub_rn(sn, bv)), __fsub_rn(pr, bv));
        S = sn;
        Er += pe + se;
    }
    return (double)S + (double)Er;
}

// Correlation from the co-moment and the windows' 1 / sqrt(M2) (flat
// partner: 0).
__device__ __forceinline__ double corr_isd(double c, double isdi, double isdj, bool flat_j)
{
    return flat_j ? 0.0 : clamp_q(c * isdi * isdj);
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
    if (em.audit) return true;
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

// A row's stored entries during one length, held in registers: PM is a
// compile-time bound on p (8, 16 or 64) so that every loop over entries
// unrolls with constant indices (for PM = 64 the loops stay rolled and the
// arrays live in local memory). Entry e sits in index e (its storage slot);
// j < 0 marks an empty one. Orders are taken by counting, not by moving
// entries.
template <int PM> struct RowEnts {
    double q[PM];    // correlation (estimate)
    long long qk[PM];  // q as an order-preserving integer (ranking on the integer pipe)
    float dq[PM];    // its error bound
    int32_t j[PM];   // partner offset, -1 = empty
};

// Order-preserving map of a double (not NaN) to a signed 64-bit integer:
// comparisons of the images order like the doubles, on the integer pipe
// instead of GB300's 1/64-rate FP64 pipe.
__device__ __forceinline__ long long ord64(double v)
{
    const long long b = __double_as_longlong(v);
    return b >= 0 ? b : (b ^ 0x7fffffffffffffffLL);
}

template <int PM, typename F>
__device__ __forceinline__ void for_pm(F &&f)
{
    if constexpr (PM <= 16) {
#pragma unroll
        for (int a = 0; a < PM; ++a) f(a);
    } else {
#pragma unroll 1
        for (int a = 0; a < PM; ++a) f(a);
    }
}

// (key desc, j asc) on the integer images of q.
__device__ __forceinline__ bool qk_before(long long ka, int32_t ja, long long kb, int32_t jb)
{
    return ka > kb || (ka == kb && ja < jb);
}

// Rank of every entry in (q desc, j asc) order (0 = best).
template <int PM>
__device__ __forceinline__ void corr_ranks(const RowEnts<PM> &r, int (&rk)[PM])
{
    for_pm<PM>([&](int a) {
        int k = 0;
        for_pm<PM>([&](int b) { k += (r.j[b] >= 0 && qk_before(r.qk[b], r.j[b], r.qk[a], r.j[a])); });
        rk[a] = k;
    });
}

// Re-evaluate in FP64, one at a time, the best-ranked entry among the first
// m (correlation order) whose distance error could exceed half the
// tolerance, until none is left (a re-evaluation can reorder entries).
// An entry is re-evaluated first by the compensated FP32 co-moment, which
// it keeps (with error bound DQ_COMP) if that bound meets half the tolerance
// (only with an absolute tolerance, i.e. the FP32 path), else in FP64.
template <int PM>
__device__ void refine_reported(const double *x, const float *xh, const float *xl, int64_t i, int l, double mui,
                                double isdi, const double *mu, const double *isd, const ErrModel &em, RowState st,
                                int64_t n0, RowEnts<PM> &r, int m, unsigned long long *stat_dq,
                                unsigned long long *stat_ratio)
{
    double dqmax = 0.0, ratio = 0.0;
    for (int pass = 0; pass <= PM; ++pass) {
        int rk[PM];
        corr_ranks(r, rk);
        int hit = -1, hr = 1 << 30;
        int32_t j = -1;
        double qold = 0.0;
        for_pm<PM>([&](int a) {
            if (r.j[a] >= 0 && (rk[a] < m || em.audit) && rk[a] < hr &&
                needs_refine(em, dist_from_q(r.q[a], l), r.dq[a], l)) {
                hit = a;
                hr = rk[a];
                j = r.j[a];
                qold = r.q[a];
            }
        });
        if (hit < 0) break;
        double c = 0.0, q = 0.0;
        float dqn = 0.0f;
        bool done = false;
        if (em.abs_coef > 0.0 && !em.audit) {
            c = comoment_comp(xh, xl, i, j, l, mui, mu[j]);
            q = clamp_q(c * isdi * isd[j]);
            dqn = (float)DQ_COMP;
            done = !needs_refine(em, dist_from_q(q, l), DQ_COMP, l);
        }
        if (!done) {
            c = comoment(x, i, j, l, mui, mu[j]);
            q = clamp_q(c * isdi * isd[j]);
            dqn = 0.0f;
        }
        dqmax = fmax(dqmax, fabs(q - qold));
        // the entry's observed error over its own bound (<= 1 while the bound
        // holds); against the compensated value the error is known to within
        // DQ_COMP, which is added (an upper estimate)
        float dqb = 0.0f;
        for_pm<PM>([&](int a) { if (a == hit) dqb = r.dq[a]; });
        if (dqb > 0.0f) ratio = fmax(ratio, (fabs(q - qold) + (double)dqn) / (double)dqb);
        st.ent_c[(int64_t)hit * n0 + i] = c;
        st.ent_dq[(int64_t)hit * n0 + i] = dqn;
        for_pm<PM>([&](int a) {
            if (a == hit) {
                r.q[a] = q;
                r.qk[a] = ord64(q);
                r.dq[a] = dqn;
            }
        });
    }
    if (dqmax > 0.0 && stat_dq) atomicMax(stat_dq, (unsigned long long)__double_as_longlong(dqmax));
    if (ratio > 0.0 && stat_ratio) atomicMax(stat_ratio, (unsigned long long)__double_as_longlong(ratio));
}

// The row's m-th best matches (first m entries in correlation order), +inf
// past the last of its cnt entries, and VALMP from the best (Algorithm 2).
template <int PM>
__device__ double report_row(const LenOut &o, const Valmp &vm, int64_t n0, int64_t i, int l, const RowEnts<PM> &r,
                             int cnt, int m)
{
    int rk[PM];
    corr_ranks(r, rk);
    double best = pinf();
    for_pm<PM>([&](int a) {
        if (r.j[a] >= 0 && rk[a] < m) {
            const double d = dist_from_q(r.q[a], l);
            o.nnd[(int64_t)rk[a] * n0 + i] = d;
            o.nnj[(int64_t)rk[a] * n0 + i] = r.j[a];
            if (rk[a] == 0) {
                valmp_update(vm, i, d, r.j[a], l);
                best = d;
            }
        }
    });
    for (int t = cnt; t < m; ++t) {
        o.nnd[(int64_t)t * n0 + i] = pinf();
        o.nnj[(int64_t)t * n0 + i] = -1;
    }
    return best;
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
// The row's loads are all issued before its stores.
// Motif mode: dbest / lb receive the row's certified distance or its bound
// (a flat row has no usable bound: 0).
template <typename T, int PM>
__device__ __forceinline__ int extend_row(const ExtArgs<T> &A, int64_t i, double &dbest, double &lb)
{
    const int l = A.l;
    const int64_t n0 = A.n0, E = A.E;
    const int p = A.p;
    if (A.run[i] >= l) {                 // flat at l: handled by k_flat_rows
        A.st.flag[i] = ROW_FLAT;
        A.thr[i] = T(pinf());
        if (A.lbmax) {
            A.lbmax[i] = 0.0;
            lb = 0.0;
        }
        if (A.obs_gap) {
            A.obs_gap[i] = __longlong_as_double(0x7ff8000000000000LL);
            A.obs_tlb[i] = __longlong_as_double(0x7ff8000000000000LL);
        }
        if (A.ub_out)
            for (int c = 0; c < A.m_max; ++c) A.out.nnd[(int64_t)c * n0 + i] = pinf();
        return 2;
    }
    const double m2i = A.m2[i];
    const double isdi = A.isd[i];
    const double xi = A.x[i + l - 1] - A.mu_prev[i];
    const double wgt = (l - 1.0) / l;

    RowEnts<PM> r;
    bool dropped[PM];
    double cn[PM];
    for_pm<PM>([&](int e) {
        int32_t j = e < p ? A.st.ent_j[(int64_t)e * n0 + i] : -1;
        dropped[e] = j >= 0 && (j >= A.nl || !nontrivial(i, j, E));
        if (dropped[e]) j = -1;
        r.j[e] = j;
        r.q[e] = -pinf();
        r.qk[e] = ord64(-pinf());
        r.dq[e] = 0.0f;
        cn[e] = 0.0;
    });
    for_pm<PM>([&](int e) {
        const int32_t j = r.j[e];
        if (j < 0) return;
        const int64_t at = (int64_t)e * n0 + i;
        cn[e] = fma(wgt * xi, A.x[j + l - 1] - A.mu_prev[j], A.st.ent_c[at]);
        const bool flat_j = A.run[j] >= l;
        r.q[e] = corr_isd(cn[e], isdi, A.isd[j], flat_j);
        r.qk[e] = ord64(r.q[e]);
        r.dq[e] = flat_j ? 0.0f : A.st.ent_dq[at];
    });
    int cnt = 0;
    for_pm<PM>([&](int e) {
        const int64_t at = (int64_t)e * n0 + i;
        if (dropped[e]) A.st.ent_j[at] = -1;
        if (r.j[e] >= 0) {
            A.st.ent_c[at] = cn[e];
            ++cnt;
        }
    });
    const double sig = sqrt(m2i / l);
    const double B = A.st.bnum[i] / sig;
    const int m = A.m_max;
    if (A.obs_gap) {
        // maxLB - minED and the mean tightness LB / ED of the stored entries
        // (Eq. LB with each entry's correlation at the row's base length)
        const double lbb = (double)A.st.base[i], sb = A.st.sigb[i];
        double dmin = pinf(), tsum = 0.0;
        int tc = 0;
        for_pm<PM>([&](int a) {
            if (r.j[a] < 0) return;
            const double d = dist_from_q(r.q[a], l);
            dmin = fmin(dmin, d);
            if (d > 0.0) {
                const double qb = A.st.ent_qb[(int64_t)a * n0 + i];
                const double base = qb <= 0.0 ? sqrt(lbb) : sqrt(lbb * (1.0 - qb * qb));
                tsum += base * sb / sig / d;
                ++tc;
            }
        });
        const double nan = __longlong_as_double(0x7ff8000000000000LL);
        A.obs_gap[i] = cnt > 0 ? B - dmin : nan;
        A.obs_tlb[i] = tc > 0 ? tsum / tc : nan;
    }
    // the m-th smallest true distance is at most the m-th smallest pessimistic
    // one (compared as squared distances 2 l (1 - q))
    bool ok = false;
    if (cnt >= m) {
        double dp[PM];
        long long dk[PM];
        for_pm<PM>([&](int a) {
            dp[a] = r.j[a] >= 0 ? 2.0 * l * (1.0 - clamp_q(r.q[a] - r.dq[a])) : pinf();
            dk[a] = ord64(dp[a]);
        });
        double dm = pinf();
        for_pm<PM>([&](int a) {
            int k = 0;
            for_pm<PM>([&](int b) { k += (r.j[b] >= 0 && (dk[b] < dk[a] || (dk[b] == dk[a] && b < a))); });
            if (r.j[a] >= 0 && k == m - 1) dm = dp[a];
        });
        ok = dm < B * B;
    }
    if (ok) {
        refine_reported<PM>(A.x, A.xh, A.xl, i, l, A.mu[i], isdi, A.mu, A.isd, A.em, A.st, n0, r, m,
                            &A.out.stats[3], &A.out.stats[12]);
        dbest = report_row<PM>(A.out, A.vm, n0, i, l, r, cnt, m);
        A.st.flag[i] = ROW_DONE;
        A.thr[i] = T(pinf());
        return 1;
    }
    if (A.lbmax) {
        A.lbmax[i] = B;
        lb = B;
    }
    if (A.ub_out) {
        // upper values: the c-th smallest pessimistic stored distance
        for (int c = 0; c < m; ++c) A.out.nnd[(int64_t)c * n0 + i] = pinf();
        double dp[PM];
        long long dk[PM];
        for_pm<PM>([&](int a) {
            dp[a] = r.j[a] >= 0 ? 2.0 * l * (1.0 - clamp_q(r.q[a] - r.dq[a])) : pinf();
            dk[a] = ord64(dp[a]);
        });
        for_pm<PM>([&](int a) {
            if (r.j[a] < 0) return;
            int k = 0;
            for_pm<PM>([&](int b) { k += (r.j[b] >= 0 && (dk[b] < dk[a] || (dk[b] == dk[a] && b < a))); });
            if (k < m) A.out.nnd[(int64_t)k * n0 + i] = sqrt(dp[a]);
        });
    }
    // theta_q: p-th best among p distinct partners with known lower bounds
    // on their correlation (the remaining entries lowered by their error
    // bound, then partners next to the exclusion zone evaluated in FP64).
    // There are never more than p such values, so the p-th best is the
    // smallest once there are p of them.
    double qmin = pinf();
    for_pm<PM>([&](int a) {
        if (r.j[a] >= 0) qmin = fmin(qmin, r.q[a] - r.dq[a]);
    });
    int nlow = cnt;
    const int64_t ntc = nontrivial_count(i, A.nl, E);
    double theta = -pinf();
    if (A.hint_j) {
        // hint partners not among the entries: their extended correlations,
        // lowered by their error bounds, are further known lower bounds
        double hq[PM];
        int nh = 0;
        for_pm<PM>([&](int e) {
            hq[e] = -pinf();
            if (e >= p) return;
            const int64_t at = (int64_t)e * n0 + i;
            const int32_t j = A.hint_j[at];
            if (j < 0) return;
            if (j >= A.nl || !nontrivial(i, j, E)) {
                A.hint_j[at] = -1;
                return;
            }
            const double c = fma(wgt * xi, A.x[j + l - 1] - A.mu_prev[j], A.hint_c[at]);
            A.hint_c[at] = c;
            bool dup = false;
            for_pm<PM>([&](int a) { dup |= (r.j[a] == j); });
            if (dup) return;
            const bool flat_j = A.run[j] >= l;
            hq[e] = corr_isd(c, isdi, A.isd[j], flat_j) - (flat_j ? 0.0 : (double)A.hint_dq[at]);
            ++nh;
        });
        if (cnt + nh >= p && ntc > p) {
            // the p-th largest of the union (ties by position, entries first)
            double pth = -pinf();
            for_pm<PM>([&](int a) {
                if (r.j[a] < 0) return;
                const double v = r.q[a] - r.dq[a];
                int rank = 0;
                for_pm<PM>([&](int b) {
                    if (r.j[b] >= 0) {
                        const double u = r.q[b] - r.dq[b];
                        rank += (u > v || (u == v && b < a));
                    }
                    rank += (hq[b] > v);
                });
                if (rank == p - 1) pth = v;
            });
            for_pm<PM>([&](int e) {
                if (hq[e] == -pinf()) return;
                const double v = hq[e];
                int rank = 0;
                for_pm<PM>([&](int b) {
                    if (r.j[b] >= 0) rank += (r.q[b] - r.dq[b] >= v);
                    rank += (hq[b] > v || (hq[b] == v && b < e));
                });
                if (rank == p - 1) pth = v;
            });
            theta = pth - dq_row(A.em, i);
            nlow = p;            // no partners next to the exclusion zone needed
        } else {
            for_pm<PM>([&](int e) {
                if (hq[e] != -pinf()) qmin = fmin(qmin, hq[e]);
            });
            nlow += nh;
        }
    }
    if (ntc > p && theta == -pinf()) {
        const double mui = A.mu[i];
        for (int64_t t = 1; nlow < p && t <= A.nl; ++t) {
            for (int side = 0; side < 2 && nlow < p; ++side) {
                const int64_t j = side == 0 ? i + E + t : i - E - t;
                if (j < 0 || j >= A.nl) continue;
                bool have = false;
                for_pm<PM>([&](int a) { have |= (r.j[a] == j); });
                if (A.hint_j)
                    for (int e = 0; e < p; ++e) have |= (A.hint_j[(int64_t)e * n0 + i] == j);
                if (have) continue;
                const bool flat_j = A.run[j] >= l;
                const double c = flat_j ? 0.0 : comoment(A.x, i, j, l, mui, A.mu[j]);
                qmin = fmin(qmin, corr_isd(c, isdi, A.isd[j], flat_j));
                ++nlow;
            }
        }
        if (nlow >= p) theta = qmin - dq_row(A.em, i);
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

// Row kernels: 128 threads per block. With at most 8 entries per row, four
// blocks per SM (at most 128 registers) hold every row of a 65,536-point
// series in one wave.
template <int PM> constexpr int row_min_blocks() { return PM <= 8 ? 4 : 1; }

template <typename T, int PM>
__global__ void __launch_bounds__(128, row_min_blocks<PM>()) k_extend(ExtArgs<T> A)
{
    __shared__ unsigned sc[2];
    __shared__ unsigned long long smin[2];
    if (threadIdx.x < 2) {
        sc[threadIdx.x] = 0;
        smin[threadIdx.x] = (unsigned long long)__double_as_longlong(pinf());
    }
    __syncthreads();
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int cat = 0;
    double dbest = pinf(), lb = pinf();
    if (i < A.n0) {
        if (i >= A.nl) {
            A.st.flag[i] = ROW_DONE;
            A.thr[i] = T(pinf());
        } else {
            cat = extend_row<T, PM>(A, i, dbest, lb);
        }
    }
    if (A.min_dist_abs) {
        // smallest certified distance and smallest non-valid bound: warp,
        // block, then one global atomic each (non-negative doubles order
        // like their bit patterns)
        for (int o = 16; o > 0; o >>= 1) {
            dbest = fmin(dbest, __shfl_xor_sync(0xffffffffu, dbest, o));
            lb = fmin(lb, __shfl_xor_sync(0xffffffffu, lb, o));
        }
        if ((threadIdx.x & 31) == 0) {
            atomicMin(&smin[0], (unsigned long long)__double_as_longlong(dbest));
            atomicMin(&smin[1], (unsigned long long)__double_as_longlong(lb));
        }
    }
    // certified / recomputed counts: one shared add per warp, one global per block
    const unsigned b1 = __ballot_sync(0xffffffffu, cat == 1), b2 = __ballot_sync(0xffffffffu, cat == 2);
    if ((threadIdx.x & 31) == 0) {
        if (b1) atomicAdd(&sc[0], (unsigned)__popc(b1));
        if (b2) atomicAdd(&sc[1], (unsigned)__popc(b2));
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (sc[0]) atomicAdd(&A.out.stats[1], (unsigned long long)sc[0]);
        if (sc[1]) atomicAdd(&A.out.stats[2], (unsigned long long)sc[1]);
        if (A.min_dist_abs) {
            atomicMin(A.min_dist_abs, smin[0]);
            atomicMin(A.min_lb_abs, smin[1]);
        }
    }
}

// Largest p the register-resident row code is instantiated for.
inline int row_pm(int p) { return p <= 8 ? 8 : (p <= 16 ? 16 : 64); }

template <typename T>
void launch_extend(const ExtArgs<T> &a, cudaStream_t s)
{
    const int B = 128;
    const unsigned g = (unsigned)((a.n0 + B - 1) / B);
    switch (row_pm(a.p)) {
    case 8: k_extend<T, 8><<<g, B, 0, s>>>(a); break;
    case 16: k_extend<T, 16><<<g, B, 0, s>>>(a); break;
    default: k_extend<T, 64><<<g, B, 0, s>>>(a); break;
    }
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
// The kept keys sit in registers, sorted, updated by one fixed-length
// compare-and-swap pass per offered key; the group counts are read four at
// a time (the group stride is a multiple of 4).
template <typename T>
__device__ __forceinline__ bool key_before(T ka, int32_t ja, T kb, int32_t jb)
{
    return ka > kb || (ka == kb && ja < jb);
}

template <typename T, int PM>
__global__ void __launch_bounds__(128, row_min_blocks<PM>()) k_merge(MergeArgs<T> A)
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

    // The symmetric form wrote row-side lists for the column groups from the
    // row's band diagonal on, and appended the column-side candidates (cells
    // (i', i), i' < i) to the row's candidate list.
    const bool sym_on = sym_rule(A.allow_sym, *A.nflagged, A.nl) && fl == ROW_RECOMPUTE;
    T bk[PM];
    int32_t bj[PM];
    float bd[PM];               // per-entry error bound from the direct paths (< 0: band model)
    for_pm<PM>([&](int t) {
        bk[t] = T(-pinf());
        bj[t] = INT32_MAX;
        bd[t] = -1.0f;
    });
    T lastk = T(-pinf());       // the p-th kept key (a sentinel until p are kept)
    int32_t lastj = INT32_MAX;
    // (list entries are partners of this length, 0 <= j < n_l; the guard,
    // and the clamp of the counts below, keep a slot that no kernel wrote
    // at this length from sending a read out of range)
    auto offer = [&](T v, int32_t j, float dq) {
        if (j < 0 || j >= A.nl) return;
        if (!key_before(v, j, lastk, lastj)) return;
        T cv = v;
        int32_t cj = j;
        float cd = dq;
        for_pm<PM>([&](int t) {
            if (t < p && key_before(cv, cj, bk[t], bj[t])) {
                const T tk = bk[t];
                const int32_t tj = bj[t];
                const float td = bd[t];
                bk[t] = cv;
                bj[t] = cj;
                bd[t] = cd;
                cv = tk;
                cj = tj;
                cd = td;
            }
        });
        for_pm<PM>([&](int t) {
            if (t == p - 1) {
                lastk = bk[t];
                lastj = bj[t];
            }
        });
    };
    if (fl == ROW_DIRECT) {
        const int64_t d = A.dindex[i];
        for (int g = 0; g < A.dnblk; ++g) {
            const int64_t slot = d * A.dnblk + g;
            if ((int64_t)g * direct_cols_per_block_dev() >= A.nl) break;
            const int cnt = min(max(A.dcnt[slot], 0), p);
            for (int c = 0; c < cnt; ++c) offer(A.dkey[slot * p + c], A.dj[slot * p + c], A.ddq[slot * p + c]);
        }
    } else {
        const int g0 = sym_on ? (int)(((i / A.R) * (int64_t)A.R) / A.group_w) : 0;
        const int64_t gl = (A.nl + A.group_w - 1) / A.group_w;
        const int gend = (int)(gl < A.ngroups ? gl : A.ngroups);
        const int4 *c4 = reinterpret_cast<const int4 *>(A.scnt + i * A.ngroups);
        for (int gq = g0 & ~3; gq < gend; gq += 16) {
            int4 cv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) cv[u] = gq + 4 * u < gend ? c4[(gq >> 2) + u] : make_int4(0, 0, 0, 0);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int cs[4] = {cv[u].x, cv[u].y, cv[u].z, cv[u].w};
#pragma unroll
                for (int w = 0; w < 4; ++w) {
                    const int g = gq + 4 * u + w;
                    if (g < g0 || g >= gend) continue;
                    const int64_t slot = i * A.ngroups + g;
                    const int cnt = min(max(cs[w], 0), p);
                    for (int c = 0; c < cnt; ++c) offer(A.skey[slot * p + c], A.sj[slot * p + c], -1.0f);
                }
            }
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
        for (int c = 0; c < cc; ++c) offer(A.ckey[i * A.cap + c], A.cj[i * A.cap + c], -1.0f);
    }
    int nb = 0;
    for_pm<PM>([&](int t) { nb += (t < p && bj[t] != INT32_MAX); });
    if (nb < need) {
        A.thr[i] = T(-pinf());
        A.st.flag[i] = ROW_RECOMPUTE;
        atomicAdd(A.overflow, 1ull);
        atomicAdd(A.overflow + 8, 1ull);
        return;
    }
    const double isdi = A.isd[i];
    RowEnts<PM> r;
    for_pm<PM>([&](int e) {
        r.j[e] = -1;
        r.q[e] = -pinf();
        r.qk[e] = ord64(-pinf());
        r.dq[e] = 0.0f;
        if (e >= p) return;
        const int64_t at = (int64_t)e * n0 + i;
        if (e < nb) {
            const int32_t j = bj[e];
            const double inv = (double)A.col[j].inv;
            const bool flat_j = A.run[j] >= l;
            const double c = (flat_j || inv == 0.0) ? 0.0 : (double)bk[e] / inv;
            const float dq = flat_j ? 0.0f : (bd[e] >= 0.0f ? bd[e] : (float)dq_pair(A.em, i, j));
            A.st.ent_j[at] = j;
            A.st.ent_c[at] = c;
            A.st.ent_dq[at] = dq;
            r.j[e] = j;
            r.q[e] = corr_isd(c, isdi, A.isd[j], flat_j);
            r.qk[e] = ord64(r.q[e]);
            r.dq[e] = dq;
        } else {
            A.st.ent_j[at] = -1;
            A.st.ent_c[at] = 0.0;
            A.st.ent_dq[at] = 0.0f;
        }
    });
    refine_reported<PM>(A.x, A.xh, A.xl, i, l, A.mu[i], isdi, A.mu, A.isd, A.em, A.st, n0, r, A.m_max,
                        &A.out.stats[3], &A.out.stats[12]);
    report_row<PM>(A.out, A.vm, n0, i, l, r, nb, A.m_max);
    for_pm<PM>([&](int e) {
        if (r.j[e] >= 0) A.st.ent_qb[(int64_t)e * n0 + i] = r.q[e];
    });
    A.st.base[i] = l;
    const double sqm2i = sqrt(A.m2[i]);
    const double sig = sqm2i / sqrt((double)l);
    A.st.sigb[i] = sig;
    if (ntc <= p) {
        A.st.bnum[i] = pinf();
    } else {
        // unstored partners have keys <= the p-th kept key, each within its
        // error bound (band model, or the direct paths' largest at this length)
        double dqb = dq_row(A.em, i);
        if (fl == ROW_DIRECT) dqb = fmax(dqb, (double)*A.ddq_max);
        double qp = (double)lastk / sqm2i + dqb;
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
    const unsigned g = (unsigned)((a.nl + B - 1) / B);
    switch (row_pm(a.p)) {
    case 8: k_merge<T, 8><<<g, B, 0, s>>>(a); break;
    case 16: k_merge<T, 16><<<g, B, 0, s>>>(a); break;
    default: k_merge<T, 64><<<g, B, 0, s>>>(a); break;
    }
}
template void launch_merge<float>(const MergeArgs<float> &, cudaStream_t);
template void launch_merge<double>(const MergeArgs<double> &, cudaStream_t);

template <typename T>
__global__ void k_submp_mark(SubmpArgs<T> A)
{
    const double md = __longlong_as_double((long long)*A.min_dist_abs);
    const double ml = __longlong_as_double((long long)*A.min_lb_abs);
    const int decision = md < ml ? 0 : ((double)*A.nonvalid < A.limit ? 1 : 2);
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    bool skip = false;
    if (i < A.nl) {
        const int32_t f = A.flag[i];
        if (decision == 2) {
            if (f == ROW_DONE) {                // the full profile recomputes certified rows too
                A.flag[i] = ROW_RECOMPUTE;
                A.thr[i] = T(-pinf());
            }
        } else if (f == ROW_RECOMPUTE || f == ROW_FLAT) {
            skip = !(decision == 1 && A.lbmax[i] < md);
            if (skip) {
                A.flag[i] = ROW_SKIP;
                A.thr[i] = T(pinf());
                A.nnd[i] = __longlong_as_double(0x7ff8000000000000LL);
                A.nnj[i] = -1;
            }
        }
    }
    const int c = __syncthreads_count(skip);
    if (threadIdx.x == 0 && c) atomicAdd(&A.stats[10], (unsigned long long)c);
    if (blockIdx.x == 0 && threadIdx.x == 0) A.stats[11] = decision == 2 ? 1ull : 0ull;
}

template <typename T>
void launch_submp_mark(const SubmpArgs<T> &a, cudaStream_t s)
{
    const int B = 256;
    k_submp_mark<T><<<(unsigned)((a.nl + B - 1) / B), B, 0, s>>>(a);
}
template void launch_submp_mark<float>(const SubmpArgs<float> &, cudaStream_t);
template void launch_submp_mark<double>(const SubmpArgs<double> &, cudaStream_t);

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
    // bins hold computed keys rounded down: the true p-th best key is at least
    // top[p-1] less one key error, and a cell whose true key reaches that
    // computes at most one more key error lower; and one FP32 step
    th -= 2.0 * dq_row(em, i) * sqrt(m2[i]) + fabs(th) * 1e-6;
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
            // reserve by one add on a second counter that is never undone:
            // reservations are handed out in one order and, once one
            // overflows, every later one does too, so the blocks that fit
            // hold a prefix of the positions with no hole; ndirect[0] counts
            // only them. (An add undone on overflow let a concurrent block
            // take positions past a hole nobody wrote; a compare-and-swap
            // loop on one counter costs too much under contention.)
            const int r = atomicAdd(A.ndirect + 1, cnt);
            base = r + cnt <= A.max_direct ? r : -1;
            if (base >= 0) {
                atomicAdd(A.ndirect, cnt);
                if (A.stat_direct) atomicAdd(A.stat_direct, (unsigned long long)cnt);
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
    cudaMemsetAsync(a.ndirect, 0, 2 * sizeof(int32_t), s);   // rows taken, positions reserved
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
