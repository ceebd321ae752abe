"""Pins for the CPU oracle (no GPU).

Each test ties the oracle to something other than itself: closed forms of the
z-normalised distance, a brute-force numpy evaluation of the definitions, a
numerical minimisation of the paper's lower-bound expression, the exactness
claim of the pruned method, planted structure, and the decision logic of the
paper's worked example.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------------ helpers

def znorm_windows(x, l):
    """All z-normalised windows of length l (population std), by numpy."""
    W = np.lib.stride_tricks.sliding_window_view(np.asarray(x, float), l)
    return (W - W.mean(1, keepdims=True)) / W.std(1, keepdims=True)


def brute_matrix_profile(x, l, num=1, den=4, m_max=1):
    """Brute force: Euclidean distances between z-normalised windows."""
    Z = znorm_windows(x, l)
    nl = len(Z)
    E = math.ceil(l * num / den)
    D = np.sqrt(((Z[:, None, :] - Z[None, :, :]) ** 2).sum(-1))
    I = np.arange(nl)
    D[np.abs(I[:, None] - I[None, :]) <= E] = np.inf
    order = np.lexsort((np.broadcast_to(I, D.shape), D), axis=1)
    nnj = order[:, :m_max]
    nnd = np.take_along_axis(D, nnj, 1)
    return nnd[:, 0], nnj[:, 0], nnd, nnj, D


# ---------------------------------------------------------------- distance

def test_exclusion_zone_is_ceil():
    for l in range(2, 200):
        assert oracle.excl(l, 1, 4) == math.ceil(l / 4)
        assert oracle.excl(l, 1, 2) == math.ceil(l / 2)


def test_window_stats_population():
    x = workloads.random_walk(500, 11)
    for l, i in [(7, 0), (64, 100), (128, 372)]:
        mu, sd = oracle.window_stats(x, l, i)
        assert mu == pytest.approx(np.mean(x[i:i + l]), rel=1e-13)
        assert sd == pytest.approx(np.std(x[i:i + l]), rel=1e-12)   # ddof=0


def test_distance_formula_matches_znormalised_euclidean():
    # Eq. DIST (through the correlation) against the definition of the
    # z-normalised Euclidean distance, two different formulas.
    rng = np.random.default_rng(0)
    x = workloads.random_walk(2000, 3)
    for _ in range(200):
        l = int(rng.integers(4, 300))
        i, j = rng.integers(0, len(x) - l + 1, 2)
        a = oracle.dist(x, l, i, j)
        zi, zj = znorm_windows(x[i:i + l], l)[0], znorm_windows(x[j:j + l], l)[0]
        assert a == pytest.approx(np.linalg.norm(zi - zj), rel=1e-9, abs=1e-9)
        assert a == pytest.approx(oracle.dist_direct(x, l, i, j), rel=1e-9, abs=1e-9)


def test_distance_closed_forms():
    l = 64
    t = np.arange(3 * l, dtype=float)
    s = np.sin(2 * np.pi * t / l)
    # identical windows one period apart: q = 1, d = 0
    assert oracle.dist(s, l, 0, l) == pytest.approx(0.0, abs=1e-6)
    # a quarter period apart: sin against cos over whole periods, q = 0, d = sqrt(2 l)
    assert oracle.dist(s, l, 0, l // 4) == pytest.approx(math.sqrt(2 * l), rel=1e-12)
    # half a period apart: the negated window, q = -1, d = 2 sqrt(l)
    assert oracle.dist(s, l, 0, l // 2) == pytest.approx(2 * math.sqrt(l), rel=1e-12)
    # an affine copy (positive scale) is at distance 0
    rng = np.random.default_rng(5)
    p = rng.standard_normal(40)
    x = np.concatenate([p, rng.standard_normal(30), 3.5 * p - 7.0])
    assert oracle.dist(x, 40, 0, 70) == pytest.approx(0.0, abs=1e-6)
    # a negative scale is at the maximum 2 sqrt(l)
    x2 = np.concatenate([p, rng.standard_normal(30), -0.25 * p + 1.0])
    assert oracle.dist(x2, 40, 0, 70) == pytest.approx(2 * math.sqrt(40), rel=1e-12)


def test_distance_range_symmetry_identity():
    rng = np.random.default_rng(1)
    x = workloads.ar2(1500, 9)
    for _ in range(300):
        l = int(rng.integers(3, 200))
        i, j = rng.integers(0, len(x) - l + 1, 2)
        d = oracle.dist(x, l, i, j)
        assert 0.0 <= d <= 2 * math.sqrt(l) + 1e-12
        assert d == oracle.dist(x, l, j, i)
        assert oracle.dist(x, l, i, i) == pytest.approx(0.0, abs=1e-6)


def test_flat_window_reading():
    x = np.concatenate([np.full(50, 2.5), workloads.random_walk(100, 4), np.full(50, -1.0)])
    l = 20
    assert oracle.pearson(x, l, 0, 170) == 1.0          # both flat
    assert oracle.dist(x, l, 0, 170) == 0.0
    assert oracle.pearson(x, l, 0, 80) == 0.0           # one flat
    assert oracle.dist(x, l, 0, 80) == pytest.approx(math.sqrt(2 * l))


# ---------------------------------------------------------- matrix profile

@pytest.mark.parametrize("l,num,den", [(16, 1, 4), (24, 1, 2), (9, 1, 4)])
def test_matrix_profile_brute_force(l, num, den):
    x = workloads.random_walk(180, 21)
    mp, ip, nnd, nnj = oracle.matrix_profile(x, l, m_max=3, num=num, den=den)
    bmp, bip, bnnd, bnnj, _ = brute_matrix_profile(x, l, num, den, m_max=3)
    np.testing.assert_allclose(mp, bmp, rtol=1e-9, atol=1e-9)
    np.testing.assert_allclose(nnd, bnnd, rtol=1e-9, atol=1e-9)
    # indices agree except where competing distances are within rounding
    bad = ip != bip
    assert bad.sum() <= 2


def test_matrix_profile_exclusion_respected():
    x = workloads.ar2(400, 2)
    for l in (10, 33):
        E = oracle.excl(l)
        mp, ip, nnd, nnj = oracle.matrix_profile(x, l, m_max=4)
        i = np.arange(len(mp))
        assert np.all(np.abs(nnj - i[:, None]) > E)
        prof = oracle.distance_profile(x, l, 100)
        assert np.all(np.isinf(prof[100 - E:100 + E + 1]))
        assert np.all(np.isfinite(np.delete(prof, np.arange(100 - E, 100 + E + 1))))


def test_row_matches_matrix_profile():
    x = workloads.random_walk(300, 8)
    mp, ip, nnd, nnj = oracle.matrix_profile(x, 30, m_max=2)
    for i in (0, 17, 150, 270):
        r = oracle.row(x, 30, i, m_max=2)
        assert r[0] == mp[i] and r[1] == ip[i]
        np.testing.assert_array_equal(r[2], nnd[i])


# ------------------------------------------------------------- lower bound

def _lb_numeric(x, l, k, row, other):
    """Minimise Eq. LB-min over (mu', sigma') numerically. ``row`` is the
    window whose longer extension is known, ``other`` the one whose last k
    values are treated as unknown."""
    from scipy.optimize import minimize
    tr = x[row:row + l]
    to = x[other:other + l]
    zr = (tr - tr.mean()) / tr.std()
    s_l = tr.std()
    s_lk = x[row:row + l + k].std()

    def f(v):
        mu, logs = v
        return np.sum(((to - mu) / math.exp(logs) - zr) ** 2)

    best = np.inf
    for mu0 in (to.mean(), to.mean() + to.std()):
        for ls0 in (math.log(to.std()), math.log(to.std()) + 3.0, math.log(to.std()) + 8.0):
            r = minimize(f, [mu0, ls0], method="Nelder-Mead",
                         options=dict(xatol=1e-12, fatol=1e-14, maxiter=20000, maxfev=40000))
            best = min(best, r.fun)
    return s_l / s_lk * math.sqrt(max(best, 0.0))


def test_lower_bound_closed_form_is_the_minimum():
    pytest.importorskip("scipy")
    x = workloads.random_walk(600, 12)
    rng = np.random.default_rng(3)
    checked_pos = checked_neg = 0
    for _ in range(40):
        l, k = 24, int(rng.integers(1, 10))
        row, other = rng.integers(0, len(x) - l - k, 2)
        q = oracle.pearson(x, l, row, other)
        s_l = oracle.window_stats(x, l, row)[1]
        s_lk = oracle.window_stats(x, l + k, row)[1]
        closed = oracle.lower_bound(l, q, s_l, s_lk)
        num = _lb_numeric(x, l, k, row, other)
        if q > 0:
            checked_pos += 1
            assert closed == pytest.approx(num, rel=1e-4, abs=1e-6)
        else:
            checked_neg += 1
            # q <= 0: the infimum is approached as sigma' -> inf
            assert closed <= num + 1e-6
            assert closed == pytest.approx(num, rel=2e-2)
    assert checked_pos > 5 and checked_neg > 5


def test_lower_bound_never_exceeds_true_distance():
    # The reason the bound exists: LB(d^{l+k}) <= d^{l+k} for every k >= 1,
    # with either window as the row.
    for series in (workloads.random_walk(900, 1), workloads.ar2(900, 2), workloads.ecg_like(900, 3)):
        rng = np.random.default_rng(7)
        for _ in range(300):
            l = int(rng.integers(8, 80))
            k = int(rng.integers(1, 60))
            i, j = rng.integers(0, len(series) - l - k, 2)
            if i == j:
                continue
            q = oracle.pearson(series, l, i, j)
            d = oracle.dist(series, l + k, i, j)
            for row in (i, j):
                lb = oracle.lower_bound(l, q, oracle.window_stats(series, l, row)[1],
                                        oracle.window_stats(series, l + k, row)[1])
                assert lb <= d * (1 + 1e-12) + 1e-6   # sqrt of rounding in 1-q^2


def test_lower_bound_rank_preservation():
    # The ranking of a row's lower-bound profile is the same for every k.
    x = workloads.random_walk(700, 5)
    l, row = 32, 300
    cols = [j for j in range(len(x) - l - 40) if abs(j - row) > 8]
    q = np.array([oracle.pearson(x, l, row, j) for j in cols])
    s_l = oracle.window_stats(x, l, row)[1]
    ref = None
    for k in (1, 2, 5, 17, 40):
        s_lk = oracle.window_stats(x, l + k, row)[1]
        lb = np.array([oracle.lower_bound(l, qq, s_l, s_lk) for qq in q])
        order = np.lexsort((np.array(cols), lb))
        if ref is None:
            ref = order
        assert np.array_equal(order, ref)


def test_worked_example_decisions():
    # Example 2: only the decisions are pinned (the example's series is absent).
    g = json.load(open(os.path.join(GOLDEN, "example2_certification.json")))
    for r in g["rows"]:
        assert oracle.row_valid([r["minDist"]], 1, r["maxLB"]) == r["valid"]
    gl = g["global"]
    assert (gl["minDistAbs"] < gl["minLbAbs"]) == gl["motif_found"]
    # strictness: a tie is not valid
    assert not oracle.row_valid([3.0], 1, 3.0)
    # m-th best match: needs m stored distances below the bound
    assert oracle.row_valid([1.0, 2.0, 2.9], 3, 3.0)
    assert not oracle.row_valid([1.0, 2.0], 3, 3.0)


# ------------------------------------------------------------------ VALMP

def test_valmp_single_length_is_matrix_profile():
    x = workloads.random_walk(400, 6)
    l = 40
    v = oracle.valmp_plain(x, l, l)
    mp, ip, _, _ = oracle.matrix_profile(x, l)
    np.testing.assert_array_equal(v["dist"], mp)
    np.testing.assert_array_equal(v["nn"], ip)
    np.testing.assert_allclose(v["norm"], mp / math.sqrt(l), rtol=1e-15)
    assert np.all(v["len"] == l)


def test_valmp_brute_force_all_lengths():
    x = workloads.ar2(160, 13)
    lmin, lmax = 12, 19
    v = oracle.valmp_plain(x, lmin, lmax)
    n0 = len(x) - lmin + 1
    best = np.full(n0, np.inf)
    blen = np.zeros(n0, int)
    for l in range(lmin, lmax + 1):
        bmp = brute_matrix_profile(x, l)[0]
        nd = bmp / math.sqrt(l)
        for i in range(len(bmp)):
            if nd[i] < best[i] - 1e-9:
                best[i], blen[i] = nd[i], l
    np.testing.assert_allclose(v["norm"], best, rtol=1e-9)
    assert np.mean(v["len"] == blen) > 0.98


@pytest.mark.parametrize("gen,n,lmin,lmax,p,m_max", [
    ("rw", 500, 20, 34, 5, 1),
    ("rw", 420, 16, 24, 8, 3),
    ("ar2", 450, 18, 30, 5, 2),
    ("ecg", 900, 40, 60, 4, 1),
    ("planted", 1200, 30, 44, 5, 2),
])
def test_pruned_equals_independent_lengths(gen, n, lmin, lmax, p, m_max):
    if gen == "rw":
        x = workloads.random_walk(n, 31)
    elif gen == "ar2":
        x = workloads.ar2(n, 32)
    elif gen == "ecg":
        x = workloads.ecg_like(n, 33, period=40.0)
    else:
        x, _ = workloads.planted_walk(n, 34, motif_lengths=(30, 36), lmax=60)
    pl = oracle.valmp_plain(x, lmin, lmax, m_max=m_max, keep_nn=True)
    pr = oracle.valmod_pruned(x, lmin, lmax, p, m_max=m_max, keep_nn=True)
    for key in ("dist", "norm", "len", "nn"):
        np.testing.assert_array_equal(pl[key], pr[key])
    np.testing.assert_array_equal(pl["nnd"], pr["nnd"])
    np.testing.assert_array_equal(pl["nnj"], pr["nnj"])
    st = pr["stats"]
    assert np.all(st[:, 1] + st[:, 2] == st[:, 0])
    assert st[0, 2] == st[0, 0]                   # everything computed at lmin
    assert st[1:, 1].sum() > 0                    # the bound certified some rows


def test_pruned_prunes_on_periodic_data():
    # On quasi-periodic data most rows stay certified (the paper's regime).
    x = workloads.ecg_like(2000, 40, period=50.0)
    pr = oracle.valmod_pruned(x, 50, 60, 8)
    st = pr["stats"]
    assert st[1:, 2].sum() < 0.2 * st[1:, 0].sum()


@pytest.mark.parametrize("gen,n,lmin,lmax,p", [
    ("rw", 500, 20, 34, 5),
    ("rw", 300, 12, 20, 2),       # n log p / log n = 36 rows: full-profile fallbacks
    ("ar2", 450, 18, 30, 5),
    ("ecg", 900, 40, 60, 4),
    ("planted", 1200, 30, 44, 5),
])
def test_motif_mode_finds_every_lengths_motif(gen, n, lmin, lmax, p):
    # Algorithm 4's guarantee: at every length the smallest SubMP value is the
    # exact motif distance, and every value it defines is the exact matrix
    # profile; checked against independent per-length profiles.
    if gen == "rw":
        x = workloads.random_walk(n, 41)
    elif gen == "ar2":
        x = workloads.ar2(n, 42)
    elif gen == "ecg":
        x = workloads.ecg_like(n, 43, period=40.0)
    else:
        x, _ = workloads.planted_walk(n, 34, motif_lengths=(30, 36), lmax=60)
    mo = oracle.valmod_motif(x, lmin, lmax, p)
    pl = oracle.valmp_plain(x, lmin, lmax, m_max=1, keep_nn=True)
    st = mo["stats"]
    for li, l in enumerate(range(lmin, lmax + 1)):
        nl = n - l + 1
        exact = pl["nnd"][li, :nl, 0]
        sub = mo["submp"][li, :nl]
        d = np.isfinite(sub)
        np.testing.assert_array_equal(sub[d], exact[d])
        assert sub[d].min() == exact.min()
        assert st[li, 0] == nl and st[li, 1] + st[li, 2] == nl
        if st[li, 4]:
            assert d.all()                             # full profile: every row defined
        else:
            assert d.sum() == st[li, 1] + st[li, 3]   # valid + recomputed rows
    assert st[0, 4] == 1                               # lmin: the full profile
    # the variable-length motif (best normalised VALMP entry) is exact
    assert mo["norm"].min() == pl["norm"].min()
    i = int(np.argmin(mo["norm"]))
    assert mo["dist"][i] == pl["dist"][i] and mo["len"][i] == pl["len"][i]
    if (gen, p) == ("rw", 2):
        assert st[1:, 4].sum() > 0                     # the fallback ran
    if gen == "ecg":
        computed = np.where(st[1:, 4] == 1, st[1:, 0], st[1:, 3]).sum()
        assert computed < 0.5 * st[1:, 0].sum()       # it pruned (full profiles included)


def _znorm_dist(x, l, i, j):
    a, b = x[i:i + l], x[j:j + l]
    za, zb = (a - a.mean()) / a.std(), (b - b.mean()) / b.std()
    return float(np.sqrt(((za - zb) ** 2).sum()))


def test_motif_set_contains_planted_copies():
    # four noisy copies of one pattern in a random walk: the set grown from
    # the best pair holds all four (Sec. "Finding Motif Sets")
    rng = np.random.default_rng(61)
    n, L = 3000, 40
    x = np.cumsum(rng.standard_normal(n))
    pat = 3.0 * np.sin(np.linspace(0, 4 * np.pi, L)) * np.hanning(L)
    offs = [300, 1000, 1700, 2400]
    for o in offs:
        seg = x[o:o + L]
        x[o:o + L] = seg.mean() + pat * seg.std() + 0.05 * seg.std() * rng.standard_normal(L)
    pl = oracle.valmp_plain(x, L, L)
    top = oracle.topk_motifs(pl, 1)[0]
    sets = oracle.motif_sets(x, [(top[0], top[1], top[2], top[3])], D=4.0, cap=16)
    got = sets[0]
    for o in offs:
        assert any(abs(m - o) <= oracle.excl(L) for m in got), (o, got)


def test_motif_sets_brute_force_tiny():
    # the same growth rule restated with numpy distances on a tiny series
    x = workloads.random_walk(260, 62)
    l, num, den = 12, 1, 4
    E = int(np.ceil(l * num / den))
    nl = len(x) - l + 1
    pl = oracle.valmp_plain(x, l, l + 3)
    pairs = [(a, b, L, d) for a, b, L, d, _ in oracle.topk_motifs(pl, 3)]
    got = oracle.motif_sets(x, pairs, D=1.6, cap=10)
    used = []                           # (offset, length) of earlier members
    for (a, b, L, d), g in zip(pairs, got):
        EL = int(np.ceil(L * num / den))
        nL = len(x) - L + 1
        r = 1.6 * d
        cand = []
        for j in range(nL):
            if abs(j - a) <= EL or abs(j - b) <= EL:
                continue
            dj = min(_znorm_dist(x, L, a, j), _znorm_dist(x, L, b, j))
            if dj > r + 1e-9:
                continue
            if any(abs(j - m) <= max(EL, int(np.ceil(Lm * num / den))) for m, Lm in used):
                continue
            cand.append((dj, j))
        cand.sort()
        mem = [a, b]
        for dj, j in cand:
            if len(mem) >= 10:
                break
            if all(abs(j - m) > EL for m in mem):
                mem.append(j)
        assert [int(v) for v in g] == mem
        used += [(m, L) for m in mem]


def test_motif_set_properties():
    x = workloads.ar2(2000, 63)
    lmin, lmax = 24, 32
    pl = oracle.valmp_plain(x, lmin, lmax)
    pairs = [(a, b, L, d) for a, b, L, d, _ in oracle.topk_motifs(pl, 4)]
    sets = oracle.motif_sets(x, pairs, D=2.0, cap=12)
    seen = []
    for (a, b, L, d), mem in zip(pairs, sets):
        E = oracle.excl(L)
        assert mem[0] == a and mem[1] == b and len(mem) <= 12
        for i, m in enumerate(mem[2:]):
            assert min(oracle.dist(x, L, a, m), oracle.dist(x, L, b, m)) <= 2.0 * d + 1e-9
        for i in range(len(mem)):
            for j in range(i + 1, len(mem)):
                assert abs(mem[i] - mem[j]) > E
        for m in mem[2:]:
            assert all(abs(m - u) > max(E, oracle.excl(Lu)) for u, Lu in seen)
        seen += [(m, L) for m in mem]


@pytest.mark.parametrize("gen", ["rw", "ecg"])
def test_observation_gap_and_tlb(gen):
    # maxLB - minED > 0 exactly for the rows the bound certifies, and the
    # tightness LB / ED lies in (0, 1] (Eq. LB lower-bounds the distance)
    x = workloads.random_walk(700, 81) if gen == "rw" else workloads.ecg_like(900, 82, period=40.0)
    lmin, L = 30, 36
    pr = oracle.valmod_pruned(x, lmin, L, 5, observe_len=L)
    gap, tlb = pr["gap"], pr["tlb"]
    ok = np.isfinite(gap)
    assert ok.sum() > 0.9 * len(gap)
    # certified rows at L are those with a positive gap
    assert int((gap[ok] > 0).sum()) == pr["stats"][-1, 1]
    t = tlb[np.isfinite(tlb)]
    assert np.all(t > 0) and np.all(t <= 1 + 1e-12)


def test_global_discords_brute_force():
    # the global greedy restated over all (i, l) with numpy on a small series
    x = workloads.ar2(400, 95)
    lmin, lmax, m_max, k = 16, 22, 2, 4
    pl = oracle.valmp_plain(x, lmin, lmax, m_max=m_max, keep_nn=True)
    n = len(x)
    for m in (1, 2):
        got = oracle.discords_global(n, lmin, lmax, k, m_max, m, pl["nnd"], pl["nnj"])
        cand = []
        for li, l in enumerate(range(lmin, lmax + 1)):
            for i in range(n - l + 1):
                d = pl["nnd"][li, i, m - 1]
                if np.isfinite(d):
                    cand.append((-d / np.sqrt(l), -l, i, d))
        cand.sort()
        acc = []
        for s_, nl_, i, d in cand:
            l = -nl_
            if all(abs(i - a) > max(oracle.excl(l), oracle.excl(b)) for a, b, _ in acc):
                acc.append((i, l, d))
            if len(acc) == k:
                break
        assert [(g[0], g[1]) for g in got] == [(a, b) for a, b, _ in acc]
        assert np.allclose([g[2] for g in got], [d for _, _, d in acc])


def test_global_discords_planted_spike():
    x = workloads.random_walk(1500, 96)
    x[700] += 25.0
    pl = oracle.valmp_plain(x, 20, 30, keep_nn=True)
    top = oracle.discords_global(len(x), 20, 30, 1, 1, 1, pl["nnd"], pl["nnj"])[0]
    assert top[0] <= 700 < top[0] + top[1]


def _streamed_invariants(t, E):
    offs = [int(o) for o in t["off"].ravel() if o >= 0]
    assert len(offs) == len(set(offs))                      # a window in at most one cell
    for a in range(len(offs)):
        for b in range(a):
            assert abs(offs[a] - offs[b]) > E                # pairwise non-trivial
    for c in range(t["dist"].shape[1]):
        col = t["dist"][:, c]
        assert np.all(col[:-1] >= col[1:])                   # ranked within a column


def test_streamed_dkm_pins():
    x = workloads.ar2(700, 101)
    lmin, lmax, m_max, k = 20, 23, 3, 5
    pl = oracle.valmp_plain(x, lmin, lmax, m_max=m_max, keep_nn=True)
    n = len(x)
    for li, l in enumerate(range(lmin, lmax + 1)):
        nl = n - l + 1
        nd, nj = pl["nnd"][li, :nl], pl["nnj"][li, :nl]
        for m in (1, 2, 3):
            t = oracle.dkm_streamed(nd, nj, l, k, m)
            _streamed_invariants(t, oracle.excl(l))
            assert np.all(t["off"] >= 0)
            # no exclusion zone: the last column tried first is the exact top-k
            t0 = oracle.dkm_streamed(nd, nj, l, k, m, num=0, den=1)
            top = np.argsort(-nd[:, m - 1], kind="stable")[:k]
            assert list(t0["off"][:, m - 1]) == list(top)
            assert np.array_equal(t0["dist"][:, m - 1], nd[top, m - 1])
            assert np.array_equal(t0["nn"][:, m - 1], nj[top, m - 1])
            _streamed_invariants(t0, 0)
    # Algorithm 9's merge: per cell the largest d / sqrt(l) over the lengths
    for m in (1, 3):
        g = oracle.discords_streamed(n, lmin, lmax, k, m_max, m, pl["nnd"], pl["nnj"])
        for r in range(k):
            for c in range(m):
                best = None
                for li, l in enumerate(range(lmin, lmax + 1)):
                    nl = n - l + 1
                    t = oracle.dkm_streamed(pl["nnd"][li, :nl], pl["nnj"][li, :nl], l, k, m)
                    v = t["dist"][r, c] / np.sqrt(l)
                    if best is None or v >= best[0]:
                        best = (v, int(t["off"][r, c]), l)
                assert (g["norm"][r, c], int(g["off"][r, c]), int(g["len"][r, c])) == best


def test_streamed_dkm_planted_spike():
    # a spike on a noisy sine: the window at rank 1 of column 1 covers it
    # (windows over it that are more than E apart may follow at lower ranks:
    # the streamed form only keeps present entries pairwise non-trivial)
    rng = np.random.default_rng(102)
    t_ = np.arange(3000)
    x = np.sin(2 * np.pi * t_ / 50) + 0.05 * rng.standard_normal(3000)
    x[1300] += 3.0
    l = 24
    pl = oracle.valmp_plain(x, l, l, keep_nn=True)
    nl = len(x) - l + 1
    t = oracle.dkm_streamed(pl["nnd"][0, :nl], pl["nnj"][0, :nl], l, 3, 1)
    offs = [int(o) for o in t["off"][:, 0]]
    assert offs[0] <= 1300 < offs[0] + l, offs
    _streamed_invariants(t, oracle.excl(l))


def test_pruned_discords_all_valid_equals_streamed():
    # every window stored (p at least the non-trivial count): every row is
    # valid at every length, so the pruned iteration is the streamed form on
    # exact profiles, length by length
    x = workloads.ar2(70, 103)
    lmin, lmax, k = 10, 14, 4
    pl = oracle.valmp_plain(x, lmin, lmax, m_max=2, keep_nn=True)
    n = len(x)
    for m in (1, 2):
        g = oracle.valmod_discord(x, lmin, lmax, 64, k, m)
        assert np.array_equal(g["stats"][1:, 3], np.zeros(lmax - lmin, np.int64))   # nothing recomputed
        for li, l in enumerate(range(lmin, lmax + 1)):
            nl = n - l + 1
            t = oracle.dkm_streamed(pl["nnd"][li, :nl, :m], pl["nnj"][li, :nl, :m], l, k, m)
            assert np.array_equal(g["dkm_off"][li], t["off"])
            assert np.allclose(g["dkm_d"][li], t["dist"], rtol=1e-12, atol=0)
        ref = oracle.discords_streamed(n, lmin, lmax, k, 2, m, pl["nnd"], pl["nnj"])
        assert np.array_equal(g["off"], ref["off"]) and np.array_equal(g["len"], ref["len"])


def test_pruned_discords_exact_values_and_invariants():
    x = workloads.ar2(1200, 104)
    lmin, lmax, p, k, m = 20, 30, 5, 4, 2
    g = oracle.valmod_discord(x, lmin, lmax, p, k, m)
    pl = oracle.valmp_plain(x, lmin, lmax, m_max=m, keep_nn=True)
    st = g["stats"]
    assert st[0, 3] == st[0, 0]                                  # lmin: every row
    assert np.all(st[1:, 1] + st[1:, 2] <= st[1:, 0])
    assert np.all(st[1:, 3] <= st[1:, 2])
    assert st[1:, 2].sum() > st[1:, 3].sum() > 0                 # the second pass prunes
    for li, l in enumerate(range(lmin, lmax + 1)):
        t = dict(off=g["dkm_off"][li], dist=g["dkm_d"][li])
        _streamed_invariants(t, oracle.excl(l))
        for r in range(k):
            for c in range(m):
                o = t["off"][r, c]
                if o >= 0:                                       # only exact distances enter
                    assert abs(t["dist"][r, c] - pl["nnd"][li, o, c]) <= 1e-12 * pl["nnd"][li, o, c]
    # lmin = lmax: the streamed form
    g1 = oracle.valmod_discord(x, lmin, lmin, p, k, m)
    nl = len(x) - lmin + 1
    t = oracle.dkm_streamed(pl["nnd"][0, :nl], pl["nnj"][0, :nl], lmin, k, m)
    assert np.array_equal(g1["dkm_off"][0], t["off"])


def test_pruned_discords_planted_spike():
    # the spike's windows are far from their stored partners: non-valid, then
    # recomputed in the second pass and placed at rank 1 of column 1
    rng = np.random.default_rng(105)
    t_ = np.arange(2500)
    x = np.sin(2 * np.pi * t_ / 50) + 0.05 * rng.standard_normal(2500)
    x[1300] += 3.0
    lmin, lmax = 24, 30
    g = oracle.valmod_discord(x, lmin, lmax, 5, 3, 1)
    for li, l in enumerate(range(lmin, lmax + 1)):
        o = g["dkm_off"][li, 0, 0]
        assert o <= 1300 < o + l, (l, o)
    assert g["stats"][1:, 3].sum() < g["stats"][1:, 0].sum() // 10   # few rows recomputed


# ---------------------------------------------------------------- read-outs

def test_topk_motif_planted_pair():
    rng = np.random.default_rng(17)
    pat = np.cumsum(rng.standard_normal(48))
    x = workloads.random_walk(1500, 18)
    x[300:348] = 2.0 * pat + 5.0
    x[1000:1048] = 0.5 * pat - 3.0 + 1e-4 * rng.standard_normal(48)
    v = oracle.valmp_plain(x, 40, 48)
    mot = oracle.topk_motifs(v, 3)
    a, b, L, d, nd = mot[0]
    assert (a, b) == (300, 1000) and L == 48
    assert d < 0.01


def test_topk_motif_greedy_properties():
    x = workloads.random_walk(700, 19)
    v = oracle.valmp_plain(x, 20, 30)
    k = 8
    mot = oracle.topk_motifs(v, k)
    assert len(mot) == k
    nds = [m[4] for m in mot]
    assert nds == sorted(nds)

    def conflict(m1, m2):
        E = max(oracle.excl(m1[2]), oracle.excl(m2[2]))
        return any(abs(u - w) <= E for u in m1[:2] for w in m2[:2])

    for i in range(k):
        for j in range(i):
            assert not conflict(mot[i], mot[j])
    # maximality: every VALMP entry better than the last accepted one either
    # is an accepted pair or conflicts with an accepted pair listed before it
    order = np.lexsort((np.arange(len(v["norm"])), v["norm"]))
    last = mot[-1][4]
    for i in order:
        if v["norm"][i] > last:
            break
        cand = (min(i, v["nn"][i]), max(i, v["nn"][i]), v["len"][i])
        if any(cand == m[:3] for m in mot):
            continue
        assert any(conflict(cand, m) for m in mot if m[4] <= v["norm"][i])


def test_discord_planted_spike():
    x = workloads.ecg_like(3000, 41, period=60.0)
    x[1700] += 3.0
    l = 60
    mp, ip, nnd, nnj = oracle.matrix_profile(x, l)
    top = oracle.discords_one_length(mp, l, 3)
    o = top[0][0]
    assert o <= 1700 < o + l


def test_discord_table_merge_and_exclusion():
    x = workloads.ar2(600, 23)
    lmin, lmax, k, m_max = 16, 22, 4, 2
    pl = oracle.valmp_plain(x, lmin, lmax, m_max=m_max, keep_nn=True)
    dk = oracle.discords(len(x), lmin, lmax, k, m_max, pl["nnd"], pl["nnj"])
    n0 = len(x) - lmin + 1
    for m in range(m_max):
        for r in range(k):
            L = dk["len"][r, m]
            assert lmin <= L <= lmax
            # the winning length's own ranking has this offset at rank r
            nl = len(x) - L + 1
            sc = pl["nnd"][L - lmin, :nl, m]
            per = oracle.discords_one_length(sc, L, k, pl["nnj"][L - lmin, :nl, m])
            assert per[r][0] == dk["off"][r, m]
            assert dk["norm"][r, m] == pytest.approx(per[r][1] / math.sqrt(L))
            # no other length scores higher at this rank (ties go to the later length)
            for l2 in range(lmin, lmax + 1):
                nl2 = len(x) - l2 + 1
                per2 = oracle.discords_one_length(pl["nnd"][l2 - lmin, :nl2, m], l2, k)
                if len(per2) > r:
                    v2 = per2[r][1] / math.sqrt(l2)
                    assert v2 <= dk["norm"][r, m] + 1e-15
                    if l2 > L:
                        assert v2 < dk["norm"][r, m]
        # per-length picks are pairwise non-trivial and descending
        for l2 in range(lmin, lmax + 1):
            nl2 = len(x) - l2 + 1
            per2 = oracle.discords_one_length(pl["nnd"][l2 - lmin, :nl2, m], l2, k)
            sc = [p[1] for p in per2]
            assert sc == sorted(sc, reverse=True)
            offs = [p[0] for p in per2]
            E = oracle.excl(l2)
            assert all(abs(a - b) > E for a in offs for b in offs if a != b)
    assert n0 > 0


def test_planted_workload_recovered_small():
    # A scaled-down planted series: the top motif is one of the planted pairs
    # and the top discord covers a planted discord.
    x, info = workloads.planted_walk(6000, 44, motif_lengths=(60, 80), lmax=100)
    v = oracle.valmp_plain(x, 64, 72, keep_nn=True)
    mot = oracle.topk_motifs(v, 3)
    planted = [(a, b) for a, b, L in info.motifs]
    hit = False
    for a, b, L, d, nd in mot[:2]:
        for pa, pb in planted:
            if abs(a - pa) <= 20 and abs(b - pb) <= 20:
                hit = True
    assert hit
    dk = oracle.discords(len(x), 64, 72, 3, 1, v["nnd"], v["nnj"])
    offs = dk["off"][:, 0]
    lens = dk["len"][:, 0]
    assert any(o <= info.spike < o + L or o <= info.level_shift < o + L for o, L in zip(offs, lens))
