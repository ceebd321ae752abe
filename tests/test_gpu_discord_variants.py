"""Discord read-out variants on the GPU.

Global-greedy variable-length discords: the ranking over the GPU's own kept
profiles identical to the oracle's ranking of the same profiles; against the
oracle's own profiles, identical picks (FP64) or the same scores within the
distance tolerance (FP32); pairwise separation by the larger exclusion zone;
a planted spike; argument and state errors.

Streamed dkm (Algorithms 7 and 8 as printed, merged by Algorithm 9): identical
to the oracle given the same kept profiles, for k on both sides of one warp's
32 ranks; FP64 also identical to the oracle's own profiles; errors."""
import numpy as np
import pytest

import oracle
import paper_2008_13447_gb300 as mad
import workloads

pytestmark = pytest.mark.gpu
PRECS = [pytest.param(mad.MAD_FP64, id="fp64"), pytest.param(mad.MAD_FP32, id="fp32")]


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2008_13447_gb300 import build
    build.build()
    oracle.build()


def kept_profiles(ctx, n, lmin, lmax, m_max):
    n0 = n - lmin + 1
    nnd = np.full((lmax - lmin + 1, n0, m_max), np.nan)
    nnj = np.full((lmax - lmin + 1, n0, m_max), -1, np.int64)
    for li, l in enumerate(range(lmin, lmax + 1)):
        _, _, d, j = mad.mad_matrix_profile(ctx, 0, l, n, m_max)
        nnd[li, :n - l + 1] = d
        nnj[li, :n - l + 1] = j
    return nnd, nnj


def as_cols(got, k, m):
    cols = []
    for c in range(m):
        col = [(g["off"], g["len"], g["dist"], g["norm_dist"], g["nn"]) for g in got[c::m] if g["len"] > 0]
        cols.append(col)
    return cols


@pytest.mark.parametrize("prec", PRECS)
def test_discord_variants_match_oracle(prec):
    x = workloads.ar2(2500, 97)
    n, lmin, lmax, m_max, k = len(x), 24, 40, 2, 8
    ctx = mad.mad_create(x, precision=prec, k_max=4, m_max=m_max, keep_profiles=True)
    try:
        mad.mad_profile(ctx, lmin, lmax, 5)
        got = mad.mad_discords_global(ctx, 0, k, m_max)
        streamed = {(k2, m): mad.mad_discords_streamed(ctx, 0, k2, m) for k2 in (6, 40) for m in (1, 2)}
        assert len(got) == k * m_max
        assert [(g["rank"], g["m"]) for g in got] == [(r + 1, c + 1) for r in range(k) for c in range(m_max)]
        nnd, nnj = kept_profiles(ctx, n, lmin, lmax, m_max)
    finally:
        mad.mad_destroy(ctx)
    cols = as_cols(got, k, m_max)
    pl = oracle.valmp_plain(x, lmin, lmax, m_max=m_max, keep_nn=True)
    tol = 1e-9 if prec == mad.MAD_FP64 else 1e-4
    for c in range(m_max):
        # the same ranking of the same profiles: identical
        same = oracle.discords_global(n, lmin, lmax, k, m_max, c + 1, nnd, nnj)
        assert cols[c] == same
        # pairwise apart by the larger exclusion zone
        for a in range(len(cols[c])):
            for b in range(a):
                ia, la = cols[c][a][:2]
                ib, lb = cols[c][b][:2]
                assert abs(ia - ib) > max(oracle.excl(la), oracle.excl(lb))
        # the oracle's own profiles: same scores; FP64 also the same picks
        ref = oracle.discords_global(n, lmin, lmax, k, m_max, c + 1, pl["nnd"], pl["nnj"])
        assert len(ref) == len(cols[c]) == k
        for g, r in zip(cols[c], ref):
            assert abs(g[3] - r[3]) <= tol * max(1.0, r[3]), (g, r)
            if prec == mad.MAD_FP64:
                assert g[:2] == r[:2]
        for g in got[c::m_max]:
            assert abs(g["dist"] - g["dist_recheck"]) <= tol * np.sqrt(g["len"]) * max(1.0, g["dist"])
    for (k2, m), st in streamed.items():
        assert [(g["rank"], g["m"]) for g in st] == [(r + 1, c + 1) for r in range(k2) for c in range(m)]
        got_t = [(g["off"], g["len"], g["dist"], g["norm_dist"], g["nn"]) for g in st]
        # the same profiles: identical
        ref = oracle.discords_streamed(n, lmin, lmax, k2, m_max, m, nnd, nnj)
        want = [(int(ref["off"][r, c]), int(ref["len"][r, c]), float(ref["dist"][r, c]),
                 float(ref["norm"][r, c]), int(ref["nn"][r, c])) if ref["len"][r, c] > 0
                else (-1, 0, None, None, -1) for r in range(k2) for c in range(m)]
        for g, w in zip(got_t, want):
            if w[1] == 0:
                assert (g[0], g[1], g[4]) == (-1, 0, -1)
            else:
                assert g == w
        assert sum(w[1] > 0 for w in want) >= min(k2, 6)
        if prec == mad.MAD_FP64:
            # the oracle's own profiles: the same cells, values within FP64 rounding
            ref = oracle.discords_streamed(n, lmin, lmax, k2, m_max, m, pl["nnd"], pl["nnj"])
            for r in range(k2):
                for c in range(m):
                    g = st[r * m + c]
                    assert (g["off"], g["len"]) == (ref["off"][r, c], ref["len"][r, c])
                    if g["len"] > 0:
                        assert abs(g["norm_dist"] - ref["norm"][r, c]) <= 1e-9 * max(1.0, ref["norm"][r, c])


def test_global_discords_planted_spike():
    x = workloads.random_walk(3000, 98)
    x[1700] += 30.0
    ctx = mad.mad_create(x, precision=mad.MAD_FP32, k_max=2, m_max=1, keep_profiles=True)
    try:
        mad.mad_profile(ctx, 20, 36, 5)
        top = mad.mad_discords_global(ctx, 0, 3, 1)
    finally:
        mad.mad_destroy(ctx)
    assert top[0]["off"] <= 1700 < top[0]["off"] + top[0]["len"]
    assert top[0]["norm_dist"] >= top[1]["norm_dist"] >= top[2]["norm_dist"]


def test_global_discords_more_ranks_than_candidates():
    # a short series: the exclusion zones leave fewer than k candidates
    x = workloads.ar2(120, 99)
    n, lmin, lmax = len(x), 30, 34
    ctx = mad.mad_create(x, precision=mad.MAD_FP64, k_max=2, m_max=1, keep_profiles=True)
    try:
        mad.mad_profile(ctx, lmin, lmax, 3)
        got = mad.mad_discords_global(ctx, 0, 64, 1)
        nnd, nnj = kept_profiles(ctx, n, lmin, lmax, 1)
    finally:
        mad.mad_destroy(ctx)
    same = oracle.discords_global(n, lmin, lmax, 64, 1, 1, nnd, nnj)
    filled = [g for g in got if g["len"] > 0]
    assert 0 < len(filled) == len(same) < 64
    assert [(g["off"], g["len"], g["dist"], g["norm_dist"], g["nn"]) for g in filled] == same
    assert all(g["off"] == -1 and np.isnan(g["dist"]) for g in got[len(filled):])


@pytest.mark.parametrize("fn", [mad.mad_discords_global, mad.mad_discords_streamed], ids=["global", "streamed"])
def test_discord_variants_arguments(fn):
    x = workloads.random_walk(600, 100)
    ctx = mad.mad_create(x, precision=mad.MAD_FP32, k_max=2, m_max=2, keep_profiles=True)
    try:
        with pytest.raises(mad.MadError) as e:
            fn(ctx, 0, 2, 1)                                # before mad_profile
        assert e.value.status == mad.MAD_ESTATE
        mad.mad_profile(ctx, 20, 24, 3)
        for k, m in ((0, 1), (65, 1), (2, 0), (2, 3)):
            with pytest.raises(mad.MadError) as e:
                fn(ctx, 0, k, m)
            assert e.value.status == mad.MAD_EINVAL
        assert len(fn(ctx, 0, 64, 2)) == 128                # k above k_max is allowed here
    finally:
        mad.mad_destroy(ctx)
    ctx = mad.mad_create(x, precision=mad.MAD_FP32, k_max=2, m_max=1)
    try:
        mad.mad_profile(ctx, 20, 24, 3)
        with pytest.raises(mad.MadError) as e:
            fn(ctx, 0, 2, 1)                                # no kept profiles
        assert e.value.status == mad.MAD_EINVAL
    finally:
        mad.mad_destroy(ctx)
    ctx = mad.mad_create(x, precision=mad.MAD_FP32, k_max=2, m_max=1, keep_profiles=True, mode=1)
    try:
        mad.mad_profile(ctx, 20, 24, 3)
        with pytest.raises(mad.MadError) as e:
            fn(ctx, 0, 2, 1)                                # motif mode
        assert e.value.status == mad.MAD_ESTATE
    finally:
        mad.mad_destroy(ctx)
