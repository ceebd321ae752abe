"""The other workload configurations at full size, in the launch
configuration of the benchmark (FP32, full rows): the ECG-like series
(n = 262144, l in [128, 768], p = 10), the 256 uneven series (each with its
own length range), and the 2^21-sample seismic walk (p = 10, m = 3) at the
first lengths of its range (the whole range would take minutes). Checked on
sampled windows against the oracle and by properties that hold at any size."""
import math
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import oracle
import paper_2008_13447_gb300 as mad
import workloads

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2008_13447_gb300 import build
    build.build()
    oracle.build()


def tol(l):
    return 1e-4 * math.sqrt(l)


def check_rows(x, l, mp, ip, rows):
    ref_mp, ref_ip = oracle.rows(x, l, rows)
    for i, r, rj in zip(rows, ref_mp, ref_ip):
        assert abs(mp[i] - r) <= tol(l), (l, i, mp[i], r)
        if ip[i] != rj:     # a different partner must tie within tolerance
            assert abs(oracle.dist(x, l, int(i), int(ip[i])) - r) <= tol(l)
            assert abs(int(ip[i]) - int(i)) > oracle.excl(l)


def check_readouts(mot, dis):
    for m in mot:
        assert abs(m["dist"] - m["dist_recheck"]) <= tol(m["len"])
    for d in dis:
        if d["len"] > 0:
            assert abs(d["dist"] - d["dist_recheck"]) <= tol(d["len"])


def test_ecg262k_full_range():
    w = workloads.make("ecg262k")
    x = w.series[0]
    n = len(x)
    ctx = mad.mad_create(x, precision=mad.MAD_FP32, k_max=w.k, m_max=w.m, keep_profiles=True)
    try:
        mad.mad_profile(ctx, w.lmin[0], w.lmax[0], w.p)
        rng = np.random.default_rng(31)
        for l in (128, 129, 250, 500, 767, 768):
            mp, ip, _, _ = mad.mad_matrix_profile(ctx, 0, l, n, w.m)
            check_rows(x, l, mp, ip, list(rng.integers(0, n - l + 1, 4)) + [0, n - l])
        st = mad.mad_stats(ctx, 0)
        assert [s["len"] for s in st] == list(range(w.lmin[0], w.lmax[0] + 1))
        # the quasi-periodic series is the pruned regime: most rows certified
        assert sum(s["certified"] for s in st[1:]) > 0.5 * sum(s["rows"] for s in st[1:])
        check_readouts(mad.mad_motifs(ctx, 0, w.k), mad.mad_discords(ctx, 0, w.k, w.m))
    finally:
        mad.mad_destroy(ctx)


def test_batch256_all_series():
    w = workloads.make("batch256")
    ctx = mad.mad_create_batch(w.series, precision=mad.MAD_FP32, k_max=w.k, m_max=w.m, keep_profiles=True)
    try:
        mad.mad_profile_batch(ctx, w.lmin, w.lmax, w.p)
        rng = np.random.default_rng(32)
        sizes = [len(s) for s in w.series]
        picks = sorted(set(list(rng.integers(0, len(w.series), 12)) + [int(np.argmin(sizes)), int(np.argmax(sizes))]))
        for si in picks:
            x = w.series[si]
            n = len(x)
            a, b = w.lmin[si], w.lmax[si]
            for l in (a, (a + b) // 2, b):
                mp, ip, _, _ = mad.mad_matrix_profile(ctx, si, l, n, w.m)
                check_rows(x, l, mp, ip, list(rng.integers(0, n - l + 1, 2)) + [n - l])
            vm = mad.mad_valmp(ctx, si, n - a + 1)
            assert np.all((vm["len"] >= a) & (vm["len"] <= b))
            check_readouts(mad.mad_motifs(ctx, si, w.k), mad.mad_discords(ctx, si, w.k, w.m))
    finally:
        mad.mad_destroy(ctx)


def test_seismic2m_first_lengths():
    w = workloads.make("seismic2m")
    x = w.series[0]
    n = len(x)
    lmin, lmax, m = w.lmin[0], w.lmin[0] + 2, w.m
    ctx = mad.mad_create(x, precision=mad.MAD_FP32, k_max=w.k, m_max=m, keep_profiles=True)
    try:
        mad.mad_profile(ctx, lmin, lmax, w.p)
        rng = np.random.default_rng(33)
        for l in range(lmin, lmax + 1):
            mp, ip, nnd, nnj = mad.mad_matrix_profile(ctx, 0, l, n, m)
            rows = [int(r) for r in rng.integers(0, n - l + 1, 3)] + [0, n - l]
            with ThreadPoolExecutor(len(rows)) as ex:
                profs = list(ex.map(lambda r: oracle.distance_profile(x, l, r), rows))
            for r, dp in zip(rows, profs):
                ref = np.sort(dp[np.isfinite(dp)])[:m]       # the m best matches (Def. "m-th best match")
                assert np.all(np.abs(nnd[r] - ref) <= tol(l)), (l, r, nnd[r], ref)
                for c in range(m):                          # partners: valid, distance as reported
                    j = int(nnj[r, c])
                    assert abs(j - r) > oracle.excl(l)
                    assert abs(dp[j] - nnd[r, c]) <= tol(l)
        check_readouts(mad.mad_motifs(ctx, 0, w.k), mad.mad_discords(ctx, 0, w.k, m))
    finally:
        mad.mad_destroy(ctx)
