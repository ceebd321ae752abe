"""The benchmark workload at full size (planted random walk, n = 65536,
l in [256, 512], p = 5) in the launch configuration bench.py times, on both
the FP32 and the FP64 path: every length's matrix profile is compared with
the oracle on 1000 sampled windows at 8 lengths (first, second, middle and
last lengths included), and checked by properties that hold at any size."""
import math

import numpy as np
import pytest

import oracle
import paper_2008_13447_gb300 as mad
import workloads

pytestmark = pytest.mark.gpu


LENGTHS = (256, 257, 300, 384, 450, 500, 511, 512)
SAMPLE = 1000       # windows per length compared with the oracle


@pytest.fixture(scope="module")
def workload():
    from paper_2008_13447_gb300 import build
    build.build()
    oracle.build()
    w = workloads.make("planted65k")
    x = w.series[0]
    n = len(x)
    rng = np.random.default_rng(5)
    sample = {}
    for l in LENGTHS:
        rows = sorted(set(int(r) for r in rng.integers(0, n - l + 1, SAMPLE)) | {0, n - l})
        ref_mp, ref_ip = oracle.rows(x, l, rows)
        sample[l] = (np.array(rows), ref_mp, ref_ip)
    return w, sample


@pytest.fixture(scope="module", params=[mad.MAD_FP32, mad.MAD_FP64], ids=["fp32", "fp64"])
def planted(request, workload):
    w, sample = workload
    prec = request.param
    x = w.series[0]
    ctx = mad.mad_create(x, precision=prec, k_max=w.k, m_max=w.m, keep_profiles=True)
    try:
        mad.mad_profile(ctx, w.lmin[0], w.lmax[0], w.p)
        n = len(x)
        res = dict(
            w=w, x=x, prec=prec, sample=sample,
            prof={l: mad.mad_matrix_profile(ctx, 0, l, n, 1) for l in LENGTHS},
            vm=mad.mad_valmp(ctx, 0, n - w.lmin[0] + 1),
            mot=mad.mad_motifs(ctx, 0, w.k),
            dis=mad.mad_discords(ctx, 0, w.k, w.m),
            st=mad.mad_stats(ctx, 0),
            full_at={},
        )
        # VALMP consistency needs each row's profile at its VALMP length
        vm = res["vm"]
        for l in np.unique(vm["len"][:: max(1, n // 64)]):
            res["full_at"][int(l)] = mad.mad_matrix_profile(ctx, 0, int(l), n, 1)[0]
    finally:
        mad.mad_destroy(ctx)
    return res


def tol(prec, l, d):
    """FP32: 1e-4 sqrt(l) absolute; FP64: 1e-9 relative with the floor that
    a 1e-12 correlation error puts on d near 0 (see parity_util)."""
    if prec == mad.MAD_FP32:
        return 1e-4 * math.sqrt(l)
    return 1e-9 * abs(d) + 2 * l * 1e-12 / max(2 * abs(d), math.sqrt(2 * l * 1e-12))


def test_sampled_rows_match_oracle(planted):
    x, prec = planted["x"], planted["prec"]
    flips = 0
    for l, (mp, ip, _, _) in planted["prof"].items():
        rows, ref_mp, ref_ip = planted["sample"][l]
        assert len(rows) >= SAMPLE * 0.95
        for i, r, rj in zip(rows, ref_mp, ref_ip):
            t = tol(prec, l, r)
            assert abs(mp[i] - r) <= t, (l, i, mp[i], r)
            if ip[i] != rj:
                # a different partner: valid and tied with the oracle's within tolerance
                d = oracle.dist(x, l, int(i), int(ip[i]))
                assert abs(d - r) <= t
                assert abs(int(ip[i]) - int(i)) > oracle.excl(l)
                flips += 1
    print("index near-ties:", flips)


def test_valmp_is_minimum_over_lengths(planted):
    vm = planted["vm"]
    n0 = len(vm["dist"])
    for l, mp in planted["full_at"].items():
        rows = np.nonzero(vm["len"] == l)[0]
        np.testing.assert_array_equal(vm["dist"][rows], mp[rows])
    for l, (mp, _, _, _) in planted["prof"].items():
        nl = len(mp)
        assert np.all(vm["norm"][:nl] <= mp / math.sqrt(l) + 1e-15)
    assert np.all((vm["len"] >= 256) & (vm["len"] <= 512))
    assert np.all(np.abs(vm["nn"] - np.arange(n0)) > np.ceil(vm["len"] / 4))


def test_planted_motifs_found(planted):
    info = planted["w"].info
    mot = planted["mot"]
    assert len(mot) == planted["w"].k
    found = set()
    for m in mot:
        assert abs(m["dist"] - m["dist_recheck"]) <= tol(planted["prec"], m["len"], m["dist_recheck"])
        for a, b, L in info.motifs:
            if L >= 256 and abs(m["a"] - a) <= L // 4 and abs(m["b"] - b) <= L // 4:
                found.add(L)
    assert found == {300, 400}, (mot, info.motifs)


def test_planted_discord_found(planted):
    info = planted["w"].info
    top = planted["dis"][0]
    assert top["len"] >= 256
    assert top["off"] <= info.spike < top["off"] + top["len"] or \
        top["off"] <= info.level_shift < top["off"] + top["len"]
    assert abs(top["dist"] - top["dist_recheck"]) <= tol(planted["prec"], top["len"], top["dist_recheck"])


def test_pruning_counters(planted):
    st = planted["st"]
    assert [s["len"] for s in st] == list(range(256, 513))
    for s in st:
        assert s["certified"] + s["recomputed"] == s["rows"]
        assert s["band_ms"] > 0 or s["recomputed"] == 0
    assert st[0]["recomputed"] == st[0]["rows"]
