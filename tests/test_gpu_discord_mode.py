"""Discord mode (mode 2: Algorithm 7 driving Algorithm 10) on the GPU.

Against the oracle's pruned iteration: the merged dkm table identical in
offsets and lengths (FP64; the FP32 path certifies pessimistically, so a row
near its bound can change pass, and there every reported distance is checked
against its FP64 re-check instead); with every row valid (p at least the
non-trivial count) the table equals the streamed form of the exact profiles
(mode 0 with kept profiles); a planted spike at rank 1 with few rows
recomputed; argument checks."""
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


def run_mode2(x, lmin, lmax, p, k, m, prec):
    ctx = mad.mad_create(x, precision=prec, k_max=k, m_max=m, mode=2)
    try:
        mad.mad_profile(ctx, lmin, lmax, p)
        dis = mad.mad_discords(ctx, 0, k, m)
        st = mad.mad_stats(ctx, 0)
    finally:
        mad.mad_destroy(ctx)
    return dis, st


@pytest.mark.parametrize("prec", PRECS)
def test_discord_mode_matches_oracle(prec):
    x = workloads.ar2(1500, 106)
    lmin, lmax, p, k, m = 20, 32, 5, 4, 2
    dis, st = run_mode2(x, lmin, lmax, p, k, m, prec)
    ref = oracle.valmod_discord(x, lmin, lmax, p, k, m)
    got_cells = [(d["off"], d["len"]) for d in dis]
    ref_cells = [(int(ref["off"][r, c]), int(ref["len"][r, c])) for r in range(k) for c in range(m)]
    for d in dis:
        assert d["len"] > 0
        assert abs(d["dist"] - d["dist_recheck"]) <= 1e-9 * max(1.0, d["dist_recheck"]) * (
            1.0 if prec == mad.MAD_FP64 else 1e3)
    if prec == mad.MAD_FP64:
        assert got_cells == ref_cells
        for d, (r, c) in zip(dis, [(r, c) for r in range(k) for c in range(m)]):
            assert abs(d["dist"] - ref["dist"][r, c]) <= 1e-9 * ref["dist"][r, c]
    else:
        # rank 1 of every column agrees
        for c in range(m):
            assert got_cells[c] == ref_cells[c]
    # pruning: at most the listed rows are recomputed, and fewer than all
    rec = np.array([s["recomputed"] for s in st[1:]])
    rows = np.array([s["rows"] for s in st[1:]])
    assert np.all(rec <= rows) and rec.sum() < rows.sum()
    assert st[0]["recomputed"] == st[0]["rows"]


def test_discord_mode_many_ranks_matches_oracle():
    # k above one warp's 32 ranks and three columns, a ragged series length
    x = workloads.ar2(1333, 109)
    lmin, lmax, p, k, m = 18, 26, 6, 40, 3
    dis, _ = run_mode2(x, lmin, lmax, p, k, m, mad.MAD_FP64)
    ref = oracle.valmod_discord(x, lmin, lmax, p, k, m)
    for r in range(k):
        for c in range(m):
            d = dis[r * m + c]
            if ref["len"][r, c] == 0:
                assert d["len"] == 0 and d["off"] == -1
                continue
            assert (d["off"], d["len"]) == (int(ref["off"][r, c]), int(ref["len"][r, c]))
            assert abs(d["dist"] - ref["dist"][r, c]) <= 1e-9 * ref["dist"][r, c]


def test_discord_mode_all_valid_is_streamed_form():
    # p = 64 stores every window of a short series: every row is valid, and
    # the table is the streamed form of the exact profiles
    x = workloads.ar2(72, 107)
    lmin, lmax, k, m = 10, 14, 4, 2
    dis, st = run_mode2(x, lmin, lmax, 64, k, m, mad.MAD_FP64)
    assert all(s["recomputed"] == 0 for s in st[1:])
    ctx = mad.mad_create(x, precision=mad.MAD_FP64, k_max=k, m_max=m, keep_profiles=True)
    try:
        mad.mad_profile(ctx, lmin, lmax, 64)
        ref = mad.mad_discords_streamed(ctx, 0, k, m)
    finally:
        mad.mad_destroy(ctx)
    assert [(d["off"], d["len"]) for d in dis] == [(d["off"], d["len"]) for d in ref]
    for d, e in zip(dis, ref):
        assert abs(d["dist"] - e["dist"]) <= 1e-12 * e["dist"]


@pytest.mark.parametrize("prec", PRECS)
def test_discord_mode_planted_spike(prec):
    rng = np.random.default_rng(105)
    t_ = np.arange(2500)
    x = np.sin(2 * np.pi * t_ / 50) + 0.05 * rng.standard_normal(2500)
    x[1300] += 3.0
    dis, st = run_mode2(x, 24, 30, 5, 3, 1, prec)
    assert dis[0]["off"] <= 1300 < dis[0]["off"] + dis[0]["len"]
    rec = sum(s["recomputed"] for s in st[1:])
    assert rec < sum(s["rows"] for s in st[1:]) // 10
    ref = oracle.valmod_discord(x, 24, 30, 5, 3, 1)
    assert (dis[0]["off"], dis[0]["len"]) == (int(ref["off"][0, 0]), int(ref["len"][0, 0]))


def test_discord_mode_arguments():
    x = workloads.random_walk(600, 108)
    with pytest.raises(mad.MadError) as e:
        mad.mad_create(x, precision=mad.MAD_FP32, k_max=2, m_max=1, mode=3)
    assert e.value.status == mad.MAD_EINVAL
    ctx = mad.mad_create(x, precision=mad.MAD_FP32, k_max=2, m_max=1, mode=2, keep_profiles=True)
    try:
        mad.mad_profile(ctx, 20, 24, 3)
        assert len(mad.mad_discords(ctx, 0, 2, 1)) == 2
        for fn in (mad.mad_discords_global, mad.mad_discords_streamed):
            with pytest.raises(mad.MadError) as e:
                fn(ctx, 0, 2, 1)
            assert e.value.status == mad.MAD_ESTATE
    finally:
        mad.mad_destroy(ctx)
