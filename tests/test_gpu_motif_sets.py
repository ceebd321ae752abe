"""Variable-length motif sets on the GPU against the oracle, given the same
motif pairs and radii (the pairs' FP64 distances): member lists identical,
except a window whose distance ties the radius within rounding; and the
planted-copies case."""
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


def planted_copies(n=4000, L=40, offs=(300, 1200, 2100, 3000), seed=71):
    rng = np.random.default_rng(seed)
    x = np.cumsum(rng.standard_normal(n))
    pat = 3.0 * np.sin(np.linspace(0, 4 * np.pi, L)) * np.hanning(L)
    for o in offs:
        seg = x[o:o + L]
        x[o:o + L] = seg.mean() + pat * seg.std() + 0.05 * seg.std() * rng.standard_normal(L)
    return x, L, offs


def compare_sets(x, sets, D, cap):
    pairs = [(s["a"], s["b"], s["len"], s["radius"] / D) for s in sets]
    ref = oracle.motif_sets(x, pairs, D, cap)
    for s, r in zip(sets, ref):
        got = [int(v) for v in s["members"]]
        r = [int(v) for v in r]
        if got != r:
            # allowed: a member present on one side only whose distance ties the radius
            L = s["len"]
            for j in set(got) ^ set(r):
                dj = min(oracle.dist(x, L, s["a"], j), oracle.dist(x, L, s["b"], j))
                assert abs(dj - s["radius"]) <= 1e-9 * max(1.0, s["radius"]), (got, r, j, dj)


@pytest.mark.parametrize("prec", PRECS)
def test_motif_sets_match_oracle(prec):
    x = workloads.ar2(5000, 72)
    ctx = mad.mad_create(x, precision=prec, k_max=4, m_max=1)
    try:
        mad.mad_profile(ctx, 30, 40, 5)
        for D, cap in ((1.0, 4), (2.5, 16), (4.0, 64)):
            sets = mad.mad_motif_sets(ctx, 0, 4, D, cap)
            assert 1 <= len(sets) <= 4
            for s in sets:
                assert s["members"][:2] == [s["a"], s["b"]] and len(s["members"]) <= cap
            compare_sets(x, sets, D, cap)
    finally:
        mad.mad_destroy(ctx)


@pytest.mark.parametrize("prec", PRECS)
def test_motif_set_holds_planted_copies(prec):
    x, L, offs = planted_copies()
    ctx = mad.mad_create(x, precision=prec, k_max=2, m_max=1)
    try:
        mad.mad_profile(ctx, L - 4, L + 4, 5)
        sets = mad.mad_motif_sets(ctx, 0, 1, 4.0, 16)
        got = sets[0]["members"]
        for o in offs:
            assert any(abs(m - o) <= oracle.excl(sets[0]["len"]) for m in got), (o, got)
        compare_sets(x, sets, 4.0, 16)
    finally:
        mad.mad_destroy(ctx)


def test_motif_sets_arguments():
    x = workloads.random_walk(600, 73)
    ctx = mad.mad_create(x, precision=mad.MAD_FP32, k_max=2, m_max=1)
    try:
        with pytest.raises(mad.MadError) as e:
            mad.mad_motif_sets(ctx, 0, 2, 2.0, 8)          # before mad_profile
        assert e.value.status == mad.MAD_ESTATE
        mad.mad_profile(ctx, 20, 24, 3)
        for k, D, cap in ((0, 1.0, 8), (2, -1.0, 8), (2, 1.0, 1), (2, 1.0, 257)):
            with pytest.raises(mad.MadError) as e:
                mad.mad_motif_sets(ctx, 0, k, D, cap)
            assert e.value.status == mad.MAD_EINVAL
    finally:
        mad.mad_destroy(ctx)
