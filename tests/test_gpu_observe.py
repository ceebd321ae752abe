"""Pruning observation (options.observe_len, mad_observe): maxLB - minED and
the tightness LB / ED per row at one length, against the oracle's (FP64),
and by properties (FP32)."""
import numpy as np
import pytest

import oracle
import paper_2008_13447_gb300 as mad
import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2008_13447_gb300 import build
    build.build()
    oracle.build()


@pytest.mark.parametrize("gen", ["rw", "ecg"])
def test_observation_fp64_matches_oracle(gen):
    x = workloads.random_walk(2500, 91) if gen == "rw" else workloads.ecg_like(3000, 92, period=50.0)
    lmin, lmax, L, p = 40, 48, 45, 5
    ctx = mad.mad_create(x, precision=mad.MAD_FP64, k_max=2, m_max=1, observe_len=L)
    try:
        mad.mad_profile(ctx, lmin, lmax, p)
        gap, tlb = mad.mad_observe(ctx, 0, len(x) - L + 1)
        st = mad.mad_stats(ctx, 0)
    finally:
        mad.mad_destroy(ctx)
    ref = oracle.valmod_pruned(x, lmin, lmax, p, observe_len=L)
    both = np.isfinite(gap) & np.isfinite(ref["gap"])
    assert both.sum() > 0.95 * len(gap)
    g_ok = np.abs(gap - ref["gap"]) <= 1e-9 * np.maximum(1.0, np.abs(ref["gap"]))
    t_ok = np.abs(tlb - ref["tlb"]) <= 1e-9
    assert (g_ok & t_ok)[both].mean() >= 0.995       # rows whose stored entries tie may differ
    t = tlb[np.isfinite(tlb)]
    assert np.all(t > 0) and np.all(t <= 1 + 1e-9)
    li = L - lmin
    assert abs(int((gap[np.isfinite(gap)] > 0).sum()) - st[li]["certified"]) <= max(2, 0.002 * len(gap))


def test_observation_fp32_properties():
    x = workloads.random_walk(3000, 93)
    lmin, lmax, L = 30, 40, 35
    ctx = mad.mad_create(x, precision=mad.MAD_FP32, k_max=2, m_max=1, observe_len=L)
    try:
        mad.mad_profile(ctx, lmin, lmax, 5)
        gap, tlb = mad.mad_observe(ctx, 0, len(x) - L + 1)
        st = mad.mad_stats(ctx, 0)
    finally:
        mad.mad_destroy(ctx)
    ok = np.isfinite(gap)
    # the FP32 path certifies on pessimistic distances: never more rows than a positive gap
    assert st[L - lmin]["certified"] <= int((gap[ok] > 0).sum())
    t = tlb[np.isfinite(tlb)]
    assert np.all(t > 0) and np.all(t <= 1 + 1e-3)


def test_observe_needs_a_length_in_range():
    x = workloads.random_walk(800, 94)
    ctx = mad.mad_create(x, precision=mad.MAD_FP32, k_max=2, m_max=1)
    try:
        mad.mad_profile(ctx, 20, 24, 3)
        with pytest.raises(mad.MadError) as e:
            mad.mad_observe(ctx, 0, len(x) - 20 + 1)
        assert e.value.status == mad.MAD_ESTATE
    finally:
        mad.mad_destroy(ctx)
