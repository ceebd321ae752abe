"""Repeated profiles: the workspace is reused (no device allocation by the
library) and from the second profile with the same shape on, the whole
launch sequence runs as one captured CUDA graph (its instantiation, at that
second profile, is the driver's one allocation; replays allocate nothing). Results must be identical, bit for bit, to the
eager first profile, and to a profile with graphs switched off."""
import numpy as np
import pytest

import oracle
import paper_2008_13447_gb300 as mad
import workloads
from parity_util import compare_all

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2008_13447_gb300 import build
    build.build()
    oracle.build()


def snapshot(ctx, n, lmin, lmax, k, m):
    vm = mad.mad_valmp(ctx, 0, n - lmin + 1)
    prof = [mad.mad_matrix_profile(ctx, 0, l, n, m) for l in (lmin, (lmin + lmax) // 2, lmax)]
    return dict(vm=vm, prof=prof, mot=mad.mad_motifs(ctx, 0, k), dis=mad.mad_discords(ctx, 0, k, m),
                st=mad.mad_stats(ctx, 0))


def same(a, b):
    for key in ("dist", "norm", "len", "nn"):
        assert np.array_equal(a["vm"][key], b["vm"][key]), key
    for pa, pb in zip(a["prof"], b["prof"]):
        for u, v in zip(pa, pb):
            assert np.array_equal(u, v)
    assert a["mot"] == b["mot"]
    assert a["dis"] == b["dis"]
    for sa, sb in zip(a["st"], b["st"]):
        # (list insertions are left out: units of a row share thresholds in
        # the order they finish, so the count varies, not the results)
        for key in ("certified", "recomputed", "band_cells", "direct_rows", "fp32_dq_max"):
            assert sa[key] == sb[key], key


@pytest.mark.parametrize("prec", [mad.MAD_FP32, mad.MAD_FP64], ids=["fp32", "fp64"])
def test_repeated_profiles_replay_a_graph_and_allocate_nothing(prec):
    import torch
    x = workloads.ecg_like(6000, 141, period=70.0)
    n, lmin, lmax, p, k, m = len(x), 60, 76, 6, 4, 2
    torch.cuda.init()
    mad.mad_set_graphs(1)
    ctx = mad.mad_create(x, precision=prec, k_max=k, m_max=m, keep_profiles=True)
    try:
        mad.mad_profile(ctx, lmin, lmax, p)            # eager, allocates the workspace
        first = snapshot(ctx, n, lmin, lmax, k, m)
        assert all(s["graph"] == 0 for s in first["st"])
        runs = []
        mad.mad_profile(ctx, lmin, lmax, p)            # captured (the driver takes memory for the graph)
        runs.append(snapshot(ctx, n, lmin, lmax, k, m))
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        for _ in range(2):                           # replayed: nothing allocated
            mad.mad_profile(ctx, lmin, lmax, p)
            runs.append(snapshot(ctx, n, lmin, lmax, k, m))
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
        for r in runs:
            assert all(s["graph"] == 1 for s in r["st"])
            assert sum(s["band_ms"] for s in r["st"]) > 0
            same(first, r)
        # graphs off: the same results, launched one by one
        mad.mad_set_graphs(0)
        mad.mad_profile(ctx, lmin, lmax, p + 1)        # another shape: a new workspace
        mad.mad_profile(ctx, lmin, lmax, p)            # and back: allocated again
        torch.cuda.synchronize()
        free1 = torch.cuda.mem_get_info()[0]
        mad.mad_profile(ctx, lmin, lmax, p)            # the same shape again: the workspace reused
        off = snapshot(ctx, n, lmin, lmax, k, m)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free1
        assert all(s["graph"] == 0 for s in off["st"])
        same(first, off)
    finally:
        mad.mad_set_graphs(1)
        mad.mad_destroy(ctx)


def test_replayed_profile_reads_new_series_values():
    # a caller-owned device series rewritten between profiles: the replayed
    # graph computes on the new values (checked against the oracle)
    import torch
    x1 = workloads.random_walk(4000, 142)
    x2 = workloads.ar2(4000, 143)
    xt = torch.tensor(x1, device="cuda", dtype=torch.float64)
    ctx = mad.mad_create_device(xt, precision=mad.MAD_FP64, k_max=3, m_max=1, keep_profiles=True)
    try:
        for _ in range(2):
            mad.mad_profile(ctx, 30, 36, 5)
        xt.copy_(torch.tensor(x2, dtype=torch.float64))
        torch.cuda.synchronize()
        mad.mad_profile(ctx, 30, 36, 5)
        st = mad.mad_stats(ctx, 0)
        assert st[0]["graph"] == 1
        vm = mad.mad_valmp(ctx, 0, len(x2) - 30 + 1)
        ref = oracle.valmp_plain(x2, 30, 36)
        assert np.allclose(vm["norm"], ref["norm"], rtol=1e-9, atol=1e-12)
    finally:
        mad.mad_destroy(ctx)


def test_batch_reuses_workspaces_and_matches_the_oracle():
    # uneven series, each with its own range: repeated batch profiles reuse
    # every series' workspace (eager launches, no graphs) with the same results
    series = [workloads.random_walk(1500 + 700 * s, 160 + s) if s % 2 == 0 else workloads.ar2(1800 + 500 * s, 160 + s)
              for s in range(10)]
    lmin = [20 + 3 * s for s in range(10)]
    lmax = [a + 6 for a in lmin]
    ctx = mad.mad_create_batch(series, precision=mad.MAD_FP64, k_max=3, m_max=1)
    try:
        res = []
        for rep in range(3):
            mad.mad_profile_batch(ctx, lmin, lmax, 5)
            res.append([mad.mad_valmp(ctx, s, len(series[s]) - lmin[s] + 1) for s in range(10)])
            st = [mad.mad_stats(ctx, s) for s in range(10)]
            assert all(q["graph"] == 0 for sts in st for q in sts)
        for s in range(10):
            for key in ("dist", "norm", "len", "nn"):
                assert np.array_equal(res[0][s][key], res[2][s][key])
        for s in (0, 3, 9):
            ref = oracle.valmp_plain(series[s], lmin[s], lmax[s])
            assert np.allclose(res[2][s]["norm"], ref["norm"], rtol=1e-9, atol=1e-12)
    finally:
        mad.mad_destroy(ctx)


@pytest.mark.parametrize("prec", [mad.MAD_FP32, mad.MAD_SPLIT_TC], ids=["fp32", "tc"])
def test_autotuned_launch_agrees_with_defaults(prec):
    # the tuner picks a band height (and on the tensor-core path a routing
    # threshold) per size bucket; the results agree with the defaults'
    x = workloads.ecg_like(5000, 165, period=55.0)
    out = {}
    for tune in (0, 1):
        mad.mad_set_autotune(tune)
        try:
            ctx = mad.mad_create(x, precision=prec, k_max=3, m_max=1)
            try:
                mad.mad_profile(ctx, 50, 58, 6)
                st = mad.mad_stats(ctx, 0)
                out[tune] = (mad.mad_valmp(ctx, 0, len(x) - 50 + 1), st[0]["band_rows"])
            finally:
                mad.mad_destroy(ctx)
        finally:
            mad.mad_set_autotune(1)
    assert out[0][1] == 1024 and out[1][1] in (256, 512, 1024)
    assert np.all(np.abs(out[0][0]["norm"] - out[1][0]["norm"]) <= 2e-4)
    ref = oracle.valmp_plain(x, 50, 58)
    assert np.all(np.abs(out[1][0]["norm"] - ref["norm"]) <= 1e-4)
