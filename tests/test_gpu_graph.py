"""Repeated profiles: the workspace is reused (no device allocation) and from
the second profile with the same shape on, the whole launch sequence runs as
one captured CUDA graph. Results must be identical, bit for bit, to the
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
        for key in ("certified", "recomputed", "band_cells", "inserts", "direct_rows", "fp32_dq_max"):
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
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        runs = []
        for _ in range(3):                           # captured once, then replayed
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
        mad.mad_profile(ctx, lmin, lmax, p)
        off = snapshot(ctx, n, lmin, lmax, k, m)
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
