"""The tensor-core direct path (MAD_SPLIT_TC): rows recomputed on their own
run as FP16 hi + lo split products on tcgen05 with FP32 accumulation, with a
per-entry error bound. Compared element by element with the oracle like the
other paths (FP32 tolerance 1e-4 sqrt(l)), on inputs where many rows take
the direct path: several row tiles of 128, several 4096-column blocks and a
ragged last tile."""
import numpy as np
import pytest

import oracle
import paper_2008_13447_gb300 as mad
import workloads
from parity_util import compare_all

pytestmark = pytest.mark.gpu
TC = mad.MAD_SPLIT_TC


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2008_13447_gb300 import build
    build.build()
    oracle.build()


def direct(st):
    return sum(s["direct_rows"] for s in st[1:])


def test_ecg_pruned_regime_tc():
    x = workloads.ecg_like(4500, 103, period=60.0)
    r = compare_all(x, 60, 72, 8, TC, m_max=2, k_max=3)
    st = r["stats"]
    assert direct(st) > 0
    assert sum(s["direct_ms"] for s in st[1:]) > 0


def test_many_direct_rows_several_tiles_and_blocks():
    # n_l > 4096 (several column blocks), more than 128 direct rows at a
    # length (several row tiles), l not a multiple of 64 (ragged lags)
    x = workloads.ecg_like(9000, 151, period=45.0)
    r = compare_all(x, 70, 78, 6, TC, m_max=1, k_max=4)
    st = r["stats"]
    assert max(s["direct_rows"] for s in st[1:]) > 128
    assert direct(st) > 0


def test_random_walk_tc():
    x = workloads.random_walk(5000, 101)
    compare_all(x, 40, 48, 5, TC)


def test_ar2_mth_neighbours_tc():
    x = workloads.ar2(3100, 102)
    compare_all(x, 30, 36, 6, TC, m_max=3, k_max=4, excl=(1, 2))


def test_long_windows_tc():
    # l > 128: three lag chunks of 64, the last one partial
    x = workloads.ecg_like(6000, 152, period=90.0)
    r = compare_all(x, 150, 156, 5, TC, k_max=3)
    assert direct(r["stats"]) > 0


def test_tc_matches_fp32_readouts():
    x = workloads.ecg_like(7000, 153, period=64.0)
    out = {}
    for prec in (mad.MAD_FP32, TC):
        ctx = mad.mad_create(x, precision=prec, k_max=4, m_max=1)
        try:
            mad.mad_profile(ctx, 64, 72, 6)
            out[prec] = (mad.mad_valmp(ctx, 0, len(x) - 64 + 1), mad.mad_motifs(ctx, 0, 4))
        finally:
            mad.mad_destroy(ctx)
    a, b = out[mad.MAD_FP32][0], out[TC][0]
    assert np.all(np.abs(a["norm"] - b["norm"]) <= 2e-4)


def test_large_p_takes_the_unpipelined_kernel():
    # p > 16: the one-stage kernel (per-row lists in shared memory) runs
    x = workloads.ecg_like(5200, 154, period=58.0)
    r = compare_all(x, 64, 70, 20, TC, m_max=2, k_max=3)
    assert direct(r["stats"]) > 0


def _tc_profile(x, lmin, lmax, p, tma, m_max=1, k_max=3):
    mad.mad_debug_tc_tma(tma)
    try:
        ctx = mad.mad_create(x, precision=TC, k_max=k_max, m_max=m_max, keep_profiles=True)
        try:
            mad.mad_profile(ctx, lmin, lmax, p)
            n0 = len(x) - lmin + 1
            return dict(vm=mad.mad_valmp(ctx, 0, n0),
                        prof=[mad.mad_matrix_profile(ctx, 0, l, len(x), m_max) for l in range(lmin, lmax + 1)],
                        mot=mad.mad_motifs(ctx, 0, k_max), st=mad.mad_stats(ctx, 0))
        finally:
            mad.mad_destroy(ctx)
    finally:
        mad.mad_debug_tc_tma(0)


@pytest.mark.parametrize("p", [6, 12], ids=["p6_vs_pipelined", "p12_vs_one_stage"])
def test_tma_column_tiles_match_built_tiles(p):
    # column tiles loaded by TMA from the per-length shifted copies against
    # tiles built in shared memory by the kernels without TMA (the default):
    # the same FP16 pairs and products, so the same results bit for bit
    # (ties between equal keys go to the smaller column in both)
    x = workloads.ecg_like(9000, 155, period=47.0)
    a = _tc_profile(x, 70, 76, p, 1, m_max=2)
    b = _tc_profile(x, 70, 76, p, 0, m_max=2)
    assert direct(a["st"]) > 0 and direct(a["st"]) == direct(b["st"])
    for key in ("dist", "norm", "len", "nn"):
        assert np.array_equal(a["vm"][key], b["vm"][key]), key
    for pa, pb in zip(a["prof"], b["prof"]):
        for u, v in zip(pa, pb):
            assert np.array_equal(u, v)
    assert a["mot"] == b["mot"]
    assert [s["fp32_dq_max"] for s in a["st"]] == [s["fp32_dq_max"] for s in b["st"]]


def test_tma_column_tiles_ragged_series_end():
    # TMA column tiles against the oracle: the last tile's copies run past
    # the series end (zeros), n_l not a multiple of 256, lags in three chunks
    x = workloads.ecg_like(8191, 156, period=71.0)
    mad.mad_debug_tc_tma(1)
    try:
        r = compare_all(x, 129, 133, 7, TC, k_max=3)
    finally:
        mad.mad_debug_tc_tma(0)
    assert direct(r["stats"]) > 0
