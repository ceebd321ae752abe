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
    # p > 10: the per-row lists no longer fit beside the two pipelined stages;
    # the one-stage kernel runs instead (same results)
    x = workloads.ecg_like(5200, 154, period=58.0)
    r = compare_all(x, 64, 70, 12, TC, m_max=2, k_max=3)
    assert direct(r["stats"]) > 0
