"""mad_mth_nn_dist_noalloc: the FP64 m-th best-match re-check with fixed
static scratch, against the existing entry point that computes the same
distances (mad_discords' dist_recheck) and against the oracle.

This file is collected last so that it also runs after every other test
in one process."""
import math

import numpy as np
import pytest

import oracle
import paper_2008_13447_gb300 as mad
import workloads
from parity_util import tol_for


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2008_13447_gb300 import build
    build.build()
    oracle.build()


def test_rejects_more_slots_than_the_scratch_holds():
    # checked on the host before any GPU work: the pointers are never used
    cells = np.zeros((mad.MAD_NOALLOC_MAX_SLOTS // 4 + 1, 3), np.int32)
    cells[:, 1] = 8
    cells[:, 2] = 1
    with pytest.raises(mad.MadError) as e:
        mad.mad_mth_nn_dist_noalloc(16, 100, cells, 4, 16)
    assert e.value.status == mad.MAD_EINVAL
    assert "exceeds the fixed scratch of 1024" in str(e.value)


@pytest.mark.parametrize("cell, m_max, what", [
    ((95, 8, 1), 2, "outside the series"),
    ((-1, 8, 1), 2, "outside the series"),
    ((0, 1, 1), 2, "len must be"),
    ((0, 8, 3), 2, "m must be in"),
])
def test_rejects_bad_cells(cell, m_max, what):
    with pytest.raises(mad.MadError) as e:
        mad.mad_mth_nn_dist_noalloc(16, 100, [cell], m_max, 16)
    assert e.value.status == mad.MAD_EINVAL
    assert what in str(e.value)


def test_rejects_series_beyond_32bit_offsets():
    # checked on the host before any GPU work: the pointers are never used
    with pytest.raises(mad.MadError) as e:
        mad.mad_mth_nn_dist_noalloc(16, (1 << 31) + 2, [(0, 8, 1)], 1, 16)
    assert e.value.status == mad.MAD_EINVAL
    assert "2^31" in str(e.value)


def test_empty_call_is_a_no_op():
    mad.mad_mth_nn_dist_noalloc(0, 0, np.zeros((0, 3), np.int32), 1, 0)


@pytest.mark.gpu
def test_noalloc_matches_existing_recheck_twice():
    import torch
    x = workloads.random_walk(3000, 111)
    k, m = 4, 3
    ctx = mad.mad_create(x, precision=mad.MAD_FP64, k_max=k, m_max=m)
    try:
        mad.mad_profile(ctx, 40, 48, 5)
        dis = [d for d in mad.mad_discords(ctx, 0, k, m) if d["len"] > 0]
    finally:
        mad.mad_destroy(ctx)
    assert len(dis) == k * m
    cells = np.array([(d["off"], d["len"], d["m"]) for d in dis], np.int32)
    ref = np.array([d["dist_recheck"] for d in dis])

    xt = torch.from_numpy(x).cuda()
    out = torch.empty(len(cells), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    got = []
    before = []
    for call in range(2):
        out.fill_(math.nan)
        torch.cuda.synchronize()
        before.append((torch.cuda.memory_allocated(), torch.cuda.memory_reserved(), torch.cuda.mem_get_info()[0]))
        mad.mad_mth_nn_dist_noalloc(xt.data_ptr(), len(x), cells, m, out.data_ptr(), stream=stream)
        torch.cuda.synchronize()
        got.append(out.cpu().numpy().copy())
    # nothing in the caller's allocator moved across either call ...
    after = (torch.cuda.memory_allocated(), torch.cuda.memory_reserved())
    assert after == before[0][:2] == before[1][:2]
    # ... and the second call (after the first call's set-up) left the
    # device's free memory as it was. Free memory is device-wide (another
    # process or the runtime itself can move it): one retry before failing.
    free_after = torch.cuda.mem_get_info()[0]
    if free_after != before[1][2]:
        torch.cuda.synchronize()
        f0 = torch.cuda.mem_get_info()[0]
        mad.mad_mth_nn_dist_noalloc(xt.data_ptr(), len(x), cells, m, out.data_ptr(), stream=stream)
        torch.cuda.synchronize()
        free_after, before = torch.cuda.mem_get_info()[0], [None, (None, None, f0)]
    assert free_after == before[1][2]
    for g in got:
        assert np.all(np.isfinite(g))
        for (off, L, mm), gv, rv in zip(cells, g, ref):
            tol = tol_for(mad.MAD_FP64, int(L), np.array([rv]))[0]
            assert abs(gv - rv) <= tol, (off, L, mm, gv, rv)
            # the oracle's full distance profile of the window, m-th smallest
            dp = oracle.distance_profile(x, int(L), int(off))
            want = np.sort(dp[np.isfinite(dp)])[mm - 1]
            assert abs(gv - want) <= tol, (off, L, mm, gv, want)
    assert np.array_equal(got[0], got[1])


@pytest.mark.gpu
def test_noalloc_rejects_host_series():
    import torch
    x = workloads.random_walk(500, 112)
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    with pytest.raises(mad.MadError) as e:
        mad.mad_mth_nn_dist_noalloc(x.ctypes.data, len(x), [(10, 20, 1)], 1, out.data_ptr())
    assert e.value.status == mad.MAD_EINVAL
    assert "device memory" in str(e.value)
