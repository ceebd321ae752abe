"""The FP32 paths' error model, checked on the five workloads (the 2^21-point
seismic walk on the first lengths of its range), and the tensor-core direct
path on two of them.

The library keeps, for every stored entry selected by the FP32 recurrence
(u (2R + 4) kappa_i kappa_j, a worst-case bound on the chain's rounding) or by
a direct path (the per-entry bound the kernel writes), a bound on its
correlation error. With the audit hook on, every
such entry is re-evaluated in FP64 when it is selected and the largest
observed error over its bound is recorded per length (dq_ratio_max); the
bound holds while that ratio is at most 1. Each test prints its worst ratio.
"""
import numpy as np
import pytest

import oracle
import paper_2008_13447_gb300 as mad
import workloads

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

RANGES = {
    "rw4096": None,
    "planted65k": None,
    "ecg262k": None,
    "batch256": None,
    "seismic2m": (256, 260),
}


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2008_13447_gb300 import build
    build.build()
    oracle.build()


@pytest.fixture(autouse=True)
def audit():
    mad.mad_debug_audit_error_bounds(1)
    yield
    mad.mad_debug_audit_error_bounds(0)


CASES = [(name, mad.MAD_FP32) for name in RANGES] + [("ecg262k", mad.MAD_SPLIT_TC), ("rw4096", mad.MAD_SPLIT_TC)]


@pytest.mark.parametrize("name, prec", CASES, ids=["%s-%s" % (c[0], "tc" if c[1] == mad.MAD_SPLIT_TC else "fp32")
                                                    for c in CASES])
def test_fp32_error_bound_holds(name, prec):
    w = workloads.make(name)
    worst, checked = 0.0, 0
    if len(w.series) > 1:
        ctx = mad.mad_create_batch(w.series, precision=prec, k_max=w.k, m_max=w.m)
        try:
            mad.mad_profile_batch(ctx, w.lmin, w.lmax, w.p)
            for s in range(len(w.series)):
                st = mad.mad_stats(ctx, s)
                worst = max(worst, max(q["dq_ratio_max"] for q in st))
                checked += sum(q["recomputed"] for q in st)
        finally:
            mad.mad_destroy(ctx)
    else:
        lmin, lmax = RANGES[name] or (w.lmin[0], w.lmax[0])
        ctx = mad.mad_create(w.series[0], precision=prec, k_max=w.k, m_max=w.m)
        try:
            mad.mad_profile(ctx, lmin, lmax, w.p)
            st = mad.mad_stats(ctx, 0)
            worst = max(q["dq_ratio_max"] for q in st)
            checked = sum(q["recomputed"] for q in st)
        finally:
            mad.mad_destroy(ctx)
    print("ERROR-MODEL %s %s: worst observed / bound = %.4f over %d recomputed rows"
          % (name, "tc" if prec == mad.MAD_SPLIT_TC else "fp32", worst, checked))
    assert checked > 0
    assert 0.0 < worst <= 1.0
