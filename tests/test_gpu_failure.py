"""Failure path of the band kernel's bounded waits, made on purpose without a
GPU fault: the test hook mad_debug_wavefront_wait_limit(0) makes every
wavefront wait (the hand-over of boundary values between the warps of a
block) give up at once. The kernel keeps every access in bounds, runs to its
end and records its error word; mad_profile must return MAD_ETIMEOUT, and
the next profile (default limit restored) must succeed with exact results.
The waits that hand out work units keep their own limit."""
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


@pytest.mark.parametrize("prec", [mad.MAD_FP32, mad.MAD_FP64], ids=["fp32", "fp64"])
def test_wavefront_wait_timeout_is_reported(prec):
    x = workloads.random_walk(3000, 131)
    ctx = mad.mad_create(x, precision=prec, k_max=3, m_max=1)
    try:
        mad.mad_debug_wavefront_wait_limit(0)
        try:
            with pytest.raises(mad.MadError) as e:
                mad.mad_profile(ctx, 40, 44, 5)
        finally:
            mad.mad_debug_wavefront_wait_limit(-1)
        assert e.value.status == mad.MAD_ETIMEOUT
        assert "bounded wait" in str(e.value)
        # the same context is usable again: a read-out before a good profile
        # is out of order, a new profile succeeds
        with pytest.raises(mad.MadError) as e2:
            mad.mad_motifs(ctx, 0, 3)
        assert e2.value.status == mad.MAD_ESTATE
        mad.mad_profile(ctx, 40, 44, 5)
        assert len(mad.mad_motifs(ctx, 0, 3)) == 3
    finally:
        mad.mad_destroy(ctx)
    # and a fresh context on the same device gives exact results
    compare_all(x, 40, 44, 5, prec, k_max=3)
