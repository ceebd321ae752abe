"""Motif mode (mode 1, Algorithm 1 with ComputeSubMP / Algorithm 4) on the
GPU against the exact per-length oracle: every value the mode defines is the
exact matrix profile, every length's smallest defined value is that
length's motif distance, and the best length-normalised VALMP entry (the
variable-length motif) is exact. The certification decisions may differ
from the oracle's on near-ties (FP32 tests pessimistically), so these are
checked as properties, not entry by entry."""
import math

import numpy as np
import pytest

import oracle
import paper_2008_13447_gb300 as mad
import workloads
from parity_util import tol_for

pytestmark = pytest.mark.gpu
PRECS = [pytest.param(mad.MAD_FP64, id="fp64"), pytest.param(mad.MAD_FP32, id="fp32")]


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2008_13447_gb300 import build
    build.build()
    oracle.build()


def run_motif_mode(x, lmin, lmax, p, prec):
    ctx = mad.mad_create(x, precision=prec, k_max=3, m_max=1, keep_profiles=True, mode=1)
    try:
        mad.mad_profile(ctx, lmin, lmax, p)
        n = len(x)
        prof = {l: mad.mad_matrix_profile(ctx, 0, l, n, 1) for l in range(lmin, lmax + 1)}
        vm = mad.mad_valmp(ctx, 0, n - lmin + 1)
        mot = mad.mad_motifs(ctx, 0, 1)
        st = mad.mad_stats(ctx, 0)
        with pytest.raises(mad.MadError) as e:
            mad.mad_discords(ctx, 0, 1, 1)
        assert e.value.status == mad.MAD_ESTATE
    finally:
        mad.mad_destroy(ctx)
    return prof, vm, mot, st


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("gen", ["rw", "ecg", "planted"])
def test_motif_mode_properties(prec, gen):
    if gen == "rw":
        x, lmin, lmax, p = workloads.random_walk(3000, 51), 30, 40, 5
    elif gen == "ecg":
        x, lmin, lmax, p = workloads.ecg_like(4000, 52, period=60.0), 60, 72, 8
    else:
        x, _ = workloads.planted_walk(6000, 34, motif_lengths=(40, 48), lmax=80)
        lmin, lmax, p = 40, 52, 5
    n = len(x)
    prof, vm, mot, st = run_motif_mode(x, lmin, lmax, p, prec)
    pl = oracle.valmp_plain(x, lmin, lmax, m_max=1, keep_nn=True)
    computed = 0
    for li, l in enumerate(range(lmin, lmax + 1)):
        nl = n - l + 1
        mp, ip = prof[l][0], prof[l][1]
        exact = pl["nnd"][li, :nl, 0]
        d = np.isfinite(mp)
        t = tol_for(prec, l, exact[d])
        assert np.all(np.abs(mp[d] - exact[d]) <= t), l          # defined values are exact
        assert np.all(ip[~d] == -1)
        k = int(np.argmin(exact))
        assert abs(mp[d].min() - exact[k]) <= tol_for(prec, l, np.array([exact[k]]))[0], l   # the motif
        s = st[li]
        assert s["len"] == l and s["rows"] == nl
        if li == 0 or s["full_profile"]:
            assert d.all() and s["recomputed"] == nl
        else:
            assert s["certified"] + s["recomputed"] + s["skipped"] == nl
            assert d.sum() >= s["certified"]
        computed += nl if (li == 0 or s["full_profile"]) else s["recomputed"]
    # the variable-length motif
    i = int(np.argmin(pl["norm"]))
    assert abs(vm["norm"].min() - pl["norm"][i]) <= tol_for(prec, int(pl["len"][i]), np.array([pl["dist"][i]]))[0]
    assert len(mot) == 1
    ref = oracle.topk_motifs(pl, 1)[0]
    assert abs(mot[0]["norm_dist"] - ref[4]) <= 1e-4
    if gen == "ecg":
        assert computed < 0.5 * sum(s["rows"] for s in st)    # the paper's pruned regime


def test_motif_mode_needs_m_max_1():
    x = workloads.random_walk(500, 53)
    with pytest.raises(mad.MadError) as e:
        mad.mad_create(x, precision=mad.MAD_FP32, m_max=2, mode=1)
    assert e.value.status == mad.MAD_EINVAL
