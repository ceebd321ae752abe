"""CUDA path vs the CPU oracle, element by element, through the C ABI.

Sizes span several R x R tiles (R = 1024 rows) and a
ragged last band; the rw4096 case is the small configuration of the
benchmark suite in full."""
import math

import numpy as np
import pytest

import oracle
import paper_2008_13447_gb300 as mad
import workloads
from parity_util import compare_all, run_gpu

pytestmark = pytest.mark.gpu
PRECS = [pytest.param(mad.MAD_FP64, id="fp64"), pytest.param(mad.MAD_FP32, id="fp32")]


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2008_13447_gb300 import build
    build.build()
    oracle.build()


@pytest.mark.parametrize("prec", PRECS)
def test_random_walk_multi_tile(prec):
    x = workloads.random_walk(5000, 101)
    r = compare_all(x, 40, 48, 5, prec)
    assert r["stats"][0]["tiles"] >= 1


@pytest.mark.parametrize("prec", PRECS)
def test_rw4096_full(prec):
    w = workloads.make("rw4096")
    compare_all(w.series[0], w.lmin[0], w.lmax[0], w.p, prec, m_max=w.m, k_max=w.k)


@pytest.mark.parametrize("prec", PRECS)
def test_ar2_mth_neighbours_half_zone(prec):
    x = workloads.ar2(3100, 102)
    compare_all(x, 30, 36, 6, prec, m_max=3, k_max=4, excl=(1, 2))


@pytest.mark.parametrize("band_form", [0, 1], ids=["full_rows", "symmetric"])
@pytest.mark.parametrize("prec", PRECS)
def test_ecg_pruned_regime(prec, band_form):
    x = workloads.ecg_like(4500, 103, period=60.0)
    r = compare_all(x, 60, 72, 8, prec, m_max=2, k_max=3, band_form=band_form)
    st = r["stats"]
    assert sum(s["certified"] for s in st[1:]) > 0.5 * sum(s["rows"] for s in st[1:])
    # few uncertified rows per band: they take the direct path
    assert sum(s["direct_rows"] for s in st[1:]) > 0


@pytest.mark.parametrize("prec", PRECS)
def test_random_walk_symmetric_form(prec):
    x = workloads.random_walk(5000, 101)
    compare_all(x, 40, 48, 5, prec, band_form=1)


@pytest.mark.parametrize("prec", PRECS)
def test_flat_segments(prec):
    x = workloads.random_walk(2600, 104)
    x[300:380] = 3.25        # flat at every length of the range
    x[1500:1530] = -1.0      # flat only at the shorter lengths
    x[2200:2290] = 7.0
    compare_all(x, 20, 34, 4, prec, m_max=2, k_max=3)


@pytest.mark.parametrize("prec", PRECS)
def test_ragged_band_edges(prec):
    # n_lmin = R + 1 : the last band holds one row
    R = 1024
    x = workloads.random_walk(R + 16, 105)
    compare_all(x, 16, 20, 3, prec, k_max=2)


@pytest.mark.parametrize("prec", PRECS)
def test_long_windows_shared_memory_line(prec):
    # FP64 at l = 409 puts the direct kernel's dynamic shared memory just
    # under 48 KB and its static + dynamic total just over; long windows with
    # a short series also give a sparse band for the direct path
    x = workloads.random_walk(2400, 108)
    compare_all(x, 406, 412, 3, prec, k_max=2)


@pytest.mark.parametrize("prec", PRECS)
def test_smallest_valid_series(prec):
    # n - lmax + 1 = 2 E(lmax) + 3: every window has exactly one or two partners
    lmin, lmax = 8, 12
    E = oracle.excl(lmax)
    n = 2 * E + 3 + lmax - 1
    x = workloads.ar2(n, 106)
    compare_all(x, lmin, lmax, 2, prec, k_max=1)


def test_invalid_profile_arguments():
    x = workloads.random_walk(500, 1)
    ctx = mad.mad_create(x, m_max=2)
    try:
        for args in [(1, 10, 5), (20, 10, 5), (10, 499, 5), (10, 20, 0), (10, 20, 65), (10, 20, 1)]:
            with pytest.raises(mad.MadError) as e:
                mad.mad_profile(ctx, *args)
            assert e.value.status == mad.MAD_EINVAL
        with pytest.raises(mad.MadError) as e:
            mad.mad_motifs(ctx, 0, 3)
        assert e.value.status == mad.MAD_ESTATE
        mad.mad_profile(ctx, 10, 20, 4)
        with pytest.raises(mad.MadError) as e:
            mad.mad_discords(ctx, 0, 3, 3)
        assert e.value.status == mad.MAD_EINVAL
        with pytest.raises(mad.MadError) as e:
            mad.mad_matrix_profile(ctx, 0, 12, len(x))
        assert e.value.status == mad.MAD_EINVAL     # no keep_profiles
    finally:
        mad.mad_destroy(ctx)


def test_device_input_matches_host_input():
    torch = pytest.importorskip("torch")
    x = workloads.random_walk(3000, 107)
    t = torch.tensor(x, device="cuda:0")
    a = mad.mad_create(x, precision=mad.MAD_FP32)
    b = mad.mad_create_device(t, precision=mad.MAD_FP32, stream=torch.cuda.current_stream())
    try:
        for c in (a, b):
            mad.mad_profile(c, 24, 30, 4)
        va, vb = mad.mad_valmp(a, 0, 3000 - 23), mad.mad_valmp(b, 0, 3000 - 23)
        np.testing.assert_array_equal(va["dist"], vb["dist"])
        np.testing.assert_array_equal(va["nn"], vb["nn"])
    finally:
        mad.mad_destroy(a)
        mad.mad_destroy(b)


def test_batch_matches_single_series():
    xs = [workloads.random_walk(2500, 110), workloads.ar2(1800, 111)]
    lmins, lmaxs = [20, 16], [26, 24]
    ctx = mad.mad_create_batch(xs, precision=mad.MAD_FP32, k_max=3)
    try:
        mad.mad_profile_batch(ctx, lmins, lmaxs, 4)
        for s, x in enumerate(xs):
            ref = oracle.valmp_plain(x, lmins[s], lmaxs[s])
            v = mad.mad_valmp(ctx, s, len(x) - lmins[s] + 1)
            assert np.max(np.abs(v["norm"] - ref["norm"])) <= 1e-4
            same = v["len"] == ref["len"]
            assert same.mean() > 0.95
            assert np.max(np.abs(v["dist"][same] - ref["dist"][same])) <= 1e-4 * math.sqrt(lmaxs[s])
    finally:
        mad.mad_destroy(ctx)
