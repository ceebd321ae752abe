"""The seeded synthetic workloads: deterministic, of the stated shapes and
parameters, planted segments where they are said to be."""
import numpy as np
import pytest

import workloads


@pytest.mark.parametrize("name", workloads.WORKLOADS)
def test_named_workloads_are_deterministic_and_well_formed(name):
    a, b = workloads.make(name), workloads.make(name)
    assert len(a.series) == len(b.series) >= 1
    for x, y, lo, hi in zip(a.series, b.series, a.lmin, a.lmax):
        assert x.dtype == np.float64 and x.flags.c_contiguous
        assert np.array_equal(x, y)
        assert np.all(np.isfinite(x))
        assert 2 <= lo <= hi < len(x)
    assert a.cells == float(sum(len(s) ** 2 * (h - l + 1) for s, l, h in zip(a.series, a.lmin, a.lmax)))
    assert a.m <= a.p


def test_stated_sizes():
    w = workloads.make("planted65k")
    assert (len(w.series[0]), w.lmin[0], w.lmax[0], w.p, w.k, w.m) == (65536, 256, 512, 5, 5, 1)
    w = workloads.make("rw4096")
    assert (len(w.series[0]), w.lmin[0], w.lmax[0]) == (4096, 64, 80)
    w = workloads.make("batch256")
    assert len(w.series) == 256
    assert all(2048 <= len(s) <= 65536 and 32 <= a <= 256 and b == 2 * a
               for s, a, b in zip(w.series, w.lmin, w.lmax))


def test_planted_segments_apart_and_visible():
    x, info = workloads.planted_walk(65536, 2, lmax=512)
    segs = [(a, L) for a, b, L in info.motifs] + [(b, L) for a, b, L in info.motifs]
    segs += [(info.spike, 1), (info.level_shift, 1)]
    segs.sort()
    for (o1, l1), (o2, _) in zip(segs, segs[1:]):
        assert o2 - (o1 + l1) >= 2 * 512
    # the two copies of each motif are close in z-normalised distance,
    # much closer than random windows of the walk
    def znorm(v):
        return (v - v.mean()) / v.std()
    rng = np.random.default_rng(0)
    for a, b, L in info.motifs:
        d = np.linalg.norm(znorm(x[a:a + L]) - znorm(x[b:b + L]))
        r = [np.linalg.norm(znorm(x[i:i + L]) - znorm(x[j:j + L]))
             for i, j in rng.integers(0, len(x) - L, (20, 2))]
        assert d < 0.5 * min(r)
    # the spike stands out of its neighbourhood
    s = info.spike
    assert x[s] - x[s - 1] > 5 * np.std(np.diff(x[s - 256:s]))
