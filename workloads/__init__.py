"""Seeded synthetic input series for the variable-length matrix profile.

This module only *generates* float64 series (and the length-range parameters
that go with them). It holds none of the method's arithmetic, so both the CPU
oracle (``oracle/``) and the CUDA path may use it without sharing code.

The paper evaluates on real recordings (GAP, CAP/EEG, ECG, EMG, ASTRO, Sec. 7
"Datasets"); none of them is available here, so every workload below is a
synthetic stand-in with the shape, size and structure of the paper's series:
random walks (the paper's default synthetic model), ECG-like quasi-periodic
beats, seismic-like bursts, and series with planted motifs and discords.

All generators use ``numpy.random.Generator(PCG64(seed))`` and return C-contiguous
float64 arrays.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Workload", "random_walk", "ar2", "ecg_like", "seismic_walk",
    "planted_walk", "make", "WORKLOADS",
]


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def random_walk(n: int, seed: int) -> np.ndarray:
    """Cumulative sum of N(0, 1) increments."""
    return np.ascontiguousarray(np.cumsum(_rng(seed).standard_normal(n)))


def ar2(n: int, seed: int, phi=(0.6, -0.3), burn_in: int = 200) -> np.ndarray:
    """Stationary AR(2) process x_t = phi1 x_{t-1} + phi2 x_{t-2} + N(0, 1)."""
    e = _rng(seed).standard_normal(n + burn_in)
    x = np.zeros(n + burn_in)
    for t in range(2, n + burn_in):
        x[t] = phi[0] * x[t - 1] + phi[1] * x[t - 2] + e[t]
    return np.ascontiguousarray(x[burn_in:])


def ecg_like(n: int, seed: int, period: float = 250.0) -> np.ndarray:
    """Quasi-periodic ECG-like beats: five Gaussian bumps (P, Q, R, S, T) per
    beat, beat period ``period`` x U(0.9, 1.1), baseline wander
    0.2 sin(2 pi t / 3000) and N(0, 0.05) noise."""
    g = _rng(seed)
    # (amplitude, centre as a fraction of the beat, width in samples)
    waves = ((0.15, 0.20, 8.0), (-0.15, 0.36, 3.0), (1.0, 0.40, 4.0),
             (-0.25, 0.44, 4.0), (0.35, 0.65, 14.0))
    x = np.zeros(n)
    t0 = 0.0
    while t0 < n:
        L = period * g.uniform(0.9, 1.1)
        lo = int(max(0, math.floor(t0)))
        hi = int(min(n, math.ceil(t0 + L)))
        t = np.arange(lo, hi, dtype=np.float64)
        for a, c, w in waves:
            x[lo:hi] += a * np.exp(-0.5 * ((t - (t0 + c * L)) / w) ** 2)
        t0 += L
    t = np.arange(n, dtype=np.float64)
    x += 0.2 * np.sin(2 * math.pi * t / 3000.0)
    x += g.normal(0.0, 0.05, n)
    return np.ascontiguousarray(x)


def _disjoint_offsets(g, n, lengths, gap):
    """Uniform offsets for segments of the given lengths, pairwise at least
    ``gap`` apart (start to start, and never overlapping)."""
    for _ in range(10000):
        offs = [int(g.integers(gap, n - L - gap)) for L in lengths]
        ok = True
        for a in range(len(offs)):
            for b in range(a + 1, len(offs)):
                lo, hi = sorted(((offs[a], lengths[a]), (offs[b], lengths[b])))
                if hi[0] - (lo[0] + lo[1]) < gap:
                    ok = False
        if ok:
            return offs
    raise RuntimeError("could not place planted segments")


@dataclass
class Planted:
    motifs: list = field(default_factory=list)    # (offset_a, offset_b, length)
    spike: int = -1
    level_shift: int = -1


def planted_walk(n: int, seed: int, motif_lengths=(200, 300, 400),
                 lmax: int = 512):
    """Random walk with planted motif pairs and two planted discords.

    Each motif pair is two copies of ``sin(2 pi 4 t / L) * hann(L)``, scaled to
    unit standard deviation, then to 3x the local standard deviation of the
    walk at the insertion point, each copy with its own N(0, 0.1) noise (in
    units of that local standard deviation). The copy replaces the walk
    segment, sitting on the walk's level at the segment start; the rest of the
    walk is shifted so the series stays continuous. The discords are a one
    sample spike of +10 local std and a level shift of +5 local std that lasts
    to the end of the series. All planted segments are at least 2 * lmax apart.
    """
    g = _rng(seed)
    x = np.cumsum(g.standard_normal(n))
    lengths = []
    for L in motif_lengths:
        lengths += [L, L]
    lengths += [1, 1]
    offs = _disjoint_offsets(g, n, lengths, 2 * lmax)
    info = Planted()
    for k, L in enumerate(motif_lengths):
        t = np.arange(L, dtype=np.float64)
        shape = np.sin(2 * math.pi * 4 * t / L) * np.hanning(L)
        shape /= shape.std()
        pair = []
        for c in range(2):
            o = offs[2 * k + c]
            loc = float(x[o:o + L].std())
            seg = x[o] + loc * (3.0 * shape + g.normal(0.0, 0.1, L))
            step = x[o + L] - x[o + L - 1] if o + L < n else 0.0
            tail_shift = (seg[-1] + step) - (x[o + L] if o + L < n else 0.0)
            x[o:o + L] = seg
            if o + L < n:
                x[o + L:] += tail_shift
            pair.append(o)
        info.motifs.append((min(pair), max(pair), L))
    o_spike, o_shift = offs[-2], offs[-1]
    loc = float(x[max(0, o_spike - 256):o_spike + 256].std())
    x[o_spike] += 10.0 * loc
    info.spike = o_spike
    loc = float(x[max(0, o_shift - 256):o_shift + 256].std())
    x[o_shift:] += 5.0 * loc
    info.level_shift = o_shift
    return np.ascontiguousarray(x), info


def seismic_walk(n: int, seed: int, fs: float = 100.0, every: int = 100_000,
                 jitter: int = 10_000, tau: float = 200.0):
    """Random walk plus seismic-like bursts: every ``every`` +- ``jitter``
    samples a linear chirp from 5 to 40 Hz (at sampling rate ``fs``) with an
    exp(-t / tau) envelope and amplitude 5x the local standard deviation."""
    g = _rng(seed)
    x = np.cumsum(g.standard_normal(n))
    dur = int(5 * tau)
    t = np.arange(dur, dtype=np.float64) / fs
    f0, f1 = 5.0, 40.0
    T = dur / fs
    phase = 2 * math.pi * (f0 * t + 0.5 * (f1 - f0) / T * t * t)
    burst = np.sin(phase) * np.exp(-np.arange(dur) / tau)
    burst /= np.abs(burst).max()
    o = int(g.integers(every - jitter, every + jitter))
    starts = []
    while o + dur < n:
        loc = float(x[o:o + dur].std())
        x[o:o + dur] += 5.0 * loc * burst
        starts.append(o)
        o += int(g.integers(every - jitter, every + jitter))
    return np.ascontiguousarray(x), starts


@dataclass
class Workload:
    """One synthetic workload: series plus the method's parameters."""
    name: str
    series: list            # list of float64 arrays (one per series)
    lmin: list              # per series
    lmax: list              # per series
    p: int
    k: int
    m: int
    excl: tuple = (1, 4)    # exclusion zone E(l) = ceil(l * num / den)
    info: object = None

    @property
    def cells(self) -> float:
        """Sum over series of n^2 * |L| (the throughput unit)."""
        return float(sum(len(s) ** 2 * (b - a + 1)
                         for s, a, b in zip(self.series, self.lmin, self.lmax)))


def _batch(seed: int, count: int = 256):
    g = _rng(seed)
    series, lmin, lmax = [], [], []
    for s in range(count):
        n = int(math.floor(math.exp(g.uniform(math.log(2048), math.log(65536)))))
        sub = int(g.integers(0, 2**31 - 1))
        series.append(random_walk(n, sub) if s % 2 == 0 else ar2(n, sub))
        a = int(g.integers(32, 257))
        lmin.append(a)
        lmax.append(2 * a)
    return series, lmin, lmax


def make(name: str) -> Workload:
    """Build one of the named workloads.

    rw4096     : random walk n=4096, l in [64, 80], p=5, top-5 motifs, Top-5 1st discords
    planted65k : random walk n=65536 with 3 planted motif pairs and 2 discords, l in [256, 512], p=5
    ecg262k    : ECG-like n=262144, l in [128, 768], p=10
    batch256   : 256 series, n log-uniform in [2048, 65536], lmin U{32..256}, lmax=2 lmin, p=5
    seismic2m  : random walk n=2097152 with seismic bursts, l in [256, 1024], p=10, Top-10 3rd discords
    """
    if name == "rw4096":
        return Workload(name, [random_walk(4096, 1)], [64], [80], p=5, k=5, m=1)
    if name == "planted65k":
        x, info = planted_walk(65536, 2, lmax=512)
        return Workload(name, [x], [256], [512], p=5, k=5, m=1, info=info)
    if name == "ecg262k":
        return Workload(name, [ecg_like(262144, 3)], [128], [768], p=10, k=5, m=1)
    if name == "batch256":
        s, a, b = _batch(4)
        return Workload(name, s, a, b, p=5, k=5, m=1)
    if name == "seismic2m":
        x, starts = seismic_walk(2097152, 5)
        return Workload(name, [x], [256], [1024], p=10, k=10, m=3, info=starts)
    raise KeyError(name)


WORKLOADS = ("rw4096", "planted65k", "ecg262k", "batch256", "seismic2m")
