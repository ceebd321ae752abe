"""CPU FP64 oracle for the exact variable-length matrix profile.

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only users. The product (the CUDA
library and its Python binding) never imports this package, and this package
never imports the product.

The arithmetic lives in ``mad_oracle.c`` (plain C, FP64, OpenMP over windows),
loaded through ctypes. ``build()`` compiles it with gcc.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mad_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libmad_oracle.so")
_lib = None

__all__ = [
    "build", "excl", "window_stats", "pearson", "dist", "dist_direct", "lower_bound", "row_valid",
    "distance_profile", "matrix_profile", "row", "rows", "num_threads", "valmp_plain", "valmod_pruned",
    "topk_motifs", "discords_one_length", "discords",
]


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/libmad_oracle.so``.

    No FMA contraction (``-ffp-contract=off``) so x86 and Arm builds round
    identically."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
                               "-ffp-contract=off", "-fno-fast-math", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _L():
    global _lib
    if _lib is None:
        build()
        lib = C.CDLL(_LIB)
        d, i64, i32, P = C.c_double, C.c_int64, C.c_int32, C.c_void_p
        sig = {
            "orc_excl": (i64, [C.c_int, C.c_int, C.c_int]),
            "orc_window_stats": (None, [P, i64, C.c_int, i64, P, P]),
            "orc_is_flat": (C.c_int, [P, i64, C.c_int, i64]),
            "orc_pearson": (d, [P, i64, C.c_int, i64, i64]),
            "orc_dist": (d, [P, i64, C.c_int, i64, i64]),
            "orc_dist_direct": (d, [P, i64, C.c_int, i64, i64]),
            "orc_lower_bound": (d, [C.c_int, d, d, d]),
            "orc_row_valid": (C.c_int, [P, C.c_int, C.c_int, d]),
            "orc_distance_profile": (None, [P, i64, C.c_int, C.c_int, C.c_int, i64, P]),
            "orc_matrix_profile": (None, [P, i64, C.c_int, C.c_int, C.c_int, C.c_int, P, P, P, P]),
            "orc_row": (None, [P, i64, C.c_int, C.c_int, C.c_int, C.c_int, i64, P, P, P, P]),
            "orc_rows": (None, [P, i64, C.c_int, C.c_int, C.c_int, P, i64, P, P]),
            "orc_num_threads": (C.c_int, []),
            "orc_valmp_plain": (None, [P, i64, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                                       P, P, P, P, P, P]),
            "orc_valmod_pruned": (None, [P, i64, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                                         P, P, P, P, P, P, P, C.c_int, P, P]),
            "orc_valmod_motif": (None, [P, i64, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                                        P, P, P, P, P, P]),
            "orc_topk_motifs": (C.c_int, [i64, P, P, P, P, C.c_int, C.c_int, C.c_int, P, P, P, P, P]),
            "orc_motif_sets": (None, [P, i64, C.c_int, P, P, P, P, d, C.c_int, C.c_int, C.c_int, P, P]),
            "orc_discords_one_length": (C.c_int, [i64, P, P, C.c_int, C.c_int, C.c_int, C.c_int, P, P, P]),
            "orc_discords": (None, [i64, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, P, P,
                                    P, P, P, P, P]),
            "orc_discords_global": (C.c_int, [i64, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                                              C.c_int, P, P, P, P, P, P, P]),
            "orc_dkm_streamed": (None, [i64, P, P, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                                        P, P, P]),
            "orc_discords_streamed": (None, [i64, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                                             C.c_int, P, P, P, P, P, P, P]),
            "orc_valmod_discord": (None, [P, i64, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                                          C.c_int, P, P, P, P, P, P, P, P, P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


def _f64(x):
    return np.ascontiguousarray(x, dtype=np.float64)


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


def excl(l: int, num: int = 1, den: int = 4) -> int:
    return int(_L().orc_excl(l, num, den))


def window_stats(x, l: int, i: int):
    x = _f64(x)
    mu, sd = C.c_double(), C.c_double()
    _L().orc_window_stats(_p(x), len(x), l, i, C.byref(mu), C.byref(sd))
    return mu.value, sd.value


def pearson(x, l, i, j):
    x = _f64(x)
    return _L().orc_pearson(_p(x), len(x), l, i, j)


def dist(x, l, i, j):
    x = _f64(x)
    return _L().orc_dist(_p(x), len(x), l, i, j)


def dist_direct(x, l, i, j):
    x = _f64(x)
    return _L().orc_dist_direct(_p(x), len(x), l, i, j)


def lower_bound(l_b, q, sigma_row_lb, sigma_row_lnew):
    return _L().orc_lower_bound(l_b, q, sigma_row_lb, sigma_row_lnew)


def row_valid(d_sorted, m, bound):
    d = _f64(d_sorted)
    return bool(_L().orc_row_valid(_p(d), len(d), m, bound))


def distance_profile(x, l, i, num=1, den=4):
    x = _f64(x)
    out = np.empty(len(x) - l + 1)
    _L().orc_distance_profile(_p(x), len(x), l, num, den, i, _p(out))
    return out


def matrix_profile(x, l, m_max=1, num=1, den=4):
    """Per-length matrix profile: (mp, ip, nnd[n_l, m_max], nnj[n_l, m_max])."""
    x = _f64(x)
    nl = len(x) - l + 1
    mp, ip = np.empty(nl), np.empty(nl, np.int64)
    nnd, nnj = np.empty((nl, m_max)), np.empty((nl, m_max), np.int64)
    _L().orc_matrix_profile(_p(x), len(x), l, num, den, m_max, _p(mp), _p(ip), _p(nnd), _p(nnj))
    return mp, ip, nnd, nnj


def row(x, l, i, m_max=1, num=1, den=4):
    """Matrix-profile quantities of window i only: (mp, ip, nnd[m_max], nnj[m_max])."""
    x = _f64(x)
    mp, ip = C.c_double(), C.c_int64()
    nnd, nnj = np.empty(m_max), np.empty(m_max, np.int64)
    _L().orc_row(_p(x), len(x), l, num, den, m_max, i, C.byref(mp), C.byref(ip), _p(nnd), _p(nnj))
    return mp.value, ip.value, nnd, nnj


def rows(x, l, row_list, num=1, den=4):
    """Matrix-profile value and index of the listed windows at length l
    (parallel over windows): (mp, ip)."""
    x = _f64(x)
    r = np.ascontiguousarray(row_list, np.int64)
    mp, ip = np.empty(len(r)), np.empty(len(r), np.int64)
    _L().orc_rows(_p(x), len(x), l, num, den, _p(r), len(r), _p(mp), _p(ip))
    return mp, ip


def num_threads() -> int:
    return int(_L().orc_num_threads())


def _valmp_out(n0):
    return (np.empty(n0), np.empty(n0), np.zeros(n0, np.int32), np.empty(n0, np.int64))


def valmp_plain(x, lmin, lmax, m_max=1, num=1, den=4, keep_nn=False):
    """VALMP from independent per-length matrix profiles.

    Returns dict(dist, norm, len, nn[, nnd, nnj]) where nnd/nnj have shape
    (|L|, n_lmin, m_max) (NaN / -1 past n_l)."""
    x = _f64(x)
    n0 = len(x) - lmin + 1
    dist_, norm_, len_, nn_ = _valmp_out(n0)
    nnd = nnj = None
    if keep_nn:
        nnd = np.empty((lmax - lmin + 1, n0, m_max))
        nnj = np.empty((lmax - lmin + 1, n0, m_max), np.int64)
    _L().orc_valmp_plain(_p(x), len(x), lmin, lmax, num, den, m_max, _p(dist_), _p(norm_), _p(len_),
                         _p(nn_), _p(nnd) if keep_nn else None, _p(nnj) if keep_nn else None)
    out = dict(dist=dist_, norm=norm_, len=len_, nn=nn_)
    if keep_nn:
        out.update(nnd=nnd, nnj=nnj)
    return out


def valmod_pruned(x, lmin, lmax, p, m_max=1, num=1, den=4, keep_nn=False, observe_len=0):
    """Pruned VALMOD (exact-rows reading). Returns the same dict as
    valmp_plain plus ``stats`` of shape (|L|, 3): rows alive, valid rows,
    recomputed rows per length; with observe_len (> lmin) also ``gap``
    (maxLB - minED) and ``tlb`` (mean LB / ED) per row at that length."""
    if not (1 <= m_max <= p <= 64):
        raise ValueError("need 1 <= m_max <= p <= 64")
    x = _f64(x)
    n0 = len(x) - lmin + 1
    dist_, norm_, len_, nn_ = _valmp_out(n0)
    nL = lmax - lmin + 1
    stats = np.empty((nL, 3), np.int64)
    nnd = nnj = None
    if keep_nn:
        nnd = np.empty((nL, n0, m_max))
        nnj = np.empty((nL, n0, m_max), np.int64)
    gap = tlb = None
    if observe_len:
        gap, tlb = np.full(n0, np.nan), np.full(n0, np.nan)
    _L().orc_valmod_pruned(_p(x), len(x), lmin, lmax, num, den, p, m_max, _p(dist_), _p(norm_),
                           _p(len_), _p(nn_), _p(nnd) if keep_nn else None,
                           _p(nnj) if keep_nn else None, _p(stats), observe_len,
                           _p(gap) if observe_len else None, _p(tlb) if observe_len else None)
    out = dict(dist=dist_, norm=norm_, len=len_, nn=nn_, stats=stats)
    if observe_len:
        nl = len(x) - observe_len + 1
        out.update(gap=gap[:nl], tlb=tlb[:nl])
    if keep_nn:
        out.update(nnd=nnd, nnj=nnj)
    return out


def valmod_motif(x, lmin, lmax, p, num=1, den=4):
    """The paper-literal pruned iteration (motif of every length guaranteed,
    not every row). Returns VALMP as valmp_plain does, plus ``submp``
    (|L|, n_lmin) with NaN where a row's value at that length is undefined,
    and ``stats`` (|L|, 5): rows, valid, non-valid, recomputed, full."""
    if not (1 <= p <= 64):
        raise ValueError("need 1 <= p <= 64")
    x = _f64(x)
    n0 = len(x) - lmin + 1
    dist_, norm_, len_, nn_ = _valmp_out(n0)
    nL = lmax - lmin + 1
    submp = np.empty((nL, n0))
    stats = np.empty((nL, 5), np.int64)
    _L().orc_valmod_motif(_p(x), len(x), lmin, lmax, num, den, p, _p(dist_), _p(norm_), _p(len_), _p(nn_),
                          _p(submp), _p(stats))
    return dict(dist=dist_, norm=norm_, len=len_, nn=nn_, submp=submp, stats=stats)


def topk_motifs(valmp, k, num=1, den=4):
    """Top-k motif pairs from a VALMP dict: list of (a, b, len, dist, norm_dist)."""
    d, nd = _f64(valmp["dist"]), _f64(valmp["norm"])
    ln = np.ascontiguousarray(valmp["len"], np.int32)
    nn = np.ascontiguousarray(valmp["nn"], np.int64)
    a, b = np.empty(k, np.int64), np.empty(k, np.int64)
    L, od, ond = np.empty(k, np.int32), np.empty(k), np.empty(k)
    got = _L().orc_topk_motifs(len(d), _p(d), _p(nd), _p(ln), _p(nn), num, den, k,
                               _p(a), _p(b), _p(L), _p(od), _p(ond))
    return [(int(a[r]), int(b[r]), int(L[r]), float(od[r]), float(ond[r])) for r in range(got)]


def motif_sets(x, pairs, D, cap, num=1, den=4):
    """Motif sets grown from motif pairs [(a, b, len, dist), ...] with radius
    D * dist: list of member offset lists (a, b first)."""
    x = _f64(x)
    k = len(pairs)
    a = np.array([p[0] for p in pairs], np.int64)
    b = np.array([p[1] for p in pairs], np.int64)
    L = np.array([p[2] for p in pairs], np.int32)
    d = np.array([p[3] for p in pairs], np.float64)
    mem = np.zeros((k, cap), np.int64)
    cnt = np.zeros(k, np.int32)
    _L().orc_motif_sets(_p(x), len(x), k, _p(a), _p(b), _p(L), _p(d), float(D), num, den, cap, _p(mem), _p(cnt))
    return [list(mem[s, :cnt[s]]) for s in range(k)]


def discords_one_length(score, l, k, nbr=None, num=1, den=4):
    score = _f64(score)
    nb = np.ascontiguousarray(nbr if nbr is not None else np.full(len(score), -1), np.int64)
    off, dd, nn = np.empty(k, np.int64), np.empty(k), np.empty(k, np.int64)
    got = _L().orc_discords_one_length(len(score), _p(score), _p(nb), l, num, den, k, _p(off), _p(dd), _p(nn))
    return [(int(off[r]), float(dd[r]), int(nn[r])) for r in range(got)]


def discords_global(n, lmin, lmax, k, m_max, m, nnd_all, nnj_all, num=1, den=4):
    """Global-greedy variable-length m-th discords: list of (off, len, dist,
    norm_dist, nn), at most k."""
    nnd_all = _f64(nnd_all)
    nnj_all = np.ascontiguousarray(nnj_all, np.int64)
    off, ln = np.empty(k, np.int64), np.empty(k, np.int32)
    dd, nd, nn = np.empty(k), np.empty(k), np.empty(k, np.int64)
    got = _L().orc_discords_global(n, lmin, lmax, num, den, k, m_max, m, _p(nnd_all), _p(nnj_all),
                                   _p(off), _p(ln), _p(dd), _p(nd), _p(nn))
    return [(int(off[r]), int(ln[r]), float(dd[r]), float(nd[r]), int(nn[r])) for r in range(got)]


def dkm_streamed(nnd, nnj, l, k, m, num=1, den=4):
    """dkm_l as Algorithms 7 and 8 print it, from n_l x m_max best-match
    tables: arrays (k, m) off (-1 = empty), dist, nn."""
    nnd = _f64(nnd)
    nnj = np.ascontiguousarray(nnj, np.int64)
    nl, m_max = nnd.shape
    off, dd, nn = np.empty((k, m), np.int64), np.empty((k, m)), np.empty((k, m), np.int64)
    _L().orc_dkm_streamed(nl, _p(nnd), _p(nnj), m_max, l, num, den, k, m, _p(off), _p(dd), _p(nn))
    return dict(off=off, dist=dd, nn=nn)


def discords_streamed(n, lmin, lmax, k, m_max, m, nnd_all, nnj_all, num=1, den=4):
    """dkm_{lmin,lmax} from the streamed dkm_l, merged by Algorithm 9:
    arrays of shape (k, m) as discords()."""
    nnd_all = _f64(nnd_all)
    nnj_all = np.ascontiguousarray(nnj_all, np.int64)
    off, ln = np.empty((k, m), np.int64), np.empty((k, m), np.int32)
    dd, nd, nn = np.empty((k, m)), np.empty((k, m)), np.empty((k, m), np.int64)
    _L().orc_discords_streamed(n, lmin, lmax, num, den, k, m_max, m, _p(nnd_all), _p(nnj_all),
                               _p(off), _p(ln), _p(dd), _p(nd), _p(nn))
    return dict(off=off, len=ln, dist=dd, norm=nd, nn=nn)


def valmod_discord(x, lmin, lmax, p, k, m, num=1, den=4):
    """Top-k m-th discords with the paper's pruning (Algorithms 7, 10, 8, 9):
    dict(off, len, dist, norm, nn) of shape (k, m) (the merged table),
    dkm_off / dkm_d of shape (|L|, k, m) (every dkm_l), stats (|L|, 4) =
    rows, valid, listed, recomputed, and recomp (|L|, n - lmin + 1) bool: the
    rows whose full profile was computed at each length."""
    x = _f64(x)
    nL = lmax - lmin + 1
    off, ln = np.empty((k, m), np.int64), np.empty((k, m), np.int32)
    dd, nd, nn = np.empty((k, m)), np.empty((k, m)), np.empty((k, m), np.int64)
    doff, dd_l = np.empty((nL, k, m), np.int64), np.empty((nL, k, m))
    st = np.empty((nL, 4), np.int64)
    rc = np.empty((nL, len(x) - lmin + 1), np.int8)
    _L().orc_valmod_discord(_p(x), len(x), lmin, lmax, num, den, p, k, m, _p(off), _p(ln), _p(dd), _p(nd),
                            _p(nn), _p(doff), _p(dd_l), _p(st), _p(rc))
    return dict(off=off, len=ln, dist=dd, norm=nd, nn=nn, dkm_off=doff, dkm_d=dd_l, stats=st,
                recomp=rc.astype(bool))


def discords(n, lmin, lmax, k, m_max, nnd_all, nnj_all, num=1, den=4):
    """Variable-length Top-k m-th discord table: arrays of shape (k, m_max):
    off, len (0 = empty), dist, norm_dist, nn."""
    nnd_all = _f64(nnd_all)
    nnj_all = np.ascontiguousarray(nnj_all, np.int64)
    off, ln = np.empty((k, m_max), np.int64), np.empty((k, m_max), np.int32)
    dd, nd, nn = np.empty((k, m_max)), np.empty((k, m_max)), np.empty((k, m_max), np.int64)
    _L().orc_discords(n, lmin, lmax, num, den, k, m_max, _p(nnd_all), _p(nnj_all),
                      _p(off), _p(ln), _p(dd), _p(nd), _p(nn))
    return dict(off=off, len=ln, dist=dd, norm=nd, nn=nn)
