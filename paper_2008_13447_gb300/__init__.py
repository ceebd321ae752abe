"""Python binding of the GB300 exact variable-length matrix profile library.

Argument marshalling only: every step of the method runs in the CUDA library
``_build/libmad.so`` behind the C ABI of ``include/mad.h``. The functions
below carry the ABI's names. There is no CPU fallback: if the library is
missing the import of any function raises.

Typical use::

    import numpy as np, paper_2008_13447_gb300 as mad
    ctx = mad.mad_create(x, precision=mad.MAD_FP32, k_max=5, m_max=1)
    mad.mad_profile(ctx, 256, 512, 5)
    motifs = mad.mad_motifs(ctx, 0, 5)
    discords = mad.mad_discords(ctx, 0, 5, 1)
    mad.mad_destroy(ctx)
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libmad.so")

MAD_OK, MAD_EINVAL, MAD_ENOMEM, MAD_ECUDA, MAD_ESTATE, MAD_ETIMEOUT, MAD_EINTERNAL = range(7)
MAD_FP64, MAD_FP32, MAD_SPLIT_TC = 0, 1, 2
MAD_NOALLOC_MAX_SLOTS = 1024
STATUS_NAMES = {0: "MAD_OK", 1: "MAD_EINVAL", 2: "MAD_ENOMEM", 3: "MAD_ECUDA", 4: "MAD_ESTATE",
                5: "MAD_ETIMEOUT", 6: "MAD_EINTERNAL"}
ABI_FUNCTIONS = ("mad_create", "mad_create_device", "mad_create_batch", "mad_profile", "mad_profile_batch",
                 "mad_motifs", "mad_discords", "mad_discords_global", "mad_discords_streamed",
                 "mad_valmp", "mad_matrix_profile", "mad_stats",
                 "mad_mth_nn_dist_noalloc", "mad_motif_sets", "mad_observe", "mad_last_error",
                 "mad_destroy", "mad_debug_wavefront_wait_limit", "mad_debug_audit_error_bounds",
                 "mad_set_graphs", "mad_set_autotune", "mad_debug_tc_tma")


class mad_options(C.Structure):
    _fields_ = [("excl_num", C.c_int32), ("excl_den", C.c_int32), ("precision", C.c_int32),
                ("k_max", C.c_int32), ("m_max", C.c_int32), ("keep_profiles", C.c_int32),
                ("mode", C.c_int32), ("band_form", C.c_int32), ("observe_len", C.c_int32),
                ("stream", C.c_void_p)]


class mad_motif(C.Structure):
    _fields_ = [("a", C.c_int64), ("b", C.c_int64), ("len", C.c_int32), ("reserved", C.c_int32),
                ("dist", C.c_double), ("norm_dist", C.c_double), ("dist_recheck", C.c_double)]


class mad_discord(C.Structure):
    _fields_ = [("off", C.c_int64), ("nn", C.c_int64), ("len", C.c_int32), ("rank", C.c_int32),
                ("m", C.c_int32), ("reserved", C.c_int32), ("dist", C.c_double), ("norm_dist", C.c_double),
                ("dist_recheck", C.c_double)]


class mad_length_stats(C.Structure):
    _fields_ = [("len", C.c_int32), ("reserved", C.c_int32), ("rows", C.c_int64), ("certified", C.c_int64),
                ("recomputed", C.c_int64), ("tiles", C.c_int64), ("passes", C.c_int64),
                ("band_cells", C.c_int64), ("launches", C.c_int64), ("inserts", C.c_int64),
                ("col_appends", C.c_int64), ("second_pass_rows", C.c_int64), ("direct_rows", C.c_int64),
                ("band_ms", C.c_double),
                ("fp32_dq_max", C.c_double), ("skipped", C.c_int64), ("full_profile", C.c_int32),
                ("reserved2", C.c_int32), ("dq_ratio_max", C.c_double), ("direct_ms", C.c_double),
                ("rows_ms", C.c_double), ("graph", C.c_int32), ("band_rows", C.c_int32)]


class mad_motif_set(C.Structure):
    _fields_ = [("a", C.c_int64), ("b", C.c_int64), ("len", C.c_int32), ("count", C.c_int32),
                ("radius", C.c_double)]


class MadError(RuntimeError):
    def __init__(self, status, message):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), message))
        self.status = status


_lib = None


def library() -> C.CDLL:
    """Load ``libmad.so`` (built by ``build.py``). Raises if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libmad.so not built (run paper_2008_13447_gb300/build.py): %s" % LIB_PATH)
        lib = C.CDLL(LIB_PATH)
        P, i32, i64 = C.c_void_p, C.c_int32, C.c_int64
        sig = {
            "mad_create": [P, i64, C.POINTER(mad_options), C.POINTER(P)],
            "mad_create_device": [P, i32, i64, C.POINTER(mad_options), C.POINTER(P)],
            "mad_create_batch": [C.POINTER(P), C.POINTER(i64), i32, C.POINTER(mad_options), C.POINTER(P)],
            "mad_profile": [P, i32, i32, i32],
            "mad_profile_batch": [P, C.POINTER(i32), C.POINTER(i32), i32],
            "mad_motifs": [P, i32, i32, C.POINTER(mad_motif), C.POINTER(i32)],
            "mad_discords": [P, i32, i32, i32, C.POINTER(mad_discord), C.POINTER(i32)],
            "mad_discords_global": [P, i32, i32, i32, C.POINTER(mad_discord), C.POINTER(i32)],
            "mad_discords_streamed": [P, i32, i32, i32, C.POINTER(mad_discord), C.POINTER(i32)],
            "mad_valmp": [P, i32, P, P, P, P],
            "mad_matrix_profile": [P, i32, i32, P, P, P, P],
            "mad_stats": [P, i32, C.POINTER(mad_length_stats), i32, C.POINTER(i32)],
            "mad_mth_nn_dist_noalloc": [P, i64, P, i32, i32, i32, i32, P, P],
            "mad_motif_sets": [P, i32, i32, C.c_double, i32, C.POINTER(mad_motif_set), P, C.POINTER(i32)],
            "mad_observe": [P, i32, P, P],
        }
        for name, args in sig.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = C.c_int
        lib.mad_last_error.argtypes = [P]
        lib.mad_last_error.restype = C.c_char_p
        lib.mad_destroy.argtypes = [P]
        lib.mad_destroy.restype = None
        lib.mad_debug_wavefront_wait_limit.argtypes = [i32]
        lib.mad_debug_wavefront_wait_limit.restype = None
        lib.mad_debug_audit_error_bounds.argtypes = [i32]
        lib.mad_debug_audit_error_bounds.restype = None
        lib.mad_set_graphs.argtypes = [i32]
        lib.mad_set_graphs.restype = None
        lib.mad_set_autotune.argtypes = [i32]
        lib.mad_set_autotune.restype = None
        lib.mad_debug_tc_tma.argtypes = [i32]
        lib.mad_debug_tc_tma.restype = None
        _lib = lib
    return _lib


def _check(status, ctx):
    if status != MAD_OK:
        raise MadError(status, library().mad_last_error(ctx).decode())


def _options(precision=MAD_FP64, excl=(1, 4), k_max=10, m_max=1, keep_profiles=False, stream=None, band_form=0,
             mode=0, observe_len=0):
    o = mad_options()
    o.excl_num, o.excl_den = excl
    o.precision = precision
    o.k_max = k_max
    o.m_max = m_max
    o.keep_profiles = 1 if keep_profiles else 0
    o.band_form = band_form
    o.mode = mode
    o.observe_len = observe_len
    if stream is not None:
        o.stream = stream if isinstance(stream, int) else stream.cuda_stream
    return o


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


def mad_create(series, **opts):
    """Create a context from a host FP64 series (numpy array)."""
    x = np.ascontiguousarray(series, dtype=np.float64)
    o = _options(**opts)
    ctx = C.c_void_p()
    _check(library().mad_create(_p(x), len(x), C.byref(o), C.byref(ctx)), None)
    return ctx


def mad_create_device(tensor, **opts):
    """Create a context from a CUDA tensor (torch, float64 or float32,
    contiguous). The tensor must outlive the context."""
    import torch
    if not (tensor.is_cuda and tensor.is_contiguous() and tensor.dim() == 1):
        raise ValueError("need a contiguous 1-D CUDA tensor")
    dtype = {torch.float64: 0, torch.float32: 1}[tensor.dtype]
    o = _options(**opts)
    ctx = C.c_void_p()
    _check(library().mad_create_device(C.c_void_p(tensor.data_ptr()), dtype, tensor.numel(), C.byref(o),
                                       C.byref(ctx)), None)
    return ctx


def mad_create_batch(series_list, **opts):
    xs = [np.ascontiguousarray(s, dtype=np.float64) for s in series_list]
    ptrs = (C.c_void_p * len(xs))(*[x.ctypes.data for x in xs])
    ns = (C.c_int64 * len(xs))(*[len(x) for x in xs])
    o = _options(**opts)
    ctx = C.c_void_p()
    _check(library().mad_create_batch(ptrs, ns, len(xs), C.byref(o), C.byref(ctx)), None)
    return ctx


def mad_profile(ctx, lmin, lmax, p):
    _check(library().mad_profile(ctx, lmin, lmax, p), ctx)


def mad_profile_batch(ctx, lmin, lmax, p):
    a = (C.c_int32 * len(lmin))(*lmin)
    b = (C.c_int32 * len(lmax))(*lmax)
    _check(library().mad_profile_batch(ctx, a, b, p), ctx)


def mad_motifs(ctx, series, k):
    """Top-k motif pairs: list of dicts (a, b, len, dist, norm_dist, dist_recheck)."""
    out = (mad_motif * k)()
    n = C.c_int32()
    _check(library().mad_motifs(ctx, series, k, out, C.byref(n)), ctx)
    return [dict(a=m.a, b=m.b, len=m.len, dist=m.dist, norm_dist=m.norm_dist, dist_recheck=m.dist_recheck)
            for m in out[:n.value]]


def mad_motif_sets(ctx, series, k, D, cap):
    """Motif sets grown from the top-k motif pairs: list of dicts
    (a, b, len, radius, members)."""
    sets = (mad_motif_set * k)()
    mem = np.zeros((k, cap), np.int64)
    n = C.c_int32()
    _check(library().mad_motif_sets(ctx, series, k, float(D), cap, sets, _p(mem), C.byref(n)), ctx)
    return [dict(a=s.a, b=s.b, len=s.len, radius=s.radius, members=list(mem[i, :s.count]))
            for i, s in enumerate(sets[:n.value])]


def mad_observe(ctx, series, n_rows):
    """(gap, tlb) arrays of n_rows = n - observe_len + 1 entries."""
    gap, tlb = np.empty(n_rows), np.empty(n_rows)
    _check(library().mad_observe(ctx, series, _p(gap), _p(tlb)), ctx)
    return gap, tlb


def mad_discords(ctx, series, k, m):
    """The k x m block of the discord table: list (rank-major) of dicts."""
    out = (mad_discord * (k * m))()
    n = C.c_int32()
    _check(library().mad_discords(ctx, series, k, m, out, C.byref(n)), ctx)
    return [dict(off=d.off, nn=d.nn, len=d.len, rank=d.rank, m=d.m, dist=d.dist, norm_dist=d.norm_dist,
                 dist_recheck=d.dist_recheck) for d in out[:n.value]]


def mad_discords_global(ctx, series, k, m):
    """Global-greedy variable-length discords (needs keep_profiles=True):
    list (rank-major) of dicts like mad_discords."""
    out = (mad_discord * (k * m))()
    n = C.c_int32()
    _check(library().mad_discords_global(ctx, series, k, m, out, C.byref(n)), ctx)
    return [dict(off=d.off, nn=d.nn, len=d.len, rank=d.rank, m=d.m, dist=d.dist, norm_dist=d.norm_dist,
                 dist_recheck=d.dist_recheck) for d in out[:n.value]]


def mad_discords_streamed(ctx, series, k, m):
    """dkm_{lmin,lmax} in the streamed form of Algorithms 7 and 8 (needs
    keep_profiles=True): list (rank-major) of dicts like mad_discords."""
    out = (mad_discord * (k * m))()
    n = C.c_int32()
    _check(library().mad_discords_streamed(ctx, series, k, m, out, C.byref(n)), ctx)
    return [dict(off=d.off, nn=d.nn, len=d.len, rank=d.rank, m=d.m, dist=d.dist, norm_dist=d.norm_dist,
                 dist_recheck=d.dist_recheck) for d in out[:n.value]]


def mad_valmp(ctx, series, n0):
    """VALMP arrays of n0 = n - lmin + 1 entries: dict(dist, norm, len, nn)."""
    d, nd = np.empty(n0), np.empty(n0)
    ln, nn = np.empty(n0, np.int32), np.empty(n0, np.int64)
    _check(library().mad_valmp(ctx, series, _p(d), _p(nd), _p(ln), _p(nn)), ctx)
    return dict(dist=d, norm=nd, len=ln, nn=nn)


def mad_matrix_profile(ctx, series, length, n, m_max=1):
    """Matrix profile at one length (context made with keep_profiles=True):
    (mp, ip, nnd[n_l, m_max], nnj[n_l, m_max])."""
    nl = n - length + 1
    mp, ip = np.empty(nl), np.empty(nl, np.int64)
    nnd, nnj = np.empty((nl, m_max)), np.empty((nl, m_max), np.int64)
    _check(library().mad_matrix_profile(ctx, series, length, _p(mp), _p(ip), _p(nnd), _p(nnj)), ctx)
    return mp, ip, nnd, nnj


def mad_stats(ctx, series, cap=1 << 16):
    out = (mad_length_stats * cap)()
    n = C.c_int32()
    _check(library().mad_stats(ctx, series, out, cap, C.byref(n)), ctx)
    return [dict(len=s.len, rows=s.rows, certified=s.certified, recomputed=s.recomputed, tiles=s.tiles,
                 passes=s.passes, band_cells=s.band_cells, launches=s.launches, inserts=s.inserts,
                 col_appends=s.col_appends, second_pass_rows=s.second_pass_rows, direct_rows=s.direct_rows,
                 band_ms=s.band_ms, fp32_dq_max=s.fp32_dq_max, skipped=s.skipped,
                 full_profile=s.full_profile, dq_ratio_max=s.dq_ratio_max, direct_ms=s.direct_ms,
                 rows_ms=s.rows_ms, graph=s.graph, band_rows=s.band_rows) for s in out[:min(n.value, cap)]]


def mad_mth_nn_dist_noalloc(x_ptr, n, cells, m_max, out_ptr, excl=(1, 4), stream=None):
    """m-th best-match distances of the windows in ``cells`` (rows of
    (off, len, m)), recomputed in FP64, written to ``out_ptr``. ``x_ptr`` and
    ``out_ptr`` are device addresses (ints, e.g. ``tensor.data_ptr()``) of n
    and len(cells) doubles; the call allocates no device memory."""
    c = np.ascontiguousarray(cells, dtype=np.int32).reshape(-1, 3)
    st = None if stream is None else C.c_void_p(stream if isinstance(stream, int) else stream.cuda_stream)
    _check(library().mad_mth_nn_dist_noalloc(C.c_void_p(x_ptr), n, _p(c), len(c), m_max, excl[0], excl[1],
                                             C.c_void_p(out_ptr), st), None)


def mad_debug_wavefront_wait_limit(tries):
    """Test hook: tries of the band kernel's wavefront waits (< 0: default)."""
    library().mad_debug_wavefront_wait_limit(int(tries))


def mad_debug_audit_error_bounds(on):
    """Test hook: re-evaluate every bounded stored entry in FP64 (records dq_ratio_max)."""
    library().mad_debug_audit_error_bounds(1 if on else 0)


def mad_set_graphs(on):
    """CUDA-graph replay of repeated profiles (default on)."""
    library().mad_set_graphs(1 if on else 0)


def mad_set_autotune(on):
    """Launch autotuner for small series (default on)."""
    library().mad_set_autotune(1 if on else 0)


def mad_last_error(ctx=None):
    return library().mad_last_error(ctx).decode()


def mad_destroy(ctx):
    if ctx is not None:
        library().mad_destroy(ctx)


def mad_debug_tc_tma(on):
    """Tensor-core path: column tiles built by the kernel's producer warps
    (0, default) or loaded by TMA from per-length shifted copies (1)."""
    library().mad_debug_tc_tma(1 if on else 0)
