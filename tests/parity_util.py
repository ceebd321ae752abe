"""Helpers that compare the CUDA path with the CPU oracle."""
import math

import numpy as np

import oracle
import paper_2008_13447_gb300 as mad


# FP64 correlation rounding floor: d^2 = 2 l (1 - q), so an error dq in q
# moves d^2 by 2 l dq whatever d is; near d = 0 that dominates 1e-9 * d.
DQ64 = 1e-12


def tol_for(prec, l, d_ref):
    """Distance tolerance. FP64: 1e-9 relative, with the floor that a 1e-12
    error of the correlation puts on d (|d1^2 - d2^2| <= 2 l dq, i.e.
    |d1 - d2| <= 2 l dq / (d1 + d2) <= sqrt(2 l dq)). FP32: 1e-4 sqrt(l)
    absolute."""
    d = np.abs(np.asarray(d_ref, dtype=float))
    if prec == mad.MAD_FP64:
        floor = 2 * l * DQ64 / np.maximum(2 * d, math.sqrt(2 * l * DQ64))
        return 1e-9 * d + floor
    return 1e-4 * math.sqrt(l) + 0.0 * d


def check_index_choice(x, l, i, j_gpu, d_ref, tol, num, den):
    """An index that differs from the oracle's must be a valid, non-trivial
    partner whose oracle distance ties the oracle's value within tol."""
    E = oracle.excl(l, num, den)
    assert abs(int(j_gpu) - int(i)) > E, (l, i, j_gpu)
    assert 0 <= j_gpu < len(x) - l + 1
    d = oracle.dist(x, l, int(i), int(j_gpu))
    assert abs(d - d_ref) <= tol + 1e-12, (l, i, j_gpu, d, d_ref)


def run_gpu(x, lmin, lmax, p, prec, m_max=1, k_max=5, excl=(1, 4), band_form=0):
    ctx = mad.mad_create(x, precision=prec, k_max=k_max, m_max=m_max, excl=excl, keep_profiles=True,
                         band_form=band_form)
    try:
        mad.mad_profile(ctx, lmin, lmax, p)
        n = len(x)
        prof = {l: mad.mad_matrix_profile(ctx, 0, l, n, m_max) for l in range(lmin, lmax + 1)}
        vm = mad.mad_valmp(ctx, 0, n - lmin + 1)
        mot = mad.mad_motifs(ctx, 0, k_max)
        dis = mad.mad_discords(ctx, 0, k_max, m_max)
        st = mad.mad_stats(ctx, 0)
    finally:
        mad.mad_destroy(ctx)
    return prof, vm, mot, dis, st


def compare_all(x, lmin, lmax, p, prec, m_max=1, k_max=5, excl=(1, 4), band_form=0):
    num, den = excl
    ref = oracle.valmp_plain(x, lmin, lmax, m_max=m_max, num=num, den=den, keep_nn=True)
    prof, vm, mot, dis, st = run_gpu(x, lmin, lmax, p, prec, m_max, k_max, excl, band_form)
    n = len(x)
    n0 = n - lmin + 1
    worst = 0.0
    idx_mismatch = 0
    for l in range(lmin, lmax + 1):
        nl = n - l + 1
        mp, ip, nnd, nnj = prof[l]
        rd = ref["nnd"][l - lmin, :nl, :]
        rj = ref["nnj"][l - lmin, :nl, :]
        tol = tol_for(prec, l, rd)
        err = np.abs(nnd - rd)
        assert np.all(np.isfinite(nnd)), l
        bad = err > tol
        assert not bad.any(), (l, np.argwhere(bad)[:5], nnd[bad][:5], rd[bad][:5])
        worst = max(worst, float((err / (tol if np.ndim(tol) else tol)).max()))
        np.testing.assert_array_equal(mp, nnd[:, 0])
        for m in range(m_max):
            diff = np.nonzero(nnj[:, m] != rj[:, m])[0]
            idx_mismatch += len(diff)
            for i in diff:
                t = tol if np.ndim(tol) == 0 else tol[i, m]
                check_index_choice(x, l, i, nnj[i, m], rd[i, m], t, num, den)
    # VALMP
    # normalised distance d / sqrt(l): tolerance divided by sqrt(l)
    tn = 1e-4 if prec == mad.MAD_FP32 else tol_for(prec, lmax, ref["norm"] * math.sqrt(lmin)) / math.sqrt(lmin)
    assert np.all(np.abs(vm["norm"] - ref["norm"]) <= tn), np.max(np.abs(vm["norm"] - ref["norm"]))
    same = vm["len"] == ref["len"]
    tolv = tol_for(prec, lmax, ref["dist"])
    tolv = tolv[same] if np.ndim(tolv) else tolv
    assert np.all(np.abs(vm["dist"][same] - ref["dist"][same]) <= tolv)
    # a different length is only allowed on a near-tie of normalised distances,
    # and the reported distance must be that length's distance
    for i in np.nonzero(~same)[0]:
        L = int(vm["len"][i])
        assert lmin <= L <= lmax
        d = oracle.dist(x, L, i, int(vm["nn"][i]))
        assert abs(d - vm["dist"][i]) <= tol_for(prec, L, d) + 1e-12
    # stats invariants
    for s in st:
        assert s["certified"] + s["recomputed"] == s["rows"], s
    assert st[0]["recomputed"] == st[0]["rows"]
    # motifs from the oracle's VALMP: the same pairs (a, b, len) rank by rank
    rm = oracle.topk_motifs(ref, k_max, num, den)
    assert len(mot) == len(rm)
    flips = []
    flipped = False
    for rank, (g, r) in enumerate(zip(mot, rm)):
        tn = 1e-4 if prec == mad.MAD_FP32 else float(tol_for(prec, r[2], r[3])) / math.sqrt(r[2]) + 1e-15
        assert abs(g["dist"] - g["dist_recheck"]) <= float(tol_for(prec, g["len"], g["dist_recheck"]))
        if (g["a"], g["b"], g["len"]) == tuple(r[:3]):
            assert abs(g["norm_dist"] - r[4]) <= tn, (g, r)
            continue
        if abs(g["norm_dist"] - r[4]) <= tn:
            # the oracle's competing pair ties within tolerance
            flips.append(("motif", rank + 1, (g["a"], g["b"], g["len"]), tuple(r[:3]), g["norm_dist"] - r[4]))
            flipped = True
            continue
        # after an earlier near-tie the greedy may take other pairs; each is
        # still a VALMP entry of the oracle within tolerance
        assert flipped, ("motif pick differs without a near-tie", rank + 1, g, r)
        assert any(abs(ref["norm"][i] - g["norm_dist"]) <= tn for i in (g["a"], g["b"]) if i < n0), (g, r)
        flips.append(("motif-after-tie", rank + 1, (g["a"], g["b"], g["len"]), tuple(r[:3]), g["norm_dist"] - r[4]))
    # discords: the same cell (off, len) of dkm_{lmin,lmax}, cell by cell
    rdk = oracle.discords(n, lmin, lmax, k_max, m_max, ref["nnd"], ref["nnj"], num, den)
    col_flipped = set()
    for c in sorted(dis, key=lambda c: (c["m"], c["rank"])):
        r, m = c["rank"] - 1, c["m"] - 1
        if rdk["len"][r, m] == 0:
            assert c["len"] == 0
            continue
        t = 1e-4 if prec == mad.MAD_FP32 else float(tol_for(prec, c["len"], rdk["dist"][r, m])) / math.sqrt(c["len"]) + 1e-15
        assert abs(c["dist"] - c["dist_recheck"]) <= float(tol_for(prec, c["len"], c["dist_recheck"]))
        if (c["off"], c["len"]) == (int(rdk["off"][r, m]), int(rdk["len"][r, m])):
            assert abs(c["norm_dist"] - rdk["norm"][r, m]) <= t, (c, rdk["norm"][r, m])
            continue
        if abs(c["norm_dist"] - rdk["norm"][r, m]) <= t:
            flips.append(("discord", c["rank"], c["m"], (c["off"], c["len"]),
                          (int(rdk["off"][r, m]), int(rdk["len"][r, m])), c["norm_dist"] - rdk["norm"][r, m]))
            col_flipped.add(m)
            continue
        assert m in col_flipped, ("discord cell differs without a near-tie", c, rdk["off"][r, m], rdk["len"][r, m])
        # the cell still holds that window's m-th best-match distance
        L = c["len"]
        assert abs(ref["nnd"][L - lmin, c["off"], m] - c["dist"]) <= float(tol_for(prec, L, c["dist"])), c
        flips.append(("discord-after-tie", c["rank"], c["m"], (c["off"], c["len"]),
                      (int(rdk["off"][r, m]), int(rdk["len"][r, m])), c["norm_dist"] - rdk["norm"][r, m]))
    for f in flips:
        print("near-tie pick:", f)
    return dict(worst=worst, idx_mismatch=idx_mismatch, stats=st, motifs=mot, ref_motifs=rm, flips=flips)
