"""Pins for the oracle's discord read-outs (no GPU).

1. The per-length Top-k m-th discord greedy (``orc_discords_one_length``,
   Def. "Top-k m-th discord"): checked by properties that any other greedy
   would break -- the visiting order (score descending, equal scores to the
   smaller offset), pairwise non-triviality of the picks, and maximality (a
   window that was visited before the last pick, or any window when fewer
   than k were picked, is either picked or within E of a pick accepted
   before it). A greedy that rejected windows near any higher *candidate*
   instead of near an *accepted* pick fails maximality.

2. The discord mode (``orc_valmod_discord``, Algorithm 7 driving
   Algorithm 10): restated here in Python from the paper -- numpy distance
   matrices, each row's p stored entries (largest correlations at the row's
   base length, Eq. LB bound from the p-th), the validity test at every
   longer length, Algorithm 10's first pass in offset order and its second
   pass over the non-valid list (for j = m down to 1, the first stored j-th
   distance above column j's k-th entry triggers the full profile), with
   Algorithm 8's insert. It shares nothing with the C code but the seeded
   inputs, and must give the same dkm_l at every length, the same counts and
   the same set of recomputed rows.
"""
import math

import numpy as np
import pytest

import oracle
import workloads
from test_discord_mode_model import insert, trivial


# ------------------------------------------------ per-length greedy pins

def _order_key(score, i):
    return (-score, i)


@pytest.mark.parametrize("seed", range(40))
def test_discords_one_length_order_maximality_ties(seed):
    rng = np.random.default_rng(1000 + seed)
    nl = int(rng.integers(5, 400))
    l = int(rng.integers(2, 40))
    num, den = [(1, 4), (1, 2), (0, 1), (3, 4)][seed % 4]
    k = int(rng.integers(1, 12))
    # coarse values: many exact ties; a few windows without a score
    score = np.round(rng.uniform(0, 3, nl), 1)
    score[rng.random(nl) < 0.05] = np.inf
    score[rng.random(nl) < 0.05] = np.nan
    nbr = rng.integers(0, nl, nl)
    picks = oracle.discords_one_length(score, l, k, nbr, num, den)
    E = oracle.excl(l, num, den)
    assert len(picks) <= k
    # visiting order: (score desc, offset asc), strictly
    keys = [_order_key(s, o) for o, s, _ in picks]
    assert keys == sorted(keys) and len(set(keys)) == len(keys)
    for o, s, nn in picks:
        assert np.isfinite(score[o]) and s == score[o] and nn == nbr[o]
    offs = [o for o, _, _ in picks]
    for a in range(len(offs)):
        for b in range(a):
            assert abs(offs[a] - offs[b]) > E
    # maximality
    last = keys[-1] if len(picks) == k else None
    picked = set(offs)
    for i in range(nl):
        if not np.isfinite(score[i]) or i in picked:
            continue
        ki = _order_key(score[i], i)
        if last is not None and ki > last:
            continue
        assert any(abs(i - o) <= E and kk < ki for o, kk in zip(offs, keys)), (i, score[i], picks)


def test_discords_one_length_tie_goes_to_smaller_offset():
    # two equal scores far apart: both picked, the smaller offset first;
    # two equal scores within E: only the smaller offset
    score = np.zeros(100)
    score[70] = score[20] = 5.0
    score[40] = score[44] = 4.0
    picks = oracle.discords_one_length(score, 8, 3, None, 1, 2)   # E = 4
    assert [p[0] for p in picks[:3]] == [20, 70, 40]


# -------------------------------------- discord mode, Python restatement

def _profiles(x, l):
    """Correlation and distance matrices at length l (population std);
    the inputs used here have no flat window."""
    W = np.lib.stride_tricks.sliding_window_view(np.asarray(x, float), l)
    Wc = W - W.mean(1, keepdims=True)
    sd = np.sqrt((Wc ** 2).mean(1))
    assert np.all(sd > 0)
    Q = np.clip((Wc @ Wc.T) / (l * sd[:, None] * sd[None, :]), -1.0, 1.0)
    Q = 0.5 * (Q + Q.T)     # d(i, j) = d(j, i) exactly, as the definition has it (mutual pairs tie)
    D = np.sqrt(2.0 * l * (1.0 - Q))
    return Q, D, sd


def py_valmod_discord(x, lmin, lmax, p, k, m, num=1, den=4):
    n = len(x)
    n0 = n - lmin + 1
    state = [None] * n0        # (stored partners, base length, sigma at base, bound base)
    tables, stats, recomp = [], [], np.zeros((lmax - lmin + 1, n0), bool)

    def full_profile(i, l, Q, D, sd):
        E = oracle.excl(l, num, den)
        nl = n - l + 1
        cand = [j for j in range(nl) if abs(i - j) > E]
        by_d = sorted(cand, key=lambda j: (D[i, j], j))
        exact = [D[i, by_d[t]] if t < len(by_d) else np.inf for t in range(m)]
        by_q = sorted(cand, key=lambda j: (-Q[i, j], j))
        if len(cand) <= p:
            bb = np.inf
        else:
            qp = max(Q[i, by_q[p - 1]], 0.0)
            bb = math.sqrt(l * (1.0 - qp * qp))
        state[i] = (by_q[:p], l, sd[i], bb)
        return exact

    for li, l in enumerate(range(lmin, lmax + 1)):
        Q, D, sd = _profiles(x, l)
        nl = n - l + 1
        E = oracle.excl(l, num, den)
        Dk, Ok = np.full((k, m), -np.inf), np.full((k, m), -1)
        if l == lmin:
            ex = [full_profile(i, l, Q, D, sd) for i in range(nl)]
            recomp[li, :nl] = True
            for i in range(nl):
                if not trivial(Ok, i, E):
                    insert(Dk, Ok, i, ex[i])
            stats.append((nl, 0, 0, nl))
        else:
            # stored entries at l: exact distances of the live ones, sorted;
            # valid iff the m-th is below the bound (Eq. LB, Sec. 4.2)
            s, valid = [], []
            for i in range(nl):
                part, lb, sgb, bb = state[i]
                live = sorted((D[i, j], j) for j in part if j < nl and abs(i - j) > E)
                sv = [live[t][0] if t < len(live) else np.inf for t in range(m)]
                s.append(sv)
                valid.append(len(live) >= m and sv[m - 1] < bb * sgb / sd[i])
            # Algorithm 10, first pass in offset order
            listed, nvalid = [], 0
            for i in range(nl):
                if trivial(Ok, i, E):
                    continue
                if valid[i]:
                    nvalid += 1
                    insert(Dk, Ok, i, s[i])
                else:
                    listed.append(i)
            # second pass over the list
            nre = 0
            for i in listed:
                if trivial(Ok, i, E):
                    continue
                for j in range(m - 1, -1, -1):
                    if s[i][j] > Dk[k - 1, j]:
                        ex = full_profile(i, l, Q, D, sd)
                        recomp[li, i] = True
                        nre += 1
                        insert(Dk, Ok, i, ex)
                        break
            stats.append((nl, nvalid, len(listed), nre))
        tables.append((Ok.copy(), Dk.copy()))
    return tables, np.array(stats), recomp


CASES = [
    ("ar2", 420, 201, 16, 24, 4, 3, 2),
    ("ar2", 360, 202, 12, 19, 5, 4, 3),
    ("rw", 380, 203, 14, 20, 3, 3, 2),
    ("ecg", 520, 204, 20, 27, 6, 4, 2),
    ("spike", 480, 205, 18, 25, 4, 3, 3),
]


@pytest.mark.parametrize("case", CASES, ids=[c[0] + str(c[2]) for c in CASES])
def test_discord_mode_matches_restatement(case):
    kind, n, seed, lmin, lmax, p, k, m = case
    if kind == "ar2":
        x = workloads.ar2(n, seed)
    elif kind == "rw":
        x = workloads.random_walk(n, seed)
    elif kind == "ecg":
        x = workloads.ecg_like(n, seed, period=40.0)
    else:
        rng = np.random.default_rng(seed)
        t = np.arange(n)
        x = np.sin(2 * np.pi * t / 30) + 0.05 * rng.standard_normal(n)
        x[n // 2] += 3.0
    g = oracle.valmod_discord(x, lmin, lmax, p, k, m)
    tables, st, rc = py_valmod_discord(x, lmin, lmax, p, k, m)
    for li in range(lmax - lmin + 1):
        Ok, Dk = tables[li]
        assert np.array_equal(g["dkm_off"][li], Ok), (li, g["dkm_off"][li], Ok)
        fin = Ok >= 0
        np.testing.assert_allclose(g["dkm_d"][li][fin], Dk[fin], rtol=1e-9, atol=1e-12)
    assert np.array_equal(g["stats"], st), (g["stats"], st)
    assert np.array_equal(g["recomp"], rc)


def test_discord_mode_restatement_exercises_the_second_pass():
    # the cases above list non-valid rows and recompute only some of them
    listed = recomputed = 0
    for kind, n, seed, lmin, lmax, p, k, m in CASES[:2]:
        x = workloads.ar2(n, seed)
        _, st, _ = py_valmod_discord(x, lmin, lmax, p, k, m)
        listed += st[1:, 2].sum()
        recomputed += st[1:, 3].sum()
    assert listed > recomputed > 0
