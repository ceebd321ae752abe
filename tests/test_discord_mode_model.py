"""The decomposition the GPU uses for the discord mode's two passes
(Algorithm 10), checked on the CPU against the passes as printed, on many
random instances with ties, drops and trivial matches.

The GPU visits one at a time only the windows that can change dkm_l (a
distance above its column's last entry), logs every entry and exit, and
decides every other window in parallel from those logs: a non-valid row is
listed unless an offset that entered before it and had not left lies within
E; a listed row is recomputed ahead of the second pass if an upper value
beats its column's last entry after the first pass; the second pass really
needed a row iff no offset present at its visit lies within E and an upper
value beats the column minimum as it stood then. This model restates those
steps in Python and requires the same dkm_l and the same needed rows as the
literal passes."""
import numpy as np
import pytest

NEG = -np.inf


def insert(D, O, i, vals):
    """Algorithm 8 on a k x m table (D values, O offsets); returns
    (column, dropped offset) or (-1, -1)."""
    k, m = D.shape
    for j in range(m - 1, -1, -1):
        v = vals[j]
        if not np.isfinite(v):
            continue
        for r in range(k):
            if v > D[r, j]:
                dropped = O[k - 1, j]
                D[r + 1:, j] = D[r:-1, j].copy()
                O[r + 1:, j] = O[r:-1, j].copy()
                D[r, j], O[r, j] = v, i
                return j, dropped
    return -1, -1


def trivial(O, i, E):
    return any(o >= 0 and abs(i - o) <= E for o in O.ravel())


def literal(valid, ex, ub, k, m, E):
    n = len(valid)
    D, O = np.full((k, m), NEG), np.full((k, m), -1)
    listed = []
    for i in range(n):
        if trivial(O, i, E):
            continue
        if valid[i]:
            insert(D, O, i, ex[i])
        else:
            listed.append(i)
    needed = set()
    for i in listed:
        if trivial(O, i, E):
            continue
        for j in range(m - 1, -1, -1):
            if ub[i][j] > D[k - 1, j]:
                needed.add(i)
                insert(D, O, i, ex[i])
                break
    return D, O, needed


def decomposed(valid, ex, ub, k, m, E):
    n = len(valid)
    BIG = 1 << 40
    # first pass: only windows that can enter, one at a time; log entries / exits
    D, O = np.full((k, m), NEG), np.full((k, m), -1)
    ins1, drop1 = np.zeros(n, bool), np.full(n, BIG)
    for i in range(n):
        if not valid[i] or not any(np.isfinite(ex[i][j]) and ex[i][j] > D[k - 1, j] for j in range(m)):
            continue
        if trivial(O, i, E):
            continue
        j, dropped = insert(D, O, i, ex[i])
        if j >= 0:
            ins1[i], drop1[i] = True, BIG
            if dropped >= 0:
                drop1[dropped] = i
    O1, cmin1 = O.copy(), D[k - 1].copy()
    # listed / kept, in parallel from the log
    kept = np.zeros(n, bool)
    for i in range(n):
        if valid[i]:
            continue
        blocked = any(ins1[o] and drop1[o] > i for o in range(max(0, i - E), i))
        kept[i] = not blocked and any(ub[i][j] > cmin1[j] for j in range(m))
    # second pass over the kept rows with exact distances; log entries, exits, minima
    ins2, drop2 = np.zeros(n, bool), np.full(n, BIG)
    for o in O1.ravel():
        if o >= 0:
            drop2[o] = BIG
    events = []
    for i in range(n):
        if not kept[i] or not any(np.isfinite(ex[i][j]) and ex[i][j] > D[k - 1, j] for j in range(m)):
            continue
        if trivial(O, i, E):
            continue
        j, dropped = insert(D, O, i, ex[i])
        if j >= 0:
            ins2[i], drop2[i] = True, BIG
            if dropped >= 0:
                drop2[dropped] = i
            events.append((i, j, D[k - 1, j]))
    # which kept rows the second pass needed, in parallel from the logs
    needed = set()
    for i in np.nonzero(kept)[0]:
        blocked = any(o >= 0 and abs(i - o) <= E and drop2[o] > i for o in O1.ravel())
        blocked = blocked or any(ins2[o] and drop2[o] > i for o in range(max(0, i - E), i))
        if blocked:
            continue
        cm = cmin1.copy()
        for t, j, v in events:
            if t < i:
                cm[j] = v
        if any(ub[i][j] > cm[j] for j in range(m)):
            needed.add(int(i))
    return D, O, needed


@pytest.mark.parametrize("seed", range(200))
def test_decomposition_matches_the_passes(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(20, 220))
    k, m = int(rng.integers(1, 6)), int(rng.integers(1, 4))
    E = int(rng.integers(0, 6))
    valid = rng.random(n) < rng.uniform(0.1, 0.9)
    # coarse values so that ties occur; a few windows without an m-th match
    ex = np.round(rng.uniform(0, 4, (n, m)), 1)
    ex[rng.random((n, m)) < 0.03] = np.inf
    ex.sort(axis=1)
    ub = ex + np.where(valid[:, None], 0.0, np.round(rng.uniform(0, 2, (n, m)), 1))
    D1, O1, need1 = literal(valid, ex, ub, k, m, E)
    D2, O2, need2 = decomposed(valid, ex, ub, k, m, E)
    assert np.array_equal(O1, O2)
    assert np.array_equal(D1, D2)
    assert need1 == need2
