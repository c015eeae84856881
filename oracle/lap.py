"""Landmark affinity propagation, Algorithm 3 of Xia et al. (Section 4):
Steps 1 and 2 without the max_distance gate (``run``), Steps 1-4
(``run_full``) and Step 4's refinement (``refine``).

TEST INFRASTRUCTURE ONLY -- see ``oracle/__init__.py``.

Step 1: a sample M of landmarks (uniform random sampling by default, the
"simplest" choice named at the end of Section 4), S_M from Section 2 with the
off-diagonal median of S_M as preference, Algorithm 1 on S_M -> exemplars.
Step 2: every point joins the class of its nearest exemplar (squared
Euclidean distance, the negative of s; lowest exemplar index on ties);
exemplars keep themselves.  netsim over all N points: sum of s(i, c_i) over
non-exemplars plus the preference for each exemplar.
"""
from __future__ import annotations

import numpy as np

from . import ap, rng


def uniform_landmarks(n: int, count: int, seed: int) -> np.ndarray:
    """The ``count`` points with the smallest splitmix64 keys key(i) = output
    i+1 of ``seed`` (ties by index), returned in increasing point order."""
    keys = rng.outputs(seed, np.arange(1, n + 1, dtype=np.uint64))
    order = np.lexsort((np.arange(n), keys))
    return np.sort(order[:count]).astype(np.int64)


def nearest_exemplar(X, centres) -> np.ndarray:
    """Index (into ``centres``) of the closest centre for every row of X."""
    d = -ap.similarity(X, centres)
    return np.argmin(d, axis=1).astype(np.int64)


def run(X, landmarks, lam=0.5, max_iter=200, convits=15, pref="median"):
    """Returns dict(landmarks, S_L, pref, landmark_run, E (point indices of the
    exemplars), idx (length N), dpsim, expref, netsim)."""
    X = np.asarray(X)
    landmarks = np.asarray(landmarks, dtype=np.int64)
    S_L, p = ap.build_similarity(X[landmarks], pref=pref)
    res = ap.run(S_L, lam, max_iter, convits)
    ex = ap.exemplars(S_L, res["R"], res["A"])
    n = X.shape[0]
    if ex["E"].size == 0:
        return dict(landmarks=landmarks, S_L=S_L, pref=p, landmark_run=res,
                    E=ex["E"], idx=np.full(n, -1), dpsim=np.nan,
                    expref=np.nan, netsim=np.nan)
    E = landmarks[ex["E"]]
    near = nearest_exemplar(X, X[E])
    idx = E[near]
    idx[E] = E
    is_ex = np.zeros(n, dtype=bool)
    is_ex[E] = True
    s_ic = -((X[~is_ex].astype(np.float64) - X[idx[~is_ex]].astype(np.float64)) ** 2).sum(axis=1)
    dpsim = float(s_ic.sum())
    expref = float(p * E.size) if np.isscalar(p) else float(np.sum(p))
    return dict(landmarks=landmarks, S_L=S_L, pref=p, landmark_run=res, E=E,
                idx=idx, dpsim=dpsim, expref=expref, netsim=dpsim + expref)


# ---- Algorithm 3, Steps 1-4 ------------------------------------------------------------

def _rounded_points(X):
    """The bf16-rounded centred points on which the GPU takes its distance
    decisions (the level's own mean), as float64."""
    return ap.similarity_bf16_inputs(X)


def _sqdist(A, B):
    return ((A[:, None, :] - B[None, :, :]) ** 2).sum(axis=2)


def run_full(X, n_landmarks, seed, m0, lam=0.5, max_iter=200, convits=15, max_levels=8,
             refine_rounds=0):
    """Algorithm 3 Steps 1-4 (Section 4), literally:

    Step 1  uniform landmarks (``uniform_landmarks`` with the level's seed),
            Algorithm 1 on their S (preference: the off-diagonal median of the
            first level's landmark S, kept at every level) -> c classes.
    Step 2  max_distance(j) = the largest squared distance from a landmark of
            class j to its exemplar (from the landmark S); every other point i
            joins class j = its nearest exemplar when distance(i, c_j) <
            max_distance(j), else stays unassigned.
    Step 3  the m unassigned points: Algorithm 1 on them when m <= m0 (one
            point is its own exemplar), else Steps 1-3 on them recursively
            (seed + level); their exemplars join the set.
    Step 4  with refine_rounds > 0, the merged set is first refined by
            ``refine`` (a local search on net similarity); then every point
            is reassigned to its nearest exemplar of the set; exemplars keep
            themselves.

    Readings: distances are squared Euclidean (the negative of s); the nearest
    exemplar and the gate are decided on the bf16-rounded centred points of
    the level (the precision of the tensor-core assignment), lowest index on
    ties; max_distance comes from the landmark S.
    Returns dict(E, idx, levels (list of per-level dicts), pref, dpsim,
    expref, netsim)."""
    X = np.asarray(X, dtype=np.float32)
    n = X.shape[0]
    ids = np.arange(n)
    E_all = []
    levels = []
    p = None
    level = 0
    while True:
        Xl = X[ids]
        nl = Xl.shape[0]
        if level > 0 and nl <= m0:
            # Step 3 base case: Algorithm 1 on the remaining points
            if nl == 1:
                E_all.append(ids[:1])
                levels.append(dict(n=1, E=ids[:1], unassigned=np.zeros(0, dtype=np.int64)))
            else:
                S_m, _ = ap.build_similarity(Xl, pref=p)
                res = ap.run(S_m, lam, max_iter, convits)
                ex = ap.exemplars(S_m, res["R"], res["A"])
                E_all.append(ids[ex["E"]])
                levels.append(dict(n=nl, E=ids[ex["E"]], unassigned=np.zeros(0, dtype=np.int64)))
            break
        L = min(n_landmarks, nl)
        lm = uniform_landmarks(nl, L, seed + level)
        S_L, pl = ap.build_similarity(Xl[lm], pref="median" if p is None else p)
        if p is None:
            p = pl
        res = ap.run(S_L, lam, max_iter, convits)
        ex = ap.exemplars(S_L, res["R"], res["A"])
        if ex["E"].size == 0:
            levels.append(dict(n=nl, E=np.zeros(0, dtype=np.int64), unassigned=ids))
            break
        cls = ex["idx"]                                  # landmark position -> exemplar position
        Epos = ex["E"]
        slot = {int(e): j for j, e in enumerate(Epos)}
        maxd = np.zeros(Epos.size)
        for i in range(L):
            j = slot[int(cls[i])]
            maxd[j] = max(maxd[j], -S_L[i, cls[i]] if i != cls[i] else 0.0)
        Xr = _rounded_points(Xl)
        E_loc = lm[Epos]
        D = _sqdist(Xr, Xr[E_loc])
        near = np.argmin(D, axis=1)                      # first minimum: lowest exemplar position
        dmin = D[np.arange(nl), near]
        is_lm = np.zeros(nl, dtype=bool)
        is_lm[lm] = True
        ok = is_lm | (dmin < maxd[near])
        srt = np.sort(D, axis=1)
        gap = srt[:, 1] - srt[:, 0] if srt.shape[1] > 1 else np.full(nl, np.inf)
        margin = np.abs(dmin - maxd[near])
        E_all.append(ids[E_loc])
        un = ids[~ok]
        levels.append(dict(n=nl, L=L, E=ids[E_loc], maxd=maxd, unassigned=un,
                           margin=margin[~is_lm], gap=gap[~is_lm], scale=maxd.max() if maxd.size else 0.0))
        if un.size == 0 or level + 1 >= max_levels:
            break
        ids = un
        level += 1
    E = np.unique(np.concatenate(E_all)) if E_all else np.zeros(0, dtype=np.int64)
    if E.size == 0:
        return dict(E=E, idx=np.full(n, -1), levels=levels, pref=p, dpsim=np.nan,
                    expref=np.nan, netsim=np.nan)
    refine_history = []
    if refine_rounds > 0:
        E, refine_history = refine(X, E, p, refine_rounds)
    # Step 4: nearest exemplar of the merged set, on the whole set's rounded points
    Xr = _rounded_points(X)
    D = _sqdist(Xr, Xr[E])
    idx = E[np.argmin(D, axis=1)]
    idx[E] = E
    srt = np.sort(D, axis=1)
    gap4 = srt[:, 1] - srt[:, 0] if srt.shape[1] > 1 else np.full(n, np.inf)
    is_ex = np.zeros(n, dtype=bool)
    is_ex[E] = True
    s_ic = -((X[~is_ex].astype(np.float64) - X[idx[~is_ex]].astype(np.float64)) ** 2).sum(axis=1)
    dpsim = float(s_ic.sum())
    expref = float(p * E.size)
    return dict(E=E, idx=idx, levels=levels, pref=p, gap=gap4, dpsim=dpsim, expref=expref,
                netsim=dpsim + expref, refine=refine_history)


# ---- Algorithm 3 Step 4: refinement of the merged centres ------------------------------

def _top2(D):
    """Nearest and second-nearest column of every row of the distance matrix
    D (lowest column on ties), and those distances; the second is -1 / inf
    when D has one column."""
    n, c = D.shape
    j1 = np.argmin(D, axis=1)
    d1 = D[np.arange(n), j1]
    if c == 1:
        return j1, d1, np.full(n, -1), np.full(n, np.inf)
    D2 = D.copy()
    D2[np.arange(n), j1] = np.inf
    j2 = np.argmin(D2, axis=1)
    return j1, d1, j2, D2[np.arange(n), j2]


def netsim_rounded(X, E, pref):
    """Net similarity of the centre set E (every point at its nearest centre,
    centres at themselves) measured on the bf16-rounded centred points: the
    quantity the refinement's decisions are taken on."""
    Xr = _rounded_points(X)
    E = np.asarray(E, dtype=np.int64)
    D = _sqdist(Xr, Xr[E])
    d = D.min(axis=1)
    d[E] = 0.0
    return float(-d.sum() + pref * E.size)


def refine(X, E, pref, max_rounds=8):
    """Step 4 (the merged centres and their classes are to be refined, with
    the similarities recomputed; the paper gives no procedure), read as a
    local search on the net similarity of Section 2 (netsim = -E(c): the summed similarity
    of every point to its centre plus the preference p < 0 of every centre).
    One round:
      1. every point joins its nearest centre j1 (second nearest: j2), on
         the bf16-rounded centred points;
      2. removal: the cost of dropping centre e is what its class would lose
         by moving to the second choices, delta(e) = sum over the points of
         class e of d(i, j2) - d(i, j1); e is a candidate when delta(e) < -p
         (dropping it raises netsim).  Two candidates conflict when a point
         has one as j1 and the other as j2; of a conflicting pair only the
         one of smaller (delta, index) may go, so the dropped centres form an
         independent set and every member of a dropped class moves to a
         centre that stays.  Candidates no conflict blocks are dropped;
      3. every class (after the moves of 2) moves its centre to the member
         nearest the class mean: sum_i |x_i - x_k|^2 over the class equals
         n |x_k - mean|^2 plus a constant, so that member minimises the
         class's summed squared distance (unrounded points, float64; lowest
         index on ties).
    Rounds repeat until one changes nothing, or max_rounds have run.
    Returns (E sorted, list of per-round dicts: removed, moved, netsim of the
    round's input set on the rounded points, medoid_gap: the smallest
    relative margin by which a class's medoid beat its runner-up)."""
    X = np.asarray(X, dtype=np.float32)
    X64 = X.astype(np.float64)
    Xr = _rounded_points(X)
    E = np.unique(np.asarray(E, dtype=np.int64))
    history = []
    for _ in range(max_rounds):
        D = _sqdist(Xr, Xr[E])
        j1, d1, j2, d2 = _top2(D)
        c = E.size
        delta = np.zeros(c)
        np.add.at(delta, j1, d2 - d1)                   # inf when there is no second centre
        cand = delta < -pref
        key = list(zip(delta.tolist(), E.tolist()))
        blocked = np.zeros(c, dtype=bool)
        both = (j2 >= 0)
        for a, b in zip(j1[both], j2[both]):
            if cand[a] and cand[b]:
                blocked[max(a, b, key=lambda t: key[t])] = True
        removed = cand & ~blocked
        cls = np.where(removed[j1], j2, j1)              # class position of every point
        newE = []
        moved = 0
        gap = np.inf                                     # how clear the medoid choices were
        for j in np.nonzero(~removed)[0]:
            members = np.nonzero(cls == j)[0]
            if members.size == 0:
                continue                                 # a class left empty drops its centre
            mu = X64[members].mean(axis=0)
            dm = ((X64[members] - mu) ** 2).sum(axis=1)
            k = int(members[np.argmin(dm)])             # first minimum: lowest point index
            if members.size > 1:
                s2 = np.partition(dm, 1)[:2]
                gap = min(gap, float(s2[1] - s2[0]) / max(1.0, float(s2[1])))
            moved += int(k != E[j])
            newE.append(k)
        is_c = np.zeros(X.shape[0], dtype=bool)
        is_c[E] = True
        history.append(dict(removed=int(removed.sum()), moved=moved,
                            netsim=float(-d1[~is_c].sum() + pref * c), medoid_gap=gap))
        newE = np.unique(np.asarray(newE, dtype=np.int64))
        if removed.sum() == 0 and moved == 0:
            break
        E = newE
    return E, history
