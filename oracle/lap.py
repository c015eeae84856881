"""Landmark affinity propagation, Algorithm 3 of Xia et al. (Section 4),
Steps 1 and 2 without the max_distance gate.

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
