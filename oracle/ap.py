"""Affinity propagation, Algorithm 1 of Xia et al. (Section 2), in float64.

TEST INFRASTRUCTURE ONLY -- see ``oracle/__init__.py``.

Notation follows the paper: ``S`` holds s(i,k) with the preferences p(k) on
its diagonal, ``R`` the responsibilities r(i,k), ``A`` the availabilities
a(i,k), ``lam`` the damping factor lambda.

Two statements of one iteration are given:

* ``responsibility_literal`` / ``availability_literal`` -- Eq. 2, 3 and 4 typed
  as written: for every (i,k) a max over k' != k and a sum over i' not in {i,k}.
  O(N^3); for N up to a few dozen.
* ``responsibility`` / ``availability`` -- the same values computed from each
  row's two largest a+s entries and each column's sum of positive
  responsibilities; O(N^2).  The max over k' != k equals the row maximum
  unless k is the (first) arg-max, where it equals the second largest value
  (equal to the maximum on a tie); the sum over i' not in {i,k} equals the
  column sum over i' != k minus the i-th term.

Readings of points the paper leaves open:
  * R starts at zero, like A (Eq. 1 names only A).
  * Damping (Section 2): a message's new value is lambda times its old one
    plus 1-lambda times its update; R is damped first, A is then computed
    from the damped R and damped.
  * Decisions: point i's choice is the lowest k maximising a(i,k)+r(i,k);
    the exemplar set is E = {k : choice(k) == k}.
  * Termination (Step 4): stop once E has been the same, and non-empty, for
    ``convits`` consecutive iterations, or after ``max_iter`` iterations.
  * Outputs: exemplars keep idx(k)=k; every other point takes the exemplar of
    highest similarity (lowest index on ties).  dpsim sums s(i,idx(i)) over
    non-exemplars, expref sums p(k) over exemplars, netsim = dpsim + expref,
    which is -E(c) of the energy in Section 2 with s(k,k) = p(k).
"""
from __future__ import annotations

import numpy as np

from . import rng


# ----------------------------------------------------------------------------
# Similarity and preference (Section 2: s(i,k) = -||x_i - x_k||^2)
# ----------------------------------------------------------------------------

def similarity(X: np.ndarray, Y: np.ndarray | None = None) -> np.ndarray:
    """s(i,k) = -sum_j (x_ij - y_kj)^2 in float64, by explicit differences."""
    X = np.asarray(X, dtype=np.float64)
    Y = X if Y is None else np.asarray(Y, dtype=np.float64)
    S = np.empty((X.shape[0], Y.shape[0]), dtype=np.float64)
    step = max(1, (1 << 22) // max(1, Y.shape[0] * X.shape[1]))
    for lo in range(0, X.shape[0], step):
        D = X[lo:lo + step, None, :] - Y[None, :, :]
        S[lo:lo + step] = -np.einsum("ikj,ikj->ik", D, D)
    return S


def similarity_gram(X) -> np.ndarray:
    """Section 2's s(i,k) = -||x_i - x_k||^2 in float64, expanded as
    2 x_i.x_k - |x_i|^2 - |x_k|^2 (one matrix product), for inputs too large
    for the explicit differences of ``similarity``.  The diagonal is 0 and
    every entry is clamped to <= 0, as the definition guarantees; it agrees
    with ``similarity`` to rounding (pinned)."""
    X = np.asarray(X, dtype=np.float64)
    nrm = np.einsum("ij,ij->i", X, X)
    S = X @ X.T
    S *= 2.0
    S -= nrm[:, None]
    S -= nrm[None, :]
    np.minimum(S, 0.0, out=S)
    np.fill_diagonal(S, 0.0)
    return S


def round_bf16(x) -> np.ndarray:
    """float32 -> nearest bfloat16 (ties to even), returned as float32: keep
    the top 16 bits after adding 0x7FFF plus the lowest kept bit."""
    u = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)


def centred(X, dtype=np.float32):
    """X minus its column mean (mean in float64, rounded to float32; the
    subtraction in float32), the translation the similarity paths apply
    before their GEMM; distances are unchanged by it."""
    X = np.asarray(X, dtype=np.float32)
    mean = X.astype(np.float64).mean(axis=0).astype(np.float32)
    return (X - mean).astype(dtype)


def similarity_bf16_inputs(X) -> np.ndarray:
    """The points whose exact negative squared distances the bf16 path
    computes: the centred features rounded to bfloat16 (as float64)."""
    return round_bf16(centred(X)).astype(np.float64)


def offdiag_median(S: np.ndarray) -> float:
    """Median of the N(N-1) off-diagonal entries: the middle order statistic,
    or the mean of the two middle ones when the count is even."""
    n = S.shape[0]
    vals = np.sort(S[~np.eye(n, dtype=bool)].astype(np.float64), kind="stable")
    m = vals.size
    if m == 0:
        raise ValueError("need at least two points")
    if m % 2 == 1:
        return float(vals[m // 2])
    return float(0.5 * (vals[m // 2 - 1] + vals[m // 2]))


def offdiag_median_select(S: np.ndarray) -> float:
    """``offdiag_median`` by selection (np.partition) instead of a full sort:
    the same order statistics of the N(N-1) off-diagonal entries, for large
    N (pinned against ``offdiag_median``)."""
    n = S.shape[0]
    vals = S[~np.eye(n, dtype=bool)].astype(np.float64)
    m = vals.size
    if m == 0:
        raise ValueError("need at least two points")
    if m % 2 == 1:
        return float(np.partition(vals, m // 2)[m // 2])
    lo = m // 2 - 1
    part = np.partition(vals, [lo, lo + 1])
    return float(0.5 * (part[lo] + part[lo + 1]))


def tiebreak_noise(n_rows: int, n_cols: int, seed: int) -> np.ndarray:
    """u(i,k) in [0,1): splitmix64 output number i*n_cols + k + 1 of ``seed``."""
    ctr = np.arange(1, n_rows * n_cols + 1, dtype=np.uint64)
    return rng.unit_interval(seed, ctr).reshape(n_rows, n_cols)


def set_preference(S: np.ndarray, pref) -> np.ndarray:
    """Write p(k) on the diagonal (scalar or per-point vector)."""
    S = S.copy()
    np.fill_diagonal(S, pref)
    return S


def build_similarity(X, pref="median", noise_rel=0.0, seed=0):
    """Full input of Algorithm 1 from features: S from Section 2, diagonal =
    preference (the off-diagonal median by default), then the tie-break noise
    s <- s + noise_rel*|s|*u(i,k) on every entry.  Returns (S, p)."""
    S = similarity(X)
    p = offdiag_median(S) if isinstance(pref, str) else pref
    S = set_preference(S, p)
    if noise_rel:
        S = S + noise_rel * np.abs(S) * tiebreak_noise(S.shape[0], S.shape[1], seed)
    return S, p


# ----------------------------------------------------------------------------
# One iteration, literal form (Eq. 2, 3, 4)
# ----------------------------------------------------------------------------

def responsibility_literal(S: np.ndarray, A: np.ndarray) -> np.ndarray:
    """Eq. 2: r(i,k) = s(i,k) - max_{k' != k} (a(i,k') + s(i,k'))."""
    n = S.shape[0]
    R = np.empty_like(S, dtype=np.float64)
    for i in range(n):
        for k in range(n):
            best = -np.inf
            for kp in range(n):
                if kp != k:
                    best = max(best, A[i, kp] + S[i, kp])
            R[i, k] = S[i, k] - best
    return R


def availability_literal(R: np.ndarray) -> np.ndarray:
    """Eq. 3 for i != k and Eq. 4 for i == k."""
    n = R.shape[0]
    A = np.empty_like(R, dtype=np.float64)
    for i in range(n):
        for k in range(n):
            if i == k:
                A[k, k] = sum(max(0.0, R[ip, k]) for ip in range(n) if ip != k)
            else:
                tot = R[k, k] + sum(max(0.0, R[ip, k]) for ip in range(n)
                                    if ip != i and ip != k)
                A[i, k] = min(0.0, tot)
    return A


# ----------------------------------------------------------------------------
# One iteration, row top-2 / column-sum form
# ----------------------------------------------------------------------------

def row_top2(M: np.ndarray):
    """Per row: largest value m1, its lowest index j1, largest value over the
    other indices m2 (equal to m1 when the maximum is tied)."""
    n = M.shape[0]
    j1 = np.argmax(M, axis=1)
    m1 = M[np.arange(n), j1]
    M2 = M.copy()
    M2[np.arange(n), j1] = -np.inf
    m2 = M2.max(axis=1)
    return m1, j1, m2


def responsibility(S: np.ndarray, A: np.ndarray) -> np.ndarray:
    """Eq. 2 via the row top-2 of a+s."""
    n = S.shape[0]
    m1, j1, m2 = row_top2(A + S)
    R = S - m1[:, None]
    R[np.arange(n), j1] = S[np.arange(n), j1] - m2
    return R


def column_sums(R: np.ndarray):
    """colp(k) = sum_{i != k} max(0, r(i,k)) and the diagonal r(k,k)."""
    P = np.maximum(R, 0.0)
    np.fill_diagonal(P, 0.0)
    return P.sum(axis=0), np.diag(R).copy()


def availability(R: np.ndarray) -> np.ndarray:
    """Eq. 3 (i != k) and Eq. 4 (i == k) via the column sums."""
    colp, rkk = column_sums(R)
    P = np.maximum(R, 0.0)
    A = np.minimum(0.0, rkk[None, :] + colp[None, :] - P)
    np.fill_diagonal(A, colp)
    return A


def iterate_once(S, R, A, lam, literal=False):
    """One damped iteration: R first (Eq. 2), then A from the new R (Eq. 3-4)."""
    rho = responsibility_literal if literal else responsibility
    alpha = availability_literal if literal else availability
    R = lam * R + (1.0 - lam) * rho(S, A)
    A = lam * A + (1.0 - lam) * alpha(R)
    return R, A


def decisions(R: np.ndarray, A: np.ndarray, dtype=np.float64) -> np.ndarray:
    """choice(i) = lowest k maximising a(i,k) + r(i,k).

    ``dtype`` is the precision in which a+r is formed before the arg-max; a
    comparison against a float32 implementation takes the decision in
    float32 on both sides."""
    T = np.asarray(A, dtype=dtype) + np.asarray(R, dtype=dtype)
    return np.argmax(T, axis=1).astype(np.int64)


def exemplar_mask(R, A, dtype=np.float64) -> np.ndarray:
    n = R.shape[0]
    return decisions(R, A, dtype) == np.arange(n)


def run(S, lam=0.5, max_iter=200, convits=15, R0=None, A0=None,
        literal=False, fixed_iters=None):
    """Algorithm 1 from (R0, A0) (zeros by default).

    With ``fixed_iters`` the loop runs exactly that many iterations (no
    convergence test).  Otherwise it stops at the first iteration t at which
    the exemplar set is non-empty and has not changed over the last
    ``convits`` iterations, or at ``max_iter``.
    Returns dict(R, A, iters, converged)."""
    S = np.asarray(S, dtype=np.float64)
    n = S.shape[0]
    R = np.zeros((n, n)) if R0 is None else np.array(R0, dtype=np.float64)
    A = np.zeros((n, n)) if A0 is None else np.array(A0, dtype=np.float64)
    if fixed_iters is not None:
        for _ in range(fixed_iters):
            R, A = iterate_once(S, R, A, lam, literal)
        return dict(R=R, A=A, iters=fixed_iters, converged=False)
    prev = None
    stable = 0
    t = 0
    converged = False
    while t < max_iter:
        t += 1
        R, A = iterate_once(S, R, A, lam, literal)
        E = exemplar_mask(R, A)
        stable = stable + 1 if (prev is not None and np.array_equal(E, prev)) else 1
        prev = E
        if stable >= convits and E.any():
            converged = True
            break
    return dict(R=R, A=A, iters=t, converged=converged)


def exemplars(S, R, A, dtype=np.float64):
    """Outputs of Algorithm 1: idx(j), dpsim, expref, netsim.

    Returns dict(idx int64[N] (-1 everywhere if there is no exemplar),
    E (sorted exemplar indices), dpsim, expref, netsim).  ``dtype`` as in
    ``decisions``."""
    S = np.asarray(S, dtype=np.float64)
    n = S.shape[0]
    E = np.nonzero(exemplar_mask(R, A, dtype))[0]
    if E.size == 0:
        return dict(idx=np.full(n, -1, dtype=np.int64), E=E,
                    dpsim=np.nan, expref=np.nan, netsim=np.nan)
    idx = E[np.argmax(S[:, E], axis=1)]
    idx[E] = E
    nonex = np.setdiff1d(np.arange(n), E)
    dpsim = float(S[nonex, idx[nonex]].sum())
    expref = float(np.diag(S)[E].sum())
    return dict(idx=idx.astype(np.int64), E=E, dpsim=dpsim, expref=expref,
                netsim=dpsim + expref)


def netsim_of_labels(S, idx) -> float:
    """-E(c) of Section 2 for a labelling c: sum_i s(i, c_i), where s(k,k) is
    the preference of exemplar k."""
    S = np.asarray(S, dtype=np.float64)
    return float(S[np.arange(S.shape[0]), np.asarray(idx)].sum())


def brute_force_best(S):
    """Exhaustive optimum over every non-empty exemplar set E (N <= ~12):
    netsim(E) = sum_{k in E} p(k) + sum_{i not in E} max_{k in E} s(i,k).
    Returns (best E as sorted array, best netsim)."""
    S = np.asarray(S, dtype=np.float64)
    n = S.shape[0]
    best, bestE = -np.inf, None
    for mask in range(1, 1 << n):
        E = np.array([k for k in range(n) if mask >> k & 1])
        inE = np.zeros(n, dtype=bool)
        inE[E] = True
        val = S[E, E].sum() + S[~inE][:, E].max(axis=1).sum()
        if val > best:
            best, bestE = val, E
    return bestE, float(best)


def undamped_residuals(S, R, A):
    """||R - rho(S,A)||_inf and ||A - alpha(R)||_inf: zero at a fixed point."""
    return (float(np.abs(R - responsibility(S, A)).max()),
            float(np.abs(A - availability(R)).max()))
