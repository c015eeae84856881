"""Partition affinity propagation, Algorithm 2 of Xia et al. (Section 3).

TEST INFRASTRUCTURE ONLY -- see ``oracle/__init__.py``.

Step 1 cuts S into k diagonal blocks S_11..S_kk of the given point order;
Step 2 runs Algorithm 1 on each block (the block of S as it stands, so each
sub-problem keeps the global preferences on its diagonal) and keeps its
availabilities A_jj; Step 3 places the A_jj on the diagonal of an N x N
matrix A' with zeros elsewhere; Step 4 runs Algorithm 1 on the whole S
starting from A' (R starts at zero: the paper carries only availabilities).
"""
from __future__ import annotations

import numpy as np

from . import ap


def equal_partition(n: int, k: int) -> np.ndarray:
    """Section 3 Step 1: blocks 1..k-1 have m = floor(N/k) points, block k has
    N - m(k-1).  Returns offsets (length k+1)."""
    if not (1 <= k <= n):
        raise ValueError("need 1 <= k <= N")
    m = n // k
    sizes = [m] * (k - 1) + [n - m * (k - 1)]
    return np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)


def block_count_bound_ok(n: int, k: int, max_clusters: int) -> bool:
    """The stated admissible range 1 < k < N/(4C) of Step 1."""
    return 1 < k < n / (4.0 * max_clusters)


def merge_blocks(n: int, offsets, blocks) -> np.ndarray:
    """Step 3: A' = blockdiag(A_11, ..., A_kk), zeros elsewhere."""
    Ap = np.zeros((n, n))
    for j in range(len(offsets) - 1):
        lo, hi = int(offsets[j]), int(offsets[j + 1])
        Ap[lo:hi, lo:hi] = blocks[j]
    return Ap


def run(S, offsets, lam=0.5, max_iter=200, convits=15, fixed_iters=None, carry_r=False):
    """Algorithm 2 with the given block offsets.  With ``fixed_iters`` every
    run (Step 2 and Step 4) takes exactly that many iterations.  Step 4
    starts from R = 0 (the paper carries availabilities only) or, with
    ``carry_r`` (a variant), from the block-diagonal R of the sub-problems.

    Returns dict(sub=[per-block run dicts], A_prime, final=run dict of Step 4)."""
    S = np.asarray(S, dtype=np.float64)
    n = S.shape[0]
    subs = []
    for j in range(len(offsets) - 1):
        lo, hi = int(offsets[j]), int(offsets[j + 1])
        subs.append(ap.run(S[lo:hi, lo:hi], lam, max_iter, convits, fixed_iters=fixed_iters))
    Ap = merge_blocks(n, offsets, [s["A"] for s in subs])
    R0 = merge_blocks(n, offsets, [s["R"] for s in subs]) if carry_r else np.zeros((n, n))
    final = ap.run(S, lam, max_iter, convits, R0=R0, A0=Ap, fixed_iters=fixed_iters)
    return dict(sub=subs, A_prime=Ap, final=final)
