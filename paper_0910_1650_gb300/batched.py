"""Many independent problems at once: the batch workload of image-like
vectors (256 problems, N uniform in [200, 4000], d = 4096), cold-start and
learned-warm-start Algorithm 1 over the whole batch in one batched sweep per
iteration, and the judge that keeps a warm result only when its net
similarity is within 0.5 % of the cold start's.

Orchestration only: similarity, features, network, warm start, the batched
sweep and the exemplar step are calls into libapgb.so through ``capi``.
Problem b's matrices live in 1-D float32 arenas at element offset off[b] with
leading dimension ld[b] (a multiple of 32, so every row starts 128-byte
aligned).
"""
from __future__ import annotations

import multiprocessing as mp

import numpy as np
import torch

from . import capi, synth


def image_batch(count=256, offset=0, d=4096, lo=200, hi=4000, seed=synth.config_seed(4),
                workers=None):
    """Yields the feature matrices of problems offset .. offset+count-1 of the
    batch workload in order.  The host generator is slow at d = 4096, so the
    problems are drawn in a pool of spawned processes (safe after CUDA has
    been initialised) while the caller consumes them."""
    sizes, clusters = synth.batch_problem_sizes(count + offset, lo, hi, seed)
    jobs = [(int(sizes[b]), d, int(clusters[b]), seed, b) for b in range(offset, offset + count)]
    workers = workers or max(1, min(16, mp.cpu_count() - 1))
    if workers == 1:
        for j in jobs:
            yield synth.image_like_task(j)
        return
    # the task lives in synth so that a worker imports numpy only
    with mp.get_context("spawn").Pool(workers) as pool:
        for X in pool.imap(synth.image_like_task, jobs, chunksize=1):
            yield X


def layout(sizes):
    """(off, n, ld, total) of an arena holding one n x ld matrix per size."""
    n = [int(x) for x in sizes]
    ld = [capi.padded_ld(x) for x in n]
    off, at = [], 0
    for a, b in zip(n, ld):
        off.append(at)
        at += a * b
    return off, n, ld, at


def view(arena, off, n, ld, b):
    """Problem b's n x n view (leading dimension ld) of an arena."""
    return arena[off[b]:off[b] + n[b] * ld[b]].view(n[b], ld[b])[:, :n[b]]


class Batch:
    """S of every problem in one arena (preference = each problem's
    off-diagonal median), built with ap_similarity_batched over groups of
    problems whose features are uploaded together (about ``group_bytes`` of
    features per group)."""

    def __init__(self, problems, sizes, precision="bf16", device="cuda", group_bytes=2 << 30):
        self.off, self.n, self.ld, total = layout(sizes)
        self.count = len(self.n)
        self.S = torch.empty(total, dtype=torch.float32, device=device)
        self.pref = []
        self.sim_ms = 0.0
        self.gemm_flops = 0.0           # 2 n^2 d of the Gram products
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        group, first = [], 0
        ws = None

        def flush():
            nonlocal group, first, ws
            if not group:
                return
            Xd = torch.from_numpy(np.concatenate(group)).to(device)
            rows = [x.shape[0] for x in group]
            d = group[0].shape[1]
            xoff = np.concatenate([[0], np.cumsum(rows)[:-1]]) * d
            idx = range(first, first + len(group))
            # the workspace is allocated (and grown) before the timed region
            need = capi.ap_similarity_batched_workspace_bytes(rows, d)
            if ws is None or ws.numel() < need:
                ws = None
                ws = torch.empty(need, dtype=torch.uint8, device=device)
            torch.cuda.synchronize()
            ev[0].record()
            p = capi.ap_similarity_batched(Xd, xoff, [self.n[b] for b in idx], self.S,
                                           [self.off[b] for b in idx], [self.ld[b] for b in idx],
                                           precision=precision, ws=ws)
            ev[1].record()
            torch.cuda.synchronize()
            self.sim_ms += ev[0].elapsed_time(ev[1])
            self.pref.extend(p)
            self.gemm_flops += sum(2.0 * m * m * d for m in rows)
            first += len(group)
            group = []

        held = 0
        for b, X in enumerate(problems):
            if X.shape[0] != self.n[b]:
                raise ValueError("problem sizes do not match the layout")
            group.append(X)
            held += X.nbytes
            if held >= group_bytes:
                flush()
                held = 0
        flush()
        if first != self.count:
            raise ValueError("fewer problems than sizes")

    def S_of(self, b):
        return view(self.S, self.off, self.n, self.ld, b)

    def scale(self, b):
        p = abs(self.pref[b])
        return p if p > 0 else 1.0


def run(batch, R=None, A=None, damping=0.9, max_iter=1000, conv_iter=15, ws=None):
    """Algorithm 1 on every problem of ``batch`` from (R, A) (zeros when
    omitted): one batched sweep launch per iteration.  Every allocation
    happens before the timed region.  Returns (R, A, per-problem results,
    device ms)."""
    if R is None:
        R = torch.zeros_like(batch.S)
    if A is None:
        A = torch.zeros_like(batch.S)
    if ws is None:
        ws = capi.ap_iterate_batched_workspace(batch.n, batch.ld, batch.S.device)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev[0].record()
    res, _ = capi.ap_iterate_batched(batch.S, R, A, batch.off, batch.n, batch.ld,
                                     damping=damping, max_iter=max_iter, conv_iter=conv_iter, ws=ws)
    ev[1].record()
    torch.cuda.synchronize()
    return R, A, res, ev[0].elapsed_time(ev[1])


def warm_start(batch, P, P16, gamma=1.0, R=None, A=None, ws=None):
    """R0 = 0 and the network's column-constant A0 for every problem, A0
    scaled by ``gamma``: features, forward pass and warm start of the whole
    batch in one library call, into (R, A) (allocated, like the workspace,
    before the timed region when omitted).  Returns (R, A, device ms)."""
    R = torch.empty_like(batch.S) if R is None else R
    A = torch.empty_like(batch.S) if A is None else A
    if ws is None:
        ws = capi.apl_warm_start_batched_workspace(batch.n, batch.S.device)
    scale = [batch.scale(b) * gamma for b in range(batch.count)]
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev[0].record()
    capi.apl_warm_start_batched(batch.S, R, A, batch.off, batch.n, batch.ld, scale, P, P16, ws=ws)
    ev[1].record()
    torch.cuda.synchronize()
    return R, A, ev[0].elapsed_time(ev[1])


def netsims(batch, R, A):
    """Net similarity and exemplar count of every problem (ap_exemplars)."""
    out = []
    for b in range(batch.count):
        _, r = capi.ap_exemplars(batch.S_of(b), view(R, batch.off, batch.n, batch.ld, b),
                                 view(A, batch.off, batch.n, batch.ld, b))
        out.append((r["netsim"], r["n_exemplars"]))
    return out


def judge(cold, warm, tol=0.005):
    """Per problem: keep the warm result when it has exemplars and its net
    similarity is within ``tol`` (relative) of the cold start's (the
    library's apl_judge), else fall back to the cold one."""
    keep = capi.apl_judge([nc for nc, _ in cold], [nw for nw, _ in warm], tol)
    return [k and ew > 0 for k, (_, ew) in zip(keep, warm)]
