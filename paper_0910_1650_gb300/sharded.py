"""Row-sharded Algorithm 1: the rows of S, R and A split between ranks (one
GPU each), with one all-reduce of 2n + 2 floats per iteration.

Why it shards: given the column vectors colp(k) = sum over i' != k of
max(0, r(i',k)) and r(k,k), both halves of an iteration are row-local (Eq. 2
reads row i of A + S; Eq. 3-4 read row i of R, colp and r(k,k)).  So every
rank sweeps its own rows with the library's fused kernel, and the ranks sum
their shares of colp, of r(k,k) and of the decision counts (exemplar-set
changes, exemplars) before each applies the stop rule of Step 4 to the same
totals.  The per-iteration O(N^2) work that Section 3 states is divided by
the rank count; the exchange is O(N).

Orchestration only: the sweep, the local reductions and the stop rule are
library calls (``capi.ap_shard_*``); the exchange is the caller's sum over
ranks (``torch.distributed.all_reduce`` over NCCL on GPUs).
"""
from __future__ import annotations

import ctypes as C

import torch

from . import capi


def row_range(n: int, world: int, rank: int):
    """Rows [r0, r1) of rank ``rank``: contiguous blocks, the first n % world
    ranks one row longer."""
    base, extra = divmod(int(n), int(world))
    r0 = rank * base + min(rank, extra)
    return r0, r0 + base + (1 if rank < extra else 0)


class LibraryShard:
    """One rank's rows [r0, r1) of an n-point problem on its GPU: S, R, A are
    (r1 - r0) x ld float32 CUDA tensors (rows of the n x n matrices; R and A
    hold the initial messages)."""

    def __init__(self, S, R, A, n, r0, r1, damping=0.9, max_iter=1000, conv_iter=15, decisions=None,
                 stream=None):
        for t, name in ((S, "S"), (R, "R"), (A, "A")):
            capi._dev_f32(t, name)
            if t.shape[0] != r1 - r0 or t.stride(0) != S.stride(0) or t.stride(1) != 1:
                raise ValueError(f"{name}: the shard's rows with one leading dimension")
        self.S, self.R, self.A = S, R, A
        self.n, self.r0, self.r1 = int(n), int(r0), int(r1)
        self.ld = S.stride(0)
        self.p = capi.ApParams(float(damping), int(max_iter), int(conv_iter), 0, 0)
        self.dec = decisions
        self.stream = stream
        self.ws = capi.workspace(capi.lib().ap_shard_workspace_size(self.n, self.ld, self.r0, self.r1),
                                 S.device)
        self.red = torch.empty(2 * self.n + 2, dtype=torch.float32, device=S.device)

    def _lead(self):
        return (capi._ptr(self.S), capi._ptr(self.R), capi._ptr(self.A), self.n, self.ld, self.r0,
                self.r1, C.byref(self.p), capi._ptr(self.dec))

    def begin(self):
        capi._check("ap_shard_begin", capi.lib().ap_shard_begin(
            *self._lead(), capi._ptr(self.ws), self.ws.numel(), capi._stream(self.stream)))

    def sweep(self):
        """One sweep of the shard's rows; returns the buffer of its shares."""
        capi._check("ap_shard_sweep", capi.lib().ap_shard_sweep(
            *self._lead(), capi._ptr(self.red), capi._ptr(self.ws), self.ws.numel(),
            capi._stream(self.stream)))
        return self.red

    def finish(self, red):
        """Applies the summed shares; returns (done, result dict or None)."""
        done = C.c_int32(0)
        res = capi.ApResult()
        st = capi.lib().ap_shard_finish(*self._lead(), capi._ptr(red), C.byref(done), C.byref(res),
                                        capi._ptr(self.ws), self.ws.numel(), capi._stream(self.stream))
        capi._check("ap_shard_finish", st)
        return bool(done.value), (res.as_dict() if done.value else None)


def iterate(shard, allreduce):
    """Algorithm 1 on a row shard: sweep, sum the shares over the ranks with
    ``allreduce`` (in place), apply them; until the stop rule ends the run on
    every rank at once.  Returns the shard's result (iters, converged)."""
    shard.begin()
    while True:
        red = shard.sweep()
        allreduce(red)
        done, res = shard.finish(red)
        if done:
            return res


def torch_allreduce(group=None):
    """The sum over the ranks of a torch.distributed process group."""
    import torch.distributed as dist

    def f(t):
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)

    return f
