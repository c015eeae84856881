"""Row-sharded Algorithm 1 (paper_0910_1650_gb300.sharded) with two gloo ranks
on the CPU: the driver's loop and its exchange (one all-reduce of the ranks'
shares of colp, r(k,k) and the decision counts per iteration) around a
float64 stand-in for the library's shard steps, written from the oracle's
update rules restricted to the rank's rows.  The sharded run must reproduce
the oracle's unsharded run: the same messages after a fixed number of
iterations, the same stopping iteration and messages at convergence."""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


class OracleShard:
    """The shard protocol of ap_shard_begin / ap_shard_sweep / ap_shard_finish
    in float64: launch t runs the availability half of iteration t-1 (Eq. 3-4,
    with the summed colp and c = r(k,k) + colp; then the decisions) and the
    responsibility half of iteration t (Eq. 2), exporting the rows' shares;
    the stop rule of Step 4 runs on the summed counts."""

    def __init__(self, S, r0, r1, lam, max_iter, conv_iter):
        from oracle import ap as oap
        self.oap = oap
        self.n = S.shape[0]
        self.r0, self.r1 = r0, r1
        self.S = np.array(S[r0:r1], dtype=np.float64)
        m = r1 - r0
        self.R = np.zeros((m, self.n))
        self.A = np.zeros((m, self.n))
        self.R_prev = self.R
        self.lam, self.max_iter, self.conv_iter = lam, max_iter, conv_iter
        self.rows = np.arange(m)
        self.diag = np.arange(r0, r1)           # global column of each row's diagonal
        self.red = torch.zeros(2 * self.n + 2, dtype=torch.float64)

    def begin(self):
        self.t, self.stable, self.done = 1, 0, False
        self.converged, self.iters = False, 0
        self.flags = np.zeros(self.r1 - self.r0, dtype=bool)

    def sweep(self):
        lam, t = self.lam, self.t
        changes = n_ex = 0
        if t >= 2:
            P = np.maximum(self.R, 0.0)
            A_new = np.minimum(0.0, self.c[None, :] - P)
            A_new[self.rows, self.diag] = self.colp[self.diag]
            self.A = lam * self.A + (1.0 - lam) * A_new
            flags = np.argmax(self.A + self.R, axis=1) == self.diag
            changes = int((flags != self.flags).sum())
            n_ex = int(flags.sum())
            self.flags = flags
        self.R_prev = self.R
        colp = np.zeros(self.n)
        rkk = np.zeros(self.n)
        if t <= self.max_iter:
            self.R = lam * self.R + (1.0 - lam) * self.oap.responsibility(self.S, self.A)
            P = np.maximum(self.R, 0.0)
            P[self.rows, self.diag] = 0.0
            colp = P.sum(axis=0)
            rkk[self.diag] = self.R[self.rows, self.diag]
        self.red.copy_(torch.from_numpy(np.concatenate([colp, rkk, [changes, n_ex]])))
        return self.red

    def finish(self, red):
        v = red.numpy()
        n = self.n
        self.colp = v[:n].copy()
        self.c = v[n:2 * n] + self.colp
        changes, n_ex = int(v[2 * n]), int(v[2 * n + 1])
        t = self.t
        if t >= 2:
            it = t - 1
            self.stable = 1 if (it == 1 or changes != 0) else self.stable + 1
            if self.conv_iter > 0 and self.stable >= self.conv_iter and n_ex > 0:
                self.done, self.converged, self.iters = True, True, it
                self.R = self.R_prev                # launch t also formed R_t: keep R_(t-1)
        if not self.done and t == self.max_iter + 1:
            self.done, self.iters = True, self.max_iter
        self.t = t + 1
        return self.done, (dict(iters=self.iters, converged=int(self.converged)) if self.done else None)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _problem(case):
    from oracle import ap as oap
    from paper_0910_1650_gb300 import synth
    if case == "mixture2d":
        X, _ = synth.gaussian_mixture_2d(per_cluster=24)              # 120 points
    else:
        X, _ = synth.gaussian_mixture(97, 6, 4, 11, 6.0, 1.0)          # odd size: uneven rows
    return oap.build_similarity(X)[0]


def _worker(rank, world, port, case, lam, max_iter, conv_iter, out):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_0910_1650_gb300 import sharded

    S = _problem(case)
    r0, r1 = sharded.row_range(S.shape[0], world, rank)
    sh = OracleShard(S, r0, r1, lam, max_iter, conv_iter)
    res = sharded.iterate(sh, sharded.torch_allreduce())
    out.put((rank, r0, r1, sh.R, sh.A, res))
    dist.barrier()
    dist.destroy_process_group()


def _run(world, case, lam, max_iter, conv_iter):
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, case, lam, max_iter, conv_iter, q))
             for r in range(world)]
    for p in procs:
        p.start()
    got = sorted((q.get(timeout=180) for _ in range(world)), key=lambda g: g[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return got


def test_row_ranges_cover_every_row_once():
    sys.path.insert(0, ROOT)
    from paper_0910_1650_gb300 import sharded
    for n in (2, 7, 97, 20000):
        for world in (1, 2, 3, 8):
            if world > n:
                continue
            rr = [sharded.row_range(n, world, r) for r in range(world)]
            assert rr[0][0] == 0 and rr[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(rr, rr[1:]))
            sizes = [b - a for a, b in rr]
            assert max(sizes) - min(sizes) <= 1 and min(sizes) >= 1


@pytest.mark.parametrize("case", ["mixture2d", "uneven"])
def test_two_ranks_fixed_iterations_equal_the_oracle(case):
    from oracle import ap as oap
    got = _run(2, case, 0.9, 25, 0)
    S = _problem(case)
    ref = oap.run(S, lam=0.9, fixed_iters=25)
    for rank, r0, r1, R, A, res in got:
        assert res["iters"] == 25 and not res["converged"]
        assert np.allclose(R, ref["R"][r0:r1], rtol=1e-12, atol=1e-9)
        assert np.allclose(A, ref["A"][r0:r1], rtol=1e-12, atol=1e-9)


def test_two_ranks_stop_together_at_the_oracles_iteration():
    from oracle import ap as oap
    got = _run(2, "mixture2d", 0.5, 200, 15)
    S = _problem("mixture2d")
    ref = oap.run(S, lam=0.5, max_iter=200, convits=15)
    assert ref["converged"]
    for rank, r0, r1, R, A, res in got:
        assert res["converged"] and res["iters"] == ref["iters"]
        assert np.allclose(R, ref["R"][r0:r1], rtol=1e-10, atol=1e-8)
        assert np.allclose(A, ref["A"][r0:r1], rtol=1e-10, atol=1e-8)
