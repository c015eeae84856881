"""The library's row-shard entries (ap_shard_begin / ap_shard_sweep /
ap_shard_finish) on one GPU.  Several shards of one problem run in one
process, one after another within each iteration; the sum of their share
buffers stands in for the all-reduce between GPUs (the shards' kernels never
wait on one another).  Against the float64 oracle after fixed iterations and
at convergence, and one shard holding every row against ap_iterate, bit for
bit (same work list, same summation order)."""
import numpy as np
import pytest
import torch

from oracle import ap as oap
from paper_0910_1650_gb300 import capi, sharded, synth

pytestmark = pytest.mark.gpu


def _rows(M, r0, r1, ld):
    t = torch.zeros(r1 - r0, ld, dtype=torch.float32, device="cuda")
    t[:, :M.shape[1]] = torch.from_numpy(np.ascontiguousarray(M[r0:r1], dtype=np.float32)).cuda()
    return t


def _run_shards(S, world, **kw):
    """Runs `world` shards of S to the end; returns the gathered R, A (n x n,
    float64), the result and the number of iterations each shard saw."""
    n = S.shape[0]
    ld = capi.padded_ld(n)
    shards = []
    for rank in range(world):
        r0, r1 = sharded.row_range(n, world, rank)
        sh = sharded.LibraryShard(_rows(S, r0, r1, ld), _rows(np.zeros_like(S), r0, r1, ld),
                                  _rows(np.zeros_like(S), r0, r1, ld), n, r0, r1, **kw)
        sh.begin()
        shards.append(sh)
    res = None
    while res is None:
        tot = sum(sh.sweep().clone() for sh in shards)       # the sum over the GPUs
        fin = [sh.finish(tot) for sh in shards]
        assert len({d for d, _ in fin}) == 1                  # every shard stops together
        if fin[0][0]:
            res = fin[0][1]
            assert all(r == res for _, r in fin)
    R = torch.cat([sh.R[:, :n] for sh in shards]).cpu().numpy().astype(np.float64)
    A = torch.cat([sh.A[:, :n] for sh in shards]).cpu().numpy().astype(np.float64)
    return R, A, res


def _rel(x, ref):
    return float(np.abs(x - ref).max() / np.abs(ref).max())


@pytest.mark.parametrize("world", [2, 3])
def test_shards_fixed_iterations_match_oracle(world):
    X, _ = synth.workload(1, scale=0.05)                     # 1000 points, 64-D
    S = oap.build_similarity(X)[0].astype(np.float32).astype(np.float64)
    R, A, res = _run_shards(S, world, damping=0.9, max_iter=30, conv_iter=0)
    ref = oap.run(S, lam=0.9, fixed_iters=30)
    assert res["iters"] == 30
    assert _rel(R, ref["R"]) <= 1e-4 and _rel(A, ref["A"]) <= 1e-4


def test_shards_converge_to_the_oracles_exemplars():
    X, _ = synth.workload(1, scale=0.1)                      # 2000 points, 64-D
    S = oap.build_similarity(X)[0].astype(np.float32).astype(np.float64)
    R, A, res = _run_shards(S, 4, damping=0.9, max_iter=1000, conv_iter=15)
    ref = oap.run(S, lam=0.9, max_iter=1000, convits=15)
    assert res["converged"] and ref["converged"]
    assert abs(res["iters"] - ref["iters"]) <= max(5, 0.15 * ref["iters"])
    got = oap.exemplars(S, R, A, dtype=np.float32)
    want = oap.exemplars(S, ref["R"], ref["A"])
    assert np.array_equal(got["E"], want["E"]) and np.array_equal(got["idx"], want["idx"])


def test_one_shard_is_ap_iterate_bit_for_bit():
    X, _ = synth.workload(1, scale=0.1)
    Sd, _ = capi.ap_similarity(torch.from_numpy(X).cuda(), precision="fp32")
    S = Sd.cpu().numpy().astype(np.float64)
    R1, A1, res = _run_shards(S, 1, damping=0.9, max_iter=1000, conv_iter=15)
    R, A, r, _ = capi.ap_iterate(Sd, damping=0.9, max_iter=1000, conv_iter=15)
    assert res["iters"] == r["iters"] and res["converged"] == r["converged"]
    assert np.array_equal(R1, R.cpu().numpy().astype(np.float64))
    assert np.array_equal(A1, A.cpu().numpy().astype(np.float64))


def test_shard_rejects_non_finite_rows():
    n = 64
    S = -np.abs(np.random.default_rng(1).normal(size=(n, n)))
    S[40, 7] = np.nan
    ld = capi.padded_ld(n)
    for rank, bad in ((0, False), (1, True)):
        r0, r1 = sharded.row_range(n, 2, rank)
        sh = sharded.LibraryShard(_rows(S, r0, r1, ld), _rows(0 * S, r0, r1, ld), _rows(0 * S, r0, r1, ld),
                                  n, r0, r1)
        if bad:
            with pytest.raises(capi.ApgbError) as e:
                sh.begin()
            assert e.value.status == -5                   # AP_ERR_NONFINITE
        else:
            sh.begin()


def test_shards_of_an_odd_sized_problem():
    """1001 points (not a multiple of 4: ragged float4 tail in every row)
    over three shards of 334, 334 and 333 rows."""
    X, _ = synth.gaussian_mixture(1001, 12, 9, 61, 5.0, 1.0)
    S = oap.build_similarity(X)[0].astype(np.float32).astype(np.float64)
    R, A, res = _run_shards(S, 3, damping=0.9, max_iter=25, conv_iter=0)
    ref = oap.run(S, lam=0.9, fixed_iters=25)
    assert _rel(R, ref["R"]) <= 1e-4 and _rel(A, ref["A"]) <= 1e-4
