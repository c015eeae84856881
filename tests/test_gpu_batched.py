"""The batch path: ap_similarity_batched against ap_similarity problem by
problem (bit for bit), and the batch driver's cold runs against single
problems."""
import numpy as np
import pytest
import torch

from oracle import ap as oap
from paper_0910_1650_gb300 import batched, capi, synth

pytestmark = pytest.mark.gpu


def _problems(sizes, d, seed):
    return [synth.image_like(int(n), d, 5 + b % 7, seed=seed, stream=b)[0] for b, n in enumerate(sizes)]


@pytest.mark.parametrize("precision", ["bf16", "fp32"])
@pytest.mark.parametrize("d", [40, 300])
def test_similarity_batched_equals_single(precision, d):
    sizes = [37, 300, 2, 517, 256, 129]
    probs = _problems(sizes, d, 901 + d)
    X = torch.from_numpy(np.concatenate(probs)).cuda()
    xoff = np.concatenate([[0], np.cumsum(sizes)[:-1]]) * d
    off, n, ld, total = batched.layout(sizes)
    S = torch.full((total,), float("nan"), dtype=torch.float32, device="cuda")
    prefs = capi.ap_similarity_batched(X, xoff, n, S, off, ld, precision=precision)
    for b, Xb in enumerate(probs):
        Sb, p = capi.ap_similarity(torch.from_numpy(Xb).cuda(), precision=precision)
        got = batched.view(S, off, n, ld, b)
        assert torch.equal(got, Sb), b
        assert prefs[b] == p
    # padding columns of the arena stay untouched
    for b in range(len(sizes)):
        pad = S[off[b]:off[b] + n[b] * ld[b]].view(n[b], ld[b])[:, n[b]:]
        assert torch.isnan(pad).all()


def test_similarity_batched_scalar_preference_and_bad_args():
    sizes = [50, 70]
    probs = _problems(sizes, 16, 77)
    X = torch.from_numpy(np.concatenate(probs)).cuda()
    off, n, ld, total = batched.layout(sizes)
    S = torch.empty(total, dtype=torch.float32, device="cuda")
    prefs = capi.ap_similarity_batched(X, [0, 50 * 16], n, S, off, ld, pref=-3.5)
    assert prefs == [-3.5, -3.5]
    for b in range(2):
        assert torch.all(torch.diagonal(batched.view(S, off, n, ld, b)) == -3.5)
    with pytest.raises(capi.ApgbError):
        capi.ap_similarity_batched(X, [0, 50 * 16], [50, 1], S, off, ld)


def test_batch_driver_cold_run_matches_single_runs():
    """The batched launch splits its clusters between problems differently
    from a single-problem launch, so column sums are added in another order:
    the messages agree to rounding, the outcome (iterations, exemplars,
    net similarity) is the same."""
    sizes = [300, 41, 1000, 257]
    probs = _problems(sizes, 64, 5150)
    B = batched.Batch(iter(probs), sizes, group_bytes=1)      # one problem per group
    R, A, res, _ = batched.run(B, damping=0.9, max_iter=300, conv_iter=15)
    sims = batched.netsims(B, R, A)
    for b, Xb in enumerate(probs):
        S, p = capi.ap_similarity(torch.from_numpy(Xb).cuda(), precision="bf16")
        assert p == B.pref[b]
        assert torch.equal(S, B.S_of(b))
        R1, A1, r1, _ = capi.ap_iterate(S, damping=0.9, max_iter=300, conv_iter=15)
        assert r1["converged"] == res[b]["converged"] == 1
        assert abs(r1["iters"] - res[b]["iters"]) <= 2
        _, e = capi.ap_exemplars(S, R1, A1)
        assert e["n_exemplars"] == sims[b][1]
        assert abs(e["netsim"] - sims[b][0]) <= 1e-6 * abs(e["netsim"])
    assert all(batched.judge(sims, sims))


def test_full_size_batch_sampled_problems_match_oracle():
    """The 256 problem sizes of the image batch (N ~ U{200..4000}) in one
    batched run: the size classes, work lists and launch configurations of
    the bench's cold run.  Four problems (the largest, the smallest, one of
    median size and the first) carry the image-like workload's S, built by
    the oracle (Section 2's similarity in its Gram form, preference the
    off-diagonal median); the other 252 carry the S of seeded points on a
    line (problems are independent and only their sizes enter the launch
    configuration).  After 10 fixed iterations the sampled problems' R and A
    match the float64 oracle within 1e-4."""
    sizes, clusters = synth.batch_problem_sizes(256)
    sizes = [int(x) for x in sizes]
    order = np.argsort(sizes, kind="stable")
    picks = sorted({int(order[-1]), int(order[0]), int(order[len(order) // 2]), 0})
    off, ld, at = [], [], 0
    for n in sizes:
        off.append(at)
        ld.append(capi.padded_ld(n))
        at += n * ld[-1]
    arena = np.zeros(at, dtype=np.float32)
    g = np.random.default_rng(4)
    ref_S = {}
    for b, n in enumerate(sizes):
        view = arena[off[b]:off[b] + n * ld[b]].reshape(n, ld[b])
        if b in picks:
            X = synth.image_like(n, 4096, int(clusters[b]), stream=b)[0]
            S64 = oap.similarity_gram(X)
            S32 = oap.set_preference(S64, oap.offdiag_median_select(S64)).astype(np.float32)
            ref_S[b] = S32
            view[:, :n] = S32
        else:
            x = np.sort(g.uniform(0.0, 10.0, n)).astype(np.float32)
            S32 = -((x[:, None] - x[None, :]) ** 2)
            np.fill_diagonal(S32, np.float32(-4.0))
            view[:, :n] = S32
    Sa = torch.from_numpy(arena).cuda()
    del arena
    Ra = torch.zeros_like(Sa)
    Aa = torch.zeros_like(Sa)
    res, _ = capi.ap_iterate_batched(Sa, Ra, Aa, off, sizes, ld, damping=0.9, max_iter=10, conv_iter=0)
    for b in picks:
        n = sizes[b]
        assert res[b]["iters"] == 10
        R = Ra[off[b]:off[b] + n * ld[b]].view(n, ld[b])[:, :n].cpu().numpy().astype(np.float64)
        A = Aa[off[b]:off[b] + n * ld[b]].view(n, ld[b])[:, :n].cpu().numpy().astype(np.float64)
        ref = oap.run(ref_S[b].astype(np.float64), lam=0.9, fixed_iters=10)
        for got, want in ((R, ref["R"]), (A, ref["A"])):
            assert np.abs(got - want).max() <= 1e-4 * np.abs(want).max(), b
