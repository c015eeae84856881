"""The batch path: ap_similarity_batched against ap_similarity problem by
problem (bit for bit), and the batch driver's cold runs against single
problems."""
import numpy as np
import pytest
import torch

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
