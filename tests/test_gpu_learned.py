"""The learned warm start through the C ABI against the float64 oracle
(oracle.mlp): features, forward, gradients, Adam, and what the trained
network gains over cold-start Algorithm 1 on held-out problems."""
import numpy as np
import pytest
import torch

from oracle import ap as oap
from oracle import mlp as omlp
from paper_0910_1650_gb300 import capi, learned, synth

pytestmark = pytest.mark.gpu


def rel_inf(x, ref):
    return float(np.abs(x - ref).max() / max(np.abs(ref).max(), 1e-300))


def _square(M):
    n = M.shape[0]
    t = capi.empty_square(n, "cuda")
    t.copy_(torch.from_numpy(np.ascontiguousarray(M, dtype=np.float32)).cuda())
    return t


def _params(seed=3):
    P = synth.mlp_init().astype(np.float32)
    g = np.random.default_rng(seed)
    d = omlp.unpack(P)
    for b in ("b1", "b2", "b3"):
        d[b] = g.normal(size=d[b].shape) * 0.05
    P = omlp.pack(d).astype(np.float32)
    Pd = torch.from_numpy(P).cuda()
    P16 = torch.empty(P.size, dtype=torch.bfloat16, device="cuda")
    capi.apl_sync_bf16(Pd, P16)
    return P.astype(np.float64), Pd, P16


@pytest.mark.parametrize("n", [10, 17, 300, 2500])
def test_features_match_oracle(n):
    X, _ = synth.gaussian_mixture(n, 5, 4, 50 + n, 4.0, 1.0)
    S = oap.build_similarity(X)[0].astype(np.float32).astype(np.float64)
    scale = abs(float(np.float32(oap.offdiag_median(S))))
    F = capi.apl_features(_square(S), scale).cpu().numpy().astype(np.float64)
    Fo = omlp.row_features(S, scale)
    assert F.shape == (n, 25)
    assert np.abs(F[:, :16] - Fo[:, :16]).max() <= 2e-7 * np.abs(Fo[:, :16]).max()
    assert rel_inf(F[:, 16:19], Fo[:, 16:19]) <= 1e-6
    # counts are integers compared in float32 on both sides; logs in float32
    assert np.abs(F[:, 19:23] - Fo[:, 19:23]).max() <= 1e-6
    assert np.abs(F[:, 23] - Fo[:, 23]).max() <= 2e-6
    assert np.array_equal(F[:, 24], Fo[:, 24])


def test_forward_matches_oracle():
    P, Pd, P16 = _params()
    F = np.random.default_rng(7).normal(size=(1000, 25)).astype(np.float32)
    Y = capi.apl_forward(Pd, P16, torch.from_numpy(F).cuda()).cpu().numpy().astype(np.float64)
    Yo, _ = omlp.forward(P, F.astype(np.float64), bf16=True)
    assert rel_inf(Y, Yo) <= 1e-4


def test_gradient_matches_oracle_and_adam_step():
    P, Pd, P16 = _params(5)
    g = np.random.default_rng(8)
    rows = 777
    F = g.normal(size=(rows, 25)).astype(np.float32)
    T = np.stack([g.normal(size=rows), np.abs(g.normal(size=rows)), (g.random(rows) < 0.2)],
                 1).astype(np.float32)
    M = torch.zeros_like(Pd)
    V = torch.zeros_like(Pd)
    P0 = Pd.clone()
    loss, grad = capi.apl_train_step(Pd, P16, M, V, 1, 1e-3, torch.from_numpy(F).cuda(),
                                     torch.from_numpy(T).cuda(), want_grad=True)
    Lo, Go = omlp.backward(P, F.astype(np.float64), T.astype(np.float64), bf16=True)
    assert abs(float(loss.item()) - Lo) <= 1e-4 * abs(Lo)
    G = grad.cpu().numpy().astype(np.float64)
    go, gg = omlp.unpack(Go), omlp.unpack(G)
    for name in ("W1", "b1", "W2", "b2", "W3", "b3"):
        assert rel_inf(gg[name], go[name]) <= 1e-3, name
    # the Adam update, from the GPU's own gradient, against the textbook step
    P1, _, _ = omlp.adam_step(P0.cpu().numpy().astype(np.float64), G, np.zeros(G.size),
                              np.zeros(G.size), 1, 1e-3)
    assert np.abs(Pd.cpu().numpy() - P1).max() <= 1e-6
    # the bf16 copy follows the master weights
    assert torch.equal(P16, Pd.to(torch.bfloat16))


def test_warm_start_matches_oracle():
    Yh = np.array([[1.0, 2.0, 0.0], [-1.0, -3.0, 0.0], [0.5, 0.25, 1.0], [-0.9, 0.1, -2.0]],
                  dtype=np.float32)
    R = capi.empty_square(4, "cuda", 7.0)
    A = capi.empty_square(4, "cuda", 7.0)
    capi.apl_warm_start(torch.from_numpy(Yh).cuda(), 2.0, R, A)
    Ro, Ao = omlp.warm_start(4, Yh.astype(np.float64), 2.0)
    assert np.array_equal(R.cpu().numpy(), Ro)
    assert np.allclose(A.cpu().numpy(), Ao, rtol=1e-6, atol=0)     # float32 vs float64 sums


def _auc(score, label):
    """Area under the ROC curve of ``score`` for the binary ``label``
    (ties count half), by ranks."""
    from scipy.stats import rankdata
    r = rankdata(score)
    pos = label.astype(bool)
    npos, nneg = pos.sum(), (~pos).sum()
    return float((r[pos].sum() - npos * (npos + 1) / 2) / (npos * nneg))


def test_training_and_what_the_network_gains(capsys):
    """Train on plain-AP runs of Gaussian-mixture problems, evaluate on
    held-out problems.  What the network gains over the method without it:
    its exemplar head ranks the points that plain AP makes exemplars (held-out
    AUC, against 0.5 without a network).  What its warm start costs: the
    warm-started runs are measured against cold-start Algorithm 1 and the
    ratio is asserted to stay in the documented band (this warm start does
    not shorten the runs: cold/warm iterations about 0.7); the judge keeps
    every reported net similarity within 0.5 % of the cold start."""
    train_p = learned.mixture_problems(24)
    test_p = learned.mixture_problems(8, offset=24)
    F, T, info = learned.make_dataset(train_p)
    P, P16, losses = learned.train(F, T, epochs=60, batch=2048, lr=2e-3)
    assert losses[-1] < 0.8 * losses[0]
    rows, aucs = [], []
    for X in test_p:
        S, p = capi.ap_similarity(torch.from_numpy(X).cuda(), precision="bf16")
        R, A, idx, r = capi.apl_ap_run(S, P, P16, abs(p), damping=0.9, max_iter=1000, conv_iter=15)
        rows.append(r)
        # the judge's guarantee
        assert abs(r["result"]["netsim"] - r["cold_netsim"]) <= 0.005 * abs(r["cold_netsim"])
        if r["used_warm"]:
            assert r["result"]["iters"] == r["warm_iters"]
        # exemplar ranking against the cold run's exemplars
        Rc, Ac, _, dec = capi.ap_iterate(S, damping=0.9, max_iter=1000, conv_iter=15)
        Y = capi.apl_forward(P, P16, capi.apl_features(S, abs(p))).cpu().numpy()
        ex = dec.cpu().numpy() == np.arange(S.shape[0])
        aucs.append(_auc(Y[:, 2], ex))
    warm = np.mean([r["warm_iters"] for r in rows])
    cold = np.mean([r["cold_iters"] for r in rows])
    used = np.mean([r["used_warm"] for r in rows])
    auc = float(np.mean(aucs))
    with capsys.disabled():
        print(f"\nlearned warm start: loss {losses[0]:.4f} -> {losses[-1]:.4f}; held-out exemplar "
              f"AUC {auc:.3f}; iterations warm {warm:.1f} vs cold {cold:.1f} (x{cold / warm:.2f}); "
              f"warm result kept on {used:.0%} of problems")
    assert auc >= 0.85
    assert 0.5 <= cold / warm <= 1.1


def test_warm_start_batched_equals_per_problem():
    """apl_warm_start_batched over three problems of an arena writes what
    apl_features -> apl_forward -> apl_warm_start write per problem, bit for
    bit (R = 0 and the column-constant A)."""
    from paper_0910_1650_gb300 import batched
    _, Pd, P16 = _params(13)
    probs = [synth.gaussian_mixture(n, 8, 5, 70 + n, 4.0, 1.0)[0] for n in (300, 37, 1029)]
    off, n, ld, total = batched.layout([x.shape[0] for x in probs])
    S = torch.zeros(total, dtype=torch.float32, device="cuda")
    scales = []
    for b, X in enumerate(probs):
        Sb, p = capi.ap_similarity(torch.from_numpy(X).cuda(), precision="fp32")
        batched.view(S, off, n, ld, b).copy_(Sb)
        scales.append(abs(p))
    R = torch.full((total,), 7.0, device="cuda")
    A = torch.full((total,), 7.0, device="cuda")
    Y = torch.empty(sum(n), 3, dtype=torch.float32, device="cuda")
    capi.apl_warm_start_batched(S, R, A, off, n, ld, scales, Pd, P16, Y=Y)
    row = 0
    for b in range(len(probs)):
        Sb = batched.view(S, off, n, ld, b)
        Fb = capi.apl_features(Sb, scales[b])
        Yb = capi.apl_forward(Pd, P16, Fb)
        assert torch.equal(Y[row:row + n[b]], Yb)
        Rr = capi.empty_square(n[b], "cuda")
        Ar = capi.empty_square(n[b], "cuda")
        capi.apl_warm_start(Yb, scales[b], Rr, Ar)
        assert torch.equal(batched.view(R, off, n, ld, b), Rr)
        assert torch.equal(batched.view(A, off, n, ld, b), Ar)
        row += n[b]


def test_standardisation_matches_oracle():
    g = np.random.default_rng(21)
    F = (g.normal(size=(5000, 25)) * g.uniform(0.0, 3.0, size=25) + g.normal(size=25)).astype(np.float32)
    F[:, 7] = 1.5                                          # a constant column: isd floored
    P = torch.from_numpy(synth.mlp_init()).cuda()
    capi.apl_set_standardisation(P, torch.from_numpy(F).cuda())
    got = omlp.unpack(P.cpu().numpy().astype(np.float64))
    ref = omlp.unpack(omlp.set_standardisation(synth.mlp_init().astype(np.float64), F))
    assert rel_inf(got["mu"], ref["mu"]) <= 1e-6
    assert rel_inf(got["isd"], ref["isd"]) <= 1e-5
    assert got["isd"][7] == pytest.approx(1e3, rel=1e-6)


def test_learned_landmark_scores_pick_from_the_pool():
    """landmark_scores: a seeded uniform pool of 2L points is scored by the
    network (features of the pool's own S), every other point scores -inf,
    and lap_run in score mode takes the L best of the pool."""
    X, _ = synth.gaussian_mixture(3000, 16, 30, 42, 4.0, 0.5, False)
    P, Pd, P16 = _params(11)
    Xd = torch.from_numpy(X).cuda()
    L = 300
    score = learned.landmark_scores(Xd, L, Pd, P16)
    sc = score.cpu().numpy()
    pool = np.isfinite(sc)
    assert pool.sum() == 2 * L
    # the pool's scores are the network's log-odds on the pool's own features
    # (same seeded pool order as inside landmark_scores, so the same bits)
    perm = synth.Stream(synth.SEED_BASE + 401, 0).permutation(X.shape[0])[:2 * L]
    assert np.array_equal(np.sort(perm), np.nonzero(pool)[0])
    Sp, p = capi.ap_similarity(Xd[torch.from_numpy(perm.copy()).cuda()].contiguous(), precision="bf16")
    Y = capi.apl_forward(Pd, P16, capi.apl_features(Sp, abs(p))).cpu().numpy()
    assert np.array_equal(sc[perm], Y[:, 2])
    idx, lm, _ = capi.lap_run(Xd, L, "score", score=score, damping=0.9, max_iter=50, conv_iter=10)
    lm = np.sort(lm.cpu().numpy())
    best = np.sort(np.lexsort((np.arange(sc.size), -sc.astype(np.float64)))[:L])
    assert np.array_equal(lm, best)
    assert pool[lm].all()
