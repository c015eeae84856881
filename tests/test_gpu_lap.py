"""Landmark AP (Algorithm 3 Steps 1-2) through the C ABI against the oracle.

Landmark selection is integer work: exact.  The landmark problem runs in the
same float32 arithmetic as ap_iterate (exemplars compared on a
well-conditioned case).  The nearest-exemplar assignment runs on bf16-rounded
centred features, so the decision is checked in that precision: against the
exact distances of the rounded points, a label must be the oracle's wherever
the best distance beats the runner-up by more than the float32 accumulation
bound, and within that bound of the best everywhere."""
import numpy as np
import pytest
import torch

from oracle import ap as oap
from oracle import lap as olap
from paper_0910_1650_gb300 import capi, synth

pytestmark = pytest.mark.gpu


def _data(n=3000, d=16, k=12, seed=31):
    X, lab = synth.gaussian_mixture(n, d, k, seed, 6.0, 1.0)
    return X


@pytest.mark.parametrize("n,L,seed", [(1000, 100, 5), (3001, 600, 99), (50000, 20000, 7)])
def test_uniform_landmarks_exact(n, L, seed):
    X = _data(n, 4, 3, 1)
    idx, lm, res = capi.lap_run(torch.from_numpy(X).cuda(), L, "uniform", seed=seed,
                                damping=0.9, max_iter=3, conv_iter=0)
    assert np.array_equal(lm.cpu().numpy().astype(np.int64), olap.uniform_landmarks(n, L, seed))


def test_score_landmarks_exact():
    n, L = 2000, 300
    X = _data(n, 4, 3, 2)
    g = np.random.default_rng(0)
    score = np.round(g.normal(size=n), 2).astype(np.float32)     # many ties
    idx, lm, res = capi.lap_run(torch.from_numpy(X).cuda(), L, "score",
                                score=torch.from_numpy(score), damping=0.9, max_iter=3, conv_iter=0)
    order = np.lexsort((np.arange(n), -score.astype(np.float64)))
    assert np.array_equal(lm.cpu().numpy().astype(np.int64), np.sort(order[:L]))


def _check_assignment(X, E_pts, labels):
    Xt = oap.round_bf16(oap.centred(X)).astype(np.float64)
    Et = Xt[E_pts]
    D = -oap.similarity(Xt, Et)
    K = (X.shape[1] + 63) // 64 * 64
    nx = (Xt ** 2).sum(axis=1)
    ne = (Et ** 2).sum(axis=1)
    tol = 4.0 * (K + 4) * 2.0 ** -24 * (nx + ne.max()) * 2.0
    pos = {int(e): j for j, e in enumerate(E_pts)}
    is_ex = np.zeros(X.shape[0], dtype=bool)
    is_ex[E_pts] = True
    got = np.array([pos[int(c)] for c in labels])
    best = D.min(axis=1)
    assert (D[np.arange(len(got)), got] <= best + tol).all()
    srt = np.sort(D, axis=1)
    clear = (srt[:, 1] - srt[:, 0] > 2 * tol) & ~is_ex
    assert np.array_equal(got[clear], D.argmin(axis=1)[clear])
    assert (labels[E_pts] == E_pts).all()
    return clear.mean()


def test_lap_matches_oracle():
    X = _data()
    L, seed = 600, 11
    idx, lm, res = capi.lap_run(torch.from_numpy(X).cuda(), L, "uniform", seed=seed,
                                damping=0.9, max_iter=1000, conv_iter=15)
    lmh = lm.cpu().numpy().astype(np.int64)
    ref = olap.run(X, lmh, lam=0.9, max_iter=1000, convits=15)
    labels = idx.cpu().numpy().astype(np.int64)
    E = np.unique(labels)
    assert np.array_equal(E, ref["E"]) and res["n_exemplars"] == E.size
    frac_clear = _check_assignment(X, E, labels)
    assert frac_clear > 0.99
    # netsim of the GPU labelling, recomputed in float64 by the oracle
    S_all = None
    dp = -((X.astype(np.float64) - X[labels].astype(np.float64)) ** 2).sum(axis=1)
    dp[E] = 0.0
    assert abs(res["dpsim"] - dp.sum()) <= 1e-9 * abs(dp.sum())
    assert abs(res["expref"] - res["pref"] * E.size) <= 1e-6 * abs(res["expref"])
    assert abs(res["netsim"] - ref["netsim"]) <= 1e-5 * abs(ref["netsim"])


def test_lap_with_every_point_a_landmark_is_ap():
    X = _data(800, 8, 5, 3)
    n = X.shape[0]
    idx, lm, res = capi.lap_run(torch.from_numpy(X).cuda(), n, "uniform", seed=1,
                                damping=0.9, max_iter=1000, conv_iter=15)
    assert np.array_equal(np.sort(lm.cpu().numpy()), np.arange(n))
    Sd, p = capi.ap_similarity(torch.from_numpy(X).cuda(), precision="fp32")
    R, A, r, _ = capi.ap_iterate(Sd, damping=0.9, max_iter=1000, conv_iter=15)
    idx_ap, ex = capi.ap_exemplars(Sd, R, A)
    assert res["n_exemplars"] == ex["n_exemplars"]
    assert np.array_equal(np.unique(idx.cpu().numpy()), np.unique(idx_ap.cpu().numpy()))
    assert abs(res["netsim"] - ex["netsim"]) <= 1e-4 * abs(ex["netsim"])


def test_lap_given_landmarks_and_bf16_landmark_similarity():
    X = _data(2000, 16, 8, 4)
    lm_in = np.sort(np.random.default_rng(3).choice(2000, 400, replace=False)).astype(np.int32)
    idx, lm, res = capi.lap_run(torch.from_numpy(X).cuda(), 400, "given",
                                landmarks=torch.from_numpy(lm_in), precision="bf16",
                                damping=0.9, max_iter=1000, conv_iter=15)
    assert np.array_equal(lm.cpu().numpy(), lm_in)
    labels = idx.cpu().numpy().astype(np.int64)
    E = np.unique(labels)
    assert set(E) <= set(lm_in.tolist())
    _check_assignment(X, E, labels)


# ---- Algorithm 3 Steps 1-4 -------------------------------------------------------------

def _far_data(seed):
    """A 10-Gaussian mixture in R^8 plus a tight group of 10 points far from
    it (indices 2990-2999), which no landmark class can hold."""
    X, _ = synth.gaussian_mixture(2990, 8, 10, 900 + seed, 6.0, 1.0)
    g = np.random.default_rng(seed)
    far = 60.0 + 0.2 * g.normal(size=(10, 8))
    return np.vstack([X, far]).astype(np.float32)


@pytest.mark.parametrize("dseed", [1, 2])
def test_lap_full_matches_oracle(dseed):
    """Steps 1-4 against the oracle on data whose gate and nearest-exemplar
    decisions are all clear of float32 rounding (asserted on the oracle's
    margins), so both sides must take every decision the same way.  Damping
    0.9: at 0.5 the landmark problem of this mixture is ill-conditioned (the
    float32 and float64 runs stop at different exemplar sets)."""
    X = _far_data(dseed)
    L, m0, seed = 300, 1000, 1
    assert not np.isin(np.arange(2990, 3000), olap.uniform_landmarks(X.shape[0], L, seed)).any()
    ref = olap.run_full(X, L, seed, m0, lam=0.9, max_iter=1000, convits=15)
    l0 = ref["levels"][0]
    assert (l0["margin"] / l0["scale"]).min() > 1e-4 and (l0["gap"] / l0["scale"]).min() > 1e-4
    assert (ref["gap"] / l0["scale"]).min() > 1e-4
    idx, level_of, res = capi.lap_run_full(torch.from_numpy(X).cuda(), L, m0, seed=seed,
                                           precision="fp32", damping=0.9, max_iter=1000,
                                           conv_iter=15)
    idx = idx.cpu().numpy().astype(np.int64)
    level_of = level_of.cpu().numpy()
    assert res["levels"] == 1 and res["base_case"] == 1 and len(ref["levels"]) == 2
    assert res["unassigned"][0] == l0["unassigned"].size
    assert np.array_equal(np.nonzero(level_of != 0)[0], l0["unassigned"])
    assert np.all(level_of[l0["unassigned"]] == 1)
    assert res["exemplars_at"] == [l0["E"].size, ref["levels"][1]["E"].size]
    assert np.array_equal(np.unique(idx), ref["E"]) and res["n_exemplars"] == ref["E"].size
    assert np.array_equal(idx, ref["idx"])
    assert np.all(idx[2990:] >= 2990)                 # the far group has its own exemplar
    assert abs(res["netsim"] - ref["netsim"]) <= 1e-5 * abs(ref["netsim"])


def test_lap_full_recursion_and_invariants():
    """m0 below the points left: Step 3 recurses (more landmark levels), the
    merged set labels every point, exemplars label themselves, labels are the
    nearest exemplar (checked in the assignment's precision)."""
    X = _far_data(1)
    idx, level_of, res = capi.lap_run_full(torch.from_numpy(X).cuda(), 100, 20, seed=4,
                                           precision="bf16", damping=0.5, max_iter=1000,
                                           conv_iter=15)
    idx = idx.cpu().numpy().astype(np.int64)
    level_of = level_of.cpu().numpy()
    assert res["levels"] >= 2
    E = np.unique(idx)
    assert E.size == res["n_exemplars"] == sum(res["exemplars_at"])
    assert np.all(idx[E] == E)
    assert np.all(idx[2990:] >= 2990)
    assert level_of.min() >= -1 and level_of.max() <= res["levels"]
    _check_assignment(X, E, idx)
