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


@pytest.mark.parametrize("n,L,seed", [(1000, 100, 5), (3001, 600, 99), (50000, 20000, 7),
                                      (600000, 20000, 13)])
def test_uniform_landmarks_exact(n, L, seed):
    """600000 points: the compaction's 256 blocks take several passes each."""
    X = _data(n, 4, 3, 1)
    idx, lm, res = capi.lap_run(torch.from_numpy(X).cuda(), L, "uniform", seed=seed,
                                damping=0.9, max_iter=3, conv_iter=0)
    assert np.array_equal(lm.cpu().numpy().astype(np.int64), olap.uniform_landmarks(n, L, seed))


@pytest.mark.parametrize("n,L", [(2000, 300), (400000, 5000)])
def test_score_landmarks_exact(n, L):
    """Ties of the score are broken by the lower index, also across the
    compaction's blocks (400000 points: 256 blocks of several passes)."""
    X = _data(n, 4, 3, 2)
    g = np.random.default_rng(0)
    score = np.round(g.normal(size=n), 2).astype(np.float32)     # many ties
    idx, lm, res = capi.lap_run(torch.from_numpy(X).cuda(), L, "score",
                                score=torch.from_numpy(score), damping=0.9, max_iter=3, conv_iter=0)
    order = np.lexsort((np.arange(n), -score.astype(np.float64)))
    assert np.array_equal(lm.cpu().numpy().astype(np.int64), np.sort(order[:L]))


def _check_assignment(X, E_pts, labels, best=None):
    """Labels against the oracle's distances of the bf16-rounded centred
    points: exact wherever the best distance beats the runner-up by more
    than the float32 accumulation bound, within that bound elsewhere.
    Returns (share of the non-centre points with a clear decision, share of
    their labels that differ from the float64 nearest centre of the unrounded
    points)."""
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
    best_d = D.min(axis=1)
    assert (D[np.arange(len(got)), got] <= best_d + tol).all()
    if D.shape[1] > 1:
        srt = np.sort(D, axis=1)
        clear = (srt[:, 1] - srt[:, 0] > 2 * tol) & ~is_ex
    else:
        clear = ~is_ex
    assert np.array_equal(got[clear], D.argmin(axis=1)[clear])
    assert (labels[E_pts] == E_pts).all()
    if best is not None:
        # the reported score is 2 x.e - |e|^2 of the chosen centre
        ref = nx - best_d
        assert np.all(np.abs(best - ref) <= tol + 1e-6 * np.abs(ref))
    # the paper's distance: plain float64 squared distance of the unrounded points
    D64 = -oap.similarity(X.astype(np.float64), X[E_pts].astype(np.float64))
    near64 = D64.argmin(axis=1)
    differ = (near64 != got) & ~is_ex
    nonex = max(1, (~is_ex).sum())
    return clear.sum() / nonex, differ.sum() / nonex


@pytest.mark.parametrize("c_case,n,c,seed", [("mix128", 8000, 700, 1), ("mix128", 3001, 257, 2),
                                           ("mix128", 513, 256, 3), ("mix128", 1000, 1, 4),
                                           ("subspace100", 5000, 600, 5), ("mix300", 3000, 500, 6)])
def test_lap_assign_full_shape(c_case, n, c, seed):
    """The assignment GEMM's arg-max mode through its own entry (Algorithm 3
    Step 2) at the shapes of the 1e6-point workload: d = 128 (two K blocks)
    or d = 100 (zero-padded K), and d = 300 (five K blocks), up to three
    256-column tiles of centres merged by the running arg-max, and dozens of
    128-row blocks."""
    if c_case == "mix128":
        X, _ = synth.workload(3, scale=n / 1_000_000)
    elif c_case == "mix300":                                  # K = 320: five K blocks
        X, _ = synth.gaussian_mixture(n, 300, 20, 41, 4.0, 1.0)
    else:
        X, _ = synth.workload(2, scale=n / 60000)
    X = np.ascontiguousarray(X[:n])
    g = np.random.default_rng(seed)
    E = g.choice(n, c, replace=False).astype(np.int64)        # list order = tie order
    idx, best = capi.lap_assign(torch.from_numpy(X).cuda(), torch.from_numpy(E), best=True)
    labels = idx.cpu().numpy().astype(np.int64)
    assert set(np.unique(labels).tolist()) <= set(E.tolist())
    frac_clear, frac_fp64 = _check_assignment(X, E, labels, best.cpu().numpy().astype(np.float64))
    print(f"\nlap_assign n={n} c={c} d={X.shape[1]}: clear {frac_clear:.4f}, "
          f"differ from float64 unrounded {frac_fp64:.2e}")
    # random centres put several centres in one cluster: near ties (within
    # rounding) are common, and every clear decision is still checked exactly
    assert frac_clear > 0.8
    assert frac_fp64 <= 0.02


@pytest.mark.parametrize("c", [700, 1024])
def test_lap_assign_norm_forms(c, monkeypatch):
    """The three ways -|e|^2/2 enters the arg-max GEMM's scores, on the same
    inputs: folded into the product by an extra MMA over the augmented
    operands (the default up to 1024 centres), subtracted in the epilogue
    from a shared-memory table, or from global memory.  Each is checked
    against the oracle; the two epilogue forms agree bit for bit."""
    n = 6000
    X, _ = synth.workload(3, scale=n / 1_000_000)
    X = np.ascontiguousarray(X[:n])
    E = np.random.default_rng(c).choice(n, c, replace=False).astype(np.int64)
    got = {}
    for form in ("folded", "shared", "global"):
        monkeypatch.setenv("APGB_ASSIGN_NORMS", form)
        idx, best = capi.lap_assign(torch.from_numpy(X).cuda(), torch.from_numpy(E), best=True)
        got[form] = (idx.cpu().numpy().astype(np.int64), best.cpu().numpy().astype(np.float64))
        frac_clear, _ = _check_assignment(X, E, got[form][0], got[form][1])
        assert frac_clear > 0.8, form
    assert np.array_equal(got["shared"][0], got["global"][0])
    assert np.array_equal(got["shared"][1], got["global"][1])


def test_lap_assign_at_full_size_sampled_points():
    """All 1e6 points of the 128-D workload against 1000 seeded centres (the
    exemplar count of the bench's landmark run): the assignment GEMM at full
    size (7813 row blocks, four column tiles, the norms folded into the
    product).  4000 sampled points against the oracle's distances of the
    rounded centred points: exact where the decision is clear, within the
    float32 accumulation bound elsewhere, with the reported score."""
    X, _ = synth.workload(3)
    n, dd = X.shape
    g = np.random.default_rng(12)
    E = g.choice(n, 1000, replace=False).astype(np.int64)
    idx, best = capi.lap_assign(torch.from_numpy(X).cuda(), torch.from_numpy(E), best=True)
    rows = g.choice(n, 4000, replace=False)
    labels = idx.cpu().numpy().astype(np.int64)[rows]
    bst = best.cpu().numpy().astype(np.float64)[rows]
    Xt = oap.round_bf16(oap.centred(X))
    Et = Xt[E].astype(np.float64)
    Xr = Xt[rows].astype(np.float64)
    D = -oap.similarity(Xr, Et)
    K = (dd + 63) // 64 * 64
    nx = (Xr ** 2).sum(axis=1)
    tol = 4.0 * (K + 4) * 2.0 ** -24 * (nx + (Et ** 2).sum(axis=1).max()) * 2.0
    pos = {int(e): j for j, e in enumerate(E)}
    got = np.array([pos[int(c)] for c in labels])
    best_d = D.min(axis=1)
    assert (D[np.arange(rows.size), got] <= best_d + tol).all()
    srt = np.sort(D, axis=1)
    clear = (srt[:, 1] - srt[:, 0] > 2 * tol) & ~np.isin(rows, E)
    assert clear.mean() > 0.8
    assert np.array_equal(got[clear], D.argmin(axis=1)[clear])
    ref = nx - best_d
    assert np.all(np.abs(bst - ref) <= tol + 1e-6 * np.abs(ref))


def test_lap_assign_with_more_centres_than_the_shared_norm_table():
    """8000 centres: their norms (8192 padded entries) do not fit in shared
    memory beside the operand ring, so the arg-max epilogue reads them from
    global memory; 32 column tiles merged by the running arg-max."""
    n, c = 10000, 8000
    X = _data(n=n, d=16, k=40, seed=8)
    E = np.random.default_rng(8).choice(n, c, replace=False).astype(np.int64)
    idx, best = capi.lap_assign(torch.from_numpy(X).cuda(), torch.from_numpy(E), best=True)
    labels = idx.cpu().numpy().astype(np.int64)
    frac_clear, frac_fp64 = _check_assignment(X, E, labels, best.cpu().numpy().astype(np.float64))
    print(f"\nlap_assign n={n} c={c}: clear {frac_clear:.4f}, differ from float64 {frac_fp64:.2e}")
    assert frac_clear > 0.8


def test_lap_run_full_shape_assignment():
    """lap_run (Steps 1-2) on 20000 points of the 1e6-point 128-D workload
    generator with 3000 uniform landmarks: several hundred exemplars (three or
    more 256-column tiles), 157 row blocks.  The landmark problem runs on the
    GPU; Step 2's labels are checked against the oracle's nearest exemplar."""
    X, _ = synth.workload(3, scale=0.02)
    idx, lm, res = capi.lap_run(torch.from_numpy(X).cuda(), 3000, "uniform", seed=5,
                                damping=0.9, max_iter=1000, conv_iter=15)
    labels = idx.cpu().numpy().astype(np.int64)
    E = np.unique(labels)
    assert E.size == res["n_exemplars"] >= 600
    frac_clear, frac_fp64 = _check_assignment(X, E, labels)
    print(f"\nlap_run n=20000 d=128 exemplars={E.size}: clear {frac_clear:.4f}, "
          f"differ from float64 unrounded {frac_fp64:.2e}")
    assert frac_clear > 0.99
    assert frac_fp64 <= 0.001


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
    frac_clear, _ = _check_assignment(X, E, labels)
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


# ---- Algorithm 3 Step 4: the refinement ------------------------------------------------------

def _integer_clusters(seed, k=20, per=30, d=16, spread=3):
    """Integer points symmetric about the origin (k clusters mirrored): the
    column mean is exactly zero and every coordinate, product and partial
    sum is exact in bf16 / fp32, so the GPU's distances are the exact ones
    and every decision (ties included) must be the oracle's."""
    g = np.random.default_rng(seed)
    C = g.integers(-60, 61, size=(k, d))
    P = np.concatenate([c + g.integers(-spread, spread + 1, size=(per, d)) for c in C])
    return np.vstack([P, -P]).astype(np.float32)


@pytest.mark.parametrize("seed,form", [(3, None), (4, None), (6, None), (3, "shared"), (4, "global")])
def test_lap_refine_matches_oracle_exactly_on_integer_data(seed, form, monkeypatch):
    """The refinement against the oracle's, decision for decision: seeds whose
    medoid choices are all clear (two members at the same distance from the
    class mean in exact arithmetic may round apart differently under the two
    summation orders; the precondition is asserted).  On integer data every
    norm form of the top-2 GEMM (folded by default at this size, or the
    epilogue's shared or global norms) is exact."""
    if form:
        monkeypatch.setenv("APGB_ASSIGN_NORMS", form)
    X = _integer_clusters(seed, spread=5)
    n = X.shape[0]
    g = np.random.default_rng(50 + seed)
    E0 = g.choice(n, 90, replace=False)                      # about two centres per cluster
    p = -300.5                                                # half-integer: no cost ties the threshold
    E_ref, hist = olap.refine(X, E0, p, max_rounds=30)
    assert min(h["medoid_gap"] for h in hist) > 1e-9          # every medoid choice is clear
    E, idx, res = capi.lap_refine(torch.from_numpy(X).cuda(), torch.from_numpy(E0), p, rounds=30)
    E = E.cpu().numpy().astype(np.int64)
    assert np.array_equal(E, E_ref)
    assert res["rounds"] == len(hist)
    assert res["removed"] == sum(h["removed"] for h in hist)
    assert res["moved"] == sum(h["moved"] for h in hist)
    # final labels: nearest centre (exact distances, lowest index on ties); centres keep themselves
    X64 = X.astype(np.float64)
    D = ((X64[:, None, :] - X64[None, E_ref, :]) ** 2).sum(axis=2)
    lab = E_ref[np.argmin(D, axis=1)]
    lab[E_ref] = E_ref
    assert np.array_equal(idx.cpu().numpy().astype(np.int64), lab)
    dp = -D.min(axis=1)
    dp[E_ref] = 0.0
    assert res["netsim"] == pytest.approx(dp.sum() + p * E_ref.size, rel=1e-12)
    assert res["netsim"] >= hist[0]["netsim"]


def test_lap_refine_zero_rounds_is_the_assignment():
    X, _ = synth.workload(3, scale=0.005)
    E0 = np.random.default_rng(9).choice(X.shape[0], 300, replace=False)
    Xd = torch.from_numpy(X).cuda()
    E, idx, res = capi.lap_refine(Xd, torch.from_numpy(E0), -4000.0, rounds=0)
    assert res["rounds"] == 0 and res["n_exemplars"] == 300
    assert np.array_equal(E.cpu().numpy(), np.sort(E0))
    idx2 = capi.lap_assign(Xd, torch.from_numpy(np.sort(E0)))
    assert torch.equal(idx, idx2)


def test_lap_full_refinement_raises_netsim_on_the_landmark_workload():
    """Steps 1-4 on 30000 points of the 1e6-point generator: the gate leaves
    the outskirts of every class to Step 3, whose exemplars duplicate
    classes.  The refinement must not lower net similarity, must drop
    exemplars, and its labels must be the nearest of the final exemplars."""
    X, _ = synth.workload(3, scale=0.03)
    Xd = torch.from_numpy(X).cuda()
    kw = dict(seed=7, precision="bf16", damping=0.9, max_iter=1000, conv_iter=15)
    idx0, _, r0 = capi.lap_run_full(Xd, 6000, 6000, refine_rounds=0, **kw)
    idx1, _, r1 = capi.lap_run_full(Xd, 6000, 6000, refine_rounds=8, **kw)
    print(f"\nlap_run_full 30000 points: exemplars {r0['n_exemplars']} -> {r1['n_exemplars']}, "
          f"netsim {r0['netsim']:.6g} -> {r1['netsim']:.6g}, rounds {r1['refine_rounds']} "
          f"removed {r1['refine_removed']} moved {r1['refine_moved']}")
    assert r1["refine_rounds"] >= 1 and r1["refine_removed"] > 0
    assert r1["n_exemplars"] < r0["n_exemplars"]
    assert r1["netsim"] > r0["netsim"]
    labels = idx1.cpu().numpy().astype(np.int64)
    E = np.unique(labels)
    assert E.size == r1["n_exemplars"]
    frac_clear, _ = _check_assignment(X, E, labels)
    assert frac_clear > 0.95


def test_lap_refine_single_centre_only_moves_to_the_medoid():
    """One centre: nothing can be dropped (no second centre), so the
    refinement only moves the centre to the member nearest the mean of all
    points; the oracle's choice, with every point labelled by it."""
    X = _integer_clusters(8, k=1, per=40, d=8, spread=9)
    E0 = np.array([3])
    E_ref, hist = olap.refine(X, E0, -50.0, max_rounds=10)
    E, idx, res = capi.lap_refine(torch.from_numpy(X).cuda(), torch.from_numpy(E0), -50.0, rounds=10)
    assert np.array_equal(E.cpu().numpy(), E_ref) and E_ref.size == 1
    assert res["removed"] == 0 and res["moved"] == sum(h["moved"] for h in hist)
    assert np.all(idx.cpu().numpy() == E_ref[0])
