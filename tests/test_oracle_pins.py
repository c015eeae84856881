"""Pins of the float64 oracle against facts that do not come from the oracle:
a hand-worked iteration, published generator vectors, library routines,
closed forms, invariants of Eq. 2-4 and brute-force optima."""
import itertools
import json
import os

import numpy as np
import pytest
from scipy.spatial.distance import cdist

from oracle import ap, lap, pap, rng
from paper_0910_1650_gb300 import synth


def _load(golden_dir, name):
    with open(os.path.join(golden_dir, name)) as f:
        return json.load(f)


def _rand_S(n, seed, ties=False, asym=True):
    g = np.random.default_rng(seed)
    if ties:
        S = -g.integers(0, 6, size=(n, n)).astype(np.float64)
    else:
        S = -g.random((n, n)) * 10
    if not asym:
        S = 0.5 * (S + S.T)
    np.fill_diagonal(S, np.median(S[~np.eye(n, dtype=bool)]))
    return S


def _separated(n_per=3, n_clusters=3, seed=0, sep=30.0, spread=1.0, d=2):
    g = np.random.default_rng(seed)
    centres = g.normal(size=(n_clusters, d)) * sep
    X = np.concatenate([c + g.normal(size=(n_per, d)) * spread for c in centres])
    return X, np.repeat(np.arange(n_clusters), n_per)


# --- generator ----------------------------------------------------------------

def test_splitmix64_published_vectors(golden_dir):
    g = _load(golden_dir, "splitmix64_vectors.json")
    got = [rng.output(g["seed"], n) for n in range(1, 6)]
    assert got == [int(v) for v in g["outputs"]]
    vec = rng.outputs(g["seed"], np.arange(1, 6, dtype=np.uint64))
    assert [int(v) for v in vec] == [int(v) for v in g["outputs"]]


def test_unit_interval_range():
    u = rng.unit_interval(7, np.arange(1, 100001, dtype=np.uint64))
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 0.01


# --- one iteration worked by hand (Eq. 2, 3, 4) ---------------------------------

@pytest.mark.parametrize("literal", [True, False])
def test_hand_example_one_iteration(golden_dir, literal):
    g = _load(golden_dir, "ap_three_points_by_hand.json")
    S = np.array(g["S"], dtype=np.float64)
    Z = np.zeros((3, 3))
    R, A = ap.iterate_once(S, Z, Z, 0.0, literal=literal)
    assert np.array_equal(R, np.array(g["R"], dtype=np.float64))
    assert np.array_equal(A, np.array(g["A"], dtype=np.float64))
    assert list(ap.decisions(R, A)) == g["decisions"]
    ex = ap.exemplars(S, R, A)
    assert list(ex["idx"]) == g["idx"]
    assert (ex["dpsim"], ex["expref"], ex["netsim"]) == (g["dpsim"], g["expref"], g["netsim"])


def test_hand_example_damping_order(golden_dir):
    g = _load(golden_dir, "ap_three_points_by_hand.json")
    S = np.array(g["S"], dtype=np.float64)
    Z = np.zeros((3, 3))
    R, A = ap.iterate_once(S, Z, Z, 0.5)
    assert np.array_equal(R, np.array(g["R"]) / 2.0)
    assert np.array_equal(A, np.array(g["A"]) / 4.0)


# --- the two statements of Eq. 2-4 agree ---------------------------------------

@pytest.mark.parametrize("n,ties,seed", [(7, True, 1), (12, False, 2), (20, True, 3), (25, False, 4)])
def test_literal_equals_top2_form(n, ties, seed):
    S = _rand_S(n, seed, ties=ties)
    a = ap.run(S, lam=0.5, fixed_iters=6, literal=True)
    b = ap.run(S, lam=0.5, fixed_iters=6, literal=False)
    scale = np.abs(S).max()
    assert np.abs(a["R"] - b["R"]).max() <= 1e-12 * scale
    assert np.abs(a["A"] - b["A"]).max() <= 1e-12 * scale


def test_literal_equals_top2_form_nonzero_start():
    S = _rand_S(15, 9)
    g = np.random.default_rng(3)
    R0 = g.normal(size=S.shape)
    A0 = -np.abs(g.normal(size=S.shape))
    a = ap.run(S, lam=0.7, fixed_iters=3, literal=True, R0=R0, A0=A0)
    b = ap.run(S, lam=0.7, fixed_iters=3, literal=False, R0=R0, A0=A0)
    assert np.abs(a["R"] - b["R"]).max() <= 1e-12 * 10
    assert np.abs(a["A"] - b["A"]).max() <= 1e-12 * 10


# --- invariants -----------------------------------------------------------------

def test_availability_signs_every_iteration():
    S = _rand_S(40, 5)
    n = S.shape[0]
    R = np.zeros_like(S)
    A = np.zeros_like(S)
    off = ~np.eye(n, dtype=bool)
    for _ in range(30):
        R, A = ap.iterate_once(S, R, A, 0.5)
        assert (A[off] <= 0).all()
        assert (np.diag(A) >= 0).all()


def test_responsibility_undamped_row_structure():
    S = _rand_S(30, 6)
    A = -np.abs(np.random.default_rng(1).normal(size=S.shape))
    Rn = ap.responsibility(S, A)
    m1, j1, m2 = ap.row_top2(A + S)
    T = A + Rn
    n = S.shape[0]
    assert np.allclose(T[np.arange(n), j1], m1 - m2, rtol=0, atol=1e-12)
    assert (T[np.arange(n), j1] >= 0).all()
    mask = np.ones_like(T, dtype=bool)
    mask[np.arange(n), j1] = False
    assert (T[mask] <= 1e-12).all()


def test_positive_scaling():
    S = _rand_S(30, 7)
    a = ap.run(S, lam=0.5, fixed_iters=12)
    b = ap.run(3.0 * S, lam=0.5, fixed_iters=12)
    assert np.allclose(b["R"], 3.0 * a["R"], rtol=0, atol=1e-10)
    assert np.allclose(b["A"], 3.0 * a["A"], rtol=0, atol=1e-10)
    assert np.array_equal(ap.exemplar_mask(a["R"], a["A"]), ap.exemplar_mask(b["R"], b["A"]))


def test_row_shift_invariance():
    S = _rand_S(30, 8)
    c = np.random.default_rng(2).normal(size=(30, 1)) * 5
    a = ap.run(S, lam=0.5, fixed_iters=12)
    b = ap.run(S + c, lam=0.5, fixed_iters=12)
    assert np.allclose(a["R"], b["R"], atol=1e-10)
    assert np.allclose(a["A"], b["A"], atol=1e-10)


def test_permutation_equivariance():
    S = _rand_S(30, 9)
    p = np.random.default_rng(4).permutation(30)
    a = ap.run(S, lam=0.5, fixed_iters=12)
    b = ap.run(S[np.ix_(p, p)], lam=0.5, fixed_iters=12)
    assert np.allclose(b["R"], a["R"][np.ix_(p, p)], atol=1e-12)
    assert np.allclose(b["A"], a["A"][np.ix_(p, p)], atol=1e-12)


# --- convergence, fixed point, outputs ----------------------------------------------

def _separated_S(seed=0, n_per=4, n_clusters=3):
    X, lab = _separated(n_per=n_per, n_clusters=n_clusters, seed=seed)
    S, p = ap.build_similarity(X)
    return X, lab, S


def test_fixed_point_after_convergence():
    _, _, S = _separated_S(1, n_per=8, n_clusters=4)
    res = ap.run(S, lam=0.5, max_iter=2000, convits=2000)
    dr, da = ap.undamped_residuals(S, res["R"], res["A"])
    scale = np.abs(S).max()
    assert dr <= 1e-6 * scale and da <= 1e-6 * scale


def test_termination_rule():
    _, _, S = _separated_S(2, n_per=6)
    res = ap.run(S, lam=0.5, max_iter=200, convits=15)
    assert res["converged"] and res["iters"] >= 15
    masks = []
    R = np.zeros_like(S)
    A = np.zeros_like(S)
    for _ in range(res["iters"]):
        R, A = ap.iterate_once(S, R, A, 0.5)
        masks.append(ap.exemplar_mask(R, A))
    last = masks[-15:]
    assert all(np.array_equal(m, last[0]) for m in last) and last[0].any()
    # one iteration earlier the rule did not yet hold
    prev = masks[-16:-1]
    assert not (all(np.array_equal(m, prev[0]) for m in prev) and prev[0].any())
    assert np.array_equal(R, res["R"]) and np.array_equal(A, res["A"])


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_brute_force_optimum_small(seed):
    _, _, S = _separated_S(seed, n_per=3, n_clusters=3)
    res = ap.run(S, lam=0.5, max_iter=500, convits=30)
    ex = ap.exemplars(S, res["R"], res["A"])
    bestE, best = ap.brute_force_best(S)
    assert np.array_equal(ex["E"], bestE)
    assert abs(ex["netsim"] - best) <= 1e-9 * abs(best)


def test_exemplar_self_consistency_and_energy():
    X, lab, S = _separated_S(5, n_per=10, n_clusters=5)
    res = ap.run(S, lam=0.5)
    ex = ap.exemplars(S, res["R"], res["A"])
    E = ex["E"]
    idx = ex["idx"]
    assert E.size > 0
    assert np.array_equal(idx[E], E)
    nonex = np.setdiff1d(np.arange(S.shape[0]), E)
    assert np.isin(idx[nonex], E).all()
    assert np.allclose(S[nonex, idx[nonex]], S[np.ix_(nonex, E)].max(axis=1))
    # netsim = -E(c) with s(k,k) = p for exemplars (energy of Section 2)
    energy = -sum(S[i, idx[i]] for i in range(S.shape[0]))
    assert abs(ex["netsim"] - (-energy)) <= 1e-9 * abs(energy)
    assert abs(ex["netsim"] - ap.netsim_of_labels(S, idx)) <= 1e-9 * abs(energy)
    # separated clusters: one exemplar per true cluster
    assert len(set(lab[E])) == 5 and E.size == 5


def test_no_exemplar_output():
    S = np.array([[-100.0, -1.0], [-1.0, -100.0]])
    R = np.zeros((2, 2))
    A = np.array([[-5.0, 0.0], [0.0, -5.0]])   # a+r picks the other point
    ex = ap.exemplars(S, R, A)
    assert (ex["idx"] == -1).all() and np.isnan(ex["netsim"])


# --- similarity, preference, noise --------------------------------------------------

def test_similarity_closed_form_line():
    x = np.array([[0.0], [1.0], [3.0], [-2.0]])
    S = ap.similarity(x)
    want = -np.array([[(a - b) ** 2 for b in x[:, 0]] for a in x[:, 0]])
    assert np.array_equal(S, want)


def test_similarity_vs_scipy():
    X = np.random.default_rng(0).normal(size=(50, 7)).astype(np.float32)
    assert np.allclose(ap.similarity(X), -cdist(X.astype(np.float64), X.astype(np.float64), "sqeuclidean"),
                       rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("n", [2, 3, 10, 11])
def test_offdiag_median_vs_numpy(n):
    S = np.random.default_rng(n).normal(size=(n, n))
    off = S[~np.eye(n, dtype=bool)]
    assert ap.offdiag_median(S) == float(np.median(off))


def test_offdiag_median_by_hand():
    S = np.array([[9.0, 1.0, 2.0], [3.0, 9.0, 4.0], [5.0, 6.0, 9.0]])
    assert ap.offdiag_median(S) == 3.5          # values 1..6: mean of 3 and 4


def test_similarity_gram_vs_explicit_differences():
    """The expanded form used at large N against scipy's squared distances
    (an independent routine) and the explicit differences: equal to rounding,
    zero diagonal, never positive (two coincident points give exactly 0)."""
    g = np.random.default_rng(5)
    X = (g.normal(size=(300, 64)) * 3 + 10).astype(np.float32)
    X[17] = X[3]                                     # coincident points
    Sg = ap.similarity_gram(X)
    ref = -cdist(X.astype(np.float64), X.astype(np.float64), "sqeuclidean")
    scale = np.abs(ref).max()
    assert np.abs(Sg - ref).max() <= 1e-12 * scale
    assert np.abs(Sg - ap.similarity(X)).max() <= 1e-12 * scale
    assert (np.diag(Sg) == 0).all() and (Sg <= 0).all()
    assert Sg[3, 17] == 0.0 and Sg[17, 3] == 0.0


@pytest.mark.parametrize("n", [2, 3, 10, 11, 64])
def test_offdiag_median_select_equals_sorted_median(n):
    g = np.random.default_rng(100 + n)
    S = g.normal(size=(n, n))
    assert ap.offdiag_median_select(S) == ap.offdiag_median(S)
    T = np.round(S * 2) / 2                          # many ties
    assert ap.offdiag_median_select(T) == ap.offdiag_median(T)
    assert ap.offdiag_median_select(T) == float(np.median(T[~np.eye(n, dtype=bool)]))


def test_tiebreak_noise_magnitude():
    X, _ = _separated(n_per=5, seed=1)
    S0, p = ap.build_similarity(X)
    S1, _ = ap.build_similarity(X, noise_rel=1e-6, seed=11)
    d = S1 - S0
    assert (d >= 0).all()                          # rel*|s|*u is never negative
    assert (np.abs(d) <= 1e-6 * np.abs(S0) + 1e-300).all()
    u = ap.tiebreak_noise(S0.shape[0], S0.shape[1], 11)
    # S1 - S0 cancels: compare to within a few ulps of S0
    assert (np.abs(d - 1e-6 * np.abs(S0) * u) <= 4 * np.finfo(float).eps * np.abs(S0)).all()
    assert u[0, 0] == rng.unit_interval(11, np.array([1], dtype=np.uint64))[0]


# --- Algorithm 2 (PAP) -------------------------------------------------------------

@pytest.mark.parametrize("n,k", [(100, 4), (1000, 4), (2021, 16), (7, 3), (10, 1)])
def test_equal_partition_rule(n, k):
    off = pap.equal_partition(n, k)
    sizes = np.diff(off)
    m = n // k
    assert len(sizes) == k and off[0] == 0 and off[-1] == n
    assert (sizes[:-1] == m).all() and sizes[-1] == n - m * (k - 1)


def test_block_count_bound():
    assert pap.block_count_bound_ok(2021, 4, 86) is True      # 4 < 2021/344
    assert pap.block_count_bound_ok(2021, 8, 86) is False     # Table 2's k=8 lies outside
    assert pap.block_count_bound_ok(60000, 32, 50) is True
    assert pap.block_count_bound_ok(60000, 1, 50) is False


def test_merge_is_block_diagonal():
    off = np.array([0, 2, 5, 6])
    blocks = [np.full((2, 2), 1.0), np.full((3, 3), 2.0), np.full((1, 1), 3.0)]
    Ap = pap.merge_blocks(6, off, blocks)
    want = np.zeros((6, 6))
    want[0:2, 0:2] = 1
    want[2:5, 2:5] = 2
    want[5, 5] = 3
    assert np.array_equal(Ap, want)


def test_pap_step4_from_zero_is_plain_ap():
    _, _, S = _separated_S(3, n_per=6, n_clusters=4)
    a = ap.run(S, lam=0.5)
    b = ap.run(S, lam=0.5, R0=np.zeros_like(S), A0=pap.merge_blocks(S.shape[0], [0, S.shape[0]],
                                                                      [np.zeros_like(S)]))
    assert np.array_equal(a["R"], b["R"]) and a["iters"] == b["iters"]


def test_pap_single_block_subrun_is_plain_ap():
    _, _, S = _separated_S(4, n_per=5, n_clusters=3)
    r = pap.run(S, [0, S.shape[0]], lam=0.5)
    a = ap.run(S, lam=0.5)
    assert np.array_equal(r["sub"][0]["A"], a["A"])


def test_pap_netsim_close_to_ap():
    g = np.random.default_rng(11)
    centres = g.uniform(-10, 10, size=(5, 2))
    X = np.concatenate([c + g.normal(size=(40, 2)) for c in centres])
    X = X[g.permutation(len(X))]
    S, _ = ap.build_similarity(X)
    a = ap.run(S, lam=0.5, max_iter=500)
    ea = ap.exemplars(S, a["R"], a["A"])
    r = pap.run(S, pap.equal_partition(S.shape[0], 4), lam=0.5, max_iter=500)
    er = ap.exemplars(S, r["final"]["R"], r["final"]["A"])
    # Section 3: PAP's result matches plain AP's or improves on it
    assert er["netsim"] >= ea["netsim"] * (1 + 0.005)


# --- Algorithm 3 (LAP) -------------------------------------------------------------

def test_uniform_landmarks():
    lm = lap.uniform_landmarks(1000, 100, 5)
    assert lm.size == 100 and np.unique(lm).size == 100
    assert (np.diff(lm) > 0).all() and lm.max() < 1000
    assert np.array_equal(lm, lap.uniform_landmarks(1000, 100, 5))
    assert not np.array_equal(lm, lap.uniform_landmarks(1000, 100, 6))


def test_lap_all_points_as_landmarks_is_ap():
    X, _ = _separated(n_per=8, n_clusters=4, seed=7)
    r = lap.run(X, np.arange(X.shape[0]), lam=0.5)
    S, _ = ap.build_similarity(X)
    a = ap.run(S, lam=0.5)
    ea = ap.exemplars(S, a["R"], a["A"])
    assert np.array_equal(r["E"], ea["E"])
    assert np.array_equal(r["idx"], ea["idx"])
    assert abs(r["netsim"] - ea["netsim"]) <= 1e-9 * abs(ea["netsim"])


def test_lap_assignment_brute_force():
    g = np.random.default_rng(3)
    X = g.normal(size=(60, 3))
    C = g.normal(size=(7, 3))
    near = lap.nearest_exemplar(X, C)
    for i in range(60):
        d = [sum((X[i, j] - C[c, j]) ** 2 for j in range(3)) for c in range(7)]
        assert near[i] == int(np.argmin(d))


# --- the pins catch plausible mistakes planted in copies of the oracle ---------------

def _mutant_iterations():
    def rho_m1_everywhere(S, A):            # forgets the k == argmax case of Eq. 2
        return S - (A + S).max(axis=1, keepdims=True)

    def alpha_no_rkk(R):                     # drops r(k,k) in Eq. 3
        colp, _ = ap.column_sums(R)
        P = np.maximum(R, 0.0)
        A = np.minimum(0.0, colp[None, :] - P)
        np.fill_diagonal(A, colp)
        return A

    def alpha_transposed(R):                 # sums rows instead of columns
        return ap.availability(R.T).T

    def alpha_keeps_own_term(R):             # forgets to exclude i' = i in Eq. 3
        colp, rkk = ap.column_sums(R)
        A = np.minimum(0.0, rkk[None, :] + colp[None, :] + 0 * R)
        np.fill_diagonal(A, colp)
        return A

    def alpha_diag_includes_self(R):         # Eq. 4 summed over all i'
        A = ap.availability(R)
        np.fill_diagonal(A, np.maximum(R, 0).sum(axis=0))
        return A

    def damp_a_first(S, R, A, lam):          # A from the undamped R
        Rn = ap.responsibility(S, A)
        An = ap.availability(Rn)
        return lam * R + (1 - lam) * Rn, lam * A + (1 - lam) * An

    def std(rho=ap.responsibility, alpha=ap.availability):
        def it(S, R, A, lam):
            R = lam * R + (1 - lam) * rho(S, A)
            return R, lam * A + (1 - lam) * alpha(R)
        return it

    return {
        "rho_m1_everywhere": std(rho=rho_m1_everywhere),
        "alpha_no_rkk": std(alpha=alpha_no_rkk),
        "alpha_transposed": std(alpha=alpha_transposed),
        "alpha_keeps_own_term": std(alpha=alpha_keeps_own_term),
        "alpha_diag_includes_self": std(alpha=alpha_diag_includes_self),
        "damp_a_first": damp_a_first,
    }


@pytest.mark.parametrize("name", sorted(_mutant_iterations()))
def test_hand_pins_catch_planted_mistake(golden_dir, name):
    g = _load(golden_dir, "ap_three_points_by_hand.json")
    S = np.array(g["S"], dtype=np.float64)
    Z = np.zeros((3, 3))
    it = _mutant_iterations()[name]
    R0, A0 = it(S, Z, Z, 0.0)
    R5, A5 = it(S, Z, Z, 0.5)
    hand_ok = (np.array_equal(R0, np.array(g["R"], float)) and np.array_equal(A0, np.array(g["A"], float))
               and np.array_equal(R5, np.array(g["R"]) / 2.0) and np.array_equal(A5, np.array(g["A"]) / 4.0))
    # the literal statement of Eq. 2-4 is the second, independent pin
    Sr = _rand_S(12, 21)
    np.fill_diagonal(Sr, -0.01)      # high preferences: some r(k,k) > 0
    lit = ap.run(Sr, lam=0.5, fixed_iters=6, literal=True)
    R = np.zeros_like(Sr)
    A = np.zeros_like(Sr)
    for _ in range(6):
        R, A = it(Sr, R, A, 0.5)
    literal_ok = np.abs(R - lit["R"]).max() <= 1e-9 and np.abs(A - lit["A"]).max() <= 1e-9
    assert not (hand_ok and literal_ok)


def test_float32_transient_amplification():
    """Why the float32 parity points of the 500-point mixture at lambda=0.5 avoid
    t ~ 20..60: there the iteration is ill-conditioned and the same updates in
    float32 drift from float64 by more than 1e-3, then contract again."""
    from paper_0910_1650_gb300 import synth
    X, _ = synth.gaussian_mixture_2d()
    S32 = ap.build_similarity(X)[0].astype(np.float32)
    S64 = S32.astype(np.float64)
    R32 = np.zeros_like(S32)
    A32 = np.zeros_like(S32)
    R64 = np.zeros_like(S64)
    A64 = np.zeros_like(S64)
    err = {}
    for t in range(1, 101):
        R32, A32 = ap.iterate_once(S32, R32, A32, np.float32(0.5))
        R64, A64 = ap.iterate_once(S64, R64, A64, 0.5)
        if t in (10, 50, 100):
            err[t] = np.abs(R32 - R64).max() / np.abs(R64).max()
    assert err[10] < 1e-5 and err[50] > 1e-3 and err[100] < 1e-5


def test_lambda05_mixture_is_ill_conditioned_in_S():
    """A 1e-7 relative perturbation of S (the centred float32 norm form of the
    same distances) changes the exemplar set reached at lambda=0.5 but not at
    lambda=0.9 -- why end-to-end parity at lambda=0.5 checks quality, not
    identity."""
    from paper_0910_1650_gb300 import synth
    X, _ = synth.gaussian_mixture_2d()
    n = X.shape[0]
    mean = X.astype(np.float64).mean(axis=0).astype(np.float32)
    Xc = (X - mean).astype(np.float32)
    nrm = (Xc * Xc).sum(axis=1, dtype=np.float32)
    Sg = np.minimum(np.float32(2) * (Xc @ Xc.T) - nrm[:, None] - nrm[None, :],
                    np.float32(0)).astype(np.float64)
    Sg = ap.set_preference(Sg, np.float32(ap.offdiag_median(Sg)))
    S64, _ = ap.build_similarity(X)
    off = ~np.eye(n, dtype=bool)
    assert (np.abs(Sg - S64)[off] / np.abs(S64).max()).max() < 1e-6
    E = {}
    for nm, S in (("g", Sg), ("d", S64)):
        for lam, mi in ((0.5, 200), (0.9, 1000)):
            r = ap.run(S, lam=lam, max_iter=mi)
            E[nm, lam] = tuple(ap.exemplars(S, r["R"], r["A"])["E"])
    assert E["g", 0.5] != E["d", 0.5]
    assert E["g", 0.9] == E["d", 0.9]


# --- bf16 rounding used to state the tensor-core similarity's inputs ----------------

def test_round_bf16_hand_values():
    vals = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, 1.0 + 2 ** -7, -2.5, 0.0, 65504.0],
                    dtype=np.float32)
    # 1 + 2^-8 is halfway between 1 and 1 + 2^-7: ties go to the even mantissa (1.0);
    # 1 + 3*2^-8 is halfway between 1 + 2^-7 and 1 + 2^-6: even is 1 + 2^-6
    want = np.array([1.0, 1.0, 1.0 + 2 ** -6, 1.0 + 2 ** -7, -2.5, 0.0, 65536.0], dtype=np.float32)
    assert np.array_equal(ap.round_bf16(vals), want)


def test_round_bf16_vs_torch():
    torch = pytest.importorskip("torch")
    x = (np.random.default_rng(3).normal(size=20000) * 100).astype(np.float32)
    want = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    assert np.array_equal(ap.round_bf16(x), want)


def test_centring_preserves_distances():
    X = np.random.default_rng(4).normal(size=(40, 5)).astype(np.float32) + 100
    assert np.allclose(ap.similarity(ap.centred(X)), ap.similarity(X), rtol=1e-5, atol=1e-3)


# ---- Algorithm 3 Steps 1-4 (oracle.lap.run_full) ----------------------------------------

def _far_group_data(seed=0):
    g = np.random.default_rng(seed)
    A = g.normal(size=(200, 2))
    far = np.array([1000.0, 1000.0]) + 0.1 * g.normal(size=(5, 2))
    return np.vstack([A, far]).astype(np.float32)


def test_lap_full_every_point_a_landmark_is_ap():
    """L = n: Step 1 is Algorithm 1 on all points, the gate keeps every point
    (all are landmarks), Step 4 is the nearest-exemplar assignment, which at
    convergence is AP's own assignment."""
    X = synth.gaussian_mixture(120, 2, 4, 5, 8.0, 1.0)[0]
    full = lap.run_full(X, 120, seed=3, m0=50, lam=0.9, max_iter=1000, convits=15)
    S, p = ap.build_similarity(X)
    res = ap.run(S, 0.9, 1000, 15)
    ex = ap.exemplars(S, res["R"], res["A"])
    assert full["levels"][0]["unassigned"].size == 0 and len(full["levels"]) == 1
    assert np.array_equal(full["E"], ex["E"])
    assert np.array_equal(full["idx"], ex["idx"])


def test_lap_full_one_level_equals_steps_1_2_on_separated_data():
    X = synth.gaussian_mixture(600, 3, 6, 9, 20.0, 0.5, False)[0]
    lm = lap.uniform_landmarks(600, 150, 21)
    a = lap.run(X, lm, lam=0.9, max_iter=1000, convits=15)
    b = lap.run_full(X, 150, seed=21, m0=600, lam=0.9, max_iter=1000, convits=15, max_levels=1)
    assert np.array_equal(a["E"], b["E"])
    assert np.array_equal(a["idx"], b["idx"])
    assert abs(a["netsim"] - b["netsim"]) <= 1e-9 * abs(a["netsim"])


def test_lap_full_gate_gives_unreached_points_their_own_exemplar():
    """A tight group far from every landmark class fails Step 2's gate; Step 3
    (Algorithm 1 on the points left) makes an exemplar among them, where
    Steps 1-2 alone would have labelled them with a far-away exemplar."""
    X = _far_group_data()
    n = X.shape[0]
    seed = next(s for s in range(100)
                if not np.isin(np.arange(200, 205), lap.uniform_landmarks(n, 40, s)).any())
    # damping 0.5 (the paper's): at 0.9 the stop rule can fire on the points
    # left before their messages have grown (decisions constant from t = 1)
    full = lap.run_full(X, 40, seed=seed, m0=100, lam=0.5, max_iter=1000, convits=15)
    un0 = full["levels"][0]["unassigned"]
    assert set(range(200, 205)) <= set(un0.tolist())
    far_labels = full["idx"][200:205]
    assert np.all(far_labels >= 200)                  # an exemplar of the far group
    plain = lap.run(X, lap.uniform_landmarks(n, 40, seed), lam=0.5, max_iter=1000, convits=15)
    assert np.all(plain["idx"][200:205] < 200)        # Steps 1-2 alone: a far-away exemplar
    assert full["netsim"] > plain["netsim"]


def test_lap_full_recursion_when_m_exceeds_m0():
    """m0 below the number of points left forces Step 3's recursive branch:
    a second level of Steps 1-2 on the points left."""
    X = _far_group_data(1)
    n = X.shape[0]
    seed = next(s for s in range(100)
                if not np.isin(np.arange(200, 205), lap.uniform_landmarks(n, 40, s)).any())
    full = lap.run_full(X, 40, seed=seed, m0=2, lam=0.5, max_iter=1000, convits=15)
    assert len(full["levels"]) >= 2 and full["levels"][0]["unassigned"].size > 2
    assert np.all(full["idx"][200:205] >= 200)
    # every label is an exemplar of the merged set, and exemplars label themselves
    assert set(np.unique(full["idx"]).tolist()) == set(full["E"].tolist())
    assert np.all(full["idx"][full["E"]] == full["E"])


def test_pap_carry_r_single_block_continues_the_run():
    """With one block, carrying R and A into Step 4 continues the same run:
    t sub-iterations then t Step-4 iterations equal 2t plain iterations
    (the iteration is a map of (R, A) alone)."""
    g = np.random.default_rng(12)
    S, _ = ap.build_similarity(g.normal(size=(40, 3)))
    n = S.shape[0]
    t = 9
    two = pap.run(S, [0, n], lam=0.7, fixed_iters=t, carry_r=True)
    straight = ap.run(S, 0.7, fixed_iters=2 * t)
    assert np.allclose(two["final"]["R"], straight["R"], rtol=0, atol=1e-12 * np.abs(S).max())
    assert np.allclose(two["final"]["A"], straight["A"], rtol=0, atol=1e-12 * np.abs(S).max())
    # without carrying R the paper's Step 4 restarts R from 0 and does not continue the run
    one = pap.run(S, [0, n], lam=0.7, fixed_iters=t)
    assert not np.allclose(one["final"]["R"], straight["R"], rtol=0, atol=1e-6 * np.abs(S).max())


# ---- Algorithm 3 Step 4: the refinement (local search on net similarity) -----------------

def _integer_points(n_half, seed, spread=20):
    """Integer points symmetric about the origin: their column mean is exactly
    zero and every coordinate is exact in bf16, so the refinement's rounded
    distances are the exact squared distances."""
    g = np.random.default_rng(seed)
    P = g.integers(-spread, spread + 1, size=(n_half, 2)).astype(np.float32)
    return np.vstack([P, -P])


def _netsim_exact(X, E, p):
    X = X.astype(np.float64)
    D = ((X[:, None, :] - X[None, E, :]) ** 2).sum(axis=2)
    d = D.min(axis=1)
    d[E] = 0.0
    return -d.sum() + p * len(E)


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_refine_reaches_a_brute_force_local_optimum(seed):
    """At convergence no single centre's removal raises netsim (checked by
    recomputing netsim without it) and every centre minimises its class's
    summed squared distance over the class's members (checked by direct
    sums, not through the class mean); netsim never falls from round to
    round."""
    X = _integer_points(20, seed)
    n = X.shape[0]
    g = np.random.default_rng(100 + seed)
    E0 = np.sort(g.choice(n, 12, replace=False))
    p = -150.0
    E, hist = lap.refine(X, E0, p, max_rounds=100)
    assert hist[-1]["removed"] == 0 and hist[-1]["moved"] == 0          # converged
    ns = [h["netsim"] for h in hist]
    assert all(b >= a - 1e-9 for a, b in zip(ns, ns[1:]))
    assert ns[-1] == pytest.approx(_netsim_exact(X, E, p), abs=1e-9)
    base = _netsim_exact(X, E, p)
    for e in E:
        rest = E[E != e]
        if rest.size:
            assert _netsim_exact(X, rest, p) <= base + 1e-9
    X64 = X.astype(np.float64)
    D = ((X64[:, None, :] - X64[None, E, :]) ** 2).sum(axis=2)
    cls = D.argmin(axis=1)
    for j, e in enumerate(E):
        members = np.nonzero(cls == j)[0]
        sums = [((X64[members] - X64[k]) ** 2).sum() for k in members]
        best = members[int(np.argmin(sums))]
        assert e == best


def test_refine_drops_a_duplicate_centre_and_keeps_separated_ones():
    """Four far clusters (mirrored pairs, for an exact zero mean), one centre
    each plus a second centre in the first: the duplicate goes (merging its
    class costs far less than -p), every cluster keeps one centre."""
    g = np.random.default_rng(5)
    A = np.round(g.normal(size=(30, 2)) * 2) + np.array([50.0, 0.0])
    B = np.round(g.normal(size=(30, 2)) * 2) + np.array([0.0, 100.0])
    X = np.vstack([A, B, -A, -B]).astype(np.float32)
    E0 = np.array([0, 1, 30, 60, 90])
    E, hist = lap.refine(X, E0, -400.0, max_rounds=20)
    assert E.size == 4
    assert [int(((E >= 30 * q) & (E < 30 * q + 30)).sum()) for q in range(4)] == [1, 1, 1, 1]
    assert hist[0]["removed"] == 1


def test_refine_conflicting_candidates_drop_only_one():
    """Two centres of one tight group, each the other's members' second
    choice, both cheap to drop (the same for a mirrored group): dropping both
    would send the group to a far centre.  Only one of each pair goes, and
    netsim rises."""
    half = np.array([[20, 20], [21, 20], [20, 21], [21, 21], [60, -60], [61, -60]], dtype=np.float32)
    X = np.vstack([half, -half])
    E0 = np.array([0, 3, 4, 6, 9, 10])
    p = -30.0
    E, hist = lap.refine(X, E0, p, max_rounds=20)
    assert hist[0]["removed"] == 2
    assert ((E < 4).sum(), ((E >= 6) & (E < 10)).sum()) == (1, 1)
    assert _netsim_exact(X, E, p) > _netsim_exact(X, E0, p)


def test_refine_moves_a_centre_to_its_class_medoid():
    """One class on a line, x = 0, 1, 2, 3, 10 (mirrored for a zero mean, the
    mirror a second class): the mean is 3.2, so the member nearest it, 3, is
    the centre that minimises the class's summed squared distance."""
    xs = np.array([0, 1, 2, 3, 10], dtype=np.float32) + 200.0
    X = np.zeros((10, 2), dtype=np.float32)
    X[:5, 0] = xs
    X[5:, 0] = -xs
    E, hist = lap.refine(X, np.array([4, 9]), -10.0, max_rounds=10)
    assert list(E) == [3, 8]
    assert hist[0]["moved"] == 2 and hist[0]["removed"] == 0


def test_lap_full_refinement_does_not_lower_netsim():
    """Steps 1-4 with the refinement against Steps 1-4 with reassignment
    only, on a mixture whose Step 3 adds exemplars inside existing classes:
    at least as good a net similarity with no more exemplars."""
    X, _ = synth.gaussian_mixture(600, 8, 6, 4242, 6.0, 1.0)
    plain = lap.run_full(X, 80, 3, 400, lam=0.9, max_iter=1000, convits=15)
    ref = lap.run_full(X, 80, 3, 400, lam=0.9, max_iter=1000, convits=15, refine_rounds=8)
    assert ref["E"].size <= plain["E"].size
    assert ref["netsim"] >= plain["netsim"] - 1e-6 * abs(plain["netsim"])
