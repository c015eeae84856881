"""Pins of the float64 warm-start network: gradients against central finite
differences, Adam against its closed-form first step, features against a
hand-checked row, and the parameter layout."""
import numpy as np
import pytest

from oracle import ap, mlp
from paper_0910_1650_gb300 import synth


def _problem(seed=0, n=40):
    g = np.random.default_rng(seed)
    X = g.normal(size=(n, 3))
    S, p = ap.build_similarity(X)
    return S, abs(p)


def test_parameter_count_and_layout():
    assert mlp.NP == 256 * 25 + 256 + 256 * 256 + 256 + 3 * 256 + 3 + 2 * 25
    P = synth.mlp_init()
    assert P.size == mlp.NP
    d = mlp.unpack(P)
    assert np.all(d["b1"] == 0) and np.all(d["b3"] == 0)
    assert abs(d["W2"].std() - np.sqrt(2.0 / 256)) < 0.01
    assert np.array_equal(mlp.pack(d), P.astype(np.float64))


def test_features_hand_row():
    S = np.array([[-5.0, -1.0, -9.0], [-1.0, -5.0, -4.0], [-9.0, -4.0, -5.0]])
    F = mlp.row_features(S, 5.0)
    # row 0: off-diagonal -1, -9 -> top values -1, -9, then padded with -9
    assert F[0, 0] == -0.2 and F[0, 1] == -1.8 and np.all(F[0, 2:16] == -1.8)
    assert F[0, 16] == -1.0                      # mean of -1, -9 is -5, over 5
    assert abs(F[0, 17] - 0.8) < 1e-15           # std of -1, -9 is 4, over 5
    assert F[0, 18] == -1.0


def test_density_features_hand_example():
    """Four points on a line at 0, 1, 2, 10 (s = -squared distance), scale 8:
    thresholds -1, -2, -4, -8.  Counts, neighbour lists and density
    contrasts worked out by hand."""
    x = np.array([0.0, 1.0, 2.0, 10.0])
    S = -(x[:, None] - x[None, :]) ** 2
    np.fill_diagonal(S, -30.0)
    F = mlp.row_features(S, 8.0)
    l = np.log1p
    counts = {0: (1, 1, 2, 2), 1: (2, 2, 2, 2), 2: (1, 1, 2, 2), 3: (0, 0, 0, 0)}
    for k, c in counts.items():
        assert np.allclose(F[k, 19:23], l(np.array(c, dtype=float)), rtol=0, atol=1e-15)
    D = [l(1), l(2), l(1), l(0)]
    assert abs(F[0, 23] - (D[0] - D[1])) < 1e-15 and F[0, 24] == 1 / 16     # neighbours 1, 2, 3 x14
    assert abs(F[1, 23] - (D[1] - D[0])) < 1e-15 and F[1, 24] == 0.0        # 0, 2 (tie: lower j), 3
    assert abs(F[2, 23] - (D[2] - D[1])) < 1e-15 and F[2, 24] == 1 / 16     # 1, 0, 3 x14
    assert abs(F[3, 23] - (D[3] - D[1])) < 1e-15 and F[3, 24] == 1.0        # 2, 1, 0 x14
    # the top-16 values of row 1 keep both -1 entries (ties) then pad with -81
    assert np.array_equal(F[1, :4], np.array([-1, -1, -81, -81]) / 8.0)


@pytest.mark.parametrize("bf16", [False, True])
def test_gradient_vs_central_differences(bf16):
    S, p = _problem()
    F = mlp.row_features(S, p)
    g = np.random.default_rng(1)
    T = np.stack([g.normal(size=40), g.normal(size=40), (g.random(40) < 0.3).astype(float)], 1)
    P = mlp.set_standardisation(synth.mlp_init().astype(np.float64), F)
    d = mlp.unpack(P)
    d["b3"] = g.normal(size=3) * 0.1
    P = mlp.pack(d)
    L, G = mlp.backward(P, F, T, bf16=False)
    nt = mlp.NP - 2 * mlp.IN                    # trained parameters
    idx = np.concatenate([g.choice(nt, 60, replace=False), np.arange(nt - 3, nt)])
    h = 1e-6
    for i in idx:
        Pp, Pm = P.copy(), P.copy()
        Pp[i] += h
        Pm[i] -= h
        num = (mlp.loss(mlp.forward(Pp, F)[0], T) - mlp.loss(mlp.forward(Pm, F)[0], T)) / (2 * h)
        assert abs(num - G[i]) <= 1e-6 * max(1.0, abs(num)), (i, num, G[i])
    if bf16:
        # with bf16 products the gradient is that of the rounded network
        L16, G16 = mlp.backward(P, F, T, bf16=True)
        assert abs(L16 - L) < 0.05 * abs(L)


def test_adam_first_step_closed_form():
    g = np.random.default_rng(2)
    P = g.normal(size=10)
    grad = g.normal(size=10)
    P1, m, v = mlp.adam_step(P, grad, np.zeros(10), np.zeros(10), step=1, lr=1e-3)
    # after bias correction the first step is lr * g / (|g| + eps)
    assert np.allclose(P1, P - 1e-3 * grad / (np.abs(grad) + 1e-8), rtol=0, atol=1e-15)
    assert np.allclose(m, 0.1 * grad) and np.allclose(v, 0.001 * grad * grad)


def test_adam_second_step_by_hand():
    P = np.array([1.0])
    g1, g2 = np.array([0.5]), np.array([-0.25])
    P1, m1, v1 = mlp.adam_step(P, g1, np.zeros(1), np.zeros(1), 1, 0.1)
    P2, m2, v2 = mlp.adam_step(P1, g2, m1, v1, 2, 0.1)
    m = 0.9 * 0.05 + 0.1 * -0.25            # 0.02
    v = 0.999 * 0.00025 + 0.001 * 0.0625    # 0.00031225
    mh, vh = m / (1 - 0.81), v / (1 - 0.999 ** 2)
    assert np.allclose(P2, P1 - 0.1 * mh / (np.sqrt(vh) + 1e-8), rtol=1e-14)


def test_loss_and_targets():
    Y = np.array([[1.0, 2.0, 0.0], [0.0, 0.0, 10.0]])
    T = np.array([[0.0, 2.0, 1.0], [1.0, 1.0, 1.0]])
    want = ((1 + 0 + np.log(2)) + (1 + 1 + np.log1p(np.exp(-10.0)))) / 2
    assert abs(mlp.loss(Y, T) - want) < 1e-15
    S, p = _problem(3)
    r = ap.run(S, lam=0.5)
    Tt = mlp.targets(r["R"], r["A"], p)
    assert np.array_equal(Tt[:, 2] > 0, ap.exemplar_mask(r["R"], r["A"]))
    n = S.shape[0]
    R0, A0 = mlp.warm_start(n, Tt, p)
    assert np.all(R0 == 0) and np.allclose(np.diag(A0), np.maximum(0, np.diag(r["A"])))
    # off the diagonal: the fixed-point column value min(0, r(k,k) + a(k,k)),
    # which differs from the converged a(i,k) only by the i-th term of Eq. 3
    col = np.minimum(0, np.diag(r["R"]) + np.diag(r["A"]))
    off = ~np.eye(n, dtype=bool)
    assert np.allclose(A0[off], np.tile(col, (n, 1))[off])
    # ... up to the i-th term and to how far the stopped run is from a fixed point
    own = np.maximum(0, r["R"])
    np.fill_diagonal(own, 0)
    dr, da = ap.undamped_residuals(S, r["R"], r["A"])
    assert (np.abs(A0 - r["A"])[off] <= own[off] + 2 * (da + dr) + 1e-9 * p).all()


def test_standardisation_is_fixed_and_applied():
    S, p = _problem(4)
    F = mlp.row_features(S, p)
    P = mlp.set_standardisation(synth.mlp_init().astype(np.float64), F)
    d = mlp.unpack(P)
    Fn = (F - d["mu"]) * d["isd"]
    assert np.allclose(Fn.mean(axis=0)[:18], 0, atol=1e-12)
    T = np.zeros((F.shape[0], 3))
    _, G = mlp.backward(P, F, T)
    g = mlp.unpack(G)
    assert np.all(g["mu"] == 0) and np.all(g["isd"] == 0)
    # the standardised network equals the plain one fed standardised features
    P0 = P.copy()
    d0 = mlp.unpack(P0)
    d0["mu"][:] = 0
    d0["isd"][:] = 1
    assert np.allclose(mlp.forward(P, F)[0], mlp.forward(mlp.pack(d0), Fn)[0])
