"""The learned warm start, in float64 (the paper has no learned part; this is
the model the CUDA library trains and evaluates).  TEST INFRASTRUCTURE ONLY.

Per point k of a similarity matrix S with preference scale p > 0:
  features (25):
    0-15  the 16 largest off-diagonal s(k,j) in decreasing order (ties: the
          lower j first), divided by p;
    16-17 the mean and the standard deviation of the off-diagonal s(k,j), / p;
    18    s(k,k) / p;
    19-22 log(1 + the number of j != k with s(k,j) >= -q p), q = 1/8, 1/4,
          1/2, 1, the threshold -q p formed in float32 (p as float32);
    23    D(k) - the largest D(j) over the 16 j of features 0-15, D = feature 20;
    24    the fraction of those 16 j with D(j) > D(k);
  (with fewer than 16 off-diagonal entries the last one is repeated, value
  and index);
  network: 25 -> 256 -> 256 -> 3, ReLU after the two hidden layers;
  outputs: (c_hat, a_hat, logit): the predicted converged column value
  min(0, r(k,k) + a(k,k))/p (what the warm start writes into column k), the
  predicted a(k,k)/p and the log-odds that k is an exemplar;
  loss (mean over rows): (c_hat - t_c)^2 + (a_hat - t_a)^2
                         + softplus(logit) - t_e * logit   (binary cross-entropy);
  optimiser: Adam (Kingma & Ba 2015), beta1 0.9, beta2 0.999, eps 1e-8, with
  bias correction.
The network first standardises its input, x -> (x - mu) * isd, with mu and
isd fixed (set from the training features, never updated by Adam).
Parameters are one flat vector: W1 (256x25), b1, W2 (256x256), b2, W3 (3x256),
b3, mu (25), isd (25).
The matrix products may use bf16-rounded weights (``bf16=True``) to mirror
the GPU, which keeps bf16 weights for its products and fp32 master weights.
"""
from __future__ import annotations

import numpy as np

from . import ap

IN, HID, OUT = 25, 256, 3
SIZES = [("W1", (HID, IN)), ("b1", (HID,)), ("W2", (HID, HID)), ("b2", (HID,)),
         ("W3", (OUT, HID)), ("b3", (OUT,)), ("mu", (IN,)), ("isd", (IN,))]
FIXED = ("mu", "isd")     # input standardisation, set from data, never trained
NP = sum(int(np.prod(s)) for _, s in SIZES)


def unpack(P):
    out, at = {}, 0
    for name, shape in SIZES:
        k = int(np.prod(shape))
        out[name] = np.asarray(P[at:at + k], dtype=np.float64).reshape(shape)
        at += k
    return out


def pack(d):
    return np.concatenate([np.asarray(d[name], dtype=np.float64).ravel() for name, _ in SIZES])


def row_features(S, scale):
    """25 features per row of S (float64); see the module docstring."""
    S = np.asarray(S, dtype=np.float64)
    n = S.shape[0]
    sc32 = np.float32(scale)
    thr = [np.float64(np.float32(-(sc32 * np.float32(q)))) for q in (0.125, 0.25, 0.5, 1.0)]
    F = np.zeros((n, IN))
    nbr = np.zeros((n, 16), dtype=np.int64)
    for k in range(n):
        idx = np.array([j for j in range(n) if j != k])
        row = S[k, idx]
        order = np.lexsort((idx, -row))          # decreasing value, then increasing index
        top, topi = row[order][:16], idx[order][:16]
        if top.size < 16:
            top = np.concatenate([top, np.full(16 - top.size, top[-1])])
            topi = np.concatenate([topi, np.full(16 - topi.size, topi[-1])])
        F[k, :16] = top / scale
        nbr[k] = topi
        F[k, 16] = row.mean() / scale
        F[k, 17] = np.sqrt(max(0.0, (row ** 2).mean() - row.mean() ** 2)) / scale
        F[k, 18] = S[k, k] / scale
        for q, t in enumerate(thr):
            F[k, 19 + q] = np.log1p(np.count_nonzero(row >= t))
    D = F[:, 20]
    for k in range(n):
        Dn = D[nbr[k]]
        F[k, 23] = D[k] - Dn.max()
        F[k, 24] = np.count_nonzero(Dn > D[k]) / 16.0
    return F


def targets(R, A, scale):
    """(min(0, r(k,k) + a(k,k))/p, a(k,k)/p, [k is an exemplar]) from
    converged messages."""
    n = R.shape[0]
    E = ap.exemplar_mask(R, A)
    c = np.minimum(0.0, np.diag(R) + np.diag(A))
    return np.stack([c / scale, np.diag(A) / scale, E.astype(np.float64)], axis=1)


def _w(Pd, bf16):
    if not bf16:
        return Pd["W1"], Pd["W2"], Pd["W3"]
    r = lambda W: ap.round_bf16(W.astype(np.float32)).astype(np.float64)
    return r(Pd["W1"]), r(Pd["W2"]), r(Pd["W3"])


def forward(P, F, bf16=False):
    """Returns (Y, cache).  Y: (rows, 3) = (c_hat, a_hat, logit)."""
    Pd = unpack(P)
    W1, W2, W3 = _w(Pd, bf16)
    F = (np.asarray(F, dtype=np.float64) - Pd["mu"]) * Pd["isd"]
    Z1 = F @ W1.T + Pd["b1"]
    H1 = np.maximum(Z1, 0.0)
    Z2 = H1 @ W2.T + Pd["b2"]
    H2 = np.maximum(Z2, 0.0)
    Y = H2 @ W3.T + Pd["b3"]
    return Y, (F, Z1, H1, Z2, H2, W1, W2, W3)


def softplus(x):
    return np.logaddexp(0.0, x)


def loss(Y, T):
    """Mean over rows of MSE(r) + MSE(a) + BCE(exemplar)."""
    d = Y[:, 0] - T[:, 0]
    e = Y[:, 1] - T[:, 1]
    bce = softplus(Y[:, 2]) - T[:, 2] * Y[:, 2]
    return float(np.mean(d * d + e * e + bce))


def dloss(Y, T):
    rows = Y.shape[0]
    G = np.empty_like(Y)
    G[:, 0] = 2.0 * (Y[:, 0] - T[:, 0])
    G[:, 1] = 2.0 * (Y[:, 1] - T[:, 1])
    G[:, 2] = 1.0 / (1.0 + np.exp(-Y[:, 2])) - T[:, 2]
    return G / rows


def backward(P, F, T, bf16=False):
    """Loss and its gradient with respect to the flat parameters (the
    products with weights use the bf16-rounded weights when ``bf16``; the
    weight gradients are with respect to the master weights)."""
    Y, (F, Z1, H1, Z2, H2, W1, W2, W3) = forward(P, F, bf16)
    G3 = dloss(Y, T)
    g = {}
    g["W3"] = G3.T @ H2
    g["b3"] = G3.sum(axis=0)
    G2 = (G3 @ W3) * (Z2 > 0)
    g["W2"] = G2.T @ H1
    g["b2"] = G2.sum(axis=0)
    G1 = (G2 @ W2) * (Z1 > 0)
    g["W1"] = G1.T @ F
    g["b1"] = G1.sum(axis=0)
    g["mu"] = np.zeros(IN)
    g["isd"] = np.zeros(IN)
    return loss(Y, T), pack(g)


def set_standardisation(P, F):
    """mu = column means of F, isd = 1 / column standard deviations (floored at 1e-3)."""
    d = unpack(P)
    F = np.asarray(F, dtype=np.float64)
    d["mu"] = F.mean(axis=0)
    d["isd"] = 1.0 / np.maximum(F.std(axis=0), 1e-3)
    return pack(d)


def adam_step(P, grad, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (``step`` counts from 1).  Returns (P, m, v)."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mhat = m / (1.0 - beta1 ** step)
    vhat = v / (1.0 - beta2 ** step)
    return P - lr * mhat / (np.sqrt(vhat) + eps), m, v


def warm_start(n, Y, scale):
    """R0 = 0 and a column-constant A0 built from the per-point predictions:
    at a fixed point of Eq. 3-4, a(k,k) = colp(k) and, for i != k,
    a(i,k) = min(0, r(k,k) + colp(k) - max(0, r(i,k))), which is
    min(0, r(k,k) + a(k,k)) up to the i-th term -- the network's first output;
    so
        A0(i,k) = min(0, c_hat_k * p)   (i != k),
        A0(k,k) = max(0, a_hat_k * p)   (Eq. 4 is never negative)."""
    R0 = np.zeros((n, n))
    c = np.minimum(0.0, Y[:, 0] * scale)
    A0 = np.tile(c, (n, 1))
    np.fill_diagonal(A0, np.maximum(0.0, Y[:, 1] * scale))
    return R0, A0
