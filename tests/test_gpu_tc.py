"""Tensor-core (tcgen05) similarity path against the oracle.

The bf16 path computes, in fp32 accumulation, the exact negative squared
distances of the centred features rounded to bfloat16; the oracle states
those points (oracle.ap.similarity_bf16_inputs) and their distances in
float64.  Per-entry bound: 4 (K+4) 2^-24 (|x_i|^2 + |x_k|^2) with K the
padded feature count, the same float32 accumulation bound as the SIMT path."""
import numpy as np
import pytest
import torch

from oracle import ap as oap
from paper_0910_1650_gb300 import capi, synth

pytestmark = pytest.mark.gpu


def _bound(Xt, K):
    nrm = (Xt ** 2).sum(axis=1)
    return 4.0 * (K + 4) * 2.0 ** -24 * (nrm[:, None] + nrm[None, :]) + 1e-30


def _case(name):
    if name == "tiny_2d_300":
        X, _ = synth.gaussian_mixture_2d(per_cluster=60)
    elif name == "mix64_1000":
        X, _ = synth.workload(1, scale=0.05)
    elif name == "ragged_777_d100":
        X, _ = synth.workload(2, scale=777 / 60000)
    elif name == "mix64_2000":
        X, _ = synth.workload(1, scale=0.1)
    elif name == "images_300_d4096":
        X, _ = synth.image_like(300, 4096, n_clusters=7)
    else:
        raise KeyError(name)
    return X


@pytest.mark.parametrize("name", ["tiny_2d_300", "mix64_1000", "ragged_777_d100", "mix64_2000",
                                  "images_300_d4096"])
def test_bf16_similarity_matches_oracle(name):
    X = _case(name)
    n, d = X.shape
    Sd, p = capi.ap_similarity(torch.from_numpy(X).cuda(), precision="bf16")
    S = Sd.cpu().numpy().astype(np.float64)
    Xt = oap.similarity_bf16_inputs(X)
    Sref = oap.similarity(Xt)
    K = (d + 63) // 64 * 64
    off = ~np.eye(n, dtype=bool)
    err = np.abs(S - Sref)
    assert (err[off] <= _bound(Xt, K)[off]).all(), float((err / _bound(Xt, K))[off].max())
    assert (S[off] <= 0).all()
    assert p == np.float32(np.median(S[off].astype(np.float32).astype(np.float64)))
    assert (np.diag(S) == np.float32(p)).all()


def test_bf16_similarity_at_the_bench_size_sampled_rows():
    """The bench's 20000-point, 64-D build at full size (the launch the bench
    times): 66 sampled rows against the oracle's distances of the rounded
    centred points within the per-entry bound, every entry <= 0, and the
    preference the exact off-diagonal median of the S it wrote."""
    X, _ = synth.workload(1)
    n, d = X.shape
    Sd, p = capi.ap_similarity(torch.from_numpy(X).cuda(), precision="bf16")
    rows = np.unique(np.concatenate([[0, n - 1], np.random.default_rng(9).choice(n, 64, replace=False)]))
    Srows = Sd[torch.from_numpy(rows).cuda()].cpu().numpy().astype(np.float64)
    Xt = oap.similarity_bf16_inputs(X)
    Sref = oap.similarity(Xt[rows], Xt)
    nrm = (Xt ** 2).sum(axis=1)
    K = (d + 63) // 64 * 64
    bound = 4.0 * (K + 4) * 2.0 ** -24 * (nrm[rows][:, None] + nrm[None, :]) + 1e-30
    off = np.ones_like(Srows, dtype=bool)
    off[np.arange(rows.size), rows] = False
    assert (np.abs(Srows - Sref)[off] <= bound[off]).all()
    assert (Srows[off] <= 0).all()
    assert (Srows[~off] == np.float32(p)).all()
    S = Sd.cpu().numpy()
    assert p == np.float32(np.median(S[~np.eye(n, dtype=bool)].astype(np.float64)))


def test_bf16_similarity_error_vs_unrounded_points_reported():
    """The bf16 path against the float64 distances of the unrounded points:
    stated, not bounded by float32 rounding (the inputs differ by bf16
    rounding, relative 2^-9 per coordinate)."""
    X = _case("mix64_1000")
    Sd, _ = capi.ap_similarity(torch.from_numpy(X).cuda(), precision="bf16")
    S = Sd.cpu().numpy().astype(np.float64)
    S64 = oap.similarity(X)
    n = X.shape[0]
    off = ~np.eye(n, dtype=bool)
    rel = np.abs(S - S64)[off].max() / np.abs(S64[off]).max()
    assert rel < 1e-2
    print(f"bf16 S vs float64 S of unrounded points: max rel (inf-norm) {rel:.3e}")


def test_bf16_and_fp32_paths_give_same_exemplars():
    X = _case("mix64_2000")
    res = {}
    for prec in ("fp32", "bf16"):
        Sd, p = capi.ap_similarity(torch.from_numpy(X).cuda(), precision=prec)
        R, A, r, _ = capi.ap_iterate(Sd, damping=0.9, max_iter=1000, conv_iter=15)
        idx, ex = capi.ap_exemplars(Sd, R, A)
        res[prec] = (idx.cpu().numpy(), ex["netsim"])
    assert np.array_equal(res["fp32"][0], res["bf16"][0])
    assert abs(res["fp32"][1] - res["bf16"][1]) <= 1e-3 * abs(res["fp32"][1])
