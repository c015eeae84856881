"""Training and evaluation driver of the learned warm start.

Orchestration only: every numeric step (similarity, plain Algorithm 1 runs
that produce the targets, features, forward/backward/Adam, warm-started runs)
is a call into libapgb.so through ``capi``.
"""
from __future__ import annotations

import numpy as np
import torch

from . import capi, synth


def make_dataset(problems, damping=0.9, max_iter=1000, conv_iter=15, precision="bf16"):
    """Features and targets from plain (cold-start) Algorithm 1 runs on each
    feature matrix in ``problems``.  Returns (F, T, info) with one row per
    point of every problem; the preference scale is |median preference|."""
    Fs, Ts, info = [], [], []
    for X in problems:
        Xd = torch.from_numpy(X).cuda()
        S, p = capi.ap_similarity(Xd, precision=precision)
        scale = abs(p) if p != 0 else 1.0
        R, A, res, dec = capi.ap_iterate(S, damping=damping, max_iter=max_iter, conv_iter=conv_iter)
        Fs.append(capi.apl_features(S, scale))
        Ts.append(capi.apl_targets(R, A, dec, scale))
        info.append(dict(n=X.shape[0], scale=scale, iters=res["iters"]))
        del S, R, A
    return torch.cat(Fs), torch.cat(Ts), info


def train(F, T, epochs=30, batch=4096, lr=1e-3, seed=synth.SEED_BASE + 77, shuffle_seed=5):
    """Adam on (F, T) with the library's train step; minibatches follow a
    seeded permutation fixed per epoch.  Returns (P, P16, per-epoch mean loss)."""
    P = torch.from_numpy(synth.mlp_init(seed)).cuda()
    capi.apl_set_standardisation(P, F)                       # fixed input standardisation
    P16 = torch.empty(P.numel(), dtype=torch.bfloat16, device=P.device)
    capi.apl_sync_bf16(P, P16)
    M = torch.zeros_like(P)
    V = torch.zeros_like(P)
    rows = F.shape[0]
    ws = capi.workspace(capi.lib().apl_workspace_size(min(batch, rows)), F.device)
    losses, step = [], 0
    for ep in range(epochs):
        perm = torch.from_numpy(synth.Stream(shuffle_seed, ep).permutation(rows)).to(F.device)
        Fp, Tp = F[perm].contiguous(), T[perm].contiguous()
        tot, nb = 0.0, 0
        for lo in range(0, rows, batch):
            hi = min(rows, lo + batch)
            step += 1
            loss, _ = capi.apl_train_step(P, P16, M, V, step, lr, Fp[lo:hi], Tp[lo:hi], ws=ws)
            tot += float(loss.item())
            nb += 1
        losses.append(tot / nb)
    return P, P16, losses


def image_problems(count, lo=200, hi=4000, d=4096, seed=synth.config_seed(4), offset=0):
    """Feature matrices of the batch workload (image-like vectors), problem
    sizes and cluster counts from the workload's seeded draws."""
    sizes, clusters = synth.batch_problem_sizes(count + offset, lo, hi, seed)
    out = []
    for b in range(offset, offset + count):
        X, _ = synth.image_like(int(sizes[b]), d, int(clusters[b]), seed=seed, stream=b)
        out.append(X)
    return out


def mixture_problems(count, lo=500, hi=2000, d=32, seed=synth.SEED_BASE + 300, offset=0):
    """Gaussian-mixture problems of seeded sizes (10-40 clusters, centres
    N(0, 16 I), sigma 1, Dirichlet(2) weights)."""
    sizes, clusters = synth.batch_problem_sizes(count + offset, lo, hi, seed)
    out = []
    for b in range(offset, offset + count):
        k = 10 + int(clusters[b]) % 31
        X, _ = synth.gaussian_mixture(int(sizes[b]), d, k, seed + 1000 + b, 4.0, 1.0)
        out.append(X)
    return out


def landmark_training_problems(count=12, n=4000, d=128, clusters=100, seed=synth.SEED_BASE + 400):
    """Mixtures with the landmark pool's density (about 40 points per
    cluster; 1000-cluster workload, sigma 0.5, centres N(0, 16 I))."""
    return [synth.gaussian_mixture(n, d, clusters, seed + b, 4.0, 0.5, False)[0]
            for b in range(count)]


def landmark_scores(X, n_landmarks, P, P16, seed=synth.SEED_BASE + 401, pool_factor=2):
    """Scores for Algorithm 3's landmark choice by the network's exemplar
    log-odds: a uniform pool of pool_factor * n_landmarks points (seeded
    permutation) gets its own S, features and forward pass; every other
    point scores -inf, so lap_run(mode="score") keeps the best-scoring
    n_landmarks of the pool.  Returns a device float32 [n] tensor."""
    n = X.shape[0]
    m = min(n, pool_factor * int(n_landmarks))
    pool = torch.from_numpy(synth.Stream(seed, 0).permutation(n)[:m].copy()).to(X.device)
    S, p = capi.ap_similarity(X[pool].contiguous(), precision="bf16")
    F = capi.apl_features(S, abs(p) if p != 0 else 1.0)
    Y = capi.apl_forward(P, P16, F)
    score = torch.full((n,), float("-inf"), dtype=torch.float32, device=X.device)
    score[pool] = Y[:, 2]
    return score
