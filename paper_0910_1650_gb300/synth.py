"""Seeded synthetic inputs shaped like the paper's workloads (Section 5).

This module only *draws data*: it holds none of the clustering arithmetic, so
both the CUDA path and the CPU oracle can take their inputs from it.  Every
stream is counter based (splitmix64, Steele/Lea/Flood 2014 with Vigna's
constants), so a value depends only on (seed, stream, counter) and never on the
order in which arrays are requested.  Normals come from Box-Muller in float64,
Gamma(2) from -ln(u1) - ln(u2); every feature array is rounded to float32 once.

Workloads (the paper's datasets are not available, these stand in for them):

* ``gaussian_mixture_2d`` -- the random 2-D point sets of Section 5 (Table 1,
  Fig. 2): 5 isotropic Gaussians, centres U[-10,10]^2, sigma 1, 100 points each.
* ``gaussian_mixture``    -- dense AP at N=20000, d=64: 50 Gaussians, centres
  N(0, 25 I), sigma 1, Dirichlet(2) weights, multinomial counts; and the LAP
  workload N=1e6, d=128, 1000 equal-weight Gaussians, centres N(0,16 I), sigma
  0.5 (stand-in for the calligraphy set of Section 5).
* ``subspaces``           -- stand-in for the manifold sets of Section 5: points on
  10 random 5-dim linear subspaces of R^100 plus N(0, 0.01) noise, shuffled.
* ``uneven_partition``    -- 32 seeded subset sizes in [500, 4000] summing to N.
* ``image_like``          -- stand-in for the face images of Section 5: nonnegative
  [0,1] vectors from rank-20 templates plus uniform 0.05 noise.
"""
from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_TWO53 = float(2.0 ** -53)

SEED_BASE = 0xA9000000


def config_seed(c: int) -> int:
    """Seed of workload number ``c`` (0 = the 500-point 2-D mixture, ...)."""
    return SEED_BASE + int(c)


def _mix64(z: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def splitmix64_seq(seed: int, count: int, start: int = 0) -> np.ndarray:
    """Outputs ``start+1 .. start+count`` of splitmix64 seeded with ``seed``."""
    ctr = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + ctr * _GOLDEN
    return _mix64(z)


class Stream:
    """A named counter-based stream: ``Stream(seed, k)`` is independent of
    ``Stream(seed, k')`` because its key is the splitmix64 hash of (seed, k)."""

    def __init__(self, seed: int, stream: int = 0):
        key = splitmix64_seq(seed, 1, start=int(stream) * 7919)[0]
        self.key = int(key)
        self.pos = 0

    def u64(self, n: int) -> np.ndarray:
        out = splitmix64_seq(self.key, n, start=self.pos)
        self.pos += n
        return out

    def uniform(self, n: int) -> np.ndarray:
        """float64 in [0, 1) with 53 random bits."""
        return (self.u64(n) >> np.uint64(11)).astype(np.float64) * _TWO53

    def normal(self, n: int) -> np.ndarray:
        """Standard normals by Box-Muller (cosine branch only)."""
        u1 = 1.0 - self.uniform(n)          # (0, 1]
        u2 = self.uniform(n)
        return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)

    def gamma2(self, n: int) -> np.ndarray:
        """Gamma(shape 2, scale 1) as a sum of two unit exponentials."""
        return -np.log(1.0 - self.uniform(n)) - np.log(1.0 - self.uniform(n))

    def integers(self, lo: int, hi: int, n: int) -> np.ndarray:
        """Integers uniform on [lo, hi] (inclusive) by floor(u * span)."""
        span = hi - lo + 1
        return lo + np.minimum((self.uniform(n) * span).astype(np.int64), span - 1)

    def permutation(self, n: int) -> np.ndarray:
        """Seeded permutation: argsort of n random 64-bit keys (stable)."""
        return np.argsort(self.u64(n), kind="stable")


def gaussian_mixture_2d(seed: int = config_seed(0), n_clusters: int = 5,
                        per_cluster: int = 100, sigma: float = 1.0,
                        box: float = 10.0):
    """N = n_clusters*per_cluster points in 2-D; returns (X float32 [N,2], labels)."""
    st = Stream(seed, 1)
    centres = (st.uniform(n_clusters * 2).reshape(n_clusters, 2) * 2.0 - 1.0) * box
    n = n_clusters * per_cluster
    labels = np.repeat(np.arange(n_clusters), per_cluster)
    noise = st.normal(n * 2).reshape(n, 2) * sigma
    X = centres[labels] + noise
    return X.astype(np.float32), labels.astype(np.int32)


def gaussian_mixture(n: int, d: int, n_clusters: int, seed: int,
                     centre_sigma: float, sigma: float,
                     dirichlet_alpha2: bool = True):
    """Mixture of isotropic Gaussians in d dims.

    Cluster weights are Dirichlet(2,...,2) (normalised Gamma(2) draws) when
    ``dirichlet_alpha2`` else equal; each point draws its cluster from the
    weights by inverse CDF (multinomial counts).  Returns (X float32 [n,d],
    labels int32 [n])."""
    st = Stream(seed, 2)
    centres = st.normal(n_clusters * d).reshape(n_clusters, d) * centre_sigma
    if dirichlet_alpha2:
        w = st.gamma2(n_clusters)
        w = w / w.sum()
    else:
        w = np.full(n_clusters, 1.0 / n_clusters)
    cdf = np.cumsum(w)
    cdf[-1] = 1.0
    labels = np.searchsorted(cdf, st.uniform(n), side="right").astype(np.int32)
    labels = np.minimum(labels, n_clusters - 1)
    X = np.empty((n, d), dtype=np.float32)
    chunk = 1 << 16
    for lo in range(0, n, chunk):
        hi = min(n, lo + chunk)
        z = st.normal((hi - lo) * d).reshape(hi - lo, d)
        X[lo:hi] = (centres[labels[lo:hi]] + sigma * z).astype(np.float32)
    return X, labels


def subspaces(n: int = 60000, d: int = 100, n_sub: int = 10, dim: int = 5,
              noise_var: float = 0.01, seed: int = config_seed(2)):
    """Points on ``n_sub`` random ``dim``-dimensional linear subspaces of R^d
    (orthonormal bases from QR of a d x dim Gaussian), coefficients N(0,1),
    n/n_sub points each, plus N(0, noise_var) noise, in seeded shuffled order.
    Returns (X float32 [n,d], labels int32 [n])."""
    st = Stream(seed, 3)
    per = n // n_sub
    labels = np.repeat(np.arange(n_sub), per)
    labels = np.concatenate([labels, np.full(n - per * n_sub, n_sub - 1)])
    X = np.empty((n, d), dtype=np.float64)
    for j in range(n_sub):
        B, _ = np.linalg.qr(st.normal(d * dim).reshape(d, dim))
        idx = np.nonzero(labels == j)[0]
        coef = st.normal(idx.size * dim).reshape(idx.size, dim)
        X[idx] = coef @ B.T
    X += st.normal(n * d).reshape(n, d) * np.sqrt(noise_var)
    perm = st.permutation(n)
    return X[perm].astype(np.float32), labels[perm].astype(np.int32)


def uneven_partition(n: int = 60000, parts: int = 32, lo: int = 500,
                     hi: int = 4000, seed: int = config_seed(2)) -> np.ndarray:
    """Seeded subset sizes m_j in [lo, hi] with sum n.

    m_j = lo + round((n - parts*lo) * w_j / sum(w)) with w_j ~ U(0,1); sizes
    above ``hi`` are clamped and the excess is handed, in index order, to
    subsets with room; the rounding residue goes to the last subset (or is
    spread the same way if it would break a bound).  Returns int64 offsets of
    length parts+1 (offsets[0] = 0, offsets[-1] = n)."""
    if parts * lo > n or parts * hi < n:
        raise ValueError("infeasible partition bounds")
    st = Stream(seed, 4)
    w = st.uniform(parts) + 1e-3
    extra = n - parts * lo
    m = lo + np.rint(extra * w / w.sum()).astype(np.int64)
    m = np.minimum(m, hi)
    resid = n - int(m.sum())
    j = parts - 1
    while resid != 0:
        step = 1 if resid > 0 else -1
        room = (hi - m[j]) if step > 0 else (m[j] - lo)
        take = min(abs(resid), int(room))
        m[j] += step * take
        resid -= step * take
        j = (j - 1) % parts
    off = np.zeros(parts + 1, dtype=np.int64)
    off[1:] = np.cumsum(m)
    return off


def image_like(n: int, d: int = 4096, n_clusters: int = 10, rank: int = 20,
               noise: float = 0.05, seed: int = config_seed(4), stream: int = 0):
    """Nonnegative image-like vectors in [0,1]^d.

    A basis B ~ U[0,1]^{rank x d}; each cluster template t = wB / max(wB) with
    w ~ U[0,1]^rank; each member is clip(t + U[0, noise], 0, 1); members are
    spread evenly over clusters then shuffled.  Returns (X float32 [n,d],
    labels int32 [n])."""
    st = Stream(seed, 100 + stream)
    B = st.uniform(rank * d).reshape(rank, d)
    W = st.uniform(n_clusters * rank).reshape(n_clusters, rank)
    T = W @ B
    T /= T.max(axis=1, keepdims=True)
    labels = np.arange(n) % n_clusters
    labels = labels[st.permutation(n)]
    X = T[labels] + noise * st.uniform(n * d).reshape(n, d)
    return np.clip(X, 0.0, 1.0).astype(np.float32), labels.astype(np.int32)


def image_like_task(args):
    """``image_like`` for a process pool: args = (n, d, n_clusters, seed,
    stream); returns X only."""
    n, d, k, seed, stream = args
    return image_like(n, d, k, seed=seed, stream=stream)[0]


def batch_problem_sizes(count: int = 256, lo: int = 200, hi: int = 4000,
                        seed: int = config_seed(4)):
    """Sizes N_b ~ U{lo..hi} and cluster counts ~ U{5..40} of a batch of
    independent problems.  Returns (sizes int64 [count], clusters int64 [count])."""
    st = Stream(seed, 5)
    return st.integers(lo, hi, count), st.integers(5, 40, count)


def workload(c: int, scale: float = 1.0):
    """Features of workload ``c`` (0..3); ``scale`` < 1 shrinks N for parity
    cases that the oracle finishes in seconds (same generator, fewer points).
    Returns (X float32 [N,d], labels int32 [N])."""
    if c == 0:
        return gaussian_mixture_2d()
    if c == 1:
        n = max(8, int(round(20000 * scale)))
        return gaussian_mixture(n, 64, 50, config_seed(1), 5.0, 1.0, True)
    if c == 2:
        n = max(20, int(round(60000 * scale)))
        return subspaces(n=n)
    if c == 3:
        n = max(8, int(round(1_000_000 * scale)))
        return gaussian_mixture(n, 128, 1000, config_seed(3), 4.0, 0.5, False)
    raise ValueError(c)


def mlp_init(seed: int = SEED_BASE + 77, n_in: int = 25, hid: int = 256, n_out: int = 3):
    """Initial parameters of the warm-start network as one float32 vector
    (W1, b1, W2, b2, W3, b3, mu, isd): He-normal weights N(0, 2/fan_in), zero
    biases, identity input standardisation (mu = 0, isd = 1)."""
    st = Stream(seed, 200)
    parts = []
    for fan_out, fan_in in ((hid, n_in), (hid, hid), (n_out, hid)):
        parts.append(st.normal(fan_out * fan_in) * np.sqrt(2.0 / fan_in))
        parts.append(np.zeros(fan_out))
    parts.append(np.zeros(n_in))
    parts.append(np.ones(n_in))
    return np.concatenate(parts).astype(np.float32)
