"""Seeded synthetic inputs shaped like the paper's merge workloads.

This module only draws numbers: it holds none of the merge's arithmetic, and
both the CUDA library's tests and the CPU oracle's tests take their inputs from
it.  Every generator uses numpy's PCG64 with an explicit seed.

The paper measures on RAND100K, SIFT, GIST, NYTimes and other sets (Sec. 5,
Table "Overview of Datasets"); none of them is available here, so these
generators copy only their shapes, dimensionality, value ranges and metric:

* ``gaussian_mixture``: RAND-style clustered float vectors (means U[-lo, hi],
  unit-variance noise), optionally L2-normalised.
* ``clustered_mixture``: a Gaussian mixture whose components vary in their own
  random low-dimensional subspace (rank 16) plus small isotropic noise,
  L2-normalised for the cosine workload.  An isotropic 96-d Gaussian has a
  local intrinsic dimension near 96 and almost no nearest-neighbour structure
  (NN-Descent reaches recall@10 ~0.13 on it at 1M points); the paper's real
  sets sit at 16-40 (Table "Overview of Datasets": SIFT1M 16.3, GIST1M 38.1,
  GloVe1M 39.5).
* ``sift_like``: non-negative integers 0..255 stored as float32, drawn around
  256 sparse-ish centres (each centre coordinate is 0 with p=0.4, else
  Gamma(2, 20)).  Each centre spreads its points in its own random 16-d
  subspace (about 8 per coordinate), so the local intrinsic dimension is near
  the 16.3 the paper lists for SIFT; values are rounded and clipped.
* ``gist_like``: non-negative correlated vectors |M u| with M a random
  d x d matrix (entries N(0, 1/d)) and u a 64-d latent (drawn from a
  clustered mixture, rank 16) padded with small noise.
"""
from __future__ import annotations

import numpy as np


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def gaussian_mixture(n: int, d: int, n_comp: int = 16, seed: int = 0, normalize: bool = False,
                     mean_range: float = 10.0, chunk: int = 1 << 18) -> np.ndarray:
    rng = _rng(seed)
    means = rng.uniform(-mean_range, mean_range, size=(n_comp, d))
    comp = rng.integers(0, n_comp, size=n)
    X = np.empty((n, d), np.float32)
    for b in range(0, n, chunk):
        e = min(n, b + chunk)
        blk = means[comp[b:e]] + rng.standard_normal((e - b, d))
        if normalize:
            blk /= np.linalg.norm(blk, axis=1, keepdims=True)
        X[b:e] = blk
    return X


def clustered_mixture(n: int, d: int, n_comp: int = 256, rank: int = 8, spread: float = 3.0,
                      noise: float = 0.1, mean_range: float = 10.0, seed: int = 0,
                      normalize: bool = False, chunk: int = 1 << 16) -> np.ndarray:
    """Gaussian mixture whose components vary mostly inside a random `rank`-dim
    subspace (sd `spread`), plus isotropic noise of sd `noise`: the low
    intrinsic dimension of real descriptor sets (an isotropic d-dim Gaussian
    has almost no nearest-neighbour structure at d ~ 100)."""
    rng = _rng(seed)
    means = rng.uniform(-mean_range, mean_range, size=(n_comp, d))
    basis = rng.normal(0.0, spread / np.sqrt(rank), size=(n_comp, d, rank))
    which = rng.integers(0, n_comp, size=n)
    X = np.empty((n, d), np.float32)
    for b in range(0, n, chunk):
        e = min(n, b + chunk)
        z = rng.standard_normal((e - b, rank))
        blk = (means[which[b:e]] + np.einsum("ndr,nr->nd", basis[which[b:e]], z)
               + noise * rng.standard_normal((e - b, d)))
        if normalize:
            blk /= np.linalg.norm(blk, axis=1, keepdims=True)
        X[b:e] = blk
    return X


def sift_like(n: int, d: int = 128, n_centres: int = 256, seed: int = 0, rank: int = 16,
              spread: float = 8.0, chunk: int = 1 << 16) -> np.ndarray:
    rng = _rng(seed)
    zero = rng.random((n_centres, d)) < 0.4
    centres = np.where(zero, 0.0, rng.gamma(2.0, 20.0, size=(n_centres, d)))
    basis = rng.normal(0.0, spread / np.sqrt(rank), size=(n_centres, d, rank))
    which = rng.integers(0, n_centres, size=n)
    X = np.empty((n, d), np.float32)
    for b in range(0, n, chunk):
        e = min(n, b + chunk)
        z = rng.standard_normal((e - b, rank))
        blk = centres[which[b:e]] + np.einsum("ndr,nr->nd", basis[which[b:e]], z)
        X[b:e] = np.clip(np.rint(blk), 0, 255)
    return X


def sift_manifold(n: int, d: int = 128, latent: int = 16, n_comp: int = 64, sep: float = 1.5,
                  seed: int = 0, chunk: int = 1 << 16) -> np.ndarray:
    """Search stand-in for SIFT: a 16-d latent mixture of 64 overlapping unit
    Gaussians (means N(0, sep^2)), mapped to d dims by a random N(0, 1/latent)
    matrix, scaled and rounded to integers in [0, 255].  Unlike sift_like's
    well-separated clusters (whose k-NN graph splits into one component per
    cluster, which no graph search can cross), its k-NN graph is one weakly
    connected component."""
    rng = _rng(seed)
    means = rng.normal(0.0, sep, size=(n_comp, latent))
    M = rng.normal(0.0, 1.0 / np.sqrt(latent), size=(d, latent))
    which = rng.integers(0, n_comp, size=n)
    X = np.empty((n, d), np.float32)
    for b in range(0, n, chunk):
        e = min(n, b + chunk)
        z = means[which[b:e]] + rng.standard_normal((e - b, latent))
        X[b:e] = np.clip(np.rint(64.0 + 16.0 * (z @ M.T)), 0, 255)
    return X


def bovw_like(n: int, d: int = 500, n_topics: int = 64, words: float = 60.0, seed: int = 0,
              chunk: int = 1 << 16) -> np.ndarray:
    """Bag-of-visual-words stand-in (NUSWide's 500-d BoVW histograms, chi-square
    metric): each row draws Poisson counts of `words` expected words from a
    mixture of two of n_topics sparse topic distributions over d visual words;
    non-negative integers stored as float32, mostly zeros."""
    rng = _rng(seed)
    topics = rng.gamma(0.1, 1.0, size=(n_topics, d))
    topics /= topics.sum(1, keepdims=True)
    X = np.empty((n, d), np.float32)
    for b in range(0, n, chunk):
        e = min(n, b + chunk)
        t1 = rng.integers(0, n_topics, size=e - b)
        t2 = rng.integers(0, n_topics, size=e - b)
        w = rng.random((e - b, 1))
        lam = words * (w * topics[t1] + (1.0 - w) * topics[t2])
        X[b:e] = rng.poisson(lam)
    return X


def itemsets(n: int, dim: int = 27983, n_types: int = 2000, core: int = 40,
             mean_len: float = 20.0, p_core: float = 0.8, seed: int = 0):
    """Kosarak-like itemsets (Jaccard metric) as CSR arrays (offsets int64
    [n+1], items int32, ascending within a row): items have Zipf(1.2)
    popularity; each row picks one of n_types basket types with a core of
    `core` items and draws a log-normal number of items (median mean_len,
    sigma 0.6, 1..200), a share p_core from its type's core, the rest by
    popularity."""
    rng = _rng(seed)
    pop = 1.0 / np.arange(1, dim + 1) ** 1.2
    pop /= pop.sum()
    perm = rng.permutation(dim)
    cores = [perm[rng.choice(dim, size=core, replace=False, p=pop)] for _ in range(n_types)]
    lens = np.clip(np.rint(rng.lognormal(np.log(mean_len), 0.6, size=n)), 1, 200).astype(int)
    types = rng.integers(0, n_types, size=n)
    k_core = np.minimum(core, rng.binomial(lens, p_core))
    popular = perm[rng.choice(dim, size=int((lens - k_core).sum()), p=pop)]
    starts = np.concatenate([[0], np.cumsum(lens - k_core)])
    rows = []
    for i in range(n):
        a = cores[types[i]][rng.permutation(core)[:k_core[i]]]
        rows.append(np.unique(np.concatenate([a, popular[starts[i]:starts[i + 1]]])))
    offsets = np.zeros(n + 1, np.int64)
    offsets[1:] = np.cumsum([len(r) for r in rows])
    items = np.concatenate(rows).astype(np.int32) if n else np.zeros(0, np.int32)
    return offsets, items


def sets_to_rows(offsets, items, dim) -> np.ndarray:
    """0/1 rows [n][dim] of CSR sets (the oracle's input form)."""
    n = len(offsets) - 1
    X = np.zeros((n, dim), np.float32)
    for i in range(n):
        X[i, items[offsets[i]:offsets[i + 1]]] = 1.0
    return X


def gist_like(n: int, d: int = 960, latent: int = 64, seed: int = 0, n_comp: int = 256,
              rank: int = 16, chunk: int = 1 << 16) -> np.ndarray:
    """|M u|: a random d x d mixing M (entries N(0, 1/d)) of u = [z; 0.02 e],
    z a 64-d latent drawn from a clustered mixture (low intrinsic dimension),
    e isotropic noise in the other d - 64 coordinates."""
    rng = _rng(seed)
    M = rng.normal(0.0, 1.0 / np.sqrt(d), size=(d, d)).astype(np.float32)
    Z = clustered_mixture(n, latent, n_comp=n_comp, rank=rank, spread=1.0, noise=0.05,
                          mean_range=2.0, seed=seed + 7919)
    X = np.empty((n, d), np.float32)
    for b in range(0, n, chunk):
        e = min(n, b + chunk)
        u = np.empty((e - b, d), np.float32)
        u[:, :latent] = Z[b:e]
        u[:, latent:] = 0.02 * rng.standard_normal((e - b, d - latent))
        X[b:e] = np.abs(u @ M.T)
    return X


def sample_nodes(n: int, count: int, seed: int = 0) -> np.ndarray:
    """Sorted distinct node ids for sampled recall checks."""
    rng = _rng(seed)
    count = min(count, n)
    return np.sort(rng.choice(n, size=count, replace=False))


# The five workloads (sizes, metric, k, rounds).  Data seed = 1000 + index.
WORKLOADS = {
    "smerge_gmm_10k_d32_k10": dict(kind="symmetric", gen="gaussian_mixture", n=10_000, d=32,
                                   k=10, metric="l2", rounds=8, sample_rate=0.5, seed=1001,
                                   gen_args=dict(n_comp=16)),
    "smerge_sift_1m_d128_k20": dict(kind="symmetric", gen="sift_like", n=1_000_000, d=128, k=20,
                                    metric="l2", rounds=10, sample_rate=0.5, seed=1002,
                                    gen_args={}),
    "jmerge_gmm_2m_d96_k16_cos": dict(kind="joint", gen="clustered_mixture", n=2_000_000, d=96,
                                      k=16, metric="cos", rounds=10, sample_rate=0.5, seed=1003,
                                      gen_args=dict(n_comp=256, rank=16, normalize=True)),
    "serve_sift_2m_d128_k16": dict(kind="serve", gen="sift_like", n=2_000_000, d=128, k=16,
                                   metric="l2", rounds=10, sample_rate=0.5, seed=1004,
                                   gen_args={}),
    "hmerge_sift_1m_d128_k20": dict(kind="hmerge", gen="sift_like", n=1_000_000, d=128, k=20,
                                    metric="l2", rounds=10, sample_rate=0.5, seed=1006,
                                    gen_args={}),
    "hsearch_sift_1m_d128_k20": dict(kind="hsearch", gen="sift_manifold", n=1_000_000, d=128, k=20,
                                     metric="l2", rounds=10, sample_rate=0.5, seed=1007,
                                     queries=10_000, gen_args={}),
    "smerge_nuswide_260k_d500_k20_chi2": dict(kind="symmetric_chi2", gen="bovw_like", n=260_000,
                                              d=500, k=20, metric="chi2", rounds=20,
                                              sample_rate=0.5, seed=1008,
                                              gen_args=dict(words=2000.0)),
    "smerge_kosarak_75k_k20_jaccard": dict(kind="sets", gen="itemsets", n=74_962, dim=27_983,
                                           k=20, metric="jaccard", rounds=20, sample_rate=0.5,
                                           seed=1009,
                                           gen_args=dict(n_types=1500, core=24, p_core=0.9)),
    "smerge_gist_1m_d960_k20": dict(kind="symmetric", gen="gist_like", n=1_000_000, d=960,
                                    k=20, metric="l1", rounds=10, sample_rate=0.5, seed=1005,
                                    gen_args={}),
}


def serve_batch_sizes(count: int, seed: int, median: int = 8000, sigma: float = 1.0,
                      lo: int = 1000, hi: int = 64000) -> np.ndarray:
    """Raw-batch sizes of the serving workload: lognormal around `median`,
    clipped to [lo, hi]."""
    rng = np.random.default_rng(seed)
    sizes = np.exp(np.log(median) + sigma * rng.standard_normal(count))
    return np.clip(np.rint(sizes), lo, hi).astype(np.int64)


def poisson_arrivals(count: int, rate_per_s: float, seed: int) -> np.ndarray:
    """Arrival times (seconds from 0) of a Poisson process of the given rate."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate_per_s, count))


def generate(name: str, n: int | None = None) -> np.ndarray:
    w = WORKLOADS[name]
    gen = {"gaussian_mixture": gaussian_mixture, "sift_like": sift_like,
           "sift_manifold": sift_manifold, "bovw_like": bovw_like,
           "gist_like": gist_like, "clustered_mixture": clustered_mixture}[w["gen"]]
    return gen(n if n is not None else w["n"], w["d"], seed=w["seed"], **w["gen_args"])
