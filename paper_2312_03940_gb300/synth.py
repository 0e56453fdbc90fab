"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws random numbers: it holds none of the clustering
method's arithmetic, so both the CUDA path and the CPU oracle can be fed from
it. Every generator is deterministic in its seed (numpy PCG64).

Workloads (the paper's real datasets are not available; these stand in for
them by shape and structure):

* ``gaussian_mixture``: isotropic Gaussian clusters (the paper's synthetic
  ``gaussian`` family, Sec. 6.1).
* ``u8_mixture``: uint8 Gaussian mixture with Zipf weights, per-cluster
  sigma and uniform noise points (a SIFT-like byte workload).
* ``vmf_like``: unit-norm clusters around random directions (stands in for
  image embeddings such as ImageNet).
* ``powerlaw_sphere``: unit-norm rows with a power-law covariance spectrum and
  Pareto cluster sizes (stands in for text embeddings).
* ``batched_sets``: many independent Gaussian mixtures of uneven sizes.
* ``insertion_order``: the random insertion permutation of the graph build.
"""
from __future__ import annotations

import numpy as np

SEED_BASE = 231203940


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def gaussian_mixture(n: int = 10_000, d: int = 32, components: int = 10, sigma: float = 1.0,
                     box: float = 10.0, seed: int = SEED_BASE + 1):
    """n points from `components` equal-weight isotropic Gaussians (std sigma)
    with centres uniform in [-box, box]^d. Returns (X float32 (n, d), labels)."""
    g = rng(seed)
    centres = g.uniform(-box, box, size=(components, d))
    labels = np.sort(g.integers(0, components, size=n))
    labels = g.permutation(labels)
    X = centres[labels] + sigma * g.standard_normal((n, d))
    return X.astype(np.float32), labels.astype(np.int64)


def u8_mixture(n: int = 1_000_000, d: int = 128, components: int = 100, zipf: float = 1.1,
               sigma_lo: float = 5.0, sigma_hi: float = 20.0, noise_frac: float = 0.05,
               centre_lo: float = 32.0, centre_hi: float = 224.0, seed: int = SEED_BASE + 2,
               chunk: int = 1 << 18):
    """uint8 Gaussian mixture: weights proportional to c^-zipf (c = 1..components),
    per-component sigma ~ U[sigma_lo, sigma_hi], centres U[centre_lo, centre_hi]^d,
    rounded and clipped to [0, 255]; plus noise_frac uniform-integer points
    (label = components). Rows are shuffled. Returns (X uint8 (n, d), labels)."""
    g = rng(seed)
    n_noise = int(round(noise_frac * n))
    n_mix = n - n_noise
    w = np.arange(1, components + 1, dtype=np.float64) ** (-zipf)
    w /= w.sum()
    centres = g.uniform(centre_lo, centre_hi, size=(components, d)).astype(np.float32)
    sig = g.uniform(sigma_lo, sigma_hi, size=components).astype(np.float32)
    lab = g.choice(components, size=n_mix, p=w)
    labels = np.concatenate([lab, np.full(n_noise, components)]).astype(np.int64)
    perm = g.permutation(n)
    labels = labels[perm]
    X = np.empty((n, d), np.uint8)
    for c0 in range(0, n, chunk):
        c1 = min(n, c0 + chunk)
        lb = labels[c0:c1]
        z = g.standard_normal((c1 - c0, d), dtype=np.float32)
        is_noise = lb == components
        lbm = np.where(is_noise, 0, lb)
        v = centres[lbm] + sig[lbm][:, None] * z
        v = np.where(is_noise[:, None], g.integers(0, 256, size=(c1 - c0, d)).astype(np.float32), v)
        X[c0:c1] = np.clip(np.rint(v), 0, 255).astype(np.uint8)
    return X, labels


def _normalise(X):
    return X / np.linalg.norm(X, axis=1, keepdims=True)


def vmf_like(n: int = 1_280_000, d: int = 1024, components: int = 1000, kappa_lo: float = 20.0,
             kappa_hi: float = 200.0, seed: int = SEED_BASE + 3, chunk: int = 1 << 16):
    """Unit-norm rows: mu_c uniform on the sphere, kappa_c log-uniform in
    [kappa_lo, kappa_hi], x = normalise(mu_c + g / sqrt(kappa_c)) with
    g ~ N(0, I_d). Cluster sizes ~ lognormal(0, 1) normalised to n.
    Returns (X float32, labels)."""
    g = rng(seed)
    mu = _normalise(g.standard_normal((components, d))).astype(np.float32)
    kappa = np.exp(g.uniform(np.log(kappa_lo), np.log(kappa_hi), size=components)).astype(np.float32)
    sz = g.lognormal(0.0, 1.0, size=components)
    cnt = np.floor(sz / sz.sum() * n).astype(np.int64)
    cnt[: n - cnt.sum()] += 1
    labels = g.permutation(np.repeat(np.arange(components), cnt))
    X = np.empty((n, d), np.float32)
    for c0 in range(0, n, chunk):
        c1 = min(n, c0 + chunk)
        lb = labels[c0:c1]
        v = mu[lb] + g.standard_normal((c1 - c0, d), dtype=np.float32) / np.sqrt(kappa[lb])[:, None]
        X[c0:c1] = _normalise(v)
    return X, labels.astype(np.int64)


def powerlaw_sphere(n: int = 1_000_000, d: int = 384, components: int = 10_000, decay: float = 1.2,
                    pareto: float = 1.5, spread: float = 0.35, seed: int = SEED_BASE + 5,
                    chunk: int = 1 << 16):
    """Unit-norm rows with a power-law covariance spectrum: eigenvalue i
    proportional to i^-decay in a random orthonormal basis Q (QR of a Gaussian
    matrix). Cluster centres and within-cluster offsets are both drawn from
    that covariance (offsets scaled by `spread`); cluster sizes ~ Pareto(pareto)
    normalised to n. Returns (X float32, labels)."""
    g = rng(seed)
    Q, _ = np.linalg.qr(g.standard_normal((d, d)))
    scale = (np.arange(1, d + 1, dtype=np.float64) ** (-decay / 2.0))
    A = (Q * scale[None, :]).astype(np.float32)  # x = A z has covariance Q diag(i^-decay) Q^T
    centres = g.standard_normal((components, d), dtype=np.float32) @ A.T
    sz = g.pareto(pareto, size=components) + 1.0
    cnt = np.floor(sz / sz.sum() * n).astype(np.int64)
    cnt[: n - cnt.sum()] += 1
    labels = g.permutation(np.repeat(np.arange(components), cnt))
    X = np.empty((n, d), np.float32)
    for c0 in range(0, n, chunk):
        c1 = min(n, c0 + chunk)
        lb = labels[c0:c1]
        off = (g.standard_normal((c1 - c0, d), dtype=np.float32) @ A.T) * spread
        X[c0:c1] = _normalise(centres[lb] + off)
    return X, labels.astype(np.int64)


def batched_sets(count: int = 64, n_lo: int = 2_000, n_hi: int = 200_000, dims=(96, 128, 256, 384),
                 comp_lo: int = 5, comp_hi: int = 500, seed: int = SEED_BASE + 4):
    """`count` independent Gaussian mixtures: n log-uniform in [n_lo, n_hi],
    d uniform over `dims`, components uniform in [comp_lo, comp_hi].
    Returns a list of (X float32, labels, components)."""
    g = rng(seed)
    out = []
    for _ in range(count):
        n = int(round(np.exp(g.uniform(np.log(n_lo), np.log(n_hi)))))
        d = int(g.choice(dims))
        comp = int(g.integers(comp_lo, comp_hi + 1))
        X, lab = gaussian_mixture(n, d, comp, sigma=1.0, box=10.0, seed=int(g.integers(1 << 31)))
        out.append((X, lab, comp))
    return out


def random_neighbours(n: int, K: int, repeats: int = 1, seed: int = SEED_BASE + 19) -> np.ndarray:
    """Initial neighbour lists of an NN-Descent build: for every repeat and
    point, K distinct ids drawn uniformly from the other n - 1 points.
    Returns int32 (repeats, n, K)."""
    if not 1 <= K < n:
        raise ValueError("need 1 <= K < n")
    g = rng(seed)
    out = np.empty((repeats, n, K), np.int32)
    rows = np.arange(n)[:, None]
    for r in range(repeats):
        draw = g.integers(0, n - 1, size=(n, 2 * K))
        draw = np.where(draw >= rows, draw + 1, draw)  # skip the point itself
        srt = np.sort(draw, axis=1)
        first = np.ones_like(srt, dtype=bool)
        first[:, 1:] = srt[:, 1:] != srt[:, :-1]
        # the K smallest distinct draws of each row (rows short of K are redrawn below)
        order = np.argsort(~first, axis=1, kind="stable")
        pick = np.take_along_axis(srt, order, 1)[:, :K]
        short = np.flatnonzero(first.sum(1) < K)
        for i in short:
            choice = g.choice(n - 1, size=K, replace=False)
            pick[i] = np.where(choice >= i, choice + 1, choice)
        out[r] = pick
    return out


def insertion_order(n: int, seed: int = SEED_BASE + 17) -> np.ndarray:
    """Random insertion permutation for the graph build (int32)."""
    return rng(seed).permutation(n).astype(np.int32)


def sample_ids(n: int, m: int, seed: int = SEED_BASE + 23) -> np.ndarray:
    """m distinct ids of [0, n) in increasing order (query samples)."""
    m = min(m, n)
    return np.sort(rng(seed).choice(n, size=m, replace=False)).astype(np.int64)
