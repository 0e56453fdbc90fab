"""Exact density-peaks clustering in FP64 by brute force -- TEST INFRASTRUCTURE ONLY.

This is the paper's ``BruteForce`` instance ("exact DPC", Sec. 6.1): exact
k-NN, the density functions of Sec. 4.2 / Appendix A, Definition 2.1 for the
dependent point, and the noise / center / union-find steps of Algorithm 2.
Everything is in float64 numpy; nothing here is shared with the GPU library.
Also: the Adjusted Rand Index (Sec. 6.1, Hubert and Arabie) and a tie-aware
k-NN recall.
"""
from __future__ import annotations

import numpy as np

L2, IP = 0, 1


def _block_dist(X: np.ndarray, Y: np.ndarray, metric: int) -> np.ndarray:
    """Exact FP64 distances D between the rows of X and Y."""
    X = X.astype(np.float64)
    Y = Y.astype(np.float64)
    if metric == IP:
        return 1.0 - X @ Y.T
    d2 = (X * X).sum(1)[:, None] + (Y * Y).sum(1)[None, :] - 2.0 * (X @ Y.T)
    # the expansion above can lose a few ulps; recompute the small ones exactly
    np.maximum(d2, 0.0, out=d2)
    return np.sqrt(d2)


def exact_dist_rows(X: np.ndarray, rows: np.ndarray, metric: int = L2) -> np.ndarray:
    """D(x_i, x_j) for i in rows and all j, computed as sum of squared
    differences (no cancellation) -- slow but exact to FP64 rounding."""
    Xd = X.astype(np.float64)
    out = np.empty((len(rows), X.shape[0]))
    for t, i in enumerate(rows):
        if metric == IP:
            out[t] = 1.0 - Xd @ Xd[i]
        else:
            diff = Xd - Xd[i]
            out[t] = np.sqrt(np.einsum("ij,ij->i", diff, diff))
    return out


def exact_knn(X: np.ndarray, k: int, metric: int = L2, block: int = 512):
    """Exact k nearest neighbours of every point over P minus itself, sorted by
    (D, id). Returns ids (n,k) int64, dist (n,k) float64."""
    n = X.shape[0]
    ids = np.empty((n, k), np.int64)
    dist = np.empty((n, k))
    for b0 in range(0, n, block):
        rows = np.arange(b0, min(n, b0 + block))
        D = exact_dist_rows(X, rows, metric)
        D[np.arange(len(rows)), rows] = np.inf  # exclude the point itself
        # stable sort on D keeps smaller ids first among equal distances
        order = np.argsort(D, axis=1, kind="stable")[:, :k]
        ids[rows] = order
        dist[rows] = np.take_along_axis(D, order, 1)
    return ids, dist


def exact_knn_queries(X: np.ndarray, rows: np.ndarray, k: int, metric: int = L2, chunk: int = 65536):
    """Exact k nearest neighbours (FP64, self excluded, ties by smaller id) of
    the sampled points `rows` over all of X, scanning X in chunks.
    Returns ids (m,k) int64 and dist (m,k) float64."""
    rows = np.asarray(rows, dtype=np.int64)
    Q = X[rows].astype(np.float64)
    qn = (Q * Q).sum(1)
    best_d = np.full((len(rows), k), np.inf)
    best_i = np.full((len(rows), k), -1, np.int64)
    for c0 in range(0, X.shape[0], chunk):
        Y = X[c0:c0 + chunk].astype(np.float64)
        if metric == IP:
            D = 1.0 - Q @ Y.T
        else:
            D = qn[:, None] + (Y * Y).sum(1)[None, :] - 2.0 * (Q @ Y.T)
            np.maximum(D, 0.0, out=D)
        ids = np.arange(c0, c0 + Y.shape[0])
        D[rows[:, None] == ids[None, :]] = np.inf
        cand_d = np.concatenate([best_d, D], 1)
        cand_i = np.concatenate([best_i, np.broadcast_to(ids, D.shape)], 1)
        # sort each row by (distance, id): a stable sort keeps the earlier
        # (smaller) ids first among equal distances
        idx = np.argsort(cand_d, axis=1, kind="stable")
        cand_d = np.take_along_axis(cand_d, idx, 1)
        cand_i = np.take_along_axis(cand_i, idx, 1)
        best_d, best_i = cand_d[:, :k], cand_i[:, :k]
    if metric == L2:
        best_d = np.sqrt(best_d)
    return best_i, best_d


def density(dist: np.ndarray, fn: str = "kth", normalize: bool = False, ids: np.ndarray | None = None):
    """Density from the sorted k-NN distances (Sec. 4.2, Appendix A).
    Returns (rho, key): key ranks the points (equal to rho except for exp-sum,
    whose key is the exponent)."""
    k = dist.shape[1]
    if fn == "kth":
        with np.errstate(divide="ignore"):
            rho = 1.0 / dist[:, -1]
        key = rho
    elif fn == "exp-sum":
        key = -(dist ** 2).sum(1) / k
        rho = np.exp(key)
    elif fn == "sum-exp":
        rho = np.exp(-(dist ** 2)).sum(1) / k
        key = rho
    elif fn == "sum":
        rho = -dist.sum(1)
        key = rho
    else:
        raise ValueError(fn)
    if normalize:
        rho = rho * k / rho[ids].sum(1)
        key = rho
    return rho, key


def rank_order(key: np.ndarray) -> np.ndarray:
    """Points from highest to lowest rank: key descending, smaller id first."""
    n = key.size
    return np.lexsort((np.arange(n), -key))


def exact_dependent(X: np.ndarray, key: np.ndarray, metric: int = L2, block: int = 512):
    """Definition 2.1: lambda_i = the closest point ranked above i (ties: the
    smaller id); delta_i = D(x_i, lambda_i), +inf when there is none."""
    n = X.shape[0]
    order = rank_order(key)
    rank = np.empty(n, np.int64)
    rank[order] = np.arange(n)  # 0 = highest
    lam = np.full(n, -1, np.int64)
    delta = np.full(n, np.inf)
    for b0 in range(0, n, block):
        rows = np.arange(b0, min(n, b0 + block))
        D = exact_dist_rows(X, rows, metric)
        higher = rank[None, :] < rank[rows][:, None]
        D = np.where(higher, D, np.inf)
        j = np.argmin(D, axis=1)  # first minimum = smallest id
        ok = np.isfinite(D[np.arange(len(rows)), j])
        lam[rows[ok]] = j[ok]
        delta[rows[ok]] = D[np.arange(len(rows)), j][ok]
    return lam, delta


def cluster(rho, lam, delta, center: str = "product", rho_min: float = 0.0, delta_min: float = 0.0,
            n_clusters: int = 1):
    """Noise (rho < rho_min), centers (delta > delta_min, or the n_clusters
    largest delta * rho), then every other point joins its dependent point's
    cluster. A cluster is named by its root: the member whose dependent edge
    was cut. Implemented by following dependent pointers (the union-find of
    Algorithm 2 yields the same partition)."""
    n = rho.size
    noise = rho < rho_min
    if center == "threshold":
        cen = ~noise & (delta > delta_min)
    else:
        prod = np.where((delta == 0) | (rho == 0), 0.0, delta * rho)
        cand = np.flatnonzero(~noise)
        order = cand[np.lexsort((cand, -prod[cand]))]
        cen = np.zeros(n, bool)
        cen[order[:n_clusters]] = True
    cut = noise | cen | (lam < 0)
    parent = np.where(cut, np.arange(n), lam)
    # pointer jumping until every point points at its root
    while True:
        nxt = parent[parent]
        if np.array_equal(nxt, parent):
            break
        parent = nxt
    return parent.astype(np.int64), int(cut.sum())


def exact_dpc(X: np.ndarray, k: int, metric: int = L2, density_fn: str = "kth", **cluster_kw):
    ids, dist = exact_knn(X, k, metric)
    rho, key = density(dist, density_fn, ids=ids)
    lam, delta = exact_dependent(X, key, metric)
    labels, nc = cluster(rho, lam, delta, **cluster_kw)
    return dict(ids=ids, dist=dist, rho=rho, key=key, lam=lam, delta=delta, labels=labels, n_clusters=nc)


def ari(a: np.ndarray, b: np.ndarray) -> float:
    """Adjusted Rand Index (Hubert and Arabie; the printed formula of Sec. 6.1
    lacks a product sign, the standard definition is used).

    With n_ij the contingency counts, a_i and b_j its row and column sums and
    T = C(n, 2) the number of pairs:
        ARI = (sum_ij C(n_ij, 2) - E) / ((S_a + S_b) / 2 - E),  E = S_a S_b / T,
    S_a = sum_i C(a_i, 2), S_b = sum_j C(b_j, 2). Multiplying through by 2T
    gives the integer ratio (2 T S_ij - 2 S_a S_b) / (T (S_a + S_b) - 2 S_a S_b),
    evaluated here in Python integers (exact at any n: the products pass 2^63
    near n = 10^5) and divided once in floating point. Two identical
    partitions give 1.0, including the degenerate 0/0 case."""
    a = np.asarray(a).reshape(-1)
    b = np.asarray(b).reshape(-1)
    n = int(a.size)
    _, ai = np.unique(a, return_inverse=True)
    _, bi = np.unique(b, return_inverse=True)
    # sparse contingency table: one entry per occupied (cluster, class) cell
    cell = ai.astype(np.int64) * (int(bi.max()) + 1) + bi.astype(np.int64)
    _, cont = np.unique(cell, return_counts=True)

    def c2(counts) -> int:
        # each term x (x - 1) / 2 < 2^62 for x < 2^31; the sum in Python ints
        x = np.asarray(counts, np.int64)
        return sum(int(v) for v in (x * (x - 1) // 2))

    s_ij = c2(cont)
    s_a = c2(np.bincount(ai))
    s_b = c2(np.bincount(bi))
    total = n * (n - 1) // 2
    num = 2 * total * s_ij - 2 * s_a * s_b
    den = total * (s_a + s_b) - 2 * s_a * s_b
    if den == 0:
        return 1.0
    return num / den  # correctly rounded quotient of two Python integers


def homogeneity_completeness(pred: np.ndarray, true: np.ndarray) -> tuple:
    """Homogeneity 1 - H(T|C) / H(T) and completeness 1 - H(C|T) / H(C) of
    predicted clusters C against ground-truth classes T (Sec. 6 metrics).
    The printed symbols swap C and T against the prose that defines them; the
    prose and its example (every point its own cluster: homogeneity 1, low
    completeness) are followed. Natural logarithms; a zero entropy in a
    denominator gives 1."""
    pred = np.asarray(pred).reshape(-1)
    true = np.asarray(true).reshape(-1)
    n = pred.size
    _, ci = np.unique(pred, return_inverse=True)
    _, ti = np.unique(true, return_inverse=True)
    cont = np.zeros((ti.max() + 1, ci.max() + 1), np.int64)
    np.add.at(cont, (ti, ci), 1)
    a = cont.sum(1).astype(np.float64)  # class sizes
    b = cont.sum(0).astype(np.float64)  # cluster sizes
    nz = cont > 0
    nij = cont[nz].astype(np.float64)
    ii, jj = np.nonzero(nz)

    def entropy(sizes):
        q = sizes[sizes > 0] / n
        return float(-(q * np.log(q)).sum())

    h_t, h_c = entropy(a), entropy(b)
    h_t_given_c = float(-((nij / n) * np.log(nij / b[jj])).sum())
    h_c_given_t = float(-((nij / n) * np.log(nij / a[ii])).sum())
    hom = 1.0 if h_t == 0.0 else 1.0 - h_t_given_c / h_t
    com = 1.0 if h_c == 0.0 else 1.0 - h_c_given_t / h_c
    return hom, com


def knn_recall(found_dist: np.ndarray, exact_dist: np.ndarray, rel: float = 1e-5) -> float:
    """Tie-aware recall: per query, the fraction of the k returned points whose
    distance is within (1 + rel) of the exact k-th distance; averaged."""
    kth = exact_dist[:, -1:]
    ok = found_dist <= kth * (1.0 + rel) + 1e-30
    return float(ok.mean())
