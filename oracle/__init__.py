"""CPU oracle for PECANN density-peaks clustering -- TEST INFRASTRUCTURE ONLY.

Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. It shares no code with the CUDA library
and never calls it.

Two layers:

* ``oracle/pecann_oracle.c`` (loaded here through ctypes): the paper's method
  step by step in plain C -- Algorithm 1 (greedy beam search), Algorithm 2
  (framework: k-NN, density, noise, centers, union-find), Algorithm 3
  (dependent points with doubling rounds), RobustPrune and the batched Vamana
  construction of Sec. 3.2 / Sec. 4.1. All decisions are taken on FP32
  values computed in one fixed ("canonical") summation order, which is the
  precision the GPU path decides in.
* :mod:`oracle.exact`: exact DPC in FP64 by brute force (Definition 2.1), and
  the Adjusted Rand Index.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pecann_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None

F32, U8 = 0, 1
L2, IP = 0, 1
DENS_KTH, DENS_EXPSUM, DENS_SUMEXP, DENS_SUM = 0, 1, 2, 3
CENTER_THRESHOLD, CENTER_PRODUCT, CENTER_LOCAL = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (no FP contraction, so every fused
    multiply-add is the explicit fmaf of the canonical distance)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                           "-o", tmp, _SRC, "-lm", "-lpthread"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Points(ctypes.Structure):
    _fields_ = [("X", ctypes.c_void_p), ("n", ctypes.c_int64), ("d", ctypes.c_int32),
                ("dtype", ctypes.c_int32), ("metric", ctypes.c_int32)]


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        P = ctypes.POINTER(_Points)
        vp = ctypes.c_void_p
        i32, i64, f32 = ctypes.c_int32, ctypes.c_int64, ctypes.c_float
        _lib.orc_dis.argtypes = [P, i64, i64]
        _lib.orc_dis.restype = f32
        _lib.orc_greedy_search.argtypes = [P, vp, i32, i64, vp, i64, i32, i32, vp, vp, vp, vp, i64, vp]
        _lib.orc_greedy_search.restype = i64
        _lib.orc_knn_density.argtypes = [P, vp, i32, i32, i32, i32, i32, vp, vp, vp, vp, vp, ctypes.c_int]
        _lib.orc_knn_density.restype = ctypes.c_int
        _lib.orc_knn_density_rows.argtypes = [P, vp, i32, i32, i32, i32, vp, i64, vp, vp, vp, vp, vp,
                                              ctypes.c_int]
        _lib.orc_knn_density_rows.restype = ctypes.c_int
        _lib.orc_nndescent.argtypes = [P, i32, i32, vp, i32, f32, i32, vp, vp, vp, ctypes.c_int]
        _lib.orc_nndescent.restype = ctypes.c_int
        u64 = ctypes.c_uint64
        _lib.orc_hcnng.argtypes = [P, i32, i32, i32, f32, i32, u64, vp, vp, ctypes.c_int]
        _lib.orc_hcnng.restype = ctypes.c_int
        _lib.orc_hcnng_partition.argtypes = [P, i32, i32, u64, vp, vp]
        _lib.orc_hcnng_partition.restype = i64
        _lib.orc_hcnng_leaf_mst.argtypes = [P, vp, i64, i32, vp]
        _lib.orc_hcnng_leaf_mst.restype = i64
        _lib.orc_splitmix64.argtypes = [u64]
        _lib.orc_splitmix64.restype = u64
        _lib.orc_hcnng_draw.argtypes = [u64, i32, i64, i64, i32]
        _lib.orc_hcnng_draw.restype = u64
        _lib.orc_dependent_points.argtypes = [P, vp, i32, vp, vp, i32, i32, i32, i32, i32, vp, vp, vp,
                                              ctypes.c_int]
        _lib.orc_dependent_points.restype = ctypes.c_int
        _lib.orc_cluster.argtypes = [i64, vp, vp, vp, i32, f32, f32, i32, vp]
        _lib.orc_cluster.restype = i64
        _lib.orc_cluster_local.argtypes = [i64, i32, vp, vp, vp, vp, f32, vp]
        _lib.orc_cluster_local.restype = i64
        _lib.orc_robust_prune.argtypes = [P, i64, vp, i64, f32, i32, vp]
        _lib.orc_robust_prune.restype = i32
        _lib.orc_build_graph.argtypes = [P, i32, i32, f32, vp, i32, f32, i32, i32, vp, ctypes.c_int]
        _lib.orc_build_graph.restype = ctypes.c_int
        _lib.orc_search_counts.argtypes = [P, vp, i32, i32, vp, i64, vp, vp, ctypes.c_int]
        _lib.orc_search_counts.restype = ctypes.c_int
        _lib.orc_batch_cap.argtypes = [i64, f32]
        _lib.orc_batch_cap.restype = i64
    return _lib


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


class Points:
    """A point set as the oracle sees it: n x d, FP32 or uint8, L2 or inner
    product. Keeps a C-contiguous copy alive for the duration of the calls."""

    def __init__(self, X: np.ndarray, metric: int = L2):
        if X.dtype == np.uint8:
            dt = U8
        else:
            X = X.astype(np.float32, copy=False)
            dt = F32
        self.X = np.ascontiguousarray(X)
        n, d = self.X.shape
        if d % 4:
            raise ValueError("d must be a multiple of 4")
        self.n, self.d, self.metric = n, d, metric
        self._s = _Points(self.X.ctypes.data, n, d, dt, metric)

    @property
    def ptr(self):
        return ctypes.byref(self._s)


def _p(a: np.ndarray):
    return a.ctypes.data


def dis(P: Points, a: int, b: int) -> float:
    """Canonical FP32 dissimilarity (squared L2, or 1 - <x, y>)."""
    return float(np.float32(_load().orc_dis(P.ptr, a, b)))


def out_dist(P: Points, d: np.ndarray) -> np.ndarray:
    d = np.asarray(d, dtype=np.float32)
    return np.sqrt(d).astype(np.float32) if P.metric == L2 else d


def greedy_search(P: Points, G: np.ndarray, q: int, S, L: int, k: int, visit_cap: int = 0):
    """Algorithm 1 for one query. Returns (ids, dis) of the k closest points
    of (L u V) minus q, and the visited set sorted by (dis, id) when
    visit_cap > 0 (as (ids, dis, |V|))."""
    G = np.ascontiguousarray(G, dtype=np.int32)
    S = np.ascontiguousarray(np.asarray(S, dtype=np.int32).reshape(-1))
    ids = np.full(max(k, 1), -1, np.int32)
    ds = np.zeros(max(k, 1), np.float32)
    nv = ctypes.c_int64(0)
    vi = np.full(max(visit_cap, 1), -1, np.int32)
    vd = np.zeros(max(visit_cap, 1), np.float32)
    cnt = _load().orc_greedy_search(P.ptr, _p(G), G.shape[1], q, _p(S), S.size, L, k, _p(ids), _p(ds),
                                    _p(vi) if visit_cap > 0 else None,
                                    _p(vd) if visit_cap > 0 else None, visit_cap, ctypes.byref(nv))
    res = (ids[:cnt].copy(), ds[:cnt].copy())
    if visit_cap > 0:
        m = min(nv.value, visit_cap)
        return res, (vi[:m].copy(), vd[:m].copy(), nv.value)
    return res


def knn_density(P: Points, G: np.ndarray, L: int, k: int, density: int = DENS_KTH,
                normalize: bool = False, threads: int | None = None):
    """k-NN of every point on G (start = the point itself) and its density.
    G None: no index (Sec. 5.1, brute force), the exact k-NN of every point.
    Returns dict ids (n,k) int32, dist (n,k) f32, rho (n,) f32, key (n,) f32,
    fallback (n,) int32."""
    G = np.ascontiguousarray(G, dtype=np.int32) if G is not None else None
    n = P.n
    ids = np.empty((n, k), np.int32)
    dist = np.empty((n, k), np.float32)
    rho = np.empty(n, np.float32)
    key = np.empty(n, np.float32)
    fb = np.empty(n, np.int32)
    rc = _load().orc_knn_density(P.ptr, _p(G) if G is not None else None, G.shape[1] if G is not None else 0, L,
                                 k, density, int(normalize), _p(ids), _p(dist),
                                 _p(rho), _p(key), _p(fb), threads or default_threads())
    if rc:
        raise ValueError("orc_knn_density: bad arguments")
    return dict(ids=ids, dist=dist, rho=rho, key=key, fallback=fb)


def knn_density_rows(P: Points, G, rows, L: int, k: int, density: int = DENS_KTH, threads: int | None = None):
    """knn_density for the listed points only (no normalisation). G None: the
    brute-force index. Returns dict ids (m,k), dist (m,k), rho (m,), key (m,),
    fallback (m,)."""
    G = np.ascontiguousarray(G, dtype=np.int32) if G is not None else None
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    m = len(rows)
    ids = np.empty((m, k), np.int32)
    dist = np.empty((m, k), np.float32)
    rho = np.empty(m, np.float32)
    key = np.empty(m, np.float32)
    fb = np.empty(m, np.int32)
    rc = _load().orc_knn_density_rows(P.ptr, _p(G) if G is not None else None, G.shape[1] if G is not None else 0,
                                      L, k, density, _p(rows), m, _p(ids), _p(dist), _p(rho), _p(key), _p(fb),
                                      threads or default_threads())
    if rc:
        raise ValueError("orc_knn_density_rows: bad arguments")
    return dict(ids=ids, dist=dist, rho=rho, key=key, fallback=fb)


def nndescent(P: Points, K: int, init: np.ndarray, rounds: int, alpha: float, R: int, threads: int | None = None):
    """NN-Descent graph index (the paper's PyNNDescent option, Sec. 5.1):
    synchronous rounds from the given initial lists (repeats x n x K), the
    repeats merged, then RobustPrune and reverse edges. Returns dict knn (n,K)
    int32, G (n,R) int32, changes (repeats, rounds) int64."""
    init = np.ascontiguousarray(init, dtype=np.int32)
    repeats = init.shape[0]
    n = P.n
    knn = np.empty((n, K), np.int32)
    G = np.empty((n, R), np.int32)
    ch = np.zeros((repeats, max(rounds, 1)), np.int64)
    rc = _load().orc_nndescent(P.ptr, K, repeats, _p(init), rounds, alpha, R, _p(knn), _p(G), _p(ch),
                               threads or default_threads())
    if rc:
        raise ValueError("orc_nndescent: bad arguments")
    return dict(knn=knn, G=G, changes=ch[:, :rounds])


def hcnng(P: Points, repeats: int, leaf_size: int, mst_deg: int, alpha: float, R: int, seed: int = 0,
          threads: int | None = None):
    """HCNNG graph index (the paper's HCNNG option, Sec. 5.1): per repeat a
    random hierarchical split into leaves of at most leaf_size points and a
    degree-bounded minimum spanning forest in every leaf; the union of the
    forests, pruned by RobustPrune. Returns dict G (n,R) int32, leaves
    (repeats,) int64."""
    G = np.empty((P.n, R), np.int32)
    leaves = np.zeros(repeats, np.int64)
    rc = _load().orc_hcnng(P.ptr, repeats, leaf_size, mst_deg, alpha, R, seed, _p(G), _p(leaves),
                           threads or default_threads())
    if rc:
        raise ValueError("orc_hcnng: bad arguments")
    return dict(G=G, leaves=leaves)


def splitmix64(x: int) -> int:
    """SplitMix64's output for the state x (the HCNNG pivot generator)."""
    return int(_load().orc_splitmix64(x))


def hcnng_draw(seed: int, t: int, b: int, m: int, j: int) -> int:
    """Draw j of the HCNNG node [b, b + m) of tree t."""
    return int(_load().orc_hcnng_draw(seed, t, b, m, j))


def hcnng_partition(P: Points, t: int, leaf_size: int, seed: int = 0):
    """The leaves of HCNNG tree t: list of int32 id arrays, in order."""
    order = np.empty(P.n, np.int32)
    begin = np.empty(P.n + 1, np.int64)
    nl = _load().orc_hcnng_partition(P.ptr, t, leaf_size, seed, _p(order), _p(begin))
    return [order[begin[i]:begin[i + 1]].copy() for i in range(nl)]


def hcnng_leaf_mst(P: Points, ids: np.ndarray, mst_deg: int):
    """Degree-bounded minimum spanning forest of the points ids (ascending):
    (e, 2) int32 id pairs in the order they were taken."""
    ids = np.ascontiguousarray(ids, dtype=np.int32)
    edges = np.empty((max(len(ids) - 1, 1), 2), np.int32)
    ne = _load().orc_hcnng_leaf_mst(P.ptr, _p(ids), len(ids), mst_deg, _p(edges))
    return edges[:ne]


def dependent_points(P: Points, G: np.ndarray, key: np.ndarray, knn_ids: np.ndarray, Ld: int,
                     threshold: int = 300, max_rounds: int = 30, max_beam: int = 1 << 30,
                     threads: int | None = None):
    """Algorithm 3. G None: no index (Sec. 5.1, brute force), FindKnn is the
    exact k_dep-NN. Returns dict lam (n,) int32, delta (n,) f32, stats."""
    G = np.ascontiguousarray(G, dtype=np.int32) if G is not None else None
    key = np.ascontiguousarray(key, dtype=np.float32)
    knn_ids = np.ascontiguousarray(knn_ids, dtype=np.int32)
    n, k = knn_ids.shape
    lam = np.empty(n, np.int32)
    delta = np.empty(n, np.float32)
    stats = np.zeros(64, np.int64)
    _load().orc_dependent_points(P.ptr, _p(G) if G is not None else None, G.shape[1] if G is not None else 0,
                                 _p(key), _p(knn_ids), k, Ld, threshold, max_rounds,
                                 max_beam, _p(lam), _p(delta), _p(stats), threads or default_threads())
    rounds = int(stats[0])
    return dict(lam=lam, delta=delta, rounds=rounds, unfinished_round0=int(stats[1]),
                unfinished=[int(x) for x in stats[2:2 + rounds]], tail=int(stats[63]))


def cluster(rho, lam, delta, center: int = CENTER_PRODUCT, rho_min: float = 0.0,
            delta_min: float = 0.0, n_clusters: int = 1, knn_ids=None, rank_key=None):
    """Noise, centers and union-find (Algorithm 2 lines 5-7). Returns
    (labels, number_of_clusters); labels name each cluster by its root.
    The local center function (Appendix, center functions) also needs the
    k-NN lists (n x k) and the rank keys."""
    rho = np.ascontiguousarray(rho, dtype=np.float32)
    lam = np.ascontiguousarray(lam, dtype=np.int32)
    delta = np.ascontiguousarray(delta, dtype=np.float32)
    n = rho.size
    labels = np.empty(n, np.int32)
    if center == CENTER_LOCAL:
        knn_ids = np.ascontiguousarray(knn_ids, dtype=np.int32).reshape(n, -1)
        rank_key = np.ascontiguousarray(rank_key, dtype=np.float32)
        nc = _load().orc_cluster_local(n, knn_ids.shape[1], _p(knn_ids), _p(rank_key), _p(rho), _p(lam),
                                       np.float32(rho_min), _p(labels))
    else:
        nc = _load().orc_cluster(n, _p(rho), _p(lam), _p(delta), center, np.float32(rho_min),
                                 np.float32(delta_min), n_clusters, _p(labels))
    if nc < 0:
        raise ValueError("orc_cluster: the dependent forest is inconsistent")
    return labels, int(nc)


def robust_prune(P: Points, p: int, cand, alpha: float, R: int) -> np.ndarray:
    cand = np.ascontiguousarray(np.asarray(cand, dtype=np.int32).reshape(-1))
    out = np.full(R, -1, np.int32)
    m = _load().orc_robust_prune(P.ptr, p, _p(cand), cand.size, np.float32(alpha), R, _p(out))
    return out[:m].copy()


def search_counts(P: Points, G: np.ndarray, queries, L: int, threads: int | None = None):
    """Per query: (expansions incl. the query's own out-list, distinct
    distance evaluations) of Algorithm 1 with start set {q}, beam L."""
    G = np.ascontiguousarray(G, dtype=np.int32)
    q = np.ascontiguousarray(np.asarray(queries, dtype=np.int32).reshape(-1))
    e = np.zeros(q.size, np.int64)
    c = np.zeros(q.size, np.int64)
    _load().orc_search_counts(P.ptr, _p(G), G.shape[1], L, _p(q), q.size, _p(e), _p(c),
                              threads or default_threads())
    return e, c


def batch_cap(n: int, batch_frac: float) -> int:
    return int(_load().orc_batch_cap(n, np.float32(batch_frac)))


def build_graph(P: Points, R: int, L: int, alpha: float, perm: np.ndarray, n_start: int,
                batch_frac: float = 0.02, visit_cap: int | None = None, threads: int | None = None,
                passes: int = 1):
    """Batched Vamana construction (passes = 2: first pass with alpha = 1).
    Returns G (n x R int32, -1 padded)."""
    perm = np.ascontiguousarray(perm, dtype=np.int32)
    G = np.empty((P.n, R), np.int32)
    rc = _load().orc_build_graph(P.ptr, R, L, np.float32(alpha), _p(perm), n_start, np.float32(batch_frac),
                                 visit_cap if visit_cap else 2 * L, passes, _p(G), threads or default_threads())
    if rc:
        raise ValueError("orc_build_graph: bad arguments")
    return G
