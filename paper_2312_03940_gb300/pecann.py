"""Python binding of the C ABI declared in include/pecann.h.

Argument marshalling only: each function checks and converts torch tensors
to raw device pointers and calls the entry point of the same name in
libpecann.so. Every step of the computation runs in the library's CUDA
kernels; there is no CPU fallback. If the library has not been built, the
first call raises.
"""
from __future__ import annotations

import ctypes
import os

import torch

from . import build as _build

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, EUNSUPPORTED, EINTERNAL = range(7)
F32, U8, BF16, FP8E4M3 = 0, 1, 2, 3
L2, IP = 0, 1
DENS_KTH, DENS_EXPSUM, DENS_SUMEXP, DENS_SUM = 0, 1, 2, 3
CENTER_THRESHOLD, CENTER_PRODUCT, CENTER_LOCAL = 0, 1, 2
INDEX_GRAPH, INDEX_BRUTE_FORCE = 0, 1

_DTYPES = {torch.float32: F32, torch.uint8: U8, torch.bfloat16: BF16}
if hasattr(torch, "float8_e4m3fn"):
    _DTYPES[torch.float8_e4m3fn] = FP8E4M3


class PecannParams(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int32), ("R", ctypes.c_int32), ("L_build", ctypes.c_int32),
                ("L_search", ctypes.c_int32), ("L_dep", ctypes.c_int32), ("alpha", ctypes.c_float),
                ("n_start", ctypes.c_int32), ("batch_frac", ctypes.c_float), ("visit_cap", ctypes.c_int32),
                ("dep_threshold", ctypes.c_int32), ("max_dep_rounds", ctypes.c_int32),
                ("max_dep_beam", ctypes.c_int32), ("density", ctypes.c_int32),
                ("normalize_density", ctypes.c_int32), ("center", ctypes.c_int32), ("rho_min", ctypes.c_float),
                ("delta_min", ctypes.c_float), ("n_clusters", ctypes.c_int32), ("hash_slots", ctypes.c_int32),
                ("collect_work", ctypes.c_int32), ("build_passes", ctypes.c_int32), ("rerank_k", ctypes.c_int32), ("block_warps", ctypes.c_int32),
                ("index", ctypes.c_int32),
                ("seed", ctypes.c_uint64)]


class PecannDataset(ctypes.Structure):
    _fields_ = [("data", ctypes.c_void_p), ("n", ctypes.c_int64), ("d", ctypes.c_int32),
                ("dtype", ctypes.c_int32), ("metric", ctypes.c_int32), ("reserved0", ctypes.c_int32),
                ("dim_scale", ctypes.c_void_p), ("data_f32", ctypes.c_void_p)]


class PecannClusterSetting(ctypes.Structure):
    _fields_ = [("center", ctypes.c_int32), ("rho_min", ctypes.c_float), ("delta_min", ctypes.c_float),
                ("n_clusters", ctypes.c_int32)]


EXPORTS = ["pecann_params_default", "pecann_status_string", "pecann_last_error", "pecann_version",
           "pecann_kernel_launches",
           "pecann_workspace_size", "pecann_search", "pecann_build_graph", "pecann_nndescent_workspace_size",
           "pecann_build_nndescent", "pecann_hcnng_workspace_size", "pecann_build_hcnng", "pecann_density",
           "pecann_dependent_points", "pecann_cluster", "pecann_density_noalloc", "pecann_batch_workspace_size",
           "pecann_batch_prepare", "pecann_run_batched", "pecann_cluster_workspace_size", "pecann_cluster_sweep"]

NOALLOC_MAX_POINTS = 1 << 20

_lib = None


def library_path() -> str:
    return _build.LIB


def load_library(path: str | None = None):
    """Load libpecann.so (no GPU needed) and declare every entry point."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    path = path or _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"the CUDA library is not built ({path} is missing); "
                           "run `python -m paper_2312_03940_gb300.build`")
    lib = ctypes.CDLL(path)
    P = ctypes.POINTER(PecannParams)
    D = ctypes.POINTER(PecannDataset)
    vp, i32, i64, sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t
    lib.pecann_params_default.argtypes = [P]
    lib.pecann_params_default.restype = None
    lib.pecann_status_string.argtypes = [ctypes.c_int]
    lib.pecann_status_string.restype = ctypes.c_char_p
    lib.pecann_last_error.argtypes = []
    lib.pecann_last_error.restype = ctypes.c_char_p
    lib.pecann_version.argtypes = []
    lib.pecann_version.restype = i32
    lib.pecann_kernel_launches.argtypes = []
    lib.pecann_kernel_launches.restype = i64
    lib.pecann_workspace_size.argtypes = [D, P, ctypes.POINTER(sz)]
    lib.pecann_search.argtypes = [D, vp, i32, vp, i64, vp, i32, i32, i32, vp, vp, vp, P, vp, sz, vp]
    lib.pecann_build_graph.argtypes = [D, P, vp, vp, vp, vp, sz, vp]
    lib.pecann_nndescent_workspace_size.argtypes = [D, P, i32, i32, ctypes.POINTER(sz)]
    lib.pecann_build_nndescent.argtypes = [D, P, i32, i32, vp, i32, vp, vp, vp, vp, vp, sz, vp]
    lib.pecann_hcnng_workspace_size.argtypes = [D, P, i32, i32, i32, ctypes.POINTER(sz)]
    lib.pecann_build_hcnng.argtypes = [D, P, i32, i32, i32, vp, vp, vp, vp, sz, vp]
    lib.pecann_density.argtypes = [D, vp, P, vp, vp, vp, vp, vp, sz, vp]
    lib.pecann_dependent_points.argtypes = [D, vp, P, vp, vp, vp, vp, vp, ctypes.POINTER(i64), vp, sz, vp]
    lib.pecann_cluster.argtypes = [i64, vp, vp, vp, P, vp, ctypes.POINTER(i64), vp, sz, vp]
    lib.pecann_density_noalloc.argtypes = [D, vp, P, vp, vp, vp, vp, vp]
    lib.pecann_cluster_workspace_size.argtypes = [i64, i32, ctypes.POINTER(sz)]
    lib.pecann_cluster_sweep.argtypes = [i64, vp, vp, vp, vp, i32, vp, i32, ctypes.POINTER(PecannClusterSetting),
                                         vp, ctypes.POINTER(i64), vp, sz, vp]
    for f in ["pecann_workspace_size", "pecann_search", "pecann_build_graph", "pecann_nndescent_workspace_size",
              "pecann_build_nndescent", "pecann_hcnng_workspace_size", "pecann_build_hcnng", "pecann_density",
              "pecann_dependent_points", "pecann_cluster", "pecann_density_noalloc", "pecann_batch_workspace_size",
              "pecann_batch_prepare", "pecann_run_batched", "pecann_cluster_workspace_size", "pecann_cluster_sweep"]:
        getattr(lib, f).restype = ctypes.c_int
    if path == _build.LIB:
        _lib = lib
    return lib


class PecannError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(msg)
        self.status = status


def _check(status: int):
    if status != OK:
        lib = load_library()
        raise PecannError(status, f"{lib.pecann_status_string(status).decode()}: "
                                  f"{lib.pecann_last_error().decode()}")


def params(**kw) -> PecannParams:
    """The library defaults with the given fields replaced."""
    p = PecannParams()
    load_library().pecann_params_default(ctypes.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def _cuda(t: torch.Tensor, name: str, dtype=None) -> torch.Tensor:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


class Dataset:
    """A point set on the GPU as the library sees it (keeps tensors alive)."""

    def __init__(self, X: torch.Tensor, metric: int = L2, dim_scale: torch.Tensor | None = None,
                 data_f32: torch.Tensor | None = None):
        _cuda(X, "X")
        if X.dim() != 2 or X.dtype not in _DTYPES:
            raise ValueError("X must be a 2-D float32 / uint8 / bfloat16 / float8_e4m3fn tensor")
        self.X, self.dim_scale, self.data_f32 = X, dim_scale, data_f32
        self.n, self.d = X.shape
        self.metric = metric
        self.c = PecannDataset(X.data_ptr(), self.n, self.d, _DTYPES[X.dtype], metric, 0,
                               dim_scale.data_ptr() if dim_scale is not None else None,
                               data_f32.data_ptr() if data_f32 is not None else None)

    @property
    def ref(self):
        return ctypes.byref(self.c)


def pecann_kernel_launches() -> int:
    """Kernels launched by the library so far in this process."""
    return int(load_library().pecann_kernel_launches())


def pecann_workspace_size(ds: Dataset, p: PecannParams) -> int:
    b = ctypes.c_size_t(0)
    _check(load_library().pecann_workspace_size(ds.ref, ctypes.byref(p), ctypes.byref(b)))
    return b.value


def work_counters(ws: torch.Tensor):
    """(expansions, distance evaluations, beam insertions) left in the workspace by the last
    pecann_search / pecann_density call made with collect_work = 1."""
    v = ws[80:104].cpu().view(torch.int64)
    return int(v[0]), int(v[1]), int(v[2])


def workspace(ds: Dataset, p: PecannParams) -> torch.Tensor:
    return torch.empty(pecann_workspace_size(ds, p), dtype=torch.uint8, device=ds.X.device)


def pecann_search(ds: Dataset, graph: torch.Tensor, queries: torch.Tensor, L: int, k: int,
                  start: torch.Tensor | None = None, p: PecannParams | None = None,
                  ws: torch.Tensor | None = None, stream=None):
    """Algorithm 1 for the given query ids. Returns (ids (m,k), dis (m,k), count (m,))."""
    _cuda(graph, "graph", torch.int32)
    _cuda(queries, "queries", torch.int32)
    if start is not None:
        _cuda(start, "start", torch.int32)
    p = p or params()
    ws = ws if ws is not None else workspace(ds, p)
    m = queries.numel()
    ids = torch.empty((m, k), dtype=torch.int32, device=ds.X.device)
    dis = torch.empty((m, k), dtype=torch.float32, device=ds.X.device)
    cnt = torch.empty(m, dtype=torch.int32, device=ds.X.device)
    _check(load_library().pecann_search(ds.ref, _ptr(graph), graph.shape[1], _ptr(queries), m, _ptr(start),
                                        0 if start is None else start.numel(), L, k, _ptr(ids), _ptr(dis),
                                        _ptr(cnt), ctypes.byref(p), _ptr(ws), ws.numel(), _stream(stream)))
    return ids, dis, cnt


def pecann_build_graph(ds: Dataset, p: PecannParams, order: torch.Tensor | None = None,
                       ws: torch.Tensor | None = None, stream=None, graph: torch.Tensor | None = None,
                       degree: torch.Tensor | None = None):
    """Batched Vamana construction. Returns (graph (n,R) int32, degree (n,) int32)."""
    if order is not None:
        _cuda(order, "order", torch.int32)
    ws = ws if ws is not None else workspace(ds, p)
    dev = ds.X.device
    graph = graph if graph is not None else torch.empty((ds.n, p.R), dtype=torch.int32, device=dev)
    degree = degree if degree is not None else torch.empty(ds.n, dtype=torch.int32, device=dev)
    _check(load_library().pecann_build_graph(ds.ref, ctypes.byref(p), _ptr(order), _ptr(graph), _ptr(degree),
                                             _ptr(ws), ws.numel(), _stream(stream)))
    return graph, degree


def pecann_build_nndescent(ds: Dataset, p: PecannParams, K: int, init: torch.Tensor, rounds: int,
                           ws: torch.Tensor | None = None, stream=None):
    """NN-Descent graph index from the initial lists init (repeats, n, K) int32
    on the device. Returns dict graph (n,R), degree (n,), knn (n,K) int32 and
    changes (repeats, rounds) int64 on the host."""
    _cuda(init, "init", torch.int32)
    if init.dim() != 3 or init.shape[1] != ds.n or init.shape[2] != K:
        raise ValueError("init must have shape (repeats, n, K)")
    repeats = init.shape[0]
    lib = load_library()
    if ws is None:
        nb = ctypes.c_size_t(0)
        _check(lib.pecann_nndescent_workspace_size(ds.ref, ctypes.byref(p), K, repeats, ctypes.byref(nb)))
        ws = torch.empty(nb.value, dtype=torch.uint8, device=ds.X.device)
    dev = ds.X.device
    graph = torch.empty((ds.n, p.R), dtype=torch.int32, device=dev)
    degree = torch.empty(ds.n, dtype=torch.int32, device=dev)
    knn = torch.empty((ds.n, K), dtype=torch.int32, device=dev)
    changes = torch.zeros((repeats, max(rounds, 1)), dtype=torch.int64)  # host
    _check(lib.pecann_build_nndescent(ds.ref, ctypes.byref(p), K, repeats, _ptr(init), rounds, _ptr(graph),
                                      _ptr(degree), _ptr(knn), ctypes.c_void_p(changes.data_ptr()),
                                      _ptr(ws), ws.numel(), _stream(stream)))
    return dict(graph=graph, degree=degree, knn=knn, changes=changes[:, :rounds].numpy())


def pecann_build_hcnng(ds: Dataset, p: PecannParams, repeats: int, leaf_size: int, mst_deg: int,
                       ws: torch.Tensor | None = None, stream=None):
    """HCNNG graph index (p.R, p.alpha, p.seed). Returns dict graph (n,R),
    degree (n,) int32 and leaves (repeats,) int64 on the host."""
    lib = load_library()
    if ws is None:
        nb = ctypes.c_size_t(0)
        _check(lib.pecann_hcnng_workspace_size(ds.ref, ctypes.byref(p), repeats, leaf_size, mst_deg,
                                               ctypes.byref(nb)))
        ws = torch.empty(nb.value, dtype=torch.uint8, device=ds.X.device)
    dev = ds.X.device
    graph = torch.empty((ds.n, p.R), dtype=torch.int32, device=dev)
    degree = torch.empty(ds.n, dtype=torch.int32, device=dev)
    leaves = torch.zeros(repeats, dtype=torch.int64)  # host
    _check(lib.pecann_build_hcnng(ds.ref, ctypes.byref(p), repeats, leaf_size, mst_deg, _ptr(graph), _ptr(degree),
                                  ctypes.c_void_p(leaves.data_ptr()), _ptr(ws), ws.numel(), _stream(stream)))
    return dict(graph=graph, degree=degree, leaves=leaves.numpy())


def pecann_density(ds: Dataset, graph: torch.Tensor, p: PecannParams, ws: torch.Tensor | None = None,
                   stream=None, out: dict | None = None):
    """k-NN and density of every point. Returns dict knn_ids, knn_dist, density, rank_key.
    graph may be None with p.index = INDEX_BRUTE_FORCE."""
    if graph is not None:
        _cuda(graph, "graph", torch.int32)
    ws = ws if ws is not None else workspace(ds, p)
    dev = ds.X.device
    if out is None:
        out = dict(knn_ids=torch.empty((ds.n, p.k), dtype=torch.int32, device=dev),
                   knn_dist=torch.empty((ds.n, p.k), dtype=torch.float32, device=dev),
                   density=torch.empty(ds.n, dtype=torch.float32, device=dev),
                   rank_key=torch.empty(ds.n, dtype=torch.float32, device=dev))
    _check(load_library().pecann_density(ds.ref, _ptr(graph), ctypes.byref(p), _ptr(out["knn_ids"]),
                                         _ptr(out["knn_dist"]), _ptr(out["density"]), _ptr(out["rank_key"]),
                                         _ptr(ws), ws.numel(), _stream(stream)))
    return out


def pecann_density_noalloc(ds: Dataset, graph: torch.Tensor, p: PecannParams, stream=None,
                           out: dict | None = None):
    """pecann_density for callers that cannot allocate GPU memory: no
    workspace; the library's fixed scratch array serves (n <= 2^20, and calls
    that overlap on the GPU must be serialised by the caller). Outputs are
    still allocated here unless `out` provides them."""
    _cuda(graph, "graph", torch.int32)
    dev = ds.X.device
    if out is None:
        out = dict(knn_ids=torch.empty((ds.n, p.k), dtype=torch.int32, device=dev),
                   knn_dist=torch.empty((ds.n, p.k), dtype=torch.float32, device=dev),
                   density=torch.empty(ds.n, dtype=torch.float32, device=dev),
                   rank_key=torch.empty(ds.n, dtype=torch.float32, device=dev))
    _check(load_library().pecann_density_noalloc(ds.ref, _ptr(graph), ctypes.byref(p), _ptr(out["knn_ids"]),
                                                 _ptr(out["knn_dist"]), _ptr(out["density"]),
                                                 _ptr(out["rank_key"]), _stream(stream)))
    return out


def pecann_dependent_points(ds: Dataset, graph: torch.Tensor, p: PecannParams, rank_key: torch.Tensor,
                            knn_ids: torch.Tensor, knn_dist: torch.Tensor, ws: torch.Tensor | None = None,
                            stream=None, out: dict | None = None):
    """Algorithm 3. Returns dict dep, dep_dist, stats (list of 64 ints).
    graph may be None with p.index = INDEX_BRUTE_FORCE."""
    if graph is not None:
        _cuda(graph, "graph", torch.int32)
    _cuda(rank_key, "rank_key", torch.float32)
    _cuda(knn_ids, "knn_ids", torch.int32)
    _cuda(knn_dist, "knn_dist", torch.float32)
    ws = ws if ws is not None else workspace(ds, p)
    dev = ds.X.device
    if out is None:
        out = dict(dep=torch.empty(ds.n, dtype=torch.int32, device=dev),
                   dep_dist=torch.empty(ds.n, dtype=torch.float32, device=dev))
    stats = (ctypes.c_int64 * 64)()
    _check(load_library().pecann_dependent_points(ds.ref, _ptr(graph), ctypes.byref(p), _ptr(rank_key),
                                                  _ptr(knn_ids), _ptr(knn_dist), _ptr(out["dep"]),
                                                  _ptr(out["dep_dist"]), stats, _ptr(ws), ws.numel(),
                                                  _stream(stream)))
    out["stats"] = list(stats)
    return out


def pecann_cluster(density: torch.Tensor, dep: torch.Tensor, dep_dist: torch.Tensor, p: PecannParams,
                   ws: torch.Tensor | None = None, stream=None, count: bool = True,
                   labels: torch.Tensor | None = None):
    """Noise, centers and union-find. Returns (labels (n,) int32, number of clusters or None)."""
    _cuda(density, "density", torch.float32)
    _cuda(dep, "dep", torch.int32)
    _cuda(dep_dist, "dep_dist", torch.float32)
    n = density.numel()
    if ws is None:
        nb = ctypes.c_size_t(0)
        _check(load_library().pecann_cluster_workspace_size(n, 1, ctypes.byref(nb)))
        ws = torch.empty(nb.value, dtype=torch.uint8, device=density.device)
    labels = labels if labels is not None else torch.empty(n, dtype=torch.int32, device=density.device)
    nc = ctypes.c_int64(0)
    _check(load_library().pecann_cluster(n, _ptr(density), _ptr(dep), _ptr(dep_dist), ctypes.byref(p),
                                         _ptr(labels), ctypes.byref(nc) if count else None, _ptr(ws),
                                         ws.numel(), _stream(stream)))
    return labels, (nc.value if count else None)


def pecann_cluster_sweep(density: torch.Tensor, dep: torch.Tensor, dep_dist: torch.Tensor, settings,
                         knn_ids: torch.Tensor | None = None, rank_key: torch.Tensor | None = None,
                         ws: torch.Tensor | None = None, stream=None, count: bool = True):
    """Many clusterings of one dependent forest. `settings`: a list of dicts with
    keys center, rho_min, delta_min, n_clusters (missing keys: 0, 0, 0, 1).
    The local center needs knn_ids (n, k) and rank_key. Returns (labels
    (len(settings), n) int32, list of cluster counts or None)."""
    _cuda(density, "density", torch.float32)
    _cuda(dep, "dep", torch.int32)
    _cuda(dep_dist, "dep_dist", torch.float32)
    k = 0
    if knn_ids is not None:
        _cuda(knn_ids, "knn_ids", torch.int32)
        k = knn_ids.shape[1]
    if rank_key is not None:
        _cuda(rank_key, "rank_key", torch.float32)
    n, m = density.numel(), len(settings)
    arr = (PecannClusterSetting * max(m, 1))()
    for i, st in enumerate(settings):
        arr[i] = PecannClusterSetting(int(st.get("center", CENTER_THRESHOLD)), float(st.get("rho_min", 0.0)),
                                      float(st.get("delta_min", 0.0)), int(st.get("n_clusters", 1)))
    lib = load_library()
    if ws is None:
        b = ctypes.c_size_t(0)
        _check(lib.pecann_cluster_workspace_size(n, m, ctypes.byref(b)))
        ws = torch.empty(b.value, dtype=torch.uint8, device=density.device)
    labels = torch.empty((m, n), dtype=torch.int32, device=density.device)
    counts = (ctypes.c_int64 * max(m, 1))()
    _check(lib.pecann_cluster_sweep(n, _ptr(density), _ptr(dep), _ptr(dep_dist), _ptr(knn_ids), k, _ptr(rank_key),
                                    m, arr, _ptr(labels), counts if count else None, _ptr(ws), ws.numel(),
                                    _stream(stream)))
    return labels, ([int(counts[i]) for i in range(m)] if count else None)


class Batch:
    """Many FP32 point sets run together (pecann_batch_prepare /
    pecann_run_batched). `datasets` are Dataset objects; `graphs` their graphs
    (each n_s x R). Outputs are concatenated over the sets in order, with
    set-local ids; `offsets[s]` is the first row of set s."""

    def __init__(self, datasets, graphs, p: PecannParams, n_clusters=None, stream=None):
        if not datasets:
            raise ValueError("no datasets")
        self.datasets, self.p = list(datasets), p
        self.n_sets = len(self.datasets)
        self.sizes = [d.n for d in self.datasets]
        self.offsets = [0]
        for n in self.sizes:
            self.offsets.append(self.offsets[-1] + n)
        self.N = self.offsets[-1]
        dev = self.datasets[0].X.device
        self.graphs = torch.cat([_cuda(g, "graph", torch.int32) for g in graphs]).contiguous()
        arr = (PecannDataset * self.n_sets)()
        for i, d in enumerate(self.datasets):
            arr[i] = d.c
        self.c_sets = arr
        b = ctypes.c_size_t(0)
        lib = load_library()
        _check(lib.pecann_batch_workspace_size(self.n_sets, arr, ctypes.byref(p), ctypes.byref(b)))
        self.ws = torch.empty(b.value, dtype=torch.uint8, device=dev)
        ncl = None
        if n_clusters is not None:
            ncl = (ctypes.c_int32 * self.n_sets)(*[int(x) for x in n_clusters])
        self._ncl = ncl
        _check(lib.pecann_batch_prepare(self.n_sets, arr, _ptr(self.graphs), ncl, ctypes.byref(p), _ptr(self.ws),
                                        self.ws.numel(), _stream(stream)))
        k = p.k
        self.out = dict(knn_ids=torch.empty((self.N, k), dtype=torch.int32, device=dev),
                        knn_dist=torch.empty((self.N, k), dtype=torch.float32, device=dev),
                        density=torch.empty(self.N, dtype=torch.float32, device=dev),
                        rank_key=torch.empty(self.N, dtype=torch.float32, device=dev),
                        dep=torch.empty(self.N, dtype=torch.int32, device=dev),
                        dep_dist=torch.empty(self.N, dtype=torch.float32, device=dev),
                        labels=torch.empty(self.N, dtype=torch.int32, device=dev))

    def run(self, stream=None):
        """pecann_run_batched: one pass over all sets (asynchronous; capturable)."""
        o = self.out
        _check(load_library().pecann_run_batched(self.n_sets, self.c_sets, ctypes.byref(self.p), _ptr(o["knn_ids"]),
                                                 _ptr(o["knn_dist"]), _ptr(o["density"]), _ptr(o["rank_key"]),
                                                 _ptr(o["dep"]), _ptr(o["dep_dist"]), _ptr(o["labels"]),
                                                 _ptr(self.ws), self.ws.numel(), _stream(stream)))
        return o
