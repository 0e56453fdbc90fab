"""Batched form: many point sets of uneven sizes and dimensions in one pass.

Each set's results must equal, element for element, what the single-set
calls give for that set (which the parity tests tie to the oracle); one set
is also compared with the oracle directly. The pass must also replay from a
CUDA graph with identical results.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2312_03940_gb300 import pecann as pc
from paper_2312_03940_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    pc.load_library()


def make_sets(seed=91):
    g = np.random.default_rng(seed)
    sets = []
    for i, (n, d) in enumerate([(1500, 96), (6000, 128), (800, 32), (3500, 256), (2500, 384), (4000, 64)]):
        X, lab = synth.gaussian_mixture(n=n, d=d, components=int(g.integers(3, 12)), seed=seed + i)
        sets.append((X, lab))
    return sets


def single(ds, G, p):
    ws = pc.workspace(ds, p)
    dens = pc.pecann_density(ds, G, p, ws=ws)
    dep = pc.pecann_dependent_points(ds, G, p, dens["rank_key"], dens["knn_ids"], dens["knn_dist"], ws=ws)
    lab, _ = pc.pecann_cluster(dens["density"], dep["dep"], dep["dep_dist"], p)
    out = {k: v.cpu().numpy() for k, v in dens.items()}
    out.update(dep=dep["dep"].cpu().numpy(), dep_dist=dep["dep_dist"].cpu().numpy(), labels=lab.cpu().numpy())
    return out


@pytest.mark.parametrize("threshold", [300, 10])
def test_batched_equals_single_set_calls(threshold):
    sets = make_sets()
    p = pc.params(k=8, R=32, L_build=96, L_search=96, L_dep=96, alpha=1.2, n_start=16, dep_threshold=threshold)
    ncl = [5, 9, 3, 7, 4, 6]
    dss, graphs = [], []
    for i, (X, _) in enumerate(sets):
        ds = pc.Dataset(torch.from_numpy(X).cuda())
        G, _ = pc.pecann_build_graph(ds, p, order=torch.from_numpy(synth.insertion_order(len(X), seed=i)).cuda())
        dss.append(ds)
        graphs.append(G)
    batch = pc.Batch(dss, graphs, p, n_clusters=ncl)
    out = {k: v.cpu().numpy() for k, v in batch.run().items()}
    for i, (ds, G) in enumerate(zip(dss, graphs)):
        pi = pc.params(k=8, R=32, L_build=96, L_search=96, L_dep=96, alpha=1.2, n_start=16, dep_threshold=threshold,
                       n_clusters=ncl[i])
        ref = single(ds, G, pi)
        a, b = batch.offsets[i], batch.offsets[i + 1]
        for key in ("knn_ids", "knn_dist", "density", "rank_key", "dep", "dep_dist", "labels"):
            assert np.array_equal(out[key][a:b], ref[key]), (i, key)
    # one set against the oracle directly
    X = sets[1][0]
    P = oracle.Points(X)
    Gh = graphs[1].cpu().numpy()
    o = oracle.knn_density(P, Gh, L=96, k=8)
    d = oracle.dependent_points(P, Gh, o["key"], o["ids"], Ld=96, threshold=threshold)
    lo, _ = oracle.cluster(o["rho"], d["lam"], d["delta"], center=oracle.CENTER_PRODUCT, n_clusters=ncl[1])
    a, b = batch.offsets[1], batch.offsets[2]
    assert np.array_equal(out["knn_ids"][a:b], o["ids"])
    assert np.array_equal(out["dep"][a:b], d["lam"])
    assert np.array_equal(out["labels"][a:b], lo)


def test_batched_replays_from_a_cuda_graph():
    sets = make_sets(seed=97)[:4]
    p = pc.params(k=8, R=32, L_build=96, L_search=96, L_dep=96, alpha=1.2, n_start=16, n_clusters=5)
    dss, graphs = [], []
    for i, (X, _) in enumerate(sets):
        ds = pc.Dataset(torch.from_numpy(X).cuda())
        G, _ = pc.pecann_build_graph(ds, p, order=torch.from_numpy(synth.insertion_order(len(X), seed=i)).cuda())
        dss.append(ds)
        graphs.append(G)
    batch = pc.Batch(dss, graphs, p)
    ref = {k: v.clone() for k, v in batch.run().items()}
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        batch.run(stream=s)  # warm-up on the capture stream
    s.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        batch.run(stream=s)
    for v in batch.out.values():
        v.fill_(0)
    graph.replay()
    torch.cuda.synchronize()
    for k in ref:
        assert torch.equal(batch.out[k], ref[k]), k
