"""BF16 traversal with exact FP32 re-rank, against the FP32 path on the same graph.

Bit-for-bit parity is not defined for the traversal itself (BF16 distances
decide the beam). What is fixed: every distance the library reports is the
canonical FP32 distance of the reported pair (checked against the oracle's
FP32 distance), k-NN recall against the FP32 path is >= 0.95, and the
clusters agree with the FP32 clusters to ARI >= 0.99.
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import exact
from paper_2312_03940_gb300 import pecann as pc
from paper_2312_03940_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    pc.load_library()


def run(ds, G, p):
    ws = pc.workspace(ds, p)
    dens = pc.pecann_density(ds, G, p, ws=ws)
    dep = pc.pecann_dependent_points(ds, G, p, dens["rank_key"], dens["knn_ids"], dens["knn_dist"], ws=ws)
    lab, nc = pc.pecann_cluster(dens["density"], dep["dep"], dep["dep_dist"], p)
    out = {k: v.cpu().numpy() for k, v in dens.items()}
    out.update(dep=dep["dep"].cpu().numpy(), dep_dist=dep["dep_dist"].cpu().numpy(), labels=lab.cpu().numpy(),
               stats=dep["stats"])
    return out


def recall_vs(ref_dist, got_dist):
    kth = ref_dist[:, -1:]
    return float((got_dist <= kth * (1 + 1e-5) + 1e-30).mean())


@pytest.mark.parametrize("kind", ["l2-384", "ip-1024"])
def test_bf16_traversal_matches_fp32(kind):
    if kind == "l2-384":
        X, gt = synth.powerlaw_sphere(n=20000, d=384, components=200, seed=81)
        metric, k, R, L, nc = pc.L2, 20, 48, 128, 200
        density = pc.DENS_KTH
    else:
        X, gt = synth.vmf_like(n=12000, d=1024, components=100, seed=82)
        metric, k, R, L, nc = pc.IP, 16, 64, 128, 100
        density = pc.DENS_KTH
    Xd = torch.from_numpy(X).cuda()
    Xb = Xd.to(torch.bfloat16).contiguous()
    p = pc.params(k=k, R=R, L_build=L, L_search=L, L_dep=L, alpha=1.2, n_start=256, build_passes=2,
                  n_clusters=nc, density=density)
    ds32 = pc.Dataset(Xd, metric=metric)
    dsb = pc.Dataset(Xb, metric=metric, data_f32=Xd)
    G, _ = pc.pecann_build_graph(ds32, p, order=torch.from_numpy(synth.insertion_order(len(X), seed=83)).cuda())
    # a BF16 dataset builds on its FP32 rows: the same graph
    Gb, _ = pc.pecann_build_graph(dsb, p, order=torch.from_numpy(synth.insertion_order(len(X), seed=83)).cuda())
    assert torch.equal(G, Gb)
    r32 = run(ds32, G, p)
    rb = run(dsb, G, p)
    # every reported distance is the exact FP32 distance of the reported pair
    P = oracle.Points(X, metric=metric)
    rows = synth.sample_ids(len(X), 300, seed=84)
    for i in rows:
        for t in range(k):
            j = int(rb["knn_ids"][i, t])
            assert rb["knn_dist"][i, t] == np.float32(oracle.out_dist(P, oracle.dis(P, int(i), j)))
        lam = int(rb["dep"][i])
        if lam >= 0:
            assert rb["dep_dist"][i] == np.float32(oracle.out_dist(P, oracle.dis(P, int(i), lam)))
    # lists are sorted by the exact distances
    assert (np.diff(rb["knn_dist"], axis=1) >= 0).all()
    assert recall_vs(r32["knn_dist"], rb["knn_dist"]) >= 0.95
    assert exact.ari(rb["labels"], r32["labels"]) >= 0.99
    # where the k-NN lists agree, the densities are identical
    same = (rb["knn_ids"] == r32["knn_ids"]).all(1)
    assert same.mean() > 0.5
    assert (rb["density"][same] == r32["density"][same]).all()


def test_bf16_requires_fp32_rows():
    X = torch.zeros((100, 256), dtype=torch.bfloat16, device="cuda")
    G = torch.zeros((100, 8), dtype=torch.int32, device="cuda")
    p = pc.params(k=4, R=8, L_search=8)
    ds = pc.Dataset(X)
    with pytest.raises(pc.PecannError) as e:
        pc.pecann_density(ds, G, p, ws=torch.empty(1 << 20, dtype=torch.uint8, device="cuda"))
    assert e.value.status == pc.EINVAL
