"""BF16 / FP8 traversal with exact FP32 re-rank, against the oracle on the same graph.

Bit-for-bit parity is not defined for the traversal itself (reduced-precision
distances decide the beam). What is fixed: every distance the library reports
is the canonical FP32 distance of the reported pair (checked against the
oracle's FP32 distance); k-NN recall against the FP64 exact k-NN is >= 0.95;
and the clusters agree with the oracle's FP32 clusters on the same graph to
ARI >= 0.99. The graph is built by the oracle, so no oracle input comes from
the CUDA path; the FP32 GPU path on it must equal the oracle exactly.
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import exact
from paper_2312_03940_gb300 import pecann as pc
from paper_2312_03940_gb300 import synth

from tests.helpers import quantize_e4m3, random_graph

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


_CASES = {}


def oracle_case(kind):
    """Data, the oracle's graph, its FP32 path on that graph (k-NN, density,
    dependent points, product-center labels) and the FP64 exact k-NN of 1,000
    sampled points. Cached: the two 1024-d variants share one case."""
    if kind in _CASES:
        return _CASES[kind]
    if kind == "l2-384":
        X, _ = synth.powerlaw_sphere(n=20000, d=384, components=200, seed=81)
        metric, k, R, L, nc, n_start = pc.L2, 20, 48, 128, 200, 256
    else:
        X, _ = synth.vmf_like(n=4000, d=1024, components=40, seed=82)
        metric, k, R, L, nc, n_start = pc.IP, 16, 64, 64, 40, 64
    P = oracle.Points(X, metric=metric)
    G = oracle.build_graph(P, R=R, L=L, alpha=1.2, perm=synth.insertion_order(len(X), seed=83),
                           n_start=n_start, passes=2)
    o = oracle.knn_density(P, G, L=L, k=k)
    d = oracle.dependent_points(P, G, o["key"], o["ids"], Ld=L, threshold=300)
    lo, _ = oracle.cluster(o["rho"], d["lam"], d["delta"], center=oracle.CENTER_PRODUCT, n_clusters=nc)
    qs = synth.sample_ids(len(X), 1000, seed=85)
    _, ex = exact.exact_knn_queries(X, qs, k, metric=metric)
    _CASES[kind] = dict(X=X, P=P, G=G, metric=metric, k=k, R=R, L=L, nc=nc, o=o, labels=lo, qs=qs, ex=ex)
    return _CASES[kind]


@pytest.mark.parametrize("kind", ["l2-384", "ip-1024", "fp8-ip-1024"])
def test_reduced_traversal_against_the_oracle(kind):
    c = oracle_case("l2-384" if kind == "l2-384" else "ip-1024")
    X, P, metric, k, R, L = c["X"], c["P"], c["metric"], c["k"], c["R"], c["L"]
    Xd = torch.from_numpy(X).cuda()
    G = torch.from_numpy(c["G"]).cuda()
    p = pc.params(k=k, R=R, L_build=L, L_search=L, L_dep=L, alpha=1.2, n_start=64, build_passes=2,
                  n_clusters=c["nc"])
    ds32 = pc.Dataset(Xd, metric=metric)
    if kind.startswith("fp8"):
        codes, s = quantize_e4m3(X)
        dsb = pc.Dataset(codes.cuda(), metric=metric, dim_scale=torch.from_numpy(s).cuda(), data_f32=Xd)
    else:
        dsb = pc.Dataset(Xd.to(torch.bfloat16).contiguous(), metric=metric, data_f32=Xd)
    # a BF16 / FP8 dataset builds on its FP32 rows: the same graph
    order = torch.from_numpy(synth.insertion_order(len(X), seed=83)).cuda()
    assert torch.equal(pc.pecann_build_graph(ds32, p, order=order)[0], pc.pecann_build_graph(dsb, p, order=order)[0])
    # the FP32 path on the oracle's graph is the oracle's, exactly
    r32 = run(ds32, G, p)
    assert (r32["knn_ids"] == c["o"]["ids"]).all() and (r32["rank_key"] == c["o"]["key"]).all()
    assert (r32["labels"] == c["labels"]).all()
    rb = run(dsb, G, p)
    # every reported distance is the exact FP32 distance of the reported pair
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
    # accuracy: recall against the FP64 exact k-NN, ARI against the oracle's FP32 clusters
    assert exact.knn_recall(rb["knn_dist"][c["qs"]], c["ex"]) >= 0.95
    assert exact.ari(rb["labels"], c["labels"]) >= 0.99
    # where the k-NN lists agree with the oracle's, the densities are identical
    same = (rb["knn_ids"] == c["o"]["ids"]).all(1)
    assert same.mean() > 0.5
    assert (rb["density"][same] == c["o"]["rho"][same]).all()


def test_bf16_requires_fp32_rows():
    X = torch.zeros((100, 256), dtype=torch.bfloat16, device="cuda")
    G = torch.zeros((100, 8), dtype=torch.int32, device="cuda")
    p = pc.params(k=4, R=8, L_search=8)
    ds = pc.Dataset(X)
    with pytest.raises(pc.PecannError) as e:
        pc.pecann_density(ds, G, p, ws=torch.empty(1 << 20, dtype=torch.uint8, device="cuda"))
    assert e.value.status == pc.EINVAL


@pytest.mark.parametrize("d", [128, 256, 512, 1024])
def test_fp8_traversal_distances(d):
    """The FP8 traversal scores 1 - sum_j (q_j s_j) code_j: checked against a
    CPU decode of the same codes (torch's float8 -> float32) and an FP64 dot
    product. FP32 rounding of the d products and sums (d/32 + 6 steps on a
    lane's path, terms summing to about 1 in magnitude) stays far below
    1e-5 for d <= 1024."""
    n, R, L, k = 3000, 16, 48, 12
    X, _ = synth.vmf_like(n=n, d=d, components=20, seed=90 + d // 128)
    codes, s = quantize_e4m3(X)
    G = random_graph(n, R, seed=91)
    ds = pc.Dataset(codes.cuda(), metric=pc.IP, dim_scale=torch.from_numpy(s).cuda(),
                    data_f32=torch.from_numpy(X).cuda())
    qs = synth.sample_ids(n, 64, seed=92).astype(np.int32)
    ids, dis, cnt = pc.pecann_search(ds, torch.from_numpy(G).cuda(), torch.from_numpy(qs).cuda(), L=L, k=k)
    ids, dis, cnt = ids.cpu().numpy(), dis.cpu().numpy(), cnt.cpu().numpy()
    dec = codes.to(torch.float32).numpy().astype(np.float64) * s.astype(np.float64)
    for r, q in enumerate(qs):
        assert cnt[r] == k
        assert (np.diff(dis[r]) >= 0).all()
        ref = 1.0 - dec[ids[r]] @ X[q].astype(np.float64)
        assert np.abs(dis[r] - ref).max() <= 1e-5, (q, np.abs(dis[r] - ref).max())


def test_fp8_argument_checks():
    X = np.zeros((100, 128), np.float32)
    X[:, 0] = 1.0
    codes, s = quantize_e4m3(X)
    G = torch.zeros((100, 8), dtype=torch.int32, device="cuda")
    p = pc.params(k=4, R=8, L_search=8)
    ws = torch.empty(1 << 20, dtype=torch.uint8, device="cuda")
    Xf = torch.from_numpy(X).cuda()
    with pytest.raises(pc.PecannError) as e:  # L2 on FP8 rows
        pc.pecann_density(pc.Dataset(codes.cuda(), metric=pc.L2, dim_scale=torch.from_numpy(s).cuda(),
                                     data_f32=Xf), G, p, ws=ws)
    assert e.value.status == pc.EUNSUPPORTED
    with pytest.raises(pc.PecannError) as e:  # no scales
        pc.pecann_density(pc.Dataset(codes.cuda(), metric=pc.IP, data_f32=Xf), G, p, ws=ws)
    assert e.value.status == pc.EINVAL
    X2 = np.zeros((100, 2048), np.float32)
    X2[:, 0] = 1.0
    c2, s2 = quantize_e4m3(X2)
    with pytest.raises(pc.PecannError) as e:  # beyond the FP32 re-rank's d <= 1024
        pc.pecann_density(pc.Dataset(c2.cuda(), metric=pc.IP, dim_scale=torch.from_numpy(s2).cuda(),
                                     data_f32=torch.from_numpy(X2).cuda()), G, p, ws=ws)
    assert e.value.status == pc.EUNSUPPORTED
