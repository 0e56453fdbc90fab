"""The brute-force index on the tensor cores (Sec. 5.1: no index, exact k-NN;
Sec. 6.1: the BruteForce instance, exact DPC) against the oracle's
brute-force index.

The GPU screens every pair with BF16 tensor-core inner products and decides
exactly on the canonical FP32 (or exact integer) distance, so k-NN ids,
distances, densities, dependent points and labels must equal the oracle's
bit for bit. The oracle runs Algorithm 3 literally with an exact FindKnn
(doubling rounds, then the tail), while the GPU sends every unfinished
point straight to DPBruteForce over all points: equality also checks that
the two give the same dependent points.

Cases cover both metrics, uint8 and FP32 rows, d below, at and above one
64-column chunk (with a partial last chunk), n below one tile and with
ragged tiles, many exact ties (the band overflows the kept list: the collect
pass and the SIMT kernels take over), and an error case.
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


def gpu_path(X, metric, p):
    ds = pc.Dataset(torch.from_numpy(np.ascontiguousarray(X)).cuda(), metric=metric)
    ws = pc.workspace(ds, p)
    dens = pc.pecann_density(ds, None, p, ws=ws)
    c_knn = ws[24:32].cpu().view(torch.int32).tolist()
    dep = pc.pecann_dependent_points(ds, None, p, dens["rank_key"], dens["knn_ids"], dens["knn_dist"], ws=ws)
    c_dep = ws[24:32].cpu().view(torch.int32).tolist()
    lab, nc = pc.pecann_cluster(dens["density"], dep["dep"], dep["dep_dist"], p)
    out = {k: v.cpu().numpy() for k, v in dens.items()}
    out.update(dep=dep["dep"].cpu().numpy(), dep_dist=dep["dep_dist"].cpu().numpy(), labels=lab.cpu().numpy(),
               n_clusters=nc, stats=dep["stats"], c_knn=c_knn, c_dep=c_dep)
    return out


def check_against_oracle(X, metric, k, n_clusters, density=pc.DENS_KTH, Ld=32, cl=0):
    p = pc.params(k=k, R=8, L_search=max(k, 8), L_dep=Ld, index=pc.INDEX_BRUTE_FORCE, center=pc.CENTER_PRODUCT,
                  n_clusters=n_clusters, density=density, block_warps=cl)
    r = gpu_path(X, metric, p)
    P = oracle.Points(X, metric=metric)
    o = oracle.knn_density(P, None, L=0, k=k, density=density)
    assert (r["knn_ids"] == o["ids"]).all()
    assert (r["knn_dist"] == o["dist"]).all()
    assert (r["rank_key"] == o["key"]).all()
    # a low threshold makes the oracle run doubling rounds with its exact
    # FindKnn before the tail
    d = oracle.dependent_points(P, None, o["key"], o["ids"], Ld=Ld, threshold=10)
    assert (r["dep"] == d["lam"]).all()
    assert (r["dep_dist"] == d["delta"]).all()
    lo, nco = oracle.cluster(o["rho"], d["lam"], d["delta"], center=oracle.CENTER_PRODUCT, n_clusters=n_clusters)
    assert (r["labels"] == lo).all() and r["n_clusters"] == nco
    # every unfinished point went to the exact search, no doubling round ran
    assert r["stats"][0] == 0 and r["stats"][1] == r["stats"][63] == d["unfinished_round0"]
    assert d["rounds"] >= 1 or d["unfinished_round0"] <= 10
    return r, o, d


def test_ip_unit_norm_1024():
    """The 1.28M x 1024 inner-product workload's shape, at 5,000 points (40
    ragged 128-query tiles, a ragged last 256-point tile)."""
    X, _ = synth.vmf_like(n=5000, d=1024, components=40, seed=201)
    r, o, _ = check_against_oracle(X, pc.IP, k=16, n_clusters=40)
    # recall against the FP64 exact k-NN: 1 (the index is exact)
    qs = synth.sample_ids(len(X), 300, seed=202)
    _, ex = exact.exact_knn_queries(X, qs, 16, metric=exact.IP)
    assert exact.knn_recall(r["knn_dist"][qs], ex) == 1.0


@pytest.mark.parametrize("cl", [1, 2, 4])
def test_cluster_forms(cl):
    """The screen's k-NN pass run by single CTAs, by CTA pairs issuing one
    256-row MMA (each CTA holding half of every point tile) and by clusters
    of 4 sharing point tiles by multicast: the same exact results. An odd
    number of query tiles leaves one pair with a CTA past the last tile."""
    X, _ = synth.vmf_like(n=2 * 128 + 77, d=256, components=6, seed=209)
    check_against_oracle(X, pc.IP, k=12, n_clusters=6, cl=cl)
    U, _ = synth.u8_mixture(n=2500, d=128, components=8, seed=210)
    check_against_oracle(U, pc.L2, k=10, n_clusters=8, cl=cl)


def test_u8_l2_128():
    """The 1M x 128 uint8 workload's shape at 6,000 points: integer distances
    are exact in the screen (uint8 is exact in BF16)."""
    X, _ = synth.u8_mixture(n=6000, d=128, components=20, seed=203)
    check_against_oracle(X, pc.L2, k=10, n_clusters=20)


@pytest.mark.parametrize("d", [32, 96, 384])
def test_f32_l2(d):
    """FP32 rows with the L2 metric: d = 32 (a chunk half zero-filled by the
    tensor map), 96 (a partial second chunk) and 384. Large norms against
    small distances widen the band, so many points take the collect pass."""
    X, _ = synth.gaussian_mixture(n=3000, d=d, components=8, seed=204 + d)
    check_against_oracle(X, pc.L2, k=6, n_clusters=8)


def test_small_n_and_exp_sum():
    """n = 40 (one partial tile each way, every point in the kept list) with
    the exp-sum density (its key is the exponent: bit-exact)."""
    X, _ = synth.gaussian_mixture(n=40, d=32, components=3, seed=207)
    check_against_oracle(X, pc.L2, k=5, n_clusters=3, density=pc.DENS_EXPSUM, Ld=8)


def test_ties_overflow_the_kept_list():
    """Coarse uint8 values: thousands of points at equal distances, so the
    band around the k-th key holds more than the 80 kept candidates. Those
    points take the collect pass (up to 1,024 candidates) or, beyond it, the
    exact SIMT kernels; the results are still the oracle's, ties broken by id."""
    X, _ = synth.u8_mixture(n=4000, d=64, components=4, seed=208)
    X = (X // 64).astype(np.uint8)  # values 0..3
    r, _, _ = check_against_oracle(X, pc.L2, k=8, n_clusters=4)
    assert r["c_knn"][0] > 0  # rows that took the collect pass
    assert r["c_knn"][1] > 0  # rows beyond its capacity (exact SIMT)


def test_bruteforce_argument_checks():
    X = torch.zeros((100, 36), dtype=torch.float32, device="cuda")  # d not a multiple of 8
    p = pc.params(k=4, R=8, L_search=8, index=pc.INDEX_BRUTE_FORCE)
    ds = pc.Dataset(X)
    with pytest.raises(pc.PecannError) as e:
        pc.pecann_density(ds, None, p)
    assert e.value.status == pc.EUNSUPPORTED
    # the graph index still needs a graph
    with pytest.raises(pc.PecannError) as e:
        pc.pecann_density(pc.Dataset(torch.zeros((100, 32), device="cuda")), None, pc.params(k=4, R=8, L_search=8))
    assert e.value.status == pc.EINVAL
