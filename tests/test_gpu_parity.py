"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

The FP32 and uint8 paths decide every comparison on the same FP32 values as
the oracle (canonical summation order), so neighbour ids, dependent points,
graph rows and labels must match exactly, and distances / densities bit for
bit (exp-based densities within 1e-5 relative: expf may differ by an ulp).
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import exact
from paper_2312_03940_gb300 import pecann as pc
from paper_2312_03940_gb300 import synth
from tests.helpers import example_arrays, random_graph

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    pc.load_library()


def t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def run_pipeline(X, G, p, metric=pc.L2):
    ds = pc.Dataset(t(X), metric=metric)
    ws = pc.workspace(ds, p)
    Gd = t(G.astype(np.int32))
    dens = pc.pecann_density(ds, Gd, p, ws=ws)
    dep = pc.pecann_dependent_points(ds, Gd, p, dens["rank_key"], dens["knn_ids"], dens["knn_dist"], ws=ws)
    lab, nc = pc.pecann_cluster(dens["density"], dep["dep"], dep["dep_dist"], p)
    out = {k: v.cpu().numpy() for k, v in dens.items()}
    out.update(dep=dep["dep"].cpu().numpy(), dep_dist=dep["dep_dist"].cpu().numpy(), stats=dep["stats"],
               labels=lab.cpu().numpy(), n_clusters=nc)
    return out


# ---------------------------------------------------------------- worked example (Sec. 3)

def test_example_through_the_abi(golden_example):
    X, G, names, idx = example_arrays(golden_example)
    p = pc.params(k=1, R=G.shape[1], L_search=1, L_dep=2, dep_threshold=0, center=pc.CENTER_THRESHOLD,
                  rho_min=float(np.float32(1) / np.sqrt(np.float32(2))), delta_min=2.5)
    r = run_pipeline(X, G, p)
    for q, nn in golden_example["nearest_neighbor"].items():
        assert names[r["knn_ids"][idx[q], 0]] == nn
    for c, lam in golden_example["dependent_point"].items():
        got = r["dep"][idx[c]]
        assert (lam is None and got < 0) or names[got] == lam
    st = r["stats"]
    assert st[0] == 2 and st[1] == 1 and st[2] == 1 and st[3] == 0 and st[63] == 0
    groups = {}
    for i, l in enumerate(r["labels"]):
        groups.setdefault(int(l), []).append(names[i])
    assert sorted(sorted(g) for g in groups.values()) == sorted(sorted(c) for c in golden_example["clusters"])
    # the doubling-round candidate sets of d through pecann_search
    ds = pc.Dataset(t(X))
    for rnd in golden_example["dependent_rounds_for_d"]:
        kd = rnd["k_dep"]
        ids, _, cnt = pc.pecann_search(ds, t(G), t(np.array([idx["d"]], np.int32)), L=kd, k=kd)
        got = sorted(names[i] for i in ids[0, :cnt[0]].cpu().numpy())
        assert got == rnd["candidates"]



def test_example_local_center_through_the_abi(golden_example):
    """The local center on the Sec. 3 example through pecann_cluster_sweep:
    centers b and d; with rho_min = 1/sqrt(2) the printed clusters, without
    noise e follows d."""
    X, G, names, idx = example_arrays(golden_example)
    p = pc.params(k=1, R=G.shape[1], L_search=1, L_dep=2, dep_threshold=0)
    ds = pc.Dataset(t(X))
    ws = pc.workspace(ds, p)
    dens = pc.pecann_density(ds, t(G), p, ws=ws)
    dep = pc.pecann_dependent_points(ds, t(G), p, dens["rank_key"], dens["knn_ids"], dens["knn_dist"], ws=ws)
    rho_min = float(np.float32(1) / np.sqrt(np.float32(2)))
    labels, counts = pc.pecann_cluster_sweep(dens["density"], dep["dep"], dep["dep_dist"],
                                             [dict(center=pc.CENTER_LOCAL, rho_min=rho_min),
                                              dict(center=pc.CENTER_LOCAL, rho_min=0.0)],
                                             knn_ids=dens["knn_ids"], rank_key=dens["rank_key"])
    labels = labels.cpu().numpy()

    def groups_of(lab):
        g = {}
        for i, l in enumerate(lab):
            g.setdefault(int(l), []).append(names[i])
        return sorted(sorted(v) for v in g.values())

    assert groups_of(labels[0]) == sorted(sorted(c) for c in golden_example["clusters"]) and counts[0] == 3
    assert groups_of(labels[1]) == [["a", "b", "c"], ["d", "e", "f"]] and counts[1] == 2


def test_cluster_sweep_matches_single_calls_and_oracle():
    """One dependent forest, nine clusterings (threshold, product and local
    centers at three noise levels): each equals the oracle's clustering of the
    oracle's own forest, and the single-setting call where it exists."""
    n = 6000
    X, _ = synth.gaussian_mixture(n=n, d=32, components=12, seed=81)
    G = random_graph(n, 16, seed=81)
    p = pc.params(k=8, R=16, L_search=32, L_dep=32, n_clusters=12)
    ds = pc.Dataset(t(X))
    ws = pc.workspace(ds, p)
    dens = pc.pecann_density(ds, t(G), p, ws=ws)
    dep = pc.pecann_dependent_points(ds, t(G), p, dens["rank_key"], dens["knn_ids"], dens["knn_dist"], ws=ws)
    P = oracle.Points(X)
    o = oracle.knn_density(P, G, L=32, k=8)
    od = oracle.dependent_points(P, G, o["key"], o["ids"], Ld=32, threshold=300)
    assert (dens["knn_ids"].cpu().numpy() == o["ids"]).all() and (dens["rank_key"].cpu().numpy() == o["key"]).all()
    assert (dep["dep"].cpu().numpy() == od["lam"]).all() and (dep["dep_dist"].cpu().numpy() == od["delta"]).all()
    qs = [float(v) for v in np.quantile(o["rho"], [0.0, 0.05, 0.25])]
    dmin = float(np.median(od["delta"][np.isfinite(od["delta"])]))
    settings = []
    for rm in qs:
        settings += [dict(center=pc.CENTER_THRESHOLD, rho_min=rm, delta_min=dmin),
                     dict(center=pc.CENTER_PRODUCT, rho_min=rm, n_clusters=12),
                     dict(center=pc.CENTER_LOCAL, rho_min=rm)]
    labels, counts = pc.pecann_cluster_sweep(dens["density"], dep["dep"], dep["dep_dist"], settings,
                                             knn_ids=dens["knn_ids"], rank_key=dens["rank_key"])
    assert labels.shape == (len(settings), n)
    for i, st in enumerate(settings):
        ol, onc = oracle.cluster(o["rho"], od["lam"], od["delta"], center=st["center"], rho_min=st["rho_min"],
                                 delta_min=st.get("delta_min", 0.0), n_clusters=st.get("n_clusters", 1),
                                 knn_ids=o["ids"], rank_key=o["key"])
        assert (labels[i].cpu().numpy() == ol).all(), st
        assert counts[i] == onc, st
        if st["center"] != pc.CENTER_LOCAL:
            p1 = pc.params(center=st["center"], rho_min=st["rho_min"], delta_min=st.get("delta_min", 0.0),
                           n_clusters=st.get("n_clusters", 1))
            l1, n1 = pc.pecann_cluster(dens["density"], dep["dep"], dep["dep_dist"], p1)
            assert torch.equal(l1, labels[i]) and n1 == counts[i]
    # all settings run in shared passes: the sweep's kernel count does not
    # grow with the number of settings (9 settings, then 27 with repeats)
    l0 = pc.pecann_kernel_launches()
    pc.pecann_cluster_sweep(dens["density"], dep["dep"], dep["dep_dist"], settings,
                            knn_ids=dens["knn_ids"], rank_key=dens["rank_key"])
    l1 = pc.pecann_kernel_launches()
    labels3, counts3 = pc.pecann_cluster_sweep(dens["density"], dep["dep"], dep["dep_dist"], settings * 3,
                                               knn_ids=dens["knn_ids"], rank_key=dens["rank_key"])
    l2 = pc.pecann_kernel_launches()
    assert l2 - l1 == l1 - l0
    assert torch.equal(labels3[: len(settings)], labels) and torch.equal(labels3[len(settings):2 * len(settings)], labels)
    assert counts3[: len(settings)] == counts
    # the local center needs the k-NN lists in the single-setting call
    with pytest.raises(pc.PecannError) as e:
        pc.pecann_cluster(dens["density"], dep["dep"], dep["dep_dist"], pc.params(center=pc.CENTER_LOCAL))
    assert e.value.status == pc.EINVAL


# ---------------------------------------------------------------- Algorithm 1

@pytest.mark.parametrize("dtype,d,metric", [("f32", 32, pc.L2), ("f32", 128, pc.L2), ("u8", 128, pc.L2),
                                            ("f32", 64, pc.IP), ("f32", 384, pc.L2), ("f32", 1024, pc.L2),
                                            ("f32", 96, pc.L2), ("u8", 256, pc.L2)])
def test_search_matches_oracle(dtype, d, metric):
    n = 2500
    g = np.random.default_rng(d + metric)
    if dtype == "u8":
        X = g.integers(0, 256, size=(n, d), dtype=np.uint8)
        X[: n // 2] = np.clip(X[: n // 2] // 4 + 100, 0, 255)  # some structure, many ties
    else:
        X, _ = synth.gaussian_mixture(n=n, d=d, components=8, seed=d)
        if metric == pc.IP:
            X = (X / np.linalg.norm(X, axis=1, keepdims=True)).astype(np.float32)
    G = random_graph(n, 24, seed=d)
    P = oracle.Points(X, metric=metric)
    ds = pc.Dataset(t(X), metric=metric)
    q = synth.sample_ids(n, 150, seed=d).astype(np.int32)
    for L in (1, 7, 64, 200):
        k = min(L, 10)
        ids, dis, cnt = pc.pecann_search(ds, t(G), t(q), L=L, k=k)
        ids, dis, cnt = ids.cpu().numpy(), dis.cpu().numpy(), cnt.cpu().numpy()
        for r, qq in enumerate(q):
            oi, od = oracle.greedy_search(P, G, int(qq), [int(qq)], L=L, k=k)
            assert cnt[r] == len(oi)
            assert (ids[r, :cnt[r]] == oi).all(), (L, qq)
            assert (dis[r, :cnt[r]] == od).all(), (L, qq)


def test_u8_row_base_alignment():
    """128-byte uint8 rows are scored by 4 lanes with one 32-byte load each
    when the row base is 32-byte aligned, and by 8 lanes of 16 bytes
    otherwise: both layouts give the oracle's results."""
    n, d = 2500, 128
    g = np.random.default_rng(77)
    X = g.integers(0, 256, size=(n, d), dtype=np.uint8)
    G = random_graph(n, 24, seed=77)
    P = oracle.Points(X)
    q = synth.sample_ids(n, 100, seed=78).astype(np.int32)
    buf = torch.empty(n * d + 64, dtype=torch.uint8, device="cuda")
    outs = []
    for off in (0, 16):
        Xv = buf[off:off + n * d].view(n, d)
        Xv.copy_(t(X))
        assert (Xv.data_ptr() % 32 == 0) == (off == 0)
        ids, dis, cnt = pc.pecann_search(pc.Dataset(Xv), t(G), t(q), L=64, k=10)
        outs.append((ids.cpu().numpy(), dis.cpu().numpy()))
    for r, qq in enumerate(q):
        oi, od = oracle.greedy_search(P, G, int(qq), [int(qq)], L=64, k=10)
        for ids, dis in outs:
            assert (ids[r] == oi).all() and (dis[r] == od).all(), qq


@pytest.mark.parametrize("n_start", [20, 700])
def test_search_with_start_set(n_start):
    """Start sets smaller and larger than the staging area (the larger one is
    merged in chunks)."""
    n = 3000
    X, _ = synth.gaussian_mixture(n=n, d=32, components=6, seed=3)
    G = random_graph(n, 16, seed=3)
    P = oracle.Points(X)
    S = synth.sample_ids(n, n_start, seed=4).astype(np.int32)
    q = np.concatenate([S[:5], synth.sample_ids(n, 60, seed=5).astype(np.int32)])  # some queries in S
    ids, dis, cnt = pc.pecann_search(pc.Dataset(t(X)), t(G), t(q), L=40, k=40, start=t(S))
    ids, cnt = ids.cpu().numpy(), cnt.cpu().numpy()
    for r, qq in enumerate(q):
        oi, _ = oracle.greedy_search(P, G, int(qq), S, L=40, k=40)
        assert (ids[r, :cnt[r]] == oi).all()


# ---------------------------------------------------------------- graph build

@pytest.mark.parametrize("kind,passes,n_start", [("f32", 1, 12), ("u8", 1, 12), ("ip", 1, 12), ("u8", 2, 12),
                                                  ("f32", 2, 300)])
def test_build_graph_matches_oracle(kind, passes, n_start):
    n = 3000
    if kind == "u8":
        X, _ = synth.u8_mixture(n=n, d=128, components=12, seed=11)
        metric, d = pc.L2, 128
    else:
        X, _ = synth.gaussian_mixture(n=n, d=32 if kind == "f32" else 64, components=10, seed=12)
        metric = pc.L2
        if kind == "ip":
            X = (X / np.linalg.norm(X, axis=1, keepdims=True)).astype(np.float32)
            metric = pc.IP
    order = synth.insertion_order(n, seed=13)
    p = pc.params(R=24, L_build=48, alpha=1.2, n_start=n_start, batch_frac=0.02, build_passes=passes)
    ds = pc.Dataset(t(X), metric=metric)
    G, deg = pc.pecann_build_graph(ds, p, order=t(order))
    G = G.cpu().numpy()
    Go = oracle.build_graph(oracle.Points(X, metric=metric), R=24, L=48, alpha=1.2, perm=order, n_start=n_start,
                            passes=passes)
    assert (G == Go).all()
    assert (deg.cpu().numpy() == (Go >= 0).sum(1)).all()


def test_build_graph_without_order_is_a_valid_graph():
    n = 2000
    X, _ = synth.gaussian_mixture(n=n, d=32, components=5, seed=21)
    p = pc.params(R=16, L_build=32, alpha=1.2, n_start=8, seed=99)
    G, _ = pc.pecann_build_graph(pc.Dataset(t(X)), p)
    G = G.cpu().numpy()
    for i in range(n):
        row = G[i][G[i] >= 0]
        assert i not in row and len(set(row.tolist())) == len(row)
        assert (G[i][len(row):] == -1).all()


# ---------------------------------------------------------------- the whole path

def test_pipeline_c1_matches_oracle():
    """10,000 x 32 FP32, 10 Gaussians, R=32, L=64, alpha=1.2, k=6."""
    X, gt = synth.gaussian_mixture()
    n = len(X)
    order = synth.insertion_order(n)
    p = pc.params(k=6, R=32, L_build=64, L_search=64, L_dep=64, alpha=1.2, n_start=16,
                  center=pc.CENTER_PRODUCT, n_clusters=10)
    ds = pc.Dataset(t(X))
    G, _ = pc.pecann_build_graph(ds, p, order=t(order))
    G = G.cpu().numpy()
    P = oracle.Points(X)
    Go = oracle.build_graph(P, R=32, L=64, alpha=1.2, perm=order, n_start=16)
    assert (G == Go).all()
    r = run_pipeline(X, G, p)
    o = oracle.knn_density(P, G, L=64, k=6)
    assert (r["knn_ids"] == o["ids"]).all()
    assert (r["knn_dist"] == o["dist"]).all()
    assert (r["density"] == o["rho"]).all() and (r["rank_key"] == o["key"]).all()
    d = oracle.dependent_points(P, G, o["key"], o["ids"], Ld=64, threshold=300)
    assert (r["dep"] == d["lam"]).all()
    assert (r["dep_dist"] == d["delta"]).all()
    assert r["stats"][0] == d["rounds"] and r["stats"][1] == d["unfinished_round0"]
    lo, nco = oracle.cluster(o["rho"], d["lam"], d["delta"], center=oracle.CENTER_PRODUCT, n_clusters=10)
    assert (r["labels"] == lo).all() and r["n_clusters"] == nco
    assert exact.ari(r["labels"], gt) == 1.0
    _, ex_d = exact.exact_knn(X, 6)
    assert exact.knn_recall(r["knn_dist"], ex_d) >= 0.95


def _near_tied(key, i, j, rel=1e-5):
    """The rank keys of i and j are within rel of each other (a near-tie whose
    order FP32 rounding of exp may flip)."""
    a, b = float(key[i]), float(key[j])
    return abs(a - b) <= rel * max(abs(a), abs(b))


@pytest.mark.parametrize("fn,norm", [(pc.DENS_EXPSUM, 0), (pc.DENS_SUMEXP, 0), (pc.DENS_SUM, 0),
                                     (pc.DENS_KTH, 1)])
def test_density_variants(fn, norm):
    """Every density function of Sec. 4.2 / Appendix A. Keys that are sums
    and quotients of FP32 values in the oracle's order (kth, sum, the
    exponent of exp-sum, the normalised kth) are bit-exact, and so are the
    dependent points that follow from them. sum-exp ranks by a sum of expf
    values, which may differ by an ulp between CUDA and the C library: there
    the keys agree to 1e-5, and a dependent point may differ from the oracle's
    only across such a near-tie (the order of i against the oracle's or the
    GPU's dependent point of i flipped); every other point is bit-exact, and
    every GPU dependent distance is the oracle's distance of the reported pair."""
    X, _ = synth.gaussian_mixture(n=4000, d=32, components=8, seed=31)
    P = oracle.Points(X)
    G = oracle.build_graph(P, R=24, L=48, alpha=1.2, perm=synth.insertion_order(4000, 32), n_start=8)
    p = pc.params(k=10, R=24, L_search=48, L_dep=48, density=fn, normalize_density=norm, n_clusters=8)
    r = run_pipeline(X, G, p)
    o = oracle.knn_density(P, G, L=48, k=10, density=fn, normalize=bool(norm))
    assert (r["knn_ids"] == o["ids"]).all()
    assert (r["knn_dist"] == o["dist"]).all()
    d = oracle.dependent_points(P, G, o["key"], o["ids"], Ld=48, threshold=300)
    if fn != pc.DENS_SUMEXP:
        assert (r["rank_key"] == o["key"]).all()
        if fn != pc.DENS_EXPSUM:
            assert (r["density"] == o["rho"]).all()
        assert np.allclose(r["density"], o["rho"], rtol=1e-5, atol=0)
        assert (r["dep"] == d["lam"]).all() and (r["dep_dist"] == d["delta"]).all()
        return
    # sum-exp: near-tie rule
    assert np.allclose(r["rank_key"], o["key"], rtol=1e-5, atol=0)
    assert np.allclose(r["density"], o["rho"], rtol=1e-5, atol=0)
    diff = np.flatnonzero(r["dep"] != d["lam"])
    assert len(diff) <= len(X) // 100, f"{len(diff)} dependent points differ"
    for i in diff:
        lo, lg = int(d["lam"][i]), int(r["dep"][i])
        assert (lo >= 0 and _near_tied(o["key"], i, lo)) or (lg >= 0 and _near_tied(o["key"], i, lg)), i
    same = r["dep"] == d["lam"]
    assert (r["dep_dist"][same] == d["delta"][same]).all()
    for i in diff:
        j = int(r["dep"][i])
        if j >= 0:
            assert r["dep_dist"][i] == oracle.out_dist(P, oracle.dis(P, int(i), j))


def test_u8_pipeline_matches_oracle():
    X, gt = synth.u8_mixture(n=20000, d=128, components=20, seed=41)
    order = synth.insertion_order(len(X), seed=42)
    p = pc.params(k=10, R=32, L_build=64, L_search=64, L_dep=64, alpha=1.2, n_start=16, n_clusters=20)
    ds = pc.Dataset(t(X))
    G, _ = pc.pecann_build_graph(ds, p, order=t(order))
    G = G.cpu().numpy()
    r = run_pipeline(X, G, p)
    P = oracle.Points(X)
    o = oracle.knn_density(P, G, L=64, k=10)
    assert (r["knn_ids"] == o["ids"]).all() and (r["rank_key"] == o["key"]).all()
    d = oracle.dependent_points(P, G, o["key"], o["ids"], Ld=64, threshold=300)
    assert (r["dep"] == d["lam"]).all() and (r["dep_dist"] == d["delta"]).all()


def test_fallback_and_tail_paths():
    """Isolated points (empty out-lists) make the k-NN search return fewer
    than k points (exact brute force takes over); a low threshold and a
    one-round cap leave many points for the brute-force tail."""
    X, _ = synth.gaussian_mixture(n=3000, d=32, components=4, seed=51)
    G = random_graph(3000, 8, seed=51)
    G[::97] = -1  # isolated points
    p = pc.params(k=8, R=8, L_search=16, L_dep=16, dep_threshold=0, max_dep_rounds=1, n_clusters=4)
    r = run_pipeline(X, G, p)
    P = oracle.Points(X)
    o = oracle.knn_density(P, G, L=16, k=8)
    assert o["fallback"].sum() >= 30
    assert (r["knn_ids"] == o["ids"]).all() and (r["rank_key"] == o["key"]).all()
    d = oracle.dependent_points(P, G, o["key"], o["ids"], Ld=16, threshold=0, max_rounds=1)
    assert d["tail"] > 0
    assert (r["dep"] == d["lam"]).all() and (r["dep_dist"] == d["delta"]).all()
    assert r["stats"][63] == d["tail"]


@pytest.mark.parametrize("d", [128, 64])
def test_u8_tail(d):
    """uint8 rows of up to 128 bytes take the one-point-per-thread brute-force
    tail (d = 64 leaves half the chunks empty); a zero threshold and a
    one-round cap send hundreds of points there. Ties are frequent (coarse
    integer data), so the id order of equal distances is exercised too."""
    n = 4000
    X, _ = synth.u8_mixture(n=n, d=d, components=6, seed=53 + d)
    X = (X // 8).astype(np.uint8)  # coarse values: many equal distances
    G = random_graph(n, 12, seed=54)
    p = pc.params(k=6, R=12, L_search=12, L_dep=12, dep_threshold=0, max_dep_rounds=1, n_clusters=6)
    r = run_pipeline(X, G, p)
    P = oracle.Points(X)
    o = oracle.knn_density(P, G, L=12, k=6)
    assert (r["knn_ids"] == o["ids"]).all() and (r["rank_key"] == o["key"]).all()
    d_ = oracle.dependent_points(P, G, o["key"], o["ids"], Ld=12, threshold=0, max_rounds=1)
    assert d_["tail"] >= 100
    assert (r["dep"] == d_["lam"]).all() and (r["dep_dist"] == d_["delta"]).all()
    assert r["stats"][63] == d_["tail"]


def test_edge_cases():
    # two points
    X = np.array([[0, 0, 0, 0], [3, 4, 0, 0]], np.float32)
    G = np.array([[1], [0]], np.int32)
    r = run_pipeline(X, G, pc.params(k=1, R=1, L_search=1, L_dep=1, n_clusters=1))
    assert list(r["knn_ids"][:, 0]) == [1, 0] and np.allclose(r["knn_dist"][:, 0], 5.0)
    assert list(r["dep"]) == [-1, 0] and list(r["labels"]) == [0, 0]
    # duplicates: every distance ties; order falls back to ids
    X = np.zeros((50, 8), np.float32)
    G = random_graph(50, 4, seed=1)
    p = pc.params(k=3, R=4, L_search=8, L_dep=8, n_clusters=1)
    r = run_pipeline(X, G, p)
    o = oracle.knn_density(oracle.Points(X), G, L=8, k=3)
    assert (r["knn_ids"] == o["ids"]).all()
    assert np.isinf(r["density"]).all()
    d = oracle.dependent_points(oracle.Points(X), G, o["key"], o["ids"], Ld=8, threshold=300)
    assert (r["dep"] == d["lam"]).all()


def test_bad_graph_entry_reported():
    """An out-of-range graph entry is skipped by the kernels (never read
    through) and reported as PECANN_EINTERNAL by every call that searches the
    graph: Algorithm 1 alone, and the k-NN + density pass (Algorithm 2 lines
    2-4), whose error word is read back at the end of the call."""
    X, _ = synth.gaussian_mixture(n=500, d=32, components=3, seed=61)
    G = random_graph(500, 8, seed=61)
    G[10, 3] = 10_000  # out of range: the kernel skips it and reports
    ds = pc.Dataset(t(X))
    with pytest.raises(pc.PecannError) as e:
        pc.pecann_search(ds, t(G), t(np.arange(500, dtype=np.int32)), L=16, k=4)
    assert e.value.status == pc.EINTERNAL
    p = pc.params(k=4, R=8, L_search=16, L_dep=16)
    with pytest.raises(pc.PecannError) as e:
        pc.pecann_density(ds, t(G), p)
    assert e.value.status == pc.EINTERNAL
    assert b"out of range" in pc.load_library().pecann_last_error()
    # the next call on a good graph succeeds (nothing stale in the error word)
    G[10, 3] = 11
    pc.pecann_density(ds, t(G), p)
