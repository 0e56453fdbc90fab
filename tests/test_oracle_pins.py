"""Pins of the CPU oracle against what the paper and the mathematics fix.

Nothing here runs the CUDA library. Each test checks the oracle against
something other than itself: the paper's worked example (tests/golden), exact
FP64 brute force written independently in numpy or pure Python, closed forms,
and the invariants of the method.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import exact
from paper_2312_03940_gb300 import synth
from tests.helpers import example_arrays, random_graph, ranks_above


# ---------------------------------------------------------------- worked example (Sec. 3)

def test_example_nearest_neighbours(golden_example):
    """Sec. 3 step 2: greedy search with k = L = 1 from the query finds c, c, b, f, d, d."""
    X, G, names, idx = example_arrays(golden_example)
    P = oracle.Points(X)
    for q, nn in golden_example["nearest_neighbor"].items():
        ids, _ = oracle.greedy_search(P, G, idx[q], [idx[q]], L=1, k=1)
        assert names[ids[0]] == nn, q


def test_example_density_and_rank(golden_example):
    """Sec. 3 step 3: kth density values and the ranking b, c, a, d, f, e."""
    X, G, names, idx = example_arrays(golden_example)
    P = oracle.Points(X)
    r = oracle.knn_density(P, G, L=1, k=1, density=oracle.DENS_KTH)
    for c, expr in golden_example["density_kth"].items():
        expected = eval(expr, {"sqrt": math.sqrt})
        assert abs(r["rho"][idx[c]] - expected) <= 1e-7 * expected
    order = exact.rank_order(r["key"].astype(np.float64))
    assert [names[i] for i in order] == golden_example["rank_high_to_low"]


def test_density_functions_closed_forms():
    """Sec. 4.2 / Appendix A densities on a configuration worked out by hand:
    a center c = (0, 0) and four vertices (+-2, 0), (0, +-2), complete graph,
    k = 4 (so every k-NN list holds the other four points, exactly). For c all
    four distances are 2; for a vertex they are 2, sqrt(8), sqrt(8) and 4.
    kth: 1/2 and 1/4. exp-sum: exp(-16/4) and exp(-36/4). sum-exp: e^-4 and
    (e^-4 + 2 e^-8 + e^-16) / 4. sum: -8 and -(6 + 4 sqrt 2). Normalised kth:
    c: (1/2)(4) / (4 / 4) = 2; a vertex: (1/4)(4) / (1/2 + 3/4) = 0.8."""
    X = np.zeros((5, 4), np.float32)  # two zero coordinates pad the rows to d = 4
    X[:, :2] = [[0, 0], [2, 0], [-2, 0], [0, 2], [0, -2]]
    G = np.array([[j for j in range(5) if j != i] for i in range(5)], np.int32)
    P = oracle.Points(X)
    e = np.exp
    cases = [
        (oracle.DENS_KTH, False, [0.5, 0.25], [0.5, 0.25]),
        (oracle.DENS_EXPSUM, False, [e(-4.0), e(-9.0)], [-4.0, -9.0]),
        (oracle.DENS_SUMEXP, False, [e(-4.0), (e(-4.0) + 2 * e(-8.0) + e(-16.0)) / 4],
         [e(-4.0), (e(-4.0) + 2 * e(-8.0) + e(-16.0)) / 4]),
        (oracle.DENS_SUM, False, [-8.0, -(6 + 4 * np.sqrt(2.0))], [-8.0, -(6 + 4 * np.sqrt(2.0))]),
        (oracle.DENS_KTH, True, [2.0, 0.8], [2.0, 0.8]),
    ]
    for fn, norm, rho, key in cases:
        r = oracle.knn_density(P, G, L=4, k=4, density=fn, normalize=norm)
        assert (r["fallback"] == 0).all()
        want_rho = np.array([rho[0]] + [rho[1]] * 4)
        want_key = np.array([key[0]] + [key[1]] * 4)
        assert np.allclose(r["rho"], want_rho, rtol=2e-6, atol=0), (fn, norm, r["rho"])
        assert np.allclose(r["key"], want_key, rtol=2e-6, atol=0), (fn, norm, r["key"])


def test_search_counts_by_hand_and_full_beam(golden_example):
    """The per-query counts behind the algorithmic bytes: E_q (expansions, the
    query's own out-list included) and C_q (distinct points scored). On the
    Sec. 3 example with L = 1, counted by hand from the Fig. 1 graph: a
    expands a, b, c and scores b, c, f (E 3, C 3); d expands d, f and scores
    f, e, c (E 2, C 3); e expands e, d and scores d, f (E 2, C 2). With L >= n
    on a connected graph every point is expanded once and every other point
    scored once: E = n, C = n - 1."""
    X, G, names, idx = example_arrays(golden_example)
    e, c = oracle.search_counts(oracle.Points(X), G, [idx["a"], idx["d"], idx["e"]], L=1)
    assert list(e) == [3, 2, 2] and list(c) == [3, 3, 2]
    n = 300
    X2, _ = synth.gaussian_mixture(n=n, d=8, components=3, seed=5)
    e2, c2 = oracle.search_counts(oracle.Points(X2), random_graph(n, 6, seed=5), np.arange(0, n, 37), L=n)
    assert (e2 == n).all() and (c2 == n - 1).all()


def test_example_dependent_points_and_rounds(golden_example):
    """Fig. 2 dependent points and the Sec. 3.1 rounds for d (L_d = 2, threshold 0)."""
    X, G, names, idx = example_arrays(golden_example)
    P = oracle.Points(X)
    r = oracle.knn_density(P, G, L=1, k=1)
    dep = oracle.dependent_points(P, G, r["key"], r["ids"], Ld=golden_example["L_d"],
                                  threshold=golden_example["threshold"])
    for c, lam in golden_example["dependent_point"].items():
        got = dep["lam"][idx[c]]
        assert (got < 0 and lam is None) or (lam is not None and names[got] == lam), c
    # round 0 leaves only d (b, the maximum, is skipped); two doubling rounds finish d
    assert dep["unfinished_round0"] == 1
    assert dep["rounds"] == 2 and dep["unfinished"] == [1, 0] and dep["tail"] == 0
    # the candidate sets of those two rounds
    for rnd in golden_example["dependent_rounds_for_d"]:
        kd = rnd["k_dep"]
        ids, _ = oracle.greedy_search(P, G, idx["d"], [idx["d"]], L=kd, k=kd)
        assert sorted(names[i] for i in ids) == rnd["candidates"]
    # delta: D(x_i, lambda_i), +inf for the maximum
    assert math.isinf(dep["delta"][idx["b"]])
    assert abs(dep["delta"][idx["d"]] - 3.0) < 1e-6


def test_example_clusters(golden_example):
    """Sec. 3 step 5 / Fig. 3: rho_min = 1/sqrt(2) makes e noise; delta_min = 2.5
    makes b and d centres; clusters {a,b,c}, {d,f}, {e}. The product centre with
    n_c = 2 picks the same centres."""
    X, G, names, idx = example_arrays(golden_example)
    P = oracle.Points(X)
    r = oracle.knn_density(P, G, L=1, k=1)
    dep = oracle.dependent_points(P, G, r["key"], r["ids"], Ld=2, threshold=0)
    rho_min = np.float32(1.0) / np.sqrt(np.float32(2.0))
    expected = sorted(sorted(c) for c in golden_example["clusters"])
    for center, kw in ((oracle.CENTER_THRESHOLD, dict(delta_min=2.5)), (oracle.CENTER_PRODUCT, dict(n_clusters=2))):
        labels, nc = oracle.cluster(r["rho"], dep["lam"], dep["delta"], center=center, rho_min=rho_min, **kw)
        groups = {}
        for i, l in enumerate(labels):
            groups.setdefault(int(l), []).append(names[i])
        assert sorted(sorted(g) for g in groups.values()) == expected
        assert nc == 3
        # the label of a cluster is its root: b, d and the noise point e
        assert {names[l] for l in labels} == {"b", "d", "e"}


def test_example_local_center(golden_example):
    """Local center function (Appendix, center functions) on the Sec. 3
    example, worked by hand from the printed k = 1 neighbours and densities:
    b ranks above its neighbour c (equal density, smaller id) and d above f
    (likewise); a, c, e and f rank below theirs. With rho_min = 1/sqrt(2) the
    clusters are the printed ones, {a,b,c}, {d,f}, {e}; without a noise
    threshold e follows its dependent point d."""
    X, G, names, idx = example_arrays(golden_example)
    P = oracle.Points(X)
    r = oracle.knn_density(P, G, L=1, k=1)
    dep = oracle.dependent_points(P, G, r["key"], r["ids"], Ld=2, threshold=0)
    rho_min = np.float32(1.0) / np.sqrt(np.float32(2.0))

    def groups_of(labels):
        g = {}
        for i, l in enumerate(labels):
            g.setdefault(int(l), []).append(names[i])
        return sorted(sorted(v) for v in g.values())

    labels, nc = oracle.cluster(r["rho"], dep["lam"], dep["delta"], center=oracle.CENTER_LOCAL,
                                rho_min=rho_min, knn_ids=r["ids"], rank_key=r["key"])
    assert groups_of(labels) == sorted(sorted(c) for c in golden_example["clusters"]) and nc == 3
    assert {names[l] for l in labels} == {"b", "d", "e"}
    labels, nc = oracle.cluster(r["rho"], dep["lam"], dep["delta"], center=oracle.CENTER_LOCAL,
                                rho_min=0.0, knn_ids=r["ids"], rank_key=r["key"])
    assert groups_of(labels) == [["a", "b", "c"], ["d", "e", "f"]] and nc == 2


def test_local_center_forest_invariants():
    """On a random mixture: every label is a root; the roots are exactly the
    noise points, the points without a dependent point and the points ranked
    above all their k nearest neighbours; every other point has its dependent
    point's label."""
    X, _ = synth.gaussian_mixture(n=1500, d=8, components=5, seed=71)
    G = random_graph(1500, 12, seed=71)
    P = oracle.Points(X)
    r = oracle.knn_density(P, G, L=24, k=6)
    dep = oracle.dependent_points(P, G, r["key"], r["ids"], Ld=24, threshold=300)
    rho_min = float(np.quantile(r["rho"], 0.05))
    labels, nc = oracle.cluster(r["rho"], dep["lam"], dep["delta"], center=oracle.CENTER_LOCAL,
                                rho_min=rho_min, knn_ids=r["ids"], rank_key=r["key"])
    key, ids, lam = r["key"], r["ids"], dep["lam"]
    n = len(labels)
    top = np.array([all(not (key[j] > key[i] or (key[j] == key[i] and j < i)) for j in ids[i] if j >= 0 and j != i)
                    for i in range(n)])
    cut = (r["rho"] < np.float32(rho_min)) | (lam < 0) | top
    assert (labels[labels] == labels).all()
    assert set(np.flatnonzero(labels == np.arange(n))) == set(np.flatnonzero(cut))
    assert nc == cut.sum()
    inner = np.flatnonzero(~cut)
    assert (labels[inner] == labels[lam[inner]]).all()


def test_homogeneity_completeness_closed_forms():
    """Sec. 6 metrics: identical partitions give (1, 1); every point its own
    cluster against K equal classes gives homogeneity 1 and completeness
    1 - log(n/K) / log(n) (the paper's example of a low completeness); one
    cluster for everything gives (0, 1); scikit-learn agrees when installed."""
    true = np.repeat(np.arange(10), 100)
    assert exact.homogeneity_completeness(true, true) == pytest.approx((1.0, 1.0))
    hom, com = exact.homogeneity_completeness(np.arange(1000), true)
    assert hom == pytest.approx(1.0) and com == pytest.approx(1.0 - np.log(100) / np.log(1000))
    assert com == pytest.approx(1.0 / 3.0)
    assert exact.homogeneity_completeness(np.zeros(1000), true) == pytest.approx((0.0, 1.0))
    g = np.random.default_rng(3)
    pred = g.integers(0, 7, size=1000)
    try:
        from sklearn.metrics import completeness_score, homogeneity_score
    except ImportError:
        return
    hom, com = exact.homogeneity_completeness(pred, true)
    assert hom == pytest.approx(homogeneity_score(true, pred), abs=1e-12)
    assert com == pytest.approx(completeness_score(true, pred), abs=1e-12)


# ---------------------------------------------------------------- distances

def test_canonical_distance_within_fp32_error_bound():
    """The FP32 canonical squared distance is within the recursive-summation
    error bound of the exact FP64 value (gamma_m with m = 4d/32 + 5 steps)."""
    g = np.random.default_rng(5)
    for d in (4, 32, 128, 1024):
        X = g.standard_normal((20, d)).astype(np.float32)
        P = oracle.Points(X)
        ex = exact.exact_dist_rows(X, np.arange(20)) ** 2
        m = d // 32 * 4 + 4 + 5 if d >= 128 else 4 + 5
        gam = m * 2.0 ** -24 / (1 - m * 2.0 ** -24)
        for a in range(20):
            for b in range(20):
                assert abs(oracle.dis(P, a, b) - ex[a, b]) <= gam * ex[a, b] * 1.0001 + 1e-30


def test_canonical_distance_u8_is_exact():
    """uint8 rows: every partial sum is an integer below 2^24, so the FP32
    result equals the exact integer sum of squared differences."""
    g = np.random.default_rng(6)
    X = g.integers(0, 256, size=(16, 128), dtype=np.uint8)
    P = oracle.Points(X)
    Xi = X.astype(np.int64)
    for a in range(16):
        for b in range(16):
            assert oracle.dis(P, a, b) == float(((Xi[a] - Xi[b]) ** 2).sum())


def test_inner_product_distance():
    g = np.random.default_rng(7)
    X = g.standard_normal((10, 64)).astype(np.float32)
    X /= np.linalg.norm(X, axis=1, keepdims=True)
    P = oracle.Points(X, metric=oracle.IP)
    for a in range(10):
        for b in range(10):
            ex = 1.0 - float(X[a].astype(np.float64) @ X[b].astype(np.float64))
            assert abs(oracle.dis(P, a, b) - ex) < 1e-6


# ---------------------------------------------------------------- Algorithm 1 special cases

@pytest.mark.parametrize("seed", [0, 1, 2])
def test_full_beam_equals_exact_knn(seed):
    """With a beam at least n wide on a connected graph, Algorithm 1 visits
    every point, so it returns the exact k nearest neighbours."""
    n, d, k = 48, 8, 5
    g = np.random.default_rng(seed)
    X = g.standard_normal((n, d)).astype(np.float32)
    G = random_graph(n, 4, seed)
    P = oracle.Points(X)
    ex_ids, ex_d = exact.exact_knn(X, k)
    for q in range(n):
        ids, dis = oracle.greedy_search(P, G, q, [q], L=n, k=k)
        assert len(ids) == k
        assert np.allclose(np.sqrt(dis), ex_d[q], rtol=1e-5)
        assert list(ids) == list(ex_ids[q])


def test_search_returns_fewer_when_component_is_small():
    """A query whose component has fewer than k other points gets fewer than k
    back from Algorithm 1 (the oracle then falls back to brute force, Sec. 4.1)."""
    X = np.arange(32, dtype=np.float32).reshape(8, 4)
    G = np.full((8, 2), -1, np.int32)
    G[0, 0], G[1, 0] = 1, 0  # component {0, 1}
    for i in range(2, 8):
        G[i, 0] = 2 + (i - 1) % 6
    P = oracle.Points(X)
    ids, _ = oracle.greedy_search(P, G, 0, [0], L=4, k=3)
    assert list(ids) == [1]
    r = oracle.knn_density(P, G, L=4, k=3)
    assert r["fallback"][0] == 1 and r["fallback"][1] == 1
    ex_ids, _ = exact.exact_knn(X, 3)
    assert (r["ids"][:2] == ex_ids[:2]).all()


def test_pure_python_beam_search_tiny():
    """Algorithm 1 restated with Python sets on a tiny input, for several
    beam widths (a second independent statement of the same steps)."""
    n, d = 30, 4
    g = np.random.default_rng(11)
    X = g.integers(-5, 6, size=(n, d)).astype(np.float32)  # integer data: exact, with ties
    G = random_graph(n, 3, 11)
    P = oracle.Points(X)
    D2 = ((X[:, None, :].astype(np.int64) - X[None, :, :].astype(np.int64)) ** 2).sum(-1)

    def key(q, j):
        return (D2[q, j], j)

    for L in (1, 2, 3, 5, 8):
        for q in range(n):
            V = {q}
            beam = set(int(y) for y in G[q] if y >= 0 and y != q)
            beam = set(sorted(beam, key=lambda j: key(q, j))[:L])
            while True:
                unv = [j for j in beam if j not in V]
                if not unv:
                    break
                p = min(unv, key=lambda j: key(q, j))
                beam |= set(int(y) for y in G[p] if y >= 0 and y != q)
                V.add(p)
                beam = set(sorted(beam, key=lambda j: key(q, j))[:L])
            res = sorted((beam | V) - {q}, key=lambda j: key(q, j))[:L]
            ids, _ = oracle.greedy_search(P, G, q, [q], L=L, k=L)
            assert list(ids) == res, (L, q)


# ---------------------------------------------------------------- Algorithm 3 and Definition 2.1

def test_dependent_points_match_definition_with_exact_knn():
    """With exact k-NN lists (beam >= n) every answer of Algorithm 3 equals
    Definition 2.1 computed by FP64 brute force from the same ranking."""
    g = np.random.default_rng(3)
    n, d, k = 400, 8, 6
    X = g.standard_normal((n, d)).astype(np.float32)
    G = random_graph(n, 8, 3)
    P = oracle.Points(X)
    r = oracle.knn_density(P, G, L=n, k=k)
    dep = oracle.dependent_points(P, G, r["key"], r["ids"], Ld=2 * k, threshold=5)
    lam, delta = exact.exact_dependent(X, r["key"].astype(np.float64))
    assert (dep["lam"] == lam).all()
    fin = np.isfinite(delta)
    assert np.allclose(dep["delta"][fin], delta[fin], rtol=1e-5)


def test_approximate_dependent_distance_is_never_shorter():
    """Given the same densities, the reported dependent point ranks above the
    point and is never closer than the exact one (Definition 2.1)."""
    g = np.random.default_rng(4)
    n, d, k = 1500, 16, 8
    X, _ = _mixture(n, d, 8, g)
    G = random_graph(n, 6, 4)
    P = oracle.Points(X)
    r = oracle.knn_density(P, G, L=16, k=k)
    dep = oracle.dependent_points(P, G, r["key"], r["ids"], Ld=16, threshold=20)
    lam_ex, delta_ex = exact.exact_dependent(X, r["key"].astype(np.float64))
    key = r["key"]
    has = dep["lam"] >= 0
    assert (has == (lam_ex >= 0)).all()
    assert has.sum() == n - 1  # exactly one point, the maximum, has none
    for i in np.flatnonzero(has):
        assert ranks_above(key, dep["lam"][i], i)
    assert (dep["delta"][has] >= delta_ex[has] * (1 - 1e-6)).all()


def _mixture(n, d, c, g, box=10.0):
    centres = g.uniform(-box, box, size=(c, d))
    lab = g.integers(0, c, size=n)
    return (centres[lab] + g.standard_normal((n, d))).astype(np.float32), lab


# ---------------------------------------------------------------- clusters and ARI

def test_ari_closed_forms():
    a = np.array([0, 0, 1, 1, 2, 2])
    assert exact.ari(a, a) == 1.0
    assert exact.ari(a, a + 7) == 1.0
    assert exact.ari(np.zeros(5), np.zeros(5)) == 1.0
    # one pair split: contingency by hand -> ARI = 0.5 * ... computed from the formula terms
    b = np.array([0, 0, 1, 1, 2, 3])
    # sum_ij = 2, sum_a = 3, sum_b = 2, total = 15 -> (2 - 6/15) / (2.5 - 6/15) = 1.6 / 2.1
    assert abs(exact.ari(a, b) - 1.6 / 2.1) < 1e-12


def test_ari_matches_sklearn():
    sk = pytest.importorskip("sklearn.metrics")
    g = np.random.default_rng(9)
    for _ in range(5):
        a = g.integers(0, 5, size=200)
        b = g.integers(0, 7, size=200)
        assert abs(exact.ari(a, b) - sk.adjusted_rand_score(a, b)) < 1e-12


def test_bruteforce_index_equals_exact_dpc():
    """The brute-force index (Sec. 5.1: no index, exact k-NN by scanning every
    point) in the oracle: its k-NN lists equal the FP64 exact k-NN, and
    Algorithm 3 run literally with that exact FindKnn (doubling rounds, then
    the tail) gives Definition 2.1's dependent points for the same keys. The
    Gaussian data leaves no FP32 near-ties among the compared distances."""
    X, _ = _mixture(3000, 32, 6, np.random.default_rng(3))
    P = oracle.Points(X)
    o = oracle.knn_density(P, None, L=0, k=8)
    ei, ed = exact.exact_knn(X, 8)
    assert (o["ids"] == ei).all()
    assert np.allclose(o["dist"], ed, rtol=1e-6, atol=0)
    assert (o["fallback"] == 0).all()
    d = oracle.dependent_points(P, None, o["key"], o["ids"], Ld=16, threshold=10)
    assert d["rounds"] >= 1 and d["unfinished_round0"] > d["tail"]  # the exact rounds did work
    lam, delta = exact.exact_dependent(X, o["key"].astype(np.float64))
    assert (d["lam"] == lam).all()
    ok = lam >= 0
    assert np.allclose(d["delta"][ok], delta[ok], rtol=1e-6, atol=0)
    # inner product on unit-norm rows (isotropic directions: no near-ties)
    Xs = np.random.default_rng(4).standard_normal((2000, 32)).astype(np.float32)
    Xs /= np.linalg.norm(Xs, axis=1, keepdims=True)
    Ps = oracle.Points(Xs, metric=oracle.IP)
    o2 = oracle.knn_density(Ps, None, L=0, k=5)
    ei2, _ = exact.exact_knn(Xs, 5, metric=exact.IP)
    assert (o2["ids"] == ei2).all()


def test_ari_closed_form_at_scale():
    """Halves against quarters nested in them, n = 4m points. By hand: S_ij =
    S_b = 2m(m-1), S_a = 2m(2m-1), T = 2m(4m-1); E = S_a S_b / T =
    2m(2m-1)(m-1)/(4m-1) and (S_a + S_b)/2 = m(3m-2), so
    ARI = 4m^2(m-1) / (m^2(8m-5)) = 4(m-1)/(8m-5). At n = 2,000,000 the
    product S_a S_b is ~5e23, far beyond int64 (a 64-bit product would wrap)."""
    for m in (1, 2, 3, 1000, 500_000, 1_250_000):
        n = 4 * m
        halves = np.arange(n) // (2 * m)
        quarters = np.arange(n) // m
        want = 4 * (m - 1) / (8 * m - 5)
        assert abs(exact.ari(halves, quarters) - want) <= 1e-15, m
        assert abs(exact.ari(quarters, halves) - want) <= 1e-15, m
    # one label against n singletons: S_ij = S_b = 0, E = 0 -> ARI = 0
    assert exact.ari(np.zeros(2_000_000, np.int64), np.arange(2_000_000)) == 0.0


def test_ari_matches_sklearn_at_one_million():
    """Random labels at n = 1,000,000 (pair counts ~1e11, their products ~1e22):
    scikit-learn's ARI (which promotes to Python integers) agrees."""
    sk = pytest.importorskip("sklearn.metrics")
    g = np.random.default_rng(10)
    n = 1_000_000
    a = g.integers(0, 5, size=n)
    b = np.where(g.random(n) < 0.8, a, g.integers(0, 7, size=n))
    assert abs(exact.ari(a, b) - sk.adjusted_rand_score(a, b)) < 1e-12
    c = g.integers(0, 1000, size=n)
    assert abs(exact.ari(a, c) - sk.adjusted_rand_score(a, c)) < 1e-12


def test_cluster_root_invariants():
    """Every label is the root of its tree: a point whose dependent edge was
    cut, labelled with itself; each non-root point shares its dependent point's label."""
    g = np.random.default_rng(12)
    n, d, k = 1000, 8, 6
    X, _ = _mixture(n, d, 5, g)
    G = random_graph(n, 6, 12)
    P = oracle.Points(X)
    r = oracle.knn_density(P, G, L=24, k=k)
    dep = oracle.dependent_points(P, G, r["key"], r["ids"], Ld=24, threshold=10)
    rho_min = float(np.quantile(r["rho"], 0.05))
    labels, nc = oracle.cluster(r["rho"], dep["lam"], dep["delta"], center=oracle.CENTER_PRODUCT,
                                rho_min=rho_min, n_clusters=5)
    noise = r["rho"] < np.float32(rho_min)
    roots = np.flatnonzero(labels == np.arange(n))
    assert len(roots) == nc
    assert nc == 5 + noise.sum()
    for i in range(n):
        if labels[i] != i:
            assert labels[i] == labels[dep["lam"][i]]
    # the numpy pointer-jumping restatement gives the same labels
    lab2, nc2 = exact.cluster(r["rho"], dep["lam"].astype(np.int64), dep["delta"], center="product",
                              rho_min=np.float32(rho_min), n_clusters=5)
    assert (lab2 == labels).all() and nc2 == nc


def test_well_separated_mixture_ari_one():
    """Well-separated Gaussians: the same-graph method, on the oracle's own
    Vamana graph, recovers the generating clusters (ARI = 1) and agrees with
    exact FP64 DPC."""
    from paper_2312_03940_gb300 import synth
    X, lab = synth.gaussian_mixture(n=3000, d=32, components=10, seed=77)
    P = oracle.Points(X)
    perm = synth.insertion_order(len(X), seed=78)
    G = oracle.build_graph(P, R=32, L=64, alpha=1.2, perm=perm, n_start=16)
    r = oracle.knn_density(P, G, L=64, k=6)
    dep = oracle.dependent_points(P, G, r["key"], r["ids"], Ld=64, threshold=300)
    labels, _ = oracle.cluster(r["rho"], dep["lam"], dep["delta"], center=oracle.CENTER_PRODUCT, n_clusters=10)
    assert exact.ari(labels, lab) == 1.0
    ex = exact.exact_dpc(X, 6, center="product", n_clusters=10)
    assert exact.ari(labels, ex["labels"]) == 1.0
    assert exact.knn_recall(r["dist"], ex["dist"]) >= 0.99


# ---------------------------------------------------------------- RobustPrune and the build

def test_robust_prune_characterisation():
    """The greedy RobustPrune output is the unique list with: (a) ascending
    (dis, id) order, (b) no kept point dominated by an earlier kept point,
    (c) every dropped candidate that precedes the last kept one (or any, if
    fewer than R were kept) dominated by an earlier kept point."""
    g = np.random.default_rng(13)
    X = g.standard_normal((300, 16)).astype(np.float32)
    P = oracle.Points(X)
    Xd = X.astype(np.float64)

    def d2(a, b):
        return float(oracle.dis(P, a, b))

    for trial in range(20):
        p = int(g.integers(300))
        cand = g.choice(300, size=80, replace=False)
        alpha, R = (1.0, 1.2, 1.5)[trial % 3], (4, 8, 16, 64)[trial % 4]
        out = list(oracle.robust_prune(P, p, cand, alpha, R))
        a2 = np.float32(alpha) * np.float32(alpha)
        cs = sorted((d2(p, c), c) for c in set(int(c) for c in cand) if c != p)
        assert out == [c for _, c in sorted((d2(p, c), c) for c in out)]
        for i, u in enumerate(out):
            for v in out[:i]:
                assert not (a2 * np.float32(d2(v, u)) <= np.float32(d2(p, u)))
        last = (d2(p, out[-1]), out[-1])
        for dc, c in cs:
            if c in out:
                continue
            if len(out) == R and (dc, c) > last:
                continue
            assert any(a2 * np.float32(d2(v, c)) <= np.float32(dc) and (d2(p, v), v) < (dc, c) for v in out)
    del Xd


def test_batch_schedule():
    """Batches of 1, 2, 4, ... capped at ceil(0.02 n) (Sec. 4.1)."""
    assert oracle.batch_cap(1_000_000, 0.02) == 20_000
    assert oracle.batch_cap(10_000, 0.02) == 200
    assert oracle.batch_cap(30, 0.02) == 1


def test_build_graph_invariants_and_recall():
    from paper_2312_03940_gb300 import synth
    X, _ = synth.gaussian_mixture(n=2000, d=32, components=10, seed=31)
    P = oracle.Points(X)
    R = 32
    perm = synth.insertion_order(len(X), seed=32)
    G = oracle.build_graph(P, R=R, L=64, alpha=1.2, perm=perm, n_start=16)
    n = len(X)
    for i in range(n):
        row = G[i]
        deg = int((row >= 0).sum())
        assert (row[:deg] >= 0).all() and (row[deg:] == -1).all()
        assert i not in row[:deg]
        assert len(set(row[:deg].tolist())) == deg
    # (almost) every point is reachable from the start points: Vamana does not
    # guarantee it, a point whose in-edges were all pruned stays unreachable
    seen = set(perm[:16].tolist())
    stack = list(seen)
    while stack:
        u = stack.pop()
        for v in G[u]:
            if v >= 0 and v not in seen:
                seen.add(int(v))
                stack.append(int(v))
    assert len(seen) >= 0.995 * n
    r = oracle.knn_density(P, G, L=64, k=10)
    _, ex_d = exact.exact_knn(X, 10)
    assert exact.knn_recall(r["dist"], ex_d) >= 0.95


def test_build_graph_deterministic_across_threads():
    from paper_2312_03940_gb300 import synth
    X, _ = synth.gaussian_mixture(n=1500, d=16, components=5, seed=41)
    P = oracle.Points(X)
    perm = synth.insertion_order(len(X), seed=42)
    G1 = oracle.build_graph(P, R=12, L=24, alpha=1.2, perm=perm, n_start=4, threads=1)
    G8 = oracle.build_graph(P, R=12, L=24, alpha=1.2, perm=perm, n_start=4, threads=8)
    assert (G1 == G8).all()


# ---------------------------------------------------------------- exact oracle vs pure Python

def test_exact_oracle_against_python_loops():
    """exact.exact_knn / exact_dependent against a direct double loop on a tiny input."""
    g = np.random.default_rng(21)
    n, d, k = 25, 3, 4
    X = g.standard_normal((n, d)).astype(np.float32)
    ids, dist = exact.exact_knn(X, k)
    rho, key = exact.density(dist, "kth")
    lam, delta = exact.exact_dependent(X, key)
    for i in range(n):
        ds = []
        for j in range(n):
            if j != i:
                ds.append((math.sqrt(sum((float(X[i, t]) - float(X[j, t])) ** 2 for t in range(d))), j))
        ds.sort()
        assert [j for _, j in ds[:k]] == list(ids[i])
        assert abs(1.0 / ds[k - 1][0] - rho[i]) < 1e-12 * rho[i]
        higher = [(dd, j) for dd, j in ds if ranks_above(key, j, i)]
        if higher:
            assert lam[i] == min(higher)[1]
        else:
            assert lam[i] == -1


def test_exact_knn_queries_and_recall():
    """exact_knn_queries (sampled rows, used at full size) equals exact_knn on
    the same rows for both metrics. knn_recall closed forms: identical lists
    give 1; two of four beyond the exact k-th distance give 0.5; a distance
    within 1e-5 relative of the k-th counts (ties), one at 5e-5 does not."""
    g = np.random.default_rng(22)
    X = g.standard_normal((400, 16)).astype(np.float32)
    Xn = (X / np.linalg.norm(X, axis=1, keepdims=True)).astype(np.float32)
    rows = np.array([0, 7, 123, 399])
    for Xm, metric in ((X, exact.L2), (Xn, exact.IP)):
        ids, dist = exact.exact_knn(Xm, 5, metric=metric)
        qi, qd = exact.exact_knn_queries(Xm, rows, 5, metric=metric)
        assert (qi == ids[rows]).all()
        assert np.allclose(qd, dist[rows], rtol=1e-12, atol=1e-15)
    ex = np.array([[1.0, 2.0, 3.0, 4.0]])
    assert exact.knn_recall(ex, ex) == 1.0
    assert exact.knn_recall(np.array([[1.0, 2.0, 5.0, 6.0]]), ex) == 0.5
    assert exact.knn_recall(np.array([[1.0, 2.0, 3.0, 4.0 * (1 + 5e-6)]]), ex) == 1.0
    assert exact.knn_recall(np.array([[1.0, 2.0, 3.0, 4.0 * (1 + 5e-5)]]), ex) == 0.75


# ---------------------------------------------------------------- NN-Descent graph index

def _nnd_rounds_python(X, init, rounds):
    """Synchronous NN-Descent rounds restated with Python sets on integer
    data (squared distances exact): R(x) = the K smallest (d, q) with x in
    N(q); C(x) = N(x) | R(x); N'(u) = the K smallest (d, id) of
    N(u) | C(u) | union of C(p) for p in C(u), without u."""
    n, K = init.shape
    d2 = lambda a, b: int(((X[a].astype(np.int64) - X[b].astype(np.int64)) ** 2).sum())
    N = [sorted(init[u].tolist(), key=lambda v: (d2(u, v), v)) for u in range(n)]
    for _ in range(rounds):
        rev = {x: [] for x in range(n)}
        for q in range(n):
            for x in N[q]:
                rev[x].append(q)
        Rv = {x: sorted(rev[x], key=lambda q: (d2(q, x), q))[:K] for x in range(n)}
        C = {x: set(N[x]) | set(Rv[x]) for x in range(n)}
        new = []
        for u in range(n):
            cand = set(N[u]) | C[u]
            for p in C[u]:
                cand |= C[p]
            cand.discard(u)
            new.append(sorted(cand, key=lambda v: (d2(u, v), v))[:K])
        N = new
    return np.array(N, np.int32)


def test_nndescent_rounds_match_a_set_restatement():
    g = np.random.default_rng(21)
    X = g.integers(0, 6, size=(40, 4)).astype(np.float32)  # coarse: many equal distances, ties by id
    init = synth.random_neighbours(40, 5, repeats=1, seed=22)
    P = oracle.Points(X)
    for rounds in (1, 3):
        r = oracle.nndescent(P, 5, init, rounds=rounds, alpha=1.2, R=8)
        assert (r["knn"] == _nnd_rounds_python(X, init[0], rounds)).all(), rounds


def test_nndescent_exact_lists_are_a_fixed_point_and_repeats_merge():
    X, _ = _mixture(600, 16, 5, np.random.default_rng(23))
    P = oracle.Points(X)
    ei, _ = exact.exact_knn(X, 8)
    r = oracle.nndescent(P, 8, ei[None].astype(np.int32), rounds=3, alpha=1.2, R=12)
    assert r["changes"][0, 0] == 0 and (r["knn"] == ei).all()
    # two repeats = the 8 smallest of the union of the two single-repeat lists
    init = synth.random_neighbours(600, 8, repeats=2, seed=24)
    a = oracle.nndescent(P, 8, init[:1], rounds=2, alpha=1.2, R=12)["knn"]
    b = oracle.nndescent(P, 8, init[1:], rounds=2, alpha=1.2, R=12)["knn"]
    both = oracle.nndescent(P, 8, init, rounds=2, alpha=1.2, R=12)["knn"]
    for u in range(600):
        cand = sorted(set(a[u]) | set(b[u]), key=lambda v: (oracle.dis(P, u, int(v)), v))[:8]
        assert list(both[u]) == cand, u


def test_nndescent_graph_invariants_and_recall():
    X, _ = _mixture(3000, 32, 8, np.random.default_rng(25))
    P = oracle.Points(X)
    r = oracle.nndescent(P, 16, synth.random_neighbours(3000, 16, repeats=2, seed=26), rounds=12, alpha=1.2, R=24)
    ch = r["changes"]
    assert (ch[:, -1] == 0).all()  # converged within 12 rounds
    _, ed = exact.exact_knn(X, 16)
    got = np.array([[np.sqrt(oracle.dis(P, u, int(v))) for v in r["knn"][u]] for u in range(3000)])
    assert exact.knn_recall(got, ed) >= 0.95
    G = r["G"]
    deg = (G >= 0).sum(1)
    assert deg.max() <= 24 and deg.min() >= 1
    for u in range(3000):
        row = G[u][: deg[u]]
        assert (G[u][deg[u]:] == -1).all() and u not in row and len(set(row.tolist())) == len(row)


# ---------------------------------------------------------------- HCNNG (Sec. 5.1, graph indices)

def _scipy_mst_edges(X):
    """The minimum spanning tree of all points under the oracle's ordering
    value, as a set of (smaller id, larger id) (scipy's routine)."""
    sparse = pytest.importorskip("scipy.sparse.csgraph")
    P = oracle.Points(X)
    n = len(X)
    W = np.zeros((n, n))
    for i in range(n):
        for j in range(i + 1, n):
            W[i, j] = oracle.dis(P, i, j)
    assert (W[np.triu_indices(n, 1)] > 0).all()  # scipy reads 0 as "no edge"
    T = sparse.minimum_spanning_tree(W).tocoo()
    return {(min(a, b), max(a, b)) for a, b in zip(T.row.tolist(), T.col.tolist())}, W


def test_hcnng_leaf_forest_without_bound_is_the_mst():
    """With a degree bound no point can reach, the leaf forest is the minimum
    spanning tree (distinct distances: it is unique), as scipy computes it."""
    X = np.random.default_rng(41).normal(size=(60, 8)).astype(np.float32)
    mst, W = _scipy_mst_edges(X)
    E = oracle.hcnng_leaf_mst(oracle.Points(X), np.arange(60), mst_deg=60)
    assert len(E) == 59
    assert {(min(a, b), max(a, b)) for a, b in E.tolist()} == mst
    # the edges come out in increasing length (Kruskal's order)
    w = [W[min(a, b), max(a, b)] for a, b in E.tolist()]
    assert w == sorted(w)


def test_hcnng_leaf_forest_degree_bound():
    """Points on a line: the MST is the path through them in coordinate
    order, whose degrees are at most 2, so the bound 2 leaves it unchanged;
    the bound 1 leaves a matching of disjoint closest pairs."""
    g = np.random.default_rng(42)
    t = np.sort(g.uniform(0, 100, size=40)).astype(np.float32)
    perm = g.permutation(40)
    X = np.zeros((40, 4), np.float32)
    X[perm, 0] = t  # point perm[i] sits at the i-th coordinate
    P = oracle.Points(X)
    E = oracle.hcnng_leaf_mst(P, np.arange(40), mst_deg=2)
    path = {(min(perm[i], perm[i + 1]), max(perm[i], perm[i + 1])) for i in range(39)}
    assert {(min(a, b), max(a, b)) for a, b in E.tolist()} == path
    M = oracle.hcnng_leaf_mst(P, np.arange(40), mst_deg=1)
    deg = np.bincount(M.ravel(), minlength=40)
    assert deg.max() == 1
    # greedy matching: the globally closest pair of the line is in it
    gaps = np.diff(t)
    i = int(np.argmin(gaps))
    assert (min(perm[i], perm[i + 1]), max(perm[i], perm[i + 1])) in {(min(a, b), max(a, b)) for a, b in M.tolist()}


def test_hcnng_partition_invariants():
    X, _ = _mixture(2000, 16, 6, np.random.default_rng(43))
    P = oracle.Points(X)
    for t in range(3):
        L = oracle.hcnng_partition(P, t, leaf_size=150, seed=7)
        allids = np.concatenate(L)
        assert sorted(allids.tolist()) == list(range(2000))       # a partition of the points
        assert max(len(l) for l in L) <= 150 and len(L) >= 14      # leaves of at most leaf_size
        assert all((np.diff(l) > 0).all() for l in L)              # each leaf in ascending id
    # the draws depend on the repeat and the seed, and on nothing else
    a = oracle.hcnng_partition(P, 0, 150, seed=7)
    b = oracle.hcnng_partition(P, 0, 150, seed=7)
    c = oracle.hcnng_partition(P, 1, 150, seed=7)
    d = oracle.hcnng_partition(P, 0, 150, seed=8)
    assert all((x == y).all() for x, y in zip(a, b))
    assert len(a) != len(c) or any(not np.array_equal(x, y) for x, y in zip(a, c))
    assert len(a) != len(d) or any(not np.array_equal(x, y) for x, y in zip(a, d))
    # one leaf when it can hold every point
    one = oracle.hcnng_partition(P, 0, 2000)
    assert len(one) == 1 and (one[0] == np.arange(2000)).all()


def test_hcnng_graph_is_the_mst_when_nothing_is_cut_or_pruned():
    """One repeat, one leaf, no degree bound and alpha so large that
    RobustPrune drops nothing: every point's list is its MST neighbours."""
    X = np.random.default_rng(44).normal(size=(50, 8)).astype(np.float32)
    mst, _ = _scipy_mst_edges(X)
    G = oracle.hcnng(oracle.Points(X), repeats=1, leaf_size=50, mst_deg=50, alpha=1e6, R=50)["G"]
    got = {(min(u, v), max(u, v)) for u in range(50) for v in G[u].tolist() if v >= 0}
    assert got == mst
    for u in range(50):  # both directions of every edge
        row = [v for v in G[u].tolist() if v >= 0]
        assert sorted(row) == sorted([b if a == u else a for a, b in mst if u in (a, b)])


def test_hcnng_graph_invariants_and_recall():
    X, _ = _mixture(3000, 32, 8, np.random.default_rng(45))
    P = oracle.Points(X)
    r = oracle.hcnng(P, repeats=3, leaf_size=200, mst_deg=3, alpha=1.2, R=24)
    G = r["G"]
    deg = (G >= 0).sum(1)
    assert deg.max() <= 9 and deg.min() >= 1  # at most mst_deg per repeat
    for u in range(3000):
        row = G[u][: deg[u]]
        assert (G[u][deg[u]:] == -1).all() and u not in row and len(set(row.tolist())) == len(row)
    _, ed = exact.exact_knn(X, 10)
    o = oracle.knn_density(P, G, L=64, k=10)
    assert exact.knn_recall(o["dist"], ed) >= 0.95


def test_hcnng_pivot_generator_is_splitmix64():
    """The published SplitMix64 outputs for the states 0, 1 and 2 golden-ratio
    increments (Steele, Lea and Flood's generator as distributed with xoshiro)."""
    gold = 0x9E3779B97F4A7C15
    assert oracle.splitmix64(0) == 0xE220A8397B1DCDAF
    assert oracle.splitmix64(gold) == 0x6E789E6AA1B965F4
    assert oracle.splitmix64((2 * gold) % (1 << 64)) == 0x06C45D188009454F


def test_hcnng_first_split_by_brute_force():
    """The root split of a 60-point set into leaves of at most 40: the pivots
    are the drawn positions of 0..59, every point is on the side of its nearer
    pivot (ties left), and each side keeps ascending ids."""
    X = np.random.default_rng(46).normal(size=(60, 8)).astype(np.float32)
    P = oracle.Points(X)
    seed, t = 12, 2  # a root split of 21 / 39 points: both sides are leaves
    i1 = oracle.hcnng_draw(seed, t, 0, 60, 0) % 60
    i2 = oracle.hcnng_draw(seed, t, 0, 60, 1) % 59
    i2 += i2 >= i1
    left = [x for x in range(60) if oracle.dis(P, x, i1) <= oracle.dis(P, x, i2)]
    right = [x for x in range(60) if x not in left]
    assert 0 < len(left) <= 40 and 0 < len(right) <= 40
    L = oracle.hcnng_partition(P, t, leaf_size=40, seed=seed)
    assert [l.tolist() for l in L] == [left, right]
