"""Full-size checks of the benchmark line: the 1,280,000 x 1024 unit-norm
inner-product workload on the exact index, in the launch configuration the
benchmark times (k = 16; the k-NN screen in CTA pairs, the default for
d >= 512).

The oracle cannot take a million points in a test, so outputs are checked on
sampled points it computes one by one (its brute-force index over all rows:
k-NN ids, distances and density keys, bit for bit) and through properties
that hold at any size (every dependent point ranks above its point, its
reported distance is the canonical distance of the pair, and no point ranked
above is closer by more than FP32 rounding). The inputs are seeded synthetic
rows; nothing the oracle sees comes from the CUDA path.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2312_03940_gb300 import pecann as pc
from paper_2312_03940_gb300 import synth

pytestmark = pytest.mark.gpu
N, D, K = 1_280_000, 1024, 16


@pytest.fixture(scope="module")
def run():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    pc.load_library()
    X, _ = synth.vmf_like(n=N, d=D, components=1000)
    ds = pc.Dataset(torch.from_numpy(X).cuda(), metric=pc.IP)
    p = pc.params(k=K, index=pc.INDEX_BRUTE_FORCE, center=pc.CENTER_PRODUCT, n_clusters=1000)
    ws = pc.workspace(ds, p)
    dens = pc.pecann_density(ds, None, p, ws=ws)
    dep = pc.pecann_dependent_points(ds, None, p, dens["rank_key"], dens["knn_ids"], dens["knn_dist"], ws=ws)
    torch.cuda.synchronize()
    out = {k: v.cpu().numpy() for k, v in dens.items()}
    out.update(dep=dep["dep"].cpu().numpy(), dep_dist=dep["dep_dist"].cpu().numpy())
    del ws, ds
    torch.cuda.empty_cache()
    return X, out


def test_sampled_knn_and_densities_equal_the_oracle(run):
    X, r = run
    P = oracle.Points(X, metric=oracle.IP)
    rows = synth.sample_ids(N, 24, seed=401)
    o = oracle.knn_density_rows(P, None, rows, L=0, k=K)
    assert (r["knn_ids"][rows] == o["ids"]).all()
    assert (r["knn_dist"][rows] == o["dist"]).all()
    assert (r["rank_key"][rows] == o["key"]).all()
    assert (r["density"][rows] == o["rho"]).all()


def test_dependent_points_properties(run):
    X, r = run
    P = oracle.Points(X, metric=oracle.IP)
    key, lam, delta = r["rank_key"], r["dep"], r["dep_dist"]
    ids = np.arange(N)
    # exactly one point (the top of the ranking) has no dependent point
    top = int(np.lexsort((ids, -key))[0])
    assert (lam < 0).sum() == 1 and lam[top] < 0
    rows = synth.sample_ids(N, 24, seed=402)
    for i in rows.tolist():
        if i == top:
            continue
        j = int(lam[i])
        assert key[j] > key[i] or (key[j] == key[i] and j < i)  # ranks above
        assert delta[i] == np.float32(oracle.out_dist(P, oracle.dis(P, i, j)))
        above = (key > key[i]) | ((key == key[i]) & (ids < i))
        dots = X @ X[i]  # FP32 products, within 1e-5 of the canonical ones for unit rows
        assert delta[i] <= 1.0 - float(dots[above].max()) + 1e-4  # no closer point ranked above
