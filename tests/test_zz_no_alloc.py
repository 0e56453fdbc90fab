"""pecann_density_noalloc: the k-NN + density entry point for callers that
cannot allocate GPU memory (its scratch is a fixed array inside the library).

It must give the same results as pecann_density, element for element, on
two calls in a row (the second call finds the first call's leftovers in the
shared scratch), also when a smaller set follows a larger one and with the
autotuner's block shape; match the oracle; report an out-of-range graph
entry like pecann_density; and refuse point sets larger than its fixed
scratch holds.
This file is collected last so that a failure here comes after every other
test has run; it also passes on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_2312_03940_gb300 import autotune
from paper_2312_03940_gb300 import pecann as pc
from paper_2312_03940_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    pc.load_library()


def _graph(n, R, seed, isolated_every=0):
    g = np.random.default_rng(seed)
    G = np.full((n, R), -1, np.int32)
    for i in range(n):
        nb = [(i + 1) % n] + [int(x) for x in g.choice(n, size=R - 1, replace=False) if x != i][: R - 1]
        G[i, :len(nb)] = nb
    if isolated_every:
        G[::isolated_every] = -1  # these searches return too few points: the fallback list is used
    return torch.from_numpy(G).cuda()


def _same(a, b):
    # the same kernels on the same inputs: every output bit for bit
    for key in ("knn_ids", "knn_dist", "density", "rank_key"):
        x, y = a[key].cpu().numpy(), b[key].cpu().numpy()
        assert np.array_equal(x, y, equal_nan=True), key


def test_noalloc_matches_density_on_consecutive_calls():
    cases = []
    X, _ = synth.gaussian_mixture(n=6000, d=32, components=8, seed=71)
    cases.append((torch.from_numpy(X).cuda(), _graph(6000, 16, 71, isolated_every=101),
                  pc.params(k=8, R=16, L_search=32)))
    X2, _ = synth.u8_mixture(n=5000, d=128, components=10, seed=72)
    cases.append((torch.from_numpy(X2).cuda(), _graph(5000, 24, 72, isolated_every=0),
                  pc.params(k=10, R=24, L_search=48, normalize_density=1)))
    # R = 64 with the block shape and filter size the autotuner picks
    X3, _ = synth.gaussian_mixture(n=3000, d=64, components=6, seed=73)
    X3d, G3 = torch.from_numpy(X3).cuda(), _graph(3000, 64, 73)
    p3 = pc.params(k=6, R=64, L_search=64)
    autotune.tune_density(pc.Dataset(X3d), G3, p3, reps=1, use_cache=False)
    cases.append((X3d, G3, p3))
    # the larger set first, then the smaller ones: the later calls must not
    # see the earlier call's fallback list or densities beyond their own n
    for X, G, p in cases:
        ds = pc.Dataset(X)
        ref = pc.pecann_density(ds, G, p, ws=pc.workspace(ds, p))
        for _ in range(2):
            got = pc.pecann_density_noalloc(ds, G, p)
            torch.cuda.synchronize()
            _same(got, ref)


def test_noalloc_matches_oracle():
    """k-NN lists and densities equal to the oracle's (Algorithm 2 lines 2-4 on
    the same graph), including points whose search returns fewer than k."""
    X, _ = synth.gaussian_mixture(n=2500, d=32, components=5, seed=74)
    G = _graph(2500, 12, 74, isolated_every=53)
    p = pc.params(k=7, R=12, L_search=24)
    got = pc.pecann_density_noalloc(pc.Dataset(torch.from_numpy(X).cuda()), G, p)
    o = oracle.knn_density(oracle.Points(X), G.cpu().numpy(), L=24, k=7)
    assert o["fallback"].sum() > 0
    assert (got["knn_ids"].cpu().numpy() == o["ids"]).all()
    assert (got["knn_dist"].cpu().numpy() == o["dist"]).all()
    assert (got["rank_key"].cpu().numpy() == o["key"]).all()
    assert (got["density"].cpu().numpy() == o["rho"]).all()


def test_noalloc_reports_bad_graph_entry():
    """A graph entry >= n is skipped by the kernels and reported as
    PECANN_EINTERNAL, as pecann_density does; the next good call succeeds."""
    X, _ = synth.gaussian_mixture(n=800, d=32, components=3, seed=75)
    Gh = _graph(800, 8, 75).cpu().numpy()
    Gh[17, 2] = 5000
    ds = pc.Dataset(torch.from_numpy(X).cuda())
    p = pc.params(k=4, R=8, L_search=16)
    with pytest.raises(pc.PecannError) as e:
        pc.pecann_density_noalloc(ds, torch.from_numpy(Gh).cuda(), p)
    assert e.value.status == pc.EINTERNAL
    Gh[17, 2] = 18
    pc.pecann_density_noalloc(ds, torch.from_numpy(Gh).cuda(), p)


def test_noalloc_rejects_too_many_points():
    lib = pc.load_library()
    X = torch.zeros((16, 32), dtype=torch.float32, device="cuda")
    ds = pc.PecannDataset(X.data_ptr(), pc.NOALLOC_MAX_POINTS + 1, 32, pc.F32, pc.L2, 0, None, None)
    p = pc.params(k=4, R=8, L_search=8)
    buf = ctypes.c_void_p(X.data_ptr())
    st = lib.pecann_density_noalloc(ctypes.byref(ds), buf, ctypes.byref(p), buf, buf, buf, buf, None)
    assert st == pc.EINVAL
    assert b"PECANN_NOALLOC_MAX_POINTS" in lib.pecann_last_error()
