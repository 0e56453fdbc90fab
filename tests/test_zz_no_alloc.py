"""pecann_density_noalloc: the k-NN + density entry point for callers that
cannot allocate GPU memory (its scratch is a fixed array inside the library).

It must give the same results as pecann_density, element for element, on
two calls in a row (the second call finds the first call's leftovers in the
shared scratch), and refuse point sets larger than its fixed scratch holds.
This file is collected last so that a failure here comes after every other
test has run; it also passes on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest
import torch

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
    for key in ("knn_ids", "knn_dist", "density", "rank_key"):
        x, y = a[key].cpu().numpy(), b[key].cpu().numpy()
        if key in ("knn_ids", "knn_dist", "rank_key"):
            assert np.array_equal(x, y), key
        else:
            assert np.allclose(x, y, rtol=1e-5, atol=0), key


def test_noalloc_matches_density_on_consecutive_calls():
    cases = []
    X, _ = synth.gaussian_mixture(n=6000, d=32, components=8, seed=71)
    cases.append((torch.from_numpy(X).cuda(), _graph(6000, 16, 71, isolated_every=101),
                  pc.params(k=8, R=16, L_search=32)))
    X2, _ = synth.u8_mixture(n=5000, d=128, components=10, seed=72)
    cases.append((torch.from_numpy(X2).cuda(), _graph(5000, 24, 72, isolated_every=0),
                  pc.params(k=10, R=24, L_search=48, normalize_density=1)))
    for X, G, p in cases:
        ds = pc.Dataset(X)
        ref = pc.pecann_density(ds, G, p, ws=pc.workspace(ds, p))
        for _ in range(2):
            got = pc.pecann_density_noalloc(ds, G, p)
            torch.cuda.synchronize()
            _same(got, ref)


def test_noalloc_rejects_too_many_points():
    lib = pc.load_library()
    X = torch.zeros((16, 32), dtype=torch.float32, device="cuda")
    ds = pc.PecannDataset(X.data_ptr(), pc.NOALLOC_MAX_POINTS + 1, 32, pc.F32, pc.L2, 0, None, None)
    p = pc.params(k=4, R=8, L_search=8)
    buf = ctypes.c_void_p(X.data_ptr())
    st = lib.pecann_density_noalloc(ctypes.byref(ds), buf, ctypes.byref(p), buf, buf, buf, buf, None)
    assert st == pc.EINVAL
    assert b"PECANN_NOALLOC_MAX_POINTS" in lib.pecann_last_error()
