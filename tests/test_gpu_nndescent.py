"""The NN-Descent graph index on the GPU (Sec. 5.1, graph indices: the
framework's PyNNDescent option with num_repeats) against the oracle's.

Both sides run the same synchronous rounds from the same initial lists and
score every pair with the canonical FP32 (or exact integer) distance, so the
k-NN lists, the per-round change counts and the pruned graph must be equal
bit for bit. Cases cover FP32 L2, FP32 inner product on unit vectors and
uint8 L2, one and several repeats, K below, at and above one warp, rounds
that stop at convergence, zero rounds (initial lists only), coarse data
with many equal distances (ties by id), and the error paths.
"""
import ctypes

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


def run_both(X, metric, K, repeats, rounds, R=16, alpha=1.2, seed=300):
    init = synth.random_neighbours(len(X), K, repeats=repeats, seed=seed)
    ds = pc.Dataset(torch.from_numpy(np.ascontiguousarray(X)).cuda(), metric=metric)
    p = pc.params(R=R, alpha=alpha)
    g = pc.pecann_build_nndescent(ds, p, K, torch.from_numpy(init).cuda(), rounds)
    o = oracle.nndescent(oracle.Points(X, metric=metric), K, init, rounds=rounds, alpha=alpha, R=R)
    knn = g["knn"].cpu().numpy()
    G = g["graph"].cpu().numpy()
    assert (g["changes"] == o["changes"]).all(), (g["changes"], o["changes"])
    assert (knn == o["knn"]).all()
    assert (G == o["G"]).all()
    assert (g["degree"].cpu().numpy() == (o["G"] >= 0).sum(1)).all()
    return g, o


def test_f32_l2_two_repeats():
    X, _ = synth.gaussian_mixture(n=3000, d=32, components=8, seed=301)
    g, _ = run_both(X, pc.L2, K=16, repeats=2, rounds=12, R=24)
    assert (g["changes"][:, -1] == 0).all()  # converged


def test_u8_l2_128():
    """The 1M x 128 uint8 workload's row shape: distances are exact integers."""
    X, _ = synth.u8_mixture(n=4000, d=128, components=20, seed=302)
    run_both(X, pc.L2, K=20, repeats=1, rounds=8, R=32)


def test_ip_unit_vectors_k40():
    """K above one warp (two 32-id chunks per list), inner-product metric."""
    X, _ = synth.vmf_like(n=2500, d=64, components=10, seed=303)
    run_both(X, pc.IP, K=40, repeats=2, rounds=6, R=48)


def test_coarse_values_ties_and_round_limit():
    """Values in 0..3: many equal distances (ties broken by id); a round limit
    of 2 stops before convergence; K = 5 below a warp."""
    X = np.random.default_rng(304).integers(0, 4, size=(1500, 16)).astype(np.float32)
    g, _ = run_both(X, pc.L2, K=5, repeats=3, rounds=2, R=8)
    assert (g["changes"][:, -1] > 0).any()


def test_zero_rounds_and_small_n():
    X, _ = synth.gaussian_mixture(n=12, d=8, components=2, seed=305)
    run_both(X, pc.L2, K=11, repeats=2, rounds=0, R=4)
    run_both(X, pc.L2, K=3, repeats=1, rounds=5, R=4)


def test_bad_initial_lists_and_arguments():
    X, _ = synth.gaussian_mixture(n=200, d=16, components=2, seed=306)
    ds = pc.Dataset(torch.from_numpy(X).cuda())
    p = pc.params(R=8)
    init = torch.from_numpy(synth.random_neighbours(200, 6, repeats=1, seed=307)).cuda()
    bad = init.clone()
    bad[0, 5, 1] = bad[0, 5, 0]  # a repeated id
    with pytest.raises(pc.PecannError) as e:
        pc.pecann_build_nndescent(ds, p, 6, bad, 3)
    assert e.value.status == pc.EINTERNAL
    bad = init.clone()
    bad[0, 7, 2] = 200  # out of range
    with pytest.raises(pc.PecannError) as e:
        pc.pecann_build_nndescent(ds, p, 6, bad, 3)
    assert e.value.status == pc.EINTERNAL
    # the context is still usable: a good call right after
    pc.pecann_build_nndescent(ds, p, 6, init, 3)
    lib = pc.load_library()
    nb = ctypes.c_size_t(0)
    for K, reps in ((0, 1), (65, 1), (200, 1), (6, 0), (6, 65)):
        assert lib.pecann_nndescent_workspace_size(ds.ref, ctypes.byref(p), K, reps, ctypes.byref(nb)) == pc.EINVAL
