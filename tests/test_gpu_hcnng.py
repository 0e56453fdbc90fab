"""The HCNNG graph index on the GPU (Sec. 5.1, graph indices: the framework's
HCNNG option with num_repeats and alpha) against the oracle's.

Both sides split the points with the same SplitMix64 pivot draws, decide
every side and every forest edge on the canonical FP32 (or exact integer)
distance with the same tie order, and prune with the same RobustPrune, so the
graphs must be equal bit for bit. Cases cover FP32 L2, FP32 inner product on
unit vectors and uint8 L2, several repeats, leaves of every size up to the
200-point limit, degree bounds of 1, 3 and more than a leaf holds, coarse
data with many equal distances and repeated points (degenerate splits),
n at or below one leaf, and the argument checks.
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


def run_both(X, metric, repeats, leaf, deg, R=24, alpha=1.2, seed=5):
    ds = pc.Dataset(torch.from_numpy(np.ascontiguousarray(X)).cuda(), metric=metric)
    g = pc.pecann_build_hcnng(ds, pc.params(R=R, alpha=alpha, seed=seed), repeats, leaf, deg)
    o = oracle.hcnng(oracle.Points(X, metric=metric), repeats, leaf, deg, alpha, R, seed=seed)
    assert (g["leaves"] == o["leaves"]).all(), (g["leaves"], o["leaves"])
    G = g["graph"].cpu().numpy()
    assert (G == o["G"]).all()
    assert (g["degree"].cpu().numpy() == (o["G"] >= 0).sum(1)).all()
    return g


def test_f32_l2_three_repeats():
    X, _ = synth.gaussian_mixture(n=5000, d=32, components=8, seed=311)
    g = run_both(X, pc.L2, repeats=3, leaf=200, deg=3)
    assert g["leaves"].min() >= 25


def test_u8_l2_128():
    """The 1M x 128 uint8 workload's row shape: integer distances."""
    X, _ = synth.u8_mixture(n=6000, d=128, components=20, seed=312)
    run_both(X, pc.L2, repeats=2, leaf=150, deg=3, R=32)


def test_ip_unit_vectors():
    X, _ = synth.vmf_like(n=3000, d=64, components=10, seed=313)
    run_both(X, pc.IP, repeats=3, leaf=100, deg=4, R=16, alpha=1.1)


def test_coarse_values_and_repeated_points():
    """Values in 0..2 over 8 dimensions: many equal distances (ties by id) and
    many identical points, so some splits leave a side empty and cut the
    node in halves instead."""
    X = np.random.default_rng(314).integers(0, 3, size=(2500, 8)).astype(np.float32)
    run_both(X, pc.L2, repeats=3, leaf=40, deg=2, R=8)
    U = np.zeros((2500, 16), np.uint8)
    U[:, :8] = X.astype(np.uint8)
    run_both(U, pc.L2, repeats=2, leaf=7, deg=1, R=4)


def test_small_sets_and_bounds():
    X, _ = synth.gaussian_mixture(n=180, d=16, components=3, seed=315)
    run_both(X, pc.L2, repeats=1, leaf=200, deg=16, R=32, alpha=1e6)  # one leaf, nothing cut
    run_both(X, pc.L2, repeats=4, leaf=2, deg=1, R=4)                  # leaves of 1-2 points
    run_both(X[:3], pc.L2, repeats=2, leaf=2, deg=3, R=2)


def test_argument_checks():
    X = torch.zeros((300, 16), dtype=torch.float32, device="cuda")
    ds = pc.Dataset(X)
    lib = pc.load_library()
    p = pc.params(R=8)
    nb = ctypes.c_size_t(0)
    for reps, leaf, deg in ((0, 50, 3), (65, 50, 3), (1, 1, 3), (1, 201, 3), (1, 50, 0), (1, 50, 17)):
        assert lib.pecann_hcnng_workspace_size(ds.ref, ctypes.byref(p), reps, leaf, deg, ctypes.byref(nb)) == pc.EINVAL
    with pytest.raises(pc.PecannError) as e:
        pc.pecann_build_hcnng(ds, pc.params(R=8, alpha=0.5), 1, 50, 3)
    assert e.value.status == pc.EINVAL
