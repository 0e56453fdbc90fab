"""Host-side logic that needs no GPU: the seeded input generators and the
autotuner's selection, result check and cache (timing faked)."""
import json
import types

import numpy as np
import pytest
import torch

from paper_2312_03940_gb300 import autotune
from paper_2312_03940_gb300 import synth


# ---------------------------------------------------------------- generators

def test_generators_are_deterministic_in_their_seed():
    a, la = synth.gaussian_mixture(n=500, d=8, components=4, seed=3)
    b, lb = synth.gaussian_mixture(n=500, d=8, components=4, seed=3)
    c, _ = synth.gaussian_mixture(n=500, d=8, components=4, seed=4)
    assert np.array_equal(a, b) and np.array_equal(la, lb) and not np.array_equal(a, c)
    u, _ = synth.u8_mixture(n=2000, d=16, components=5, seed=9)
    v, _ = synth.u8_mixture(n=2000, d=16, components=5, seed=9)
    assert np.array_equal(u, v)
    assert np.array_equal(synth.insertion_order(1000, seed=1), synth.insertion_order(1000, seed=1))


def test_generator_shapes_ranges_and_structure():
    X, lab = synth.gaussian_mixture(n=1000, d=32, components=10, seed=5)
    assert X.shape == (1000, 32) and X.dtype == np.float32 and set(np.unique(lab)) <= set(range(10))
    U, ul = synth.u8_mixture(n=4000, d=128, components=20, seed=6)
    assert U.shape == (4000, 128) and U.dtype == np.uint8
    assert (ul == 20).sum() == 200  # 5% uniform noise points, labelled `components`
    V, vl = synth.vmf_like(n=3000, d=64, components=30, seed=7)
    assert np.allclose(np.linalg.norm(V, axis=1), 1.0, atol=1e-5) and len(np.unique(vl)) <= 30
    S, sl = synth.powerlaw_sphere(n=3000, d=48, components=50, seed=8)
    assert np.allclose(np.linalg.norm(S, axis=1), 1.0, atol=1e-5) and S.shape == (3000, 48)
    perm = synth.insertion_order(777, seed=2)
    assert np.array_equal(np.sort(perm), np.arange(777))
    ids = synth.sample_ids(10_000, 300, seed=3)
    assert len(np.unique(ids)) == 300 and ids.min() >= 0 and ids.max() < 10_000


def test_batched_sets_follow_their_recipe():
    sets = synth.batched_sets(count=6, n_lo=2000, n_hi=5000, dims=(96, 128), comp_lo=5, comp_hi=20, seed=11)
    assert len(sets) == 6
    for X, lab, comps in sets:
        n, d = X.shape
        assert 2000 <= n <= 5000 and d in (96, 128) and X.dtype == np.float32
        assert 5 <= comps <= 20 and lab.shape == (n,)


# ---------------------------------------------------------------- autotuner

def _fake_run(times, p, outputs):
    """A stand-in workload: its time depends on the knobs, its output is fixed
    unless `outputs` says otherwise."""
    state = {}

    def run():
        state["last"] = (p.hash_slots, p.block_warps)

    def snapshot():
        return (outputs.get(state["last"], torch.arange(5)),)

    def fake_time(fn, reps):
        fn()
        return times[(p.hash_slots, p.block_warps)]

    return run, snapshot, fake_time


def test_autotune_picks_the_fastest_and_caches_it(tmp_path, monkeypatch):
    monkeypatch.setenv("PECANN_AUTOTUNE_CACHE", str(tmp_path / "cache.json"))
    p = types.SimpleNamespace(hash_slots=0, block_warps=0)
    cands = [(512, 4), (1024, 8), (2048, 8)]
    times = {(512, 4): 3.0, (1024, 8): 1.5, (2048, 8): 2.0}
    run, snapshot, fake_time = _fake_run(times, p, {})
    monkeypatch.setattr(autotune, "_time", fake_time)
    got = autotune._tune("sig-a", p, run, snapshot, cands, reps=1, use_cache=True)
    assert (got["hash_slots"], got["block_warps"], got["cached"]) == (1024, 8, False)
    assert (p.hash_slots, p.block_warps) == (1024, 8)
    assert len(got["tried"]) == 3
    saved = json.loads((tmp_path / "cache.json").read_text())
    assert saved["sig-a"]["hash_slots"] == 1024
    # a second call reads the cache and sets the knobs without timing anything
    p2 = types.SimpleNamespace(hash_slots=0, block_warps=0)

    def no_time(fn, reps):
        raise AssertionError("timed although cached")

    monkeypatch.setattr(autotune, "_time", no_time)
    again = autotune._tune("sig-a", p2, run, snapshot, cands, reps=1, use_cache=True)
    assert again["cached"] and (p2.hash_slots, p2.block_warps) == (1024, 8)


def test_autotune_rejects_a_candidate_that_changes_results(tmp_path, monkeypatch):
    monkeypatch.setenv("PECANN_AUTOTUNE_CACHE", str(tmp_path / "cache.json"))
    p = types.SimpleNamespace(hash_slots=0, block_warps=0)
    cands = [(512, 4), (1024, 8)]
    times = {(512, 4): 1.0, (1024, 8): 2.0}
    run, snapshot, fake_time = _fake_run(times, p, {(1024, 8): torch.arange(5) + 1})
    monkeypatch.setattr(autotune, "_time", fake_time)
    with pytest.raises(RuntimeError, match="changed the results"):
        autotune._tune("sig-b", p, run, snapshot, cands, reps=1, use_cache=False)
