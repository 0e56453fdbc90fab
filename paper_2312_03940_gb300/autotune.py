"""Autotuner for the speed-only knobs of the search kernel.

Two knobs change how fast the beam search runs but never what it returns:
the seen-filter size (`hash_slots`: a forgotten id costs a repeated distance,
never a different beam) and the warps per block (`block_warps`). The tuner
times every candidate on the caller's own workload with CUDA events, checks
that each one reproduces the first candidate's outputs exactly, keeps the
fastest, and caches the choice in a JSON file keyed by a workload signature
(`PECANN_AUTOTUNE_CACHE`, default ~/.cache/pecann_gb300/autotune.json).
"""
from __future__ import annotations

import json
import os

import torch

from . import pecann as pc

CANDIDATES = [(h, w) for h in (512, 1024, 2048) for w in (4, 8)]


def _cache_path() -> str:
    return os.environ.get("PECANN_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "pecann_gb300", "autotune.json"))


def _load_cache() -> dict:
    try:
        with open(_cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _save_cache(c: dict):
    path = _cache_path()
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(c, f, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except OSError:
        pass


def _time(fn, reps: int) -> float:
    fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def _tune(sig: str, p: pc.PecannParams, run, snapshot, candidates, reps: int, use_cache: bool) -> dict:
    cache = _load_cache() if use_cache else {}
    if sig in cache:
        p.hash_slots, p.block_warps = cache[sig]["hash_slots"], cache[sig]["block_warps"]
        return dict(cache[sig], cached=True)
    results, ref = [], None
    for h, w in candidates:
        p.hash_slots, p.block_warps = h, w
        ms = _time(run, reps)
        snap = snapshot()
        if ref is None:
            ref = snap
        elif not all(torch.equal(a, b) for a, b in zip(ref, snap)):
            raise RuntimeError(f"autotune: candidate hash_slots={h} block_warps={w} changed the results")
        results.append((ms, h, w))
    ms, h, w = min(results)
    p.hash_slots, p.block_warps = h, w
    choice = {"hash_slots": h, "block_warps": w, "ms": ms,
              "tried": [{"hash_slots": hh, "block_warps": ww, "ms": mm} for mm, hh, ww in results]}
    if use_cache:
        cache[sig] = choice
        _save_cache(cache)
    return dict(choice, cached=False)


def tune_batch(batch: pc.Batch, reps: int = 2, candidates=None, use_cache: bool = True) -> dict:
    """Pick hash_slots / block_warps for a prepared batch (sets batch.p)."""
    p = batch.p
    sig = (f"batch:sets={batch.n_sets}:N={batch.N}:dmax={max(d.d for d in batch.datasets)}:"
           f"L={p.L_search}:Ld={p.L_dep}:R={p.R}:k={p.k}:{torch.cuda.get_device_name()}")
    return _tune(sig, p, batch.run, lambda: (batch.out["knn_ids"].clone(), batch.out["dep"].clone(),
                                             batch.out["labels"].clone()),
                 candidates or CANDIDATES, reps, use_cache)


def tune_density(ds: pc.Dataset, graph: torch.Tensor, p: pc.PecannParams, reps: int = 2, candidates=None,
                 use_cache: bool = True) -> dict:
    """Pick hash_slots / block_warps for pecann_density on this dataset (sets p)."""
    ws = pc.workspace(ds, p)
    out = {}

    def run():
        out.update(pc.pecann_density(ds, graph, p, ws=ws))

    sig = (f"density:n={ds.n}:d={ds.d}:dtype={ds.X.dtype}:L={p.L_search}:R={p.R}:k={p.k}:"
           f"{torch.cuda.get_device_name()}")
    return _tune(sig, p, run, lambda: (out["knn_ids"].clone(), out["rank_key"].clone()),
                 candidates or CANDIDATES, reps, use_cache)
