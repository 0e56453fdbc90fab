"""Small shared helpers for the tests (no method arithmetic here)."""
from __future__ import annotations

import numpy as np


def example_arrays(golden):
    """The worked example of Sec. 3 as arrays: X (6 x 4 float32, the two
    coordinates padded with zeros), adjacency G (6 x R, -1 padded), names."""
    names = golden["names"]
    idx = {c: i for i, c in enumerate(names)}
    X = np.zeros((len(names), 4), np.float32)
    for c, (x, y) in golden["points"].items():
        X[idx[c], 0] = x
        X[idx[c], 1] = y
    adj = {i: [] for i in range(len(names))}
    for a, b in golden["edges"]:
        adj[idx[a]].append(idx[b])
        adj[idx[b]].append(idx[a])
    R = max(len(v) for v in adj.values())
    G = np.full((len(names), R), -1, np.int32)
    for i, v in adj.items():
        G[i, :len(v)] = v
    return X, G, names, idx


def random_graph(n: int, R: int, seed: int) -> np.ndarray:
    """A random out-degree-R graph that contains the ring i -> i+1, so every
    point is reachable from every other."""
    g = np.random.default_rng(seed)
    G = np.full((n, R), -1, np.int32)
    for i in range(n):
        nb = [(i + 1) % n]
        others = g.choice(n, size=min(n - 1, 3 * R), replace=False)
        for o in others:
            if len(nb) >= R:
                break
            if o != i and o not in nb:
                nb.append(int(o))
        G[i, :len(nb)] = nb
    return G


def ranks_above(key, j, i):
    return key[j] > key[i] or (key[j] == key[i] and j < i)


def quantize_e4m3(X: np.ndarray):
    """FP8 e4m3 codes of X / s with the per-dimension scale s_j = max_i |x_ij| / 448
    (448 is the largest e4m3 value); the decoded point is s_j * code_j.
    Returns (codes as a torch float8_e4m3fn CPU tensor, s as float32)."""
    import torch
    s = (np.abs(X).max(0) / 448.0).astype(np.float32)
    s[s == 0] = 1.0
    codes = torch.from_numpy((X.astype(np.float32) / s).astype(np.float32)).to(torch.float8_e4m3fn)
    return codes, s
