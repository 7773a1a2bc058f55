"""Independent textbook definitions used to pin the oracle (test helpers).

Nothing here is the oracle's code or formula. Modularity is taken in the
Newman-Girvan adjacency form Q = (1/2m) sum_ij [A_ij - k_i k_j / 2m]
delta(c_i, c_j) over a dense adjacency matrix with A_ii = 2 L_i (a loop adds
twice to its vertex's degree), evaluated in exact integer / Fraction
arithmetic; optima come from enumerating every set partition.
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np

import synth


def random_graph(rng: np.random.Generator, n: int, p: float, wmax: int = 1, loops: float = 0.0):
    """Seeded small random graph as (edge list, weights, loops dict, CSR Graph)."""
    edges, ws = [], []
    for u in range(n):
        for v in range(u + 1, n):
            if rng.random() < p:
                edges.append((u, v))
                ws.append(int(rng.integers(1, wmax + 1)))
    lp = {v: int(rng.integers(1, wmax + 1)) for v in range(n) if rng.random() < loops}
    g = synth.from_edge_list(n, edges, ws if (wmax > 1 or lp) else None, lp)
    return edges, ws, lp, g


def adjacency(n: int, edges, ws, loops) -> np.ndarray:
    A = np.zeros((n, n), dtype=np.int64)
    for (u, v), w in zip(edges, ws if ws else [1] * len(edges)):
        A[u, v] += w
        A[v, u] += w
    for v, L in (loops or {}).items():
        A[v, v] += 2 * L
    return A


def q_ng(A: np.ndarray, labels) -> Fraction:
    """Newman-Girvan modularity, exact."""
    labels = np.asarray(labels)
    k = A.sum(axis=1)
    two_m = int(k.sum())
    if two_m == 0:
        return Fraction(0)
    same = labels[:, None] == labels[None, :]
    num = int((A * two_m - np.outer(k, k))[same].sum())
    return Fraction(num, two_m * two_m)


def set_partitions(n: int) -> np.ndarray:
    """All set partitions of n elements as restricted growth strings."""
    out = []
    a = [0] * n

    def rec(i, m):
        if i == n:
            out.append(a.copy())
            return
        for c in range(m + 2):
            a[i] = c
            rec(i + 1, max(m, c))

    if n == 0:
        return np.zeros((1, 0), dtype=np.int64)
    a[0] = 0
    rec(1, 0)
    return np.array(out, dtype=np.int64)


def best_q(A: np.ndarray) -> Fraction:
    """Maximum modularity over all partitions (brute force)."""
    n = A.shape[0]
    k = A.sum(axis=1)
    two_m = int(k.sum())
    B = A * two_m - np.outer(k, k)
    P = set_partitions(n)
    score = np.zeros(P.shape[0], dtype=np.int64)
    for i in range(n):
        for j in range(n):
            if B[i, j]:
                score += B[i, j] * (P[:, i] == P[:, j])
    return Fraction(int(score.max()), two_m * two_m)


def label_weights(n: int, edges, ws, labels, v: int) -> dict:
    """Total edge weight from v to each neighbour label (loops excluded)."""
    out = {}
    for (a, b), w in zip(edges, ws if ws else [1] * len(edges)):
        for x, y in ((a, b), (b, a)):
            if x == v:
                out[int(labels[y])] = out.get(int(labels[y]), 0) + w
    return out
