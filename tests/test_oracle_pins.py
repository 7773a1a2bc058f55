"""Pins of the CPU oracle against facts that do not come from the oracle.

Each test fixes the oracle to something independent: closed forms derived by
hand, the Newman-Girvan adjacency form of modularity, brute force over all set
partitions or all candidate moves on tiny graphs, published reference values,
and invariants of the paper's definitions (Sec. II) and algorithms
(Algorithms 1-3).
"""
import json
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth
from tests import _textbook as tb

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _frac(q_num_den):
    q, num, den = q_num_den
    return Fraction(num, den) if den else Fraction(0)


def clique_edges(members):
    return [(a, b) for i, a in enumerate(members) for b in members[i + 1:]]


# ---------------------------------------------------------------- Sec. II-C closed forms

@pytest.mark.parametrize("n", [2, 3, 5, 8])
def test_modularity_complete_graph_singletons(n):
    # K_n: vol(c) = cut(c) = n-1 for every singleton, vol(V) = n(n-1):
    # Q = -n (n-1)^2 / (n(n-1))^2 = -1/n
    g = synth.from_edge_list(n, clique_edges(list(range(n))))
    off, cols, w = g.numpy()
    assert _frac(oracle.modularity(off, cols, w, np.arange(n))) == Fraction(-1, n)
    # one community: cut = 0, vol(c) = vol(V): Q = 1 - 1 = 0
    assert _frac(oracle.modularity(off, cols, w, np.zeros(n))) == 0


@pytest.mark.parametrize("k,m", [(2, 3), (3, 4), (5, 5)])
def test_modularity_disjoint_cliques(k, m):
    # k disjoint K_m, each its own community: Q = k (1/k - 1/k^2) = 1 - 1/k
    n = k * m
    edges = sum((clique_edges(list(range(c * m, (c + 1) * m))) for c in range(k)), [])
    g = synth.from_edge_list(n, edges)
    off, cols, w = g.numpy()
    lab = np.arange(n) // m
    assert _frac(oracle.modularity(off, cols, w, lab)) == 1 - Fraction(1, k)


@pytest.mark.parametrize("k,m", [(3, 4), (6, 5)])
def test_modularity_ring_of_cliques(k, m):
    # k cliques K_m joined in a ring by one edge each. E = k m(m-1)/2 + k.
    # Per clique: vol = m(m-1) + 2, cut = 2. Q = k m(m-1)/2E - k (m(m-1)+2)^2 / 4E^2.
    n = k * m
    edges = sum((clique_edges(list(range(c * m, (c + 1) * m))) for c in range(k)), [])
    edges += [(c * m, ((c + 1) % k) * m + 1) for c in range(k)]
    g = synth.from_edge_list(n, edges)
    off, cols, w = g.numpy()
    E = k * m * (m - 1) // 2 + k
    want = Fraction(k * m * (m - 1), 2 * E) - Fraction(k * (m * (m - 1) + 2) ** 2, 4 * E * E)
    assert _frac(oracle.modularity(off, cols, w, np.arange(n) // m)) == want


def test_modularity_loops_counted_twice():
    # Two vertices with loops L and an edge of weight x, as singletons.
    # deg_w = x + 2L each, vol(V) = 4L + 2x; per community vol - cut = 2L:
    # Q = 2 [2L / (4L + 2x) - 1/4] = 2L / (2L + x) - 1/2.
    L, x = 3, 2
    g = synth.from_edge_list(2, [(0, 1)], [x], {0: L, 1: L})
    off, cols, w = g.numpy()
    d, vol = oracle.degw(off, cols, w)
    assert d.tolist() == [x + 2 * L, x + 2 * L] and vol == 4 * L + 2 * x
    assert _frac(oracle.modularity(off, cols, w, [0, 1])) == Fraction(2 * L, 2 * L + x) - Fraction(1, 2)


def test_modularity_degenerate():
    g = synth.from_edge_list(4, [])
    off, cols, w = g.numpy()
    assert oracle.modularity(off, cols, w, np.arange(4))[0] == 0.0
    assert np.isnan(oracle.modularity(off, cols, w, [0, 1, 2, 9])[0])


# ---------------------------------------------------------------- Sec. II-C vs Newman-Girvan

@pytest.mark.parametrize("seed", range(12))
def test_modularity_equals_newman_girvan(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(2, 14))
    edges, ws, lp, g = tb.random_graph(rng, n, 0.35, wmax=5, loops=0.3)
    A = tb.adjacency(n, edges, ws, lp)
    off, cols, w = g.numpy()
    for _ in range(5):
        lab = rng.integers(0, max(1, n // 2), size=n)
        q = oracle.modularity(off, cols, w, lab)
        assert _frac(q) == tb.q_ng(A, lab)
        assert abs(q[0] - float(tb.q_ng(A, lab))) <= 1e-15


# ---------------------------------------------------------------- Eq. deltaQ

@pytest.mark.parametrize("seed", range(10))
def test_gain_equals_modularity_difference(seed):
    # Eq. deltaQ (with deg_w(V) read as deg_w(v)): dQ = 2 G / vol^2 must equal
    # Q(after) - Q(before) exactly, for every vertex and every target community.
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(2, 11))
    edges, ws, lp, g = tb.random_graph(rng, n, 0.4, wmax=4, loops=0.25)
    A = tb.adjacency(n, edges, ws, lp)
    vol = int(A.sum())
    if vol == 0:
        return
    off, cols, w = g.numpy()
    lab = rng.integers(0, max(1, n // 2), size=n).astype(np.int32)
    q0 = tb.q_ng(A, lab)
    for v in range(n):
        for B in range(n):
            after = lab.copy()
            after[v] = B
            G = oracle.move_gain(off, cols, w, lab, v, B)
            assert Fraction(2 * G, vol * vol) == tb.q_ng(A, after) - q0, (v, B)


def _round_state(A, lab):
    k = A.sum(axis=1)
    n = len(lab)
    sigma = np.bincount(lab, weights=k, minlength=n).astype(np.int64)
    size = np.bincount(lab, minlength=n).astype(np.int32)
    return k.astype(np.int64), int(k.sum()), sigma, size


@pytest.mark.parametrize("seed", range(10))
def test_louvain_decision_is_best_positive_move(seed):
    # Algorithm 2 decision vs brute force over every neighbour community with
    # exact dQ from the Newman-Girvan form; ties to the smallest id; strict > 0;
    # a singleton only joins a singleton with a smaller id.
    rng = np.random.default_rng(200 + seed)
    n = int(rng.integers(3, 12))
    edges, ws, lp, g = tb.random_graph(rng, n, 0.4, wmax=3, loops=0.2)
    A = tb.adjacency(n, edges, ws, lp)
    off, cols, w = g.numpy()
    ws_ = oracle.Workspace(n)
    for trial in range(4):
        lab = (np.arange(n) if trial == 0 else rng.integers(0, n, size=n)).astype(np.int32)
        degw, vol, sigma, size = _round_state(A, lab)
        q0 = tb.q_ng(A, lab)
        for v in range(n):
            cands = {int(lab[u]) for u in range(n) if u != v and A[v, u] > 0} - {int(lab[v])}
            best, bq = None, None
            for B in sorted(cands):
                after = lab.copy()
                after[v] = B
                dq = tb.q_ng(A, after) - q0
                if bq is None or dq > bq:
                    best, bq = B, dq
            want = int(lab[v])
            if best is not None and bq > 0:
                A_ = int(lab[v])
                if not (size[A_] == 1 and size[best] == 1 and best > A_):
                    want = best
            got = oracle.louvain_decide(off, cols, w, lab, sigma, size, degw, vol, v, 1, ws_)
            assert got == want, (trial, v)


@pytest.mark.parametrize("seed", range(10))
def test_lpa_decision_brute_force(seed):
    # Algorithm 1, PLPMove: heaviest neighbour label; keep the current label on
    # a tie with the maximum, else the smallest maximal label.
    rng = np.random.default_rng(300 + seed)
    n = int(rng.integers(2, 14))
    edges, ws, lp, g = tb.random_graph(rng, n, 0.35, wmax=3, loops=0.2)
    off, cols, w = g.numpy()
    for _ in range(4):
        lab = rng.integers(0, max(1, n // 2), size=n).astype(np.int32)
        for v in range(n):
            W = tb.label_weights(n, edges, ws, lab, v)
            if not W:
                want1 = want0 = int(lab[v])
            else:
                mx = max(W.values())
                smallest = min(c for c, x in W.items() if x == mx)
                want0 = smallest
                want1 = int(lab[v]) if W.get(int(lab[v]), 0) == mx else smallest
            assert oracle.lpa_decide(off, cols, w, lab, v, 1) == want1
            assert oracle.lpa_decide(off, cols, w, lab, v, 0) == want0


# ---------------------------------------------------------------- the deferral coin

def test_commit_coin_is_splitmix64():
    with open(os.path.join(GOLDEN, "splitmix64_seed1234567.json")) as f:
        gold = json.load(f)
    # the numpy generator matches the published vector ...
    got = synth.draw(gold["state"], np.arange(5, dtype=np.uint64)).tolist()
    assert got == gold["outputs"]
    # ... and the oracle's coin is bit 63 of that generator at the stated counter
    seed = oracle.DEFAULT_SCHED_SEED
    rng = np.random.default_rng(7)
    for _ in range(200):
        lv, r, v = int(rng.integers(0, 64)), int(rng.integers(0, 1000)), int(rng.integers(0, 2**31 - 1))
        ctr = (lv << 48) | (r << 32) | v
        want = int(synth.draw(seed, np.array([ctr], dtype=np.uint64))[0] >> np.uint64(63))
        assert oracle.commit(lv, r, v, seed) == want
    coins = [oracle.commit(0, r, v) for r in range(20) for v in range(200)]
    assert 0.45 < np.mean(coins) < 0.55


# ---------------------------------------------------------------- Algorithm 3 aggregation

@pytest.mark.parametrize("seed", range(8))
def test_aggregation_matches_cut_definition(seed):
    # Coarse edge {A,B} weight = cut_w(A,B) over the original edges; loop {A,A}
    # = internal weight (edges inside A plus loops in A). Also: vol(V) and
    # modularity are preserved, Q(G', singletons) = Q(G, C).
    rng = np.random.default_rng(400 + seed)
    n = int(rng.integers(2, 16))
    edges, ws, lp, g = tb.random_graph(rng, n, 0.3, wmax=6, loops=0.3)
    off, cols, w = g.numpy()
    lab = rng.integers(0, n, size=n).astype(np.int32)
    k, newid, coff, ccols, cw = oracle.aggregate(off, cols, w, lab)
    used = sorted(set(lab.tolist()))
    assert k == len(used) and [newid[c] for c in used] == list(range(k))
    want = {}
    for (a, b), wt in zip(edges, ws if ws else [1] * len(edges)):
        A_, B_ = newid[lab[a]], newid[lab[b]]
        if A_ == B_:
            want[(A_, A_)] = want.get((A_, A_), 0) + wt
        else:
            want[(A_, B_)] = want.get((A_, B_), 0) + wt
            want[(B_, A_)] = want.get((B_, A_), 0) + wt
    for v, L in lp.items():
        A_ = newid[lab[v]]
        want[(A_, A_)] = want.get((A_, A_), 0) + L
    got = {}
    for a in range(k):
        rows = ccols[coff[a]:coff[a + 1]]
        assert list(rows) == sorted(rows)
        for j in range(coff[a], coff[a + 1]):
            got[(a, int(ccols[j]))] = int(cw[j])
    assert got == want
    A0 = tb.adjacency(n, edges, ws, lp)
    A1 = np.zeros((k, k), dtype=np.int64)
    for (a, b), x in got.items():
        A1[a, b] += 2 * x if a == b else x
    assert A1.sum() == A0.sum()
    assert tb.q_ng(A1, np.arange(k)) == tb.q_ng(A0, newid[lab])


# ---------------------------------------------------------------- whole algorithms

def _ring_of_cliques(k, m, perm_seed=None):
    n = k * m
    edges = sum((clique_edges(list(range(c * m, (c + 1) * m))) for c in range(k)), [])
    edges += [(c * m, ((c + 1) % k) * m + 1) for c in range(k)]
    lab = np.arange(n) // m
    if perm_seed is not None:
        p = np.random.default_rng(perm_seed).permutation(n)
        edges = [(int(p[a]), int(p[b])) for a, b in edges]
        lab2 = np.empty(n, dtype=np.int64)
        lab2[p] = lab
        lab = lab2
    return n, edges, lab


def _same_partition(a, b):
    a, b = np.asarray(a), np.asarray(b)
    pairs = set(zip(a.tolist(), b.tolist()))
    return len(pairs) == len(set(a.tolist())) == len(set(b.tolist()))


@pytest.mark.parametrize("k,m,seed", [(4, 5, None), (5, 6, 1), (8, 5, 2)])
def test_louvain_recovers_clique_ring(k, m, seed):
    # A ring of k cliques K_m (k small vs m^2): the optimum puts each clique in
    # its own community. Checked against the brute-force optimum for small n.
    n, edges, planted = _ring_of_cliques(k, m, seed)
    g = synth.from_edge_list(n, edges)
    off, cols, w = g.numpy()
    lab, levels, q, _ = oracle.louvain(off, cols, w)
    assert _same_partition(lab, planted)
    A = tb.adjacency(n, edges, None, None)
    assert abs(q - float(tb.q_ng(A, planted))) < 1e-12


@pytest.mark.parametrize("seed", range(6))
def test_louvain_never_beats_brute_force_optimum(seed):
    rng = np.random.default_rng(500 + seed)
    n = int(rng.integers(4, 10))
    edges, ws, lp, g = tb.random_graph(rng, n, 0.4, wmax=3)
    A = tb.adjacency(n, edges, ws, lp)
    if A.sum() == 0:
        return
    off, cols, w = g.numpy()
    lab, levels, q, _ = oracle.louvain(off, cols, w)
    qe = tb.q_ng(A, lab)
    assert abs(q - float(qe)) < 1e-12
    assert qe <= tb.best_q(A)


def test_louvain_two_cliques_bridge_is_optimal():
    # two K_5 joined by one edge: brute-force optimum = the two cliques
    edges = clique_edges(list(range(5))) + clique_edges(list(range(5, 10))) + [(4, 5)]
    g = synth.from_edge_list(10, edges)
    off, cols, w = g.numpy()
    lab, _, q, _ = oracle.louvain(off, cols, w)
    A = tb.adjacency(10, edges, None, None)
    assert tb.q_ng(A, lab) == tb.best_q(A)
    assert _same_partition(lab, [0] * 5 + [1] * 5)


@pytest.mark.parametrize("seed", range(6))
def test_local_move_end_state_has_no_admissible_move(seed):
    # With full sweeps (every vertex re-examined each round), a level that
    # stops because no vertex changes has, for every vertex, no neighbour
    # community with dQ > 0 that the singleton rule would allow. (With the
    # needCheck frontier a vertex away from every move is not re-examined,
    # so the property is only claimed for full sweeps.)
    rng = np.random.default_rng(600 + seed)
    n = int(rng.integers(5, 30))
    edges, ws, lp, g = tb.random_graph(rng, n, 0.2, wmax=4, loops=0.1)
    A = tb.adjacency(n, edges, ws, lp)
    off, cols, w = g.numpy()
    lab, moves, tr = oracle.local_move(off, cols, w, max_iter=500, use_frontier=0)
    assert tr.rounds < 500 and tr.moved[-1] == 0 and tr.deferred[-1] == 0
    _, _, sigma, size = _round_state(A, lab)
    q0 = tb.q_ng(A, lab)
    for v in range(n):
        cands = sorted({int(lab[u]) for u in range(n) if u != v and A[v, u] > 0} - {int(lab[v])})
        best, bq = None, None
        for B in cands:
            after = lab.copy()
            after[v] = B
            dq = tb.q_ng(A, after) - q0
            if bq is None or dq > bq:
                best, bq = B, dq
        if best is not None and bq > 0:
            assert size[lab[v]] == 1 and size[best] == 1 and best > lab[v]


def test_louvain_invariants_on_components():
    # communities never span two connected components; sigma_tot sums to vol
    sp = pytest.importorskip("scipy.sparse")
    from scipy.sparse.csgraph import connected_components
    rng = np.random.default_rng(11)
    parts = []
    base = 0
    edges = []
    for size in [7, 12, 3, 20, 1, 9]:
        for a in range(size):
            for b in range(a + 1, size):
                if rng.random() < 0.4:
                    edges.append((base + a, base + b))
        base += size
    n = base
    g = synth.from_edge_list(n, edges)
    off, cols, w = g.numpy()
    lab, _, q, _ = oracle.louvain(off, cols, w)
    M = sp.csr_matrix((np.ones(len(cols)), cols, off), shape=(n, n))
    ncomp, comp = connected_components(M, directed=False)
    for c in set(lab.tolist()):
        assert len(set(comp[lab == c].tolist())) == 1
    d, vol = oracle.degw(off, cols, w)
    assert d.sum() == vol == 2 * len(edges)


@pytest.mark.parametrize("k,m", [(3, 4), (6, 7)])
def test_lpa_recovers_disjoint_cliques(k, m):
    n = k * m
    edges = sum((clique_edges(list(range(c * m, (c + 1) * m))) for c in range(k)), [])
    g = synth.from_edge_list(n, edges)
    off, cols, w = g.numpy()
    lab, tr = oracle.lpa(off, cols, w)
    assert _same_partition(lab, np.arange(n) // m)
    assert tr.moved[-1] + tr.deferred[-1] == 0


@pytest.mark.parametrize("seed", range(6))
def test_lpa_stops_at_fixed_point(seed):
    # dN = 0 means every vertex holds a label of maximal neighbour weight
    rng = np.random.default_rng(700 + seed)
    n = int(rng.integers(5, 40))
    edges, ws, lp, g = tb.random_graph(rng, n, 0.15, wmax=3)
    off, cols, w = g.numpy()
    lab, tr = oracle.lpa(off, cols, w, max_iter=1000)
    assert tr.rounds < 1000
    for v in range(n):
        W = tb.label_weights(n, edges, ws, lab, v)
        if W:
            assert W.get(int(lab[v]), 0) == max(W.values())
    assert tr.arcs[0] == len(cols)


def test_degenerate_inputs():
    for n in (0, 1, 5):
        g = synth.from_edge_list(n, [])
        off, cols, w = g.numpy()
        lab, tr = oracle.lpa(off, cols, w)
        assert lab.tolist() == list(range(n)) and tr.rounds == 1
        lab, levels, q, _ = oracle.louvain(off, cols, w)
        assert lab.tolist() == list(range(n)) and levels == 1 and q == 0.0
        lab, _, tr = oracle.local_move(off, cols, w, max_iter=0)
        assert lab.tolist() == list(range(n)) and tr.rounds == 0


def test_planted_partition_sanity():
    # The SBM workload (n = 10,000, 100 blocks, p_in = 0.1, p_out = 0.001):
    # Louvain reaches at least 95% of the planted partition's modularity.
    g = synth.sbm(10000, 100, "0.1", "0.001", seed=1)
    off, cols, w = g.numpy()
    q_planted = oracle.modularity(off, cols, w, g.planted)[0]
    lab, levels, q, _ = oracle.louvain(off, cols, w)
    assert q >= 0.95 * q_planted
    lab_lpa, tr = oracle.lpa(off, cols, w)
    assert tr.moved[-1] + tr.deferred[-1] == 0  # LPA reaches a fixed point


def test_initial_active_set():
    # Algorithm 1's V_active / Algorithm 2's needCheck started from a given set:
    # all-ones equals the default; vertices outside the set keep their label
    # in round 1, and the arcs scanned are the set's degrees.
    g = synth.sbm(3000, 30, "0.1", "0.004", seed=4, wmax=3)
    off, cols, w = g.numpy()
    ones = np.ones(g.n, dtype=np.uint8)
    a, ta = oracle.lpa(off, cols, w)
    b, tb_ = oracle.lpa(off, cols, w, active_in=ones)
    assert np.array_equal(a, b) and ta.rounds == tb_.rounds
    sub = (np.random.default_rng(1).random(g.n) < 0.2).astype(np.uint8)
    deg = np.diff(off)
    for fn in (lambda: oracle.lpa(off, cols, w, max_iter=1, active_in=sub)[::1],
               lambda: oracle.local_move(off, cols, w, max_iter=1, active_in=sub)[::2]):
        lab, tr = fn()
        assert np.all(lab[sub == 0] == np.arange(g.n)[sub == 0])
        assert tr.active[0] == sub.sum() and tr.arcs[0] == deg[sub == 1].sum()
        assert tr.moved[0] == np.count_nonzero(lab != np.arange(g.n))
