"""Pins of the oracle's synchronous round drivers (Algorithm 1 PLP,
Algorithm 2 local moving) on graphs of 2-5 vertices, worked out by hand.

The per-vertex decisions are pinned elsewhere (brute force); what these cases
fix is the schedule around them, under the readings the oracle states:
- every decision of a round reads the labels (and Sigma_tot, sizes) of the
  start of the round, and all committed moves apply together afterwards;
- a vertex whose decision differs from its label commits only when the coin
  (bit 63 of SplitMix64 draw number level<<48 | round<<32 | v) is 1, else it
  defers;
- the next round examines the moved vertices, their neighbours and the
  deferred vertices; LPA stops after a round with moved + deferred <= 0,
  local moving after a round with no move and no deferral;
- the trace counts, per round, the examined vertices, their arcs, their
  distinct neighbour labels (candidate pairs, the own label included) and
  the arcs of the vertices that moved.

The coin values are literals below, checked against the SplitMix64 stream the
published reference vector pins (tests/golden); with sched_seed = 1234567 the
round-0 coins of vertices 0-4 are bit 63 of exactly that vector's five
outputs. Every expected label, count and active set was derived by hand from
the definitions; the derivations are summarised beside each case.

The last test plants each plausible mistake of a round driver (decisions that
read labels already updated in the same round, an inverted coin, a deferred
vertex not re-examined, neighbours of a moved vertex not re-examined) into a
copy of oracle.c and checks that these pins reject it.
"""
import json
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
SEED = 1234567

# COINS[(level, round)][v] for v = 0..4 under sched_seed = SEED
COINS = {
    (0, 0): [0, 0, 1, 0, 1],
    (0, 1): [1, 1, 1, 1, 0],
    (0, 2): [1, 1, 0, 0, 1],
    (0, 3): [0, 1, 0, 1, 0],
}


def test_coin_literals_follow_splitmix64():
    with open(os.path.join(GOLDEN, "splitmix64_seed1234567.json")) as f:
        gold = json.load(f)
    assert gold["state"] == SEED
    assert [x >> 63 for x in gold["outputs"]] == COINS[(0, 0)]
    for (lv, r), bits in COINS.items():
        ctr = np.array([(lv << 48) | (r << 32) | v for v in range(5)], dtype=np.uint64)
        assert [int(x >> np.uint64(63)) for x in synth.draw(SEED, ctr)] == bits
        assert [oracle.commit(lv, r, v, SEED) for v in range(5)] == bits


def csr(n, edges):
    g = synth.from_edge_list(n, edges)
    return g.numpy()


K2 = (2, [(0, 1)])
PATH = (5, [(0, 1), (1, 2), (2, 4), (4, 3)])          # the path 0-1-2-4-3
STAR = (5, [(0, 1), (0, 2), (0, 3), (0, 4)])          # centre 0
BOWTIE = (5, [(0, 1), (0, 2), (1, 2), (2, 3), (2, 4), (3, 4)])  # triangles {0,1,2}, {2,3,4}

# LPA, tie_keep_current = 1. Per case: labels after each round, and the trace.
LPA_CASES = {
    # r0: 0 wants 1, 1 wants 0; coins 0,0: both defer. r1 (deferred re-examined):
    # coins 1,1: they swap to [1,0]. r2: coins 1,1: swap back to [0,1].
    # r3: 0 defers (coin 0), 1 commits to 0. r4: nobody wants to move.
    "k2": (K2, [[0, 1], [1, 0], [0, 1], [0, 0], [0, 0]],
           dict(moved=[0, 2, 2, 1, 0], deferred=[2, 0, 0, 1, 0], active=[2, 2, 2, 2, 2], arcs=[2] * 5,
                cands=[2] * 5, moved_arcs=[0, 2, 2, 1, 0])),
    # r0: wants 0->1, 1->0, 2->1, 3->4, 4->2 (ties to the smallest label);
    #     coins commit 2 and 4: [0,1,1,3,2].
    # r1: 1, 2 keep (their label attains the maximum); 0->1, 3->2, 4->1;
    #     coins commit 0 and 3, 4 defers: [1,1,1,2,2].
    # r2: examines {0,3} + neighbours {1,4} + deferred {4}: nobody moves.
    "path": (PATH, [[0, 1, 1, 3, 2], [1, 1, 1, 2, 2], [1, 1, 1, 2, 2]],
             dict(moved=[2, 2, 0], deferred=[3, 1, 0], active=[5, 5, 4], arcs=[8, 8, 6],
                  cands=[8, 8, 5], moved_arcs=[4, 2, 0])),
    # r0: centre wants 1, leaves want 0; coins commit 2 and 4: [0,1,0,3,0].
    # r1: centre keeps 0 (weight 2), leaves 1 and 3 commit to 0.
    # r2: examines {1,3} + centre: nobody moves.
    "star": (STAR, [[0, 1, 0, 3, 0], [0, 0, 0, 0, 0], [0, 0, 0, 0, 0]],
             dict(moved=[2, 2, 0], deferred=[3, 0, 0], active=[5, 5, 3], arcs=[8, 8, 6],
                  cands=[8, 7, 3], moved_arcs=[2, 2, 0])),
}


@pytest.mark.parametrize("case", list(LPA_CASES))
def test_lpa_rounds_by_hand(case):
    (n, edges), per_round, tr = LPA_CASES[case]
    off, cols, w = csr(n, edges)
    for r, want in enumerate(per_round, start=1):
        lab, _ = oracle.lpa(off, cols, w, max_iter=r, sched_seed=SEED)
        assert lab.tolist() == want, (case, r)
    lab, t = oracle.lpa(off, cols, w, max_iter=100, sched_seed=SEED)
    assert lab.tolist() == per_round[-1] and t.rounds == len(per_round)
    for key, vals in tr.items():
        assert getattr(t, key).tolist() == vals, (case, key)


# Local moving (Algorithm 2), singletons at the start, singleton rule on.
# Gains are G = vol(V) (k_{v,c} - k_{v,A-}) - deg_w(v) (Sigma_tot(c) - Sigma_tot(A-)).
LM_CASES = {
    # vol = 2. r0: G(0->1) = G(1->0) = 1 > 0; the singleton rule lets only 1
    # move (towards the smaller id); its coin is 0: deferred.
    # r1 examines only the deferred vertex 1; coin 1: it joins 0.
    # r2 examines 1 and its neighbour 0: nothing left to gain.
    "k2": (K2, [[0, 1], [0, 0], [0, 0]],
           dict(moved=[0, 1, 0], deferred=[1, 0, 0], active=[2, 1, 2], arcs=[2, 1, 2],
                cands=[2, 1, 2], moved_arcs=[0, 1, 0]), 1),
    # vol = 12, deg = (2,2,4,2,2).
    # r0: 0 -> 1 (G 8) and 3 -> 4 (G 8) are barred by the singleton rule;
    #     1 -> 0 (G 8), 2 -> 0 (G 4, ties to the smallest id), 4 -> 3 (G 8);
    #     coins: 1 defers, 2 and 4 commit: [0,1,0,3,3].
    # r1 (all examined): 0 -> 1 (G = 0 - 2 (2 - 4) = 4), 1 -> 0 (G = 24 - 12),
    #     2 -> 3 (G = 12 - 8 = 4 beats G(2->1) = 0), 3 and 4 stay (G = -8);
    #     coins 1,1,1: all commit: [1,0,3,3,3].
    # r2: 0 -> 0 (G 8, singleton towards the smaller id) commits; 1 -> 1 is
    #     barred; 2 stays (G -4): [0,0,3,3,3].
    # r3 examines 0 and its neighbours 1, 2: no positive gain (2 -> 0 has G = 0).
    "bowtie": (BOWTIE, [[0, 1, 0, 3, 3], [1, 0, 3, 3, 3], [0, 0, 3, 3, 3], [0, 0, 3, 3, 3]],
               dict(moved=[2, 3, 1, 0], deferred=[1, 0, 0, 0], active=[5, 5, 5, 3], arcs=[12, 12, 12, 8],
                    cands=[12, 10, 9, 6], moved_arcs=[6, 8, 2, 0]), 6),
}


@pytest.mark.parametrize("case", list(LM_CASES))
def test_local_move_rounds_by_hand(case):
    (n, edges), per_round, tr, total = LM_CASES[case]
    off, cols, w = csr(n, edges)
    for r, want in enumerate(per_round, start=1):
        lab, _, _ = oracle.local_move(off, cols, w, max_iter=r, sched_seed=SEED)
        assert lab.tolist() == want, (case, r)
    lab, moves, t = oracle.local_move(off, cols, w, max_iter=100, sched_seed=SEED)
    assert lab.tolist() == per_round[-1] and t.rounds == len(per_round) and moves == total
    for key, vals in tr.items():
        assert getattr(t, key).tolist() == vals, (case, key)


def test_bowtie_end_state_modularity():
    # communities {0,1} and {2,3,4}: vol 4 and 8, cut 2 each, vol(V) = 12:
    # Q = (2/12 - 1/9) + (6/12 - 4/9) = 1/9
    (n, edges), per_round, _, _ = LM_CASES["bowtie"]
    off, cols, w = csr(n, edges)
    q, num, den = oracle.modularity(off, cols, w, per_round[-1])
    assert num * 9 == den


# ---------------------------------------------------------------- planted mistakes

def _replace(src, old, new, count=1):
    assert src.count(old) == count, old
    return src.replace(old, new)


def _mut_in_place(src):
    # decisions read the round's output arrays, which hold every move made
    # earlier in the same round (nxt / target start equal to C)
    src = _replace(src, "for (int64_t v = 0; v < n; ++v) C[v] = (int32_t)v; /* singleton labels */",
                   "for (int64_t v = 0; v < n; ++v) C[v] = nxt[v] = (int32_t)v;")
    src = _replace(src, "orc_lpa_decide(n, off, cols, w, C, (int32_t)v", "orc_lpa_decide(n, off, cols, w, nxt, (int32_t)v")
    src = _replace(src, "    csize[C[v]] += 1;\n  }\n", "    csize[C[v]] += 1;\n    target[v] = C[v];\n  }\n")
    return _replace(src, "orc_louvain_decide(n, off, cols, w, C, sigma", "orc_louvain_decide(n, off, cols, w, target, sigma")


def _mut_coin(src):
    return _replace(src, "if (orc_commit(", "if (!orc_commit(", count=2)


def _mut_no_deferred(src):
    return _replace(src, "    if (deferred[v]) active[v] = 1;\n", "")


def _mut_no_neighbours(src):
    return _replace(src, "    for (int64_t e = off[v]; e < off[v + 1]; ++e) active[cols[e]] = 1;\n", "")


MUTATIONS = {"in_place": _mut_in_place, "inverted_coin": _mut_coin,
             "deferred_not_reexamined": _mut_no_deferred, "neighbours_not_reexamined": _mut_no_neighbours}


def _pins_pass():
    try:
        for case in LPA_CASES:
            test_lpa_rounds_by_hand(case)
        for case in LM_CASES:
            test_local_move_rounds_by_hand(case)
    except AssertionError:
        return False
    return True


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
@pytest.mark.parametrize("mutation", list(MUTATIONS))
def test_pins_reject_planted_mistakes(mutation, tmp_path, monkeypatch):
    here = os.path.dirname(oracle.__file__)
    src = open(os.path.join(here, "oracle.c")).read()
    shutil.copy(os.path.join(here, "oracle.h"), tmp_path / "oracle.h")
    (tmp_path / "oracle.c").write_text(MUTATIONS[mutation](src))
    so = tmp_path / "libmut.so"
    subprocess.check_call(["gcc", "-O1", "-std=gnu11", "-fPIC", "-shared", "-o", str(so),
                           str(tmp_path / "oracle.c"), "-lm"])
    assert _pins_pass()  # the real oracle passes ...
    monkeypatch.setattr(oracle, "_lib", oracle.load(str(so)))
    assert not _pins_pass(), mutation  # ... the altered one does not
