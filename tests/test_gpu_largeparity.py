"""Full-run parity at sizes where the oracle still finishes in about a minute:
the LFR-style benchmark graph at its stated size (n = 1,000,000, degree power
law 2.5 on [5, 1000], community sizes 1.5 on [20, 5000], mu = 0.3, weights
U{1..8}) and R-MAT at scale 20 (edge factor 16, the headline graph's recipe).
LPA to convergence and Louvain to convergence through the C ABI must give the
oracle's labels, round counts and per-round traces (LPA), and its labels,
levels, per-level rounds and moves, and modularity (Louvain)."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

GRAPHS = {
    "lfr1m_w": lambda: synth.lfr(1_000_000, seed=2),
    "rmat20": lambda: synth.rmat(20, 16, seed=3, device="cuda").to("cpu"),
}
_cache = {}


def graph(name):
    if name not in _cache:
        _cache[name] = GRAPHS[name]()
    return _cache[name]


def upload(g):
    import paper_2507_06471_gb300 as cd
    return cd.Graph(g.off.cuda(), g.cols.cuda(), None if g.w is None else g.w.cuda())


@pytest.mark.parametrize("name", list(GRAPHS))
def test_lpa_full_run(name):
    g = graph(name)
    off, cols, w = g.numpy()
    G = upload(g)
    lab, rounds = G.lpa()
    tr = G.trace()
    olab, otr = oracle.lpa(off, cols, w)
    assert rounds == otr.rounds
    np.testing.assert_array_equal(lab.cpu().numpy(), olab)
    for key in ("moved", "deferred", "active", "arcs", "cands", "moved_arcs"):
        assert [t[key] for t in tr] == getattr(otr, key).tolist(), key
    G.close()


@pytest.mark.parametrize("name", list(GRAPHS))
def test_louvain_full_run(name):
    g = graph(name)
    off, cols, w = g.numpy()
    G = upload(g)
    lab, levels, q = G.louvain()
    tr = G.trace()
    olab, olv, oq, (orounds, omoves, onv) = oracle.louvain(off, cols, w)
    assert levels == olv
    assert [sum(1 for t in tr if t["level"] == l) for l in range(levels)] == orounds.tolist()
    assert [sum(t["moved"] for t in tr if t["level"] == l) for l in range(levels)] == omoves.tolist()
    np.testing.assert_array_equal(lab.cpu().numpy(), olab)
    assert abs(q - oq) <= 1e-12 * max(1.0, abs(oq))
    G.close()
