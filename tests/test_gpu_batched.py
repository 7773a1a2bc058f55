"""Batched mode: many graphs packed block-diagonally and solved together must
give every graph exactly what a solo run gives (checked against the CPU
oracle run on each graph alone): labels, round and level counts, and the
graph's own modularity."""
import numpy as np
import pytest
import torch

import oracle
import synth
from tests import _textbook as tb

pytestmark = pytest.mark.gpu


def _batch_graphs(count=40, seed=0):
    rng = np.random.default_rng(seed)
    graphs = []
    for i in range(count):
        n = int(np.exp(rng.uniform(np.log(20), np.log(600))))
        k = int(rng.integers(2, 11))
        graphs.append(synth.sbm(n, k, "0.2", "0.002", seed=100 + i, wmax=4))
    graphs.append(synth.from_edge_list(5, []))            # edgeless
    graphs.append(synth.from_edge_list(1, []))            # one vertex
    edges, ws, lp, g = tb.random_graph(rng, 60, 0.08, wmax=3, loops=0.2)
    graphs.append(g)                                      # loops and weights
    star = [(0, x) for x in range(1, 1301)] + [(x, x + 1) for x in range(1, 1300, 2)]
    graphs.append(synth.from_edge_list(1301, star, [1 + (x % 3) for x in range(len(star))]))  # a hub
    order = rng.permutation(len(graphs))
    return [graphs[j] for j in order]


@pytest.fixture(scope="module")
def batch():
    import paper_2507_06471_gb300 as cd
    graphs = _batch_graphs()
    packed, vstart = synth.pack_batch(graphs)
    G = cd.Graph(packed.off.cuda(), packed.cols.cuda(), None if packed.w is None else packed.w.cuda())
    G.set_batches(vstart)
    return cd, graphs, vstart, G


def test_batched_lpa_equals_solo(batch):
    cd, graphs, vstart, G = batch
    lab, rounds = G.batch_lpa()
    lab = lab.cpu().numpy()
    for b, g in enumerate(graphs):
        off, cols, w = g.numpy()
        olab, otr = oracle.lpa(off, cols, w)
        assert rounds[b] == otr.rounds, b
        np.testing.assert_array_equal(lab[vstart[b]:vstart[b + 1]], olab)


@pytest.mark.parametrize("threshold", [3, 40])
def test_batched_lpa_threshold_per_graph(batch, threshold):
    cd, graphs, vstart, G = batch
    lab, rounds = G.batch_lpa(threshold=threshold)
    lab = lab.cpu().numpy()
    for b, g in enumerate(graphs):
        off, cols, w = g.numpy()
        olab, otr = oracle.lpa(off, cols, w, threshold=threshold)
        assert rounds[b] == otr.rounds, b
        np.testing.assert_array_equal(lab[vstart[b]:vstart[b + 1]], olab)


def test_batched_louvain_equals_solo(batch):
    cd, graphs, vstart, G = batch
    lab, levels, q = G.batch_louvain()
    lab = lab.cpu().numpy()
    for b, g in enumerate(graphs):
        off, cols, w = g.numpy()
        olab, olv, oq, _ = oracle.louvain(off, cols, w)
        assert levels[b] == olv, b
        np.testing.assert_array_equal(lab[vstart[b]:vstart[b + 1]], olab)
        assert abs(q[b] - oq) <= 1e-12 * max(1.0, abs(oq)), b


@pytest.mark.parametrize("kw", [dict(max_levels=1), dict(max_levels=2, max_iter=4), dict(max_levels=0)])
def test_batched_louvain_limits(batch, kw):
    cd, graphs, vstart, G = batch
    lab, levels, q = G.batch_louvain(**kw)
    lab = lab.cpu().numpy()
    for b, g in enumerate(graphs):
        off, cols, w = g.numpy()
        olab, olv, oq, _ = oracle.louvain(off, cols, w, **kw)
        assert levels[b] == olv, b
        np.testing.assert_array_equal(lab[vstart[b]:vstart[b + 1]], olab)


def test_batched_equals_solo_gpu(batch):
    # the same graphs, each uploaded and solved alone through the C ABI
    cd, graphs, vstart, G = batch
    lab, levels, q = G.batch_louvain()
    lab = lab.cpu().numpy()
    for b in range(0, len(graphs), 7):
        g = graphs[b]
        H = cd.Graph(g.off.cuda(), g.cols.cuda(), None if g.w is None else g.w.cuda())
        sl, slv, sq = H.louvain()
        assert slv == levels[b] and abs(sq - q[b]) <= 1e-12 * max(1.0, abs(sq))
        np.testing.assert_array_equal(sl.cpu().numpy(), lab[vstart[b]:vstart[b + 1]])


def test_batches_must_not_share_arcs():
    import paper_2507_06471_gb300 as cd
    g = synth.from_edge_list(6, [(0, 1), (2, 3), (3, 4)])
    G = cd.Graph(g.off.cuda(), g.cols.cuda())
    with pytest.raises(cd.CDError) as e:
        G.set_batches(np.array([0, 3, 6], dtype=np.int64))  # arc 2-3 crosses
    assert e.value.status == cd.CD_EINVAL
    G.set_batches(np.array([0, 2, 5, 6], dtype=np.int64))
    lab, levels, q = G.batch_louvain()
    assert lab.shape == (6,)


def test_device_batch_generator_matches_host_sbm():
    specs = [(300, 5, 11), (57, 2, 12), (1000, 40, 13), (2, 2, 14)]
    packed, vstart, planted = synth.sbm_batch_device(specs)
    members = synth.unpack_batch(packed.to("cpu"), vstart)
    for (n, k, sd), m in zip(specs, members):
        h = synth.sbm(n, k, "0.2", "0.002", seed=sd, wmax=4)
        assert torch.equal(m.off, h.off) and torch.equal(m.cols, h.cols) and torch.equal(m.w, h.w)
    assert np.array_equal(planted[vstart[0]:vstart[1]], synth.sbm(300, 5, "0.2", "0.002", seed=11).planted)
