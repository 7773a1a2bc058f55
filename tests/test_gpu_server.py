"""Serving engine: requests admitted continuously (several worker streams,
memory-budgeted admission, small requests packed into one batched call) must
each get exactly what a solo run of their graph gives, checked against the
CPU oracle: labels, round or level counts, modularity. Also: a request alone
equals the same request inside a mix, a bad request fails alone, and the
memory budget is honoured."""
import threading
import time

import numpy as np
import pytest

import oracle
import synth
from tests import _textbook as tb

pytestmark = pytest.mark.gpu


def _requests(count=48, seed=7):
    """(kind, synth.Graph) pairs: mostly small SBM graphs, some mid-size LFR
    and R-MAT graphs, edge cases (edgeless, one vertex, loops and weights, a
    hub), both algorithms interleaved."""
    import paper_2507_06471_gb300 as cd
    rng = np.random.default_rng(seed)
    graphs = []
    for i in range(count):
        n = int(np.exp(rng.uniform(np.log(20), np.log(1500))))
        graphs.append(synth.sbm(n, int(rng.integers(2, 9)), "0.2", "0.002", seed=300 + i, wmax=3))
    graphs.append(synth.lfr(20_000, dmax=300, seed=5))
    graphs.append(synth.rmat(13, 8, seed=9))
    graphs.append(synth.from_edge_list(7, []))
    graphs.append(synth.from_edge_list(1, []))
    edges, ws, lp, g = tb.random_graph(rng, 80, 0.07, wmax=3, loops=0.2)
    graphs.append(g)
    star = [(0, x) for x in range(1, 2001)] + [(x, x + 1) for x in range(1, 2000, 2)]
    graphs.append(synth.from_edge_list(2001, star))
    order = rng.permutation(len(graphs))
    return [(cd.CD_REQ_LPA if j % 2 else cd.CD_REQ_LOUVAIN, graphs[o]) for j, o in enumerate(order)]


def _host(g):
    off, cols, w = g.numpy()
    return off, cols, None if w is None else w.astype(np.int32)


def _expect(kind, g):
    import paper_2507_06471_gb300 as cd
    off, cols, w = g.numpy()
    if kind == cd.CD_REQ_LPA:
        lab, tr = oracle.lpa(off, cols, w)
        return lab, tr.rounds, 0.0
    lab, lv, q, _ = oracle.louvain(off, cols, w)
    return lab, lv, q


@pytest.fixture(scope="module")
def reqs():
    rs = _requests()
    return rs, [_expect(k, g) for k, g in rs]


def _check(res, labels, exp):
    lab, iters, q = exp
    assert res.status == 0
    np.testing.assert_array_equal(labels, lab)
    assert res.iters == iters
    assert abs(res.q - q) <= 1e-12 * max(1.0, abs(q))


@pytest.mark.parametrize("slots,small_n", [(1, 0), (4, 4096), (8, 1 << 20)])
def test_server_matches_oracle(reqs, slots, small_n):
    import paper_2507_06471_gb300 as cd
    rs, exp = reqs
    srv = cd.Server(slots=slots, small_n=small_n, batch_arcs=1 << 20)
    ids = [srv.submit(k, *_host(g)) for k, g in rs]
    for rid, e in zip(ids, exp):
        labels, res = srv.result(rid)
        _check(res, labels, e)
        assert res.latency_ms >= res.queue_ms >= 0.0
    st = srv.stats()
    assert st["admitted"] == st["completed"] == len(rs) and st["in_use"] == 0
    if small_n == 0:
        assert st["packed_calls"] == 0
    srv.close()


def test_server_arrivals_while_running(reqs):
    # requests arrive from another thread over time; results are collected as
    # they come, in any order
    import paper_2507_06471_gb300 as cd
    rs, exp = reqs
    srv = cd.Server(slots=4, small_n=4096, batch_arcs=1 << 18)
    ids = [None] * len(rs)

    def feed():
        for i, (k, g) in enumerate(rs):
            ids[i] = srv.submit(k, *_host(g))
            time.sleep(0.002)

    t = threading.Thread(target=feed)
    t.start()
    t.join()
    for i in reversed(range(len(rs))):
        labels, res = srv.result(ids[i])
        _check(res, labels, exp[i])
    srv.close()


def test_alone_equals_in_mix(reqs):
    import paper_2507_06471_gb300 as cd
    rs, exp = reqs
    pick = [i for i, (k, g) in enumerate(rs) if g.n > 100][:3]
    srv = cd.Server(slots=2, small_n=4096)
    alone = []
    for i in pick:
        k, g = rs[i]
        labels, res = srv.result(srv.submit(k, *_host(g)))
        assert res.batched_with == 1
        alone.append((labels, res.iters, res.q))
    ids = [srv.submit(k, *_host(g)) for k, g in rs]
    for j, i in enumerate(pick):
        labels, res = srv.result(ids[i])
        np.testing.assert_array_equal(labels, alone[j][0])
        assert res.iters == alone[j][1] and res.q == alone[j][2]
    for i, rid in enumerate(ids):
        if i not in pick:
            srv.result(rid)
    assert srv.stats()["packed_calls"] >= 1
    srv.close()


def test_bad_request_fails_alone():
    import paper_2507_06471_gb300 as cd
    good = synth.sbm(300, 4, "0.2", "0.002", seed=1)
    bad_off = np.array([0, 1, 2], dtype=np.int64)
    bad_cols = np.array([1, 5], dtype=np.int32)  # column 5 outside [0, 2)
    srv = cd.Server(slots=2, small_n=4096)
    a = srv.submit(cd.CD_REQ_LOUVAIN, *_host(good))
    b = srv.submit(cd.CD_REQ_LOUVAIN, bad_off, bad_cols)
    c = srv.submit(cd.CD_REQ_LPA, *_host(good))
    labels, res = srv.result(a)
    _check(res, labels, _expect(cd.CD_REQ_LOUVAIN, good))
    with pytest.raises(cd.CDError) as e:
        srv.result(b)
    assert e.value.status == cd.CD_EBOUNDS
    labels, res = srv.result(c)
    _check(res, labels, _expect(cd.CD_REQ_LPA, good))
    srv.close()


def test_memory_budget(reqs):
    import paper_2507_06471_gb300 as cd
    rs, exp = reqs
    biggest = max(64 * g.nnz + 96 * g.n + (16 << 20) for k, g in rs)
    srv = cd.Server(slots=8, mem_budget_bytes=biggest, small_n=4096)
    big = synth.rmat(16, 16, seed=2)
    with pytest.raises(cd.CDError) as e:  # can never fit
        srv.submit(cd.CD_REQ_LPA, *_host(big))
    assert e.value.status == cd.CD_ENOMEM
    ids = [srv.submit(k, *_host(g)) for k, g in rs]
    peak = 0
    done = threading.Event()

    def watch():
        nonlocal peak
        while not done.is_set():
            peak = max(peak, srv.stats()["in_use"])
            time.sleep(0.0005)

    t = threading.Thread(target=watch)
    t.start()
    for rid, e in zip(ids, exp):
        labels, res = srv.result(rid)
        _check(res, labels, e)
    done.set()
    t.join()
    assert peak <= biggest  # (the watcher may miss short admissions; it must never see more)
    st = srv.stats()
    assert st["admitted"] == st["completed"] == len(rs) and st["in_use"] == 0
    srv.close()


def test_wait_timeout_and_unknown_id():
    import paper_2507_06471_gb300 as cd
    srv = cd.Server(slots=1)
    g = synth.sbm(200, 2, "0.2", "0.01", seed=3)
    rid = srv.submit(cd.CD_REQ_LPA, *_host(g))
    try:
        labels, res = srv.result(rid, timeout_ms=0)  # may or may not be done yet
    except cd.CDError as e:
        assert e.status == cd.CD_ETIMEOUT
        labels, res = srv.result(rid)
    _check(res, labels, _expect(cd.CD_REQ_LPA, g))
    with pytest.raises(cd.CDError) as e:
        cd.cd_server_wait(srv.h, 12345, 1, 0)
    assert e.value.status == cd.CD_EINVAL
    srv.close()


def test_destroy_drains_queue():
    import paper_2507_06471_gb300 as cd
    srv = cd.Server(slots=2)
    gs = [synth.sbm(400, 3, "0.2", "0.002", seed=40 + i) for i in range(6)]
    for g in gs:
        srv.submit(cd.CD_REQ_LOUVAIN, *_host(g))
    cd.cd_server_destroy(srv.h)  # returns after every queued request ran
    srv.h = None


def test_served_generators_device_equals_host():
    for n, k, sd in [(5000, 7, 1), (777, 2, 2), (100, 50, 3)]:
        h = synth.sbm_sparse(n, k, 16, seed=sd)
        d = synth.sbm_sparse(n, k, 16, seed=sd, device="cuda").to("cpu")
        assert torch_equal(h, d)
    for n, sd in [(3000, 4), (4096, 5), (100, 6)]:
        assert torch_equal(synth.rmat_n(n, 8, seed=sd), synth.rmat_n(n, 8, seed=sd, device="cuda").to("cpu"))


def torch_equal(a, b):
    import torch
    return a.n == b.n and torch.equal(a.off, b.off) and torch.equal(a.cols, b.cols) and (a.w is None) == (b.w is None)


def test_served_mix_matches_oracle():
    # the served recipe with sizes capped so the oracle stays quick
    import paper_2507_06471_gb300 as cd
    specs = synth.serve_specs(40, seed=9, nmax=30_000)
    srv = cd.Server(slots=4, small_n=8192, batch_arcs=1 << 20)
    items = []
    for sp in specs:
        g = synth.serve_graph(sp, "cuda").to("cpu")
        kind = cd.CD_REQ_LOUVAIN if sp[0] == "louvain" else cd.CD_REQ_LPA
        items.append((srv.submit(kind, *_host(g)), kind, g))
    for rid, kind, g in items:
        labels, res = srv.result(rid)
        _check(res, labels, _expect(kind, g))
    srv.close()
