"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Labels, round counts and per-round traces must be bit-identical (integer
work); modularity is compared within 1e-12 relative (it is computed from the
same exact integers on both sides, so it is in fact equal). Graphs span every
degree bin of the scan (sub-warp tiles, warp and CTA shared-memory tables,
multi-CTA hub tables), weighted and unweighted inputs, loops, isolated
vertices and the degenerate sizes.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from tests import _textbook as tb

pytestmark = pytest.mark.gpu

cd = None


def setup_module(module):
    global cd
    import paper_2507_06471_gb300 as _cd
    cd = _cd
    assert torch.cuda.is_available()


def upload(g, device=True):
    if device:
        return cd.Graph(g.off.cuda(), g.cols.cuda(), None if g.w is None else g.w.cuda())
    w = None if g.w is None else g.w.numpy()
    return cd.Graph(g.off.numpy(), g.cols.numpy(), w)


def merged(n, *edge_arrays, wmax=1, seed=0):
    """Canonical CSR of the union of (u, v) edge arrays, optional weights."""
    u = torch.cat([torch.as_tensor(a, dtype=torch.int64) for a, _ in edge_arrays])
    v = torch.cat([torch.as_tensor(b, dtype=torch.int64) for _, b in edge_arrays])
    keys = synth.canonical_keys(u, v)
    w = synth.edge_weights(keys, seed, wmax) if wmax > 1 else None
    return synth.csr_from_edge_keys(keys, n, w)


def bins_graph(wmax=1):
    """A planted-partition base plus hubs of degree ~9000 (several build
    chunks and evaluate slices) and ~2500 (one of each), a vertex of degree
    ~700 (128 threads per vertex), warp-bin vertices (40..250) and isolated
    vertices."""
    rng = np.random.default_rng(5)
    n = 20000
    base = synth.sbm(n, 200, "0.03", "0.0002", seed=11)
    bu = np.repeat(np.arange(n), np.diff(base.off.numpy()))
    bv = base.cols.numpy().astype(np.int64)
    hub = (np.zeros(9000, np.int64), rng.choice(np.arange(1, 15000), 9000, replace=False))
    blk = (np.ones(700, np.int64), rng.choice(np.arange(3, 19000), 700, replace=False))
    blk2 = (np.full(2500, 2, np.int64), rng.choice(np.arange(3, 19000), 2500, replace=False))
    warp_u, warp_v = [], []
    for x in range(3, 60):
        k = int(rng.integers(40, 250))
        warp_u.append(np.full(k, x))
        warp_v.append(rng.choice(np.arange(60, 19000), k, replace=False))
    wu = (np.concatenate(warp_u), np.concatenate(warp_v))
    keep = (bu < 19500) & (bv < 19500)  # the last 500 vertices stay isolated
    return merged(n, (bu[keep], bv[keep]), hub, blk, blk2, wu, wmax=wmax, seed=3)


def loops_graph(seed):
    rng = np.random.default_rng(seed)
    n = 300
    edges, ws, lp, _ = tb.random_graph(rng, n, 0.03, wmax=5, loops=0.2)
    return synth.from_edge_list(n, edges, ws, lp)


GRAPHS = {
    "sbm10k": lambda: synth.sbm(10000, 100, "0.1", "0.001", seed=1),
    "sbm2k_w": lambda: synth.sbm(2000, 20, "0.1", "0.004", seed=7, wmax=4),
    "rmat12": lambda: synth.rmat(12, 16, seed=3),
    "rmat16": lambda: synth.rmat(16, 16, seed=3),
    "lfr50k_w": lambda: synth.lfr(50000, seed=2),
    "bins": lambda: bins_graph(),
    "bins_w": lambda: bins_graph(wmax=7),
    "loops_w": lambda: loops_graph(1),
}
_cache = {}


def graph(name):
    if name not in _cache:
        _cache[name] = GRAPHS[name]()
    return _cache[name]


def same_trace(gpu_trace, otr, level=0):
    rows = [t for t in gpu_trace if t["level"] == level]
    assert len(rows) == otr.rounds
    assert [t["moved"] for t in rows] == otr.moved.tolist()
    assert [t["deferred"] for t in rows] == otr.deferred.tolist()
    assert [t["active"] for t in rows] == otr.active.tolist()
    assert [t["arcs"] for t in rows] == otr.arcs.tolist()
    assert [t["cands"] for t in rows] == otr.cands.tolist()
    assert [t["moved_arcs"] for t in rows] == otr.moved_arcs.tolist()


@pytest.mark.parametrize("name", list(GRAPHS))
def test_lpa_parity(name):
    g = graph(name)
    off, cols, w = g.numpy()
    G = upload(g)
    lab, rounds = G.lpa()
    olab, otr = oracle.lpa(off, cols, w)
    assert rounds == otr.rounds
    np.testing.assert_array_equal(lab.cpu().numpy(), olab)
    same_trace(G.trace(), otr)


@pytest.mark.parametrize("name", list(GRAPHS))
def test_local_move_parity(name):
    g = graph(name)
    off, cols, w = g.numpy()
    G = upload(g)
    lab, moves, rounds = G.local_move()
    olab, omoves, otr = oracle.local_move(off, cols, w)
    assert (moves, rounds) == (omoves, otr.rounds)
    np.testing.assert_array_equal(lab.cpu().numpy(), olab)
    same_trace(G.trace(), otr)


@pytest.mark.parametrize("name", list(GRAPHS))
def test_louvain_parity(name):
    g = graph(name)
    off, cols, w = g.numpy()
    G = upload(g)
    lab, levels, q = G.louvain()
    olab, olv, oq, (orounds, omoves, onv) = oracle.louvain(off, cols, w)
    assert levels == olv
    np.testing.assert_array_equal(lab.cpu().numpy(), olab)
    assert abs(q - oq) <= 1e-12 * max(1.0, abs(oq))
    tr = G.trace()
    assert [sum(1 for t in tr if t["level"] == l) for l in range(levels)] == orounds.tolist()
    assert [sum(t["moved"] for t in tr if t["level"] == l) for l in range(levels)] == omoves.tolist()


def rows_sorted(off, cols, w):
    """(cols, w) with every row's entries sorted by column."""
    rows = np.repeat(np.arange(len(off) - 1), np.diff(off))
    order = np.lexsort((cols, rows))
    return np.asarray(cols)[order], np.asarray(w)[order]


@pytest.mark.parametrize("name", ["sbm2k_w", "rmat12", "bins_w", "loops_w", "lfr50k_w"])
def test_aggregate_parity(name):
    g = graph(name)
    off, cols, w = g.numpy()
    G = upload(g)
    rng = np.random.default_rng(9)
    olm, _, _ = oracle.local_move(off, cols, w, max_iter=3)
    for labels in [olm, rng.integers(0, g.n, g.n).astype(np.int32),
                   (np.arange(g.n) % 7).astype(np.int32)]:
        k, newid, coff, ccols, cw = oracle.aggregate(off, cols, w, labels)
        newid_gpu = torch.empty(g.n, dtype=torch.int32, device="cuda")
        C, kg = G.aggregate(torch.from_numpy(labels).cuda(), newid_gpu)
        assert kg == k
        np.testing.assert_array_equal(newid_gpu.cpu().numpy(), newid)
        goff, gcols, gw = C.download()
        np.testing.assert_array_equal(goff, coff)
        # columns come in no particular order inside a row: compare rows as sets
        gc, gwt = rows_sorted(goff, gcols, gw)
        oc, owt = rows_sorted(coff, ccols, cw)
        np.testing.assert_array_equal(gc, oc)
        np.testing.assert_array_equal(gwt, owt)
        # the coarse graph's modularity of singletons equals Q(G, C)
        qc = C.modularity(torch.arange(k, dtype=torch.int32, device="cuda"))
        qg = oracle.modularity(off, cols, w, labels)[0]
        assert abs(qc - qg) <= 1e-12 * max(1.0, abs(qg))
        C.close()


@pytest.mark.parametrize("name", ["sbm10k", "bins_w", "loops_w", "rmat16"])
def test_modularity_parity(name):
    g = graph(name)
    off, cols, w = g.numpy()
    G = upload(g)
    rng = np.random.default_rng(4)
    for labels in [np.arange(g.n), rng.integers(0, 50, g.n), np.zeros(g.n),
                   rng.integers(0, g.n, g.n)]:
        labels = labels.astype(np.int32)
        q = G.modularity(torch.from_numpy(labels).cuda())
        oq = oracle.modularity(off, cols, w, labels)[0]
        assert q == oq or abs(q - oq) <= 1e-12 * max(1.0, abs(oq))


@pytest.mark.parametrize("kw", [dict(tie_keep_current=0), dict(use_frontier=0), dict(threshold=25),
                                dict(sched_seed=12345), dict(max_iter=1), dict(max_iter=3)])
def test_lpa_parameters(kw):
    g = graph("bins_w")
    off, cols, w = g.numpy()
    G = upload(g)
    lab, rounds = G.lpa(**kw)
    okw = dict(kw)
    olab, otr = oracle.lpa(off, cols, w, **okw)
    assert rounds == otr.rounds
    np.testing.assert_array_equal(lab.cpu().numpy(), olab)


@pytest.mark.parametrize("kw", [dict(singleton_rule=0), dict(use_frontier=0), dict(sched_seed=99),
                                dict(max_iter=1), dict(max_iter=2)])
def test_local_move_parameters(kw):
    g = graph("bins")
    off, cols, w = g.numpy()
    G = upload(g)
    lab, moves, rounds = G.local_move(**kw)
    olab, omoves, otr = oracle.local_move(off, cols, w, **kw)
    assert (moves, rounds) == (omoves, otr.rounds)
    np.testing.assert_array_equal(lab.cpu().numpy(), olab)


def test_louvain_parameters():
    g = graph("sbm2k_w")
    off, cols, w = g.numpy()
    G = upload(g)
    for kw in [dict(max_levels=1), dict(max_levels=2, max_iter=5), dict(singleton_rule=0)]:
        lab, levels, q = G.louvain(**kw)
        olab, olv, oq, _ = oracle.louvain(off, cols, w, **kw)
        assert levels == olv
        np.testing.assert_array_equal(lab.cpu().numpy(), olab)


def test_local_move_from_given_partition():
    g = graph("sbm2k_w")
    off, cols, w = g.numpy()
    G = upload(g)
    start = (np.arange(g.n) // 3).astype(np.int32)
    lab, moves, rounds = G.local_move(labels=torch.from_numpy(start).cuda())
    olab, omoves, otr = oracle.local_move(off, cols, w, labels_in=start)
    assert (moves, rounds) == (omoves, otr.rounds)
    np.testing.assert_array_equal(lab.cpu().numpy(), olab)


def test_host_pointers_end_to_end():
    g = graph("sbm2k_w")
    off, cols, w = g.numpy()
    G = upload(g, device=False)
    out = np.zeros(g.n, dtype=np.int32)
    rounds = cd.cd_lpa_run(G.h, cd.cd_params_default(), out)
    olab, otr = oracle.lpa(off, cols, w)
    assert rounds == otr.rounds and np.array_equal(out, olab)
    levels, q = cd.cd_louvain_run(G.h, cd.cd_params_default(), out)
    olab, olv, oq, _ = oracle.louvain(off, cols, w)
    assert levels == olv and np.array_equal(out, olab)
    # int32 offsets are accepted too
    G32 = cd.Graph(g.off.numpy().astype(np.int32), g.cols.numpy(), g.w.numpy())
    lab, _ = G32.lpa()
    assert np.array_equal(lab.cpu().numpy(), oracle.lpa(off, cols, w)[0])


def test_repeated_runs_are_identical():
    g = graph("bins_w")
    G = upload(g)
    a = G.louvain()[0].cpu().numpy()
    b = G.louvain()[0].cpu().numpy()
    c = G.lpa()[0].cpu().numpy()
    d = G.lpa()[0].cpu().numpy()
    assert np.array_equal(a, b) and np.array_equal(c, d)


@pytest.mark.parametrize("n", [0, 1, 7])
def test_degenerate_sizes(n):
    g = synth.from_edge_list(n, [])
    off, cols, w = g.numpy()
    G = cd.Graph(g.off.cuda(), g.cols.cuda())
    lab, rounds = G.lpa()
    olab, otr = oracle.lpa(off, cols, w)
    assert rounds == otr.rounds and lab.cpu().numpy().tolist() == olab.tolist()
    lab, levels, q = G.louvain()
    olab, olv, oq, _ = oracle.louvain(off, cols, w)
    assert levels == olv and q == oq == 0.0 and lab.cpu().numpy().tolist() == olab.tolist()


def test_loops_only_and_pairs():
    # a vertex with only a loop, a pair of singletons (swap case), a triangle
    g = synth.from_edge_list(6, [(1, 2), (3, 4), (4, 5), (3, 5)], [1, 1, 1, 1], {0: 3, 3: 2})
    off, cols, w = g.numpy()
    G = upload(g)
    lab, levels, q = G.louvain()
    olab, olv, oq, _ = oracle.louvain(off, cols, w)
    assert np.array_equal(lab.cpu().numpy(), olab) and abs(q - oq) < 1e-12
    lab, rounds = G.lpa()
    assert np.array_equal(lab.cpu().numpy(), oracle.lpa(off, cols, w)[0])


def test_input_errors_are_reported():
    off = torch.tensor([0, 2, 3, 4], dtype=torch.int64, device="cuda")
    cols = torch.tensor([1, 2, 0, 0], dtype=torch.int32, device="cuda")
    bad_cols = torch.tensor([1, 7, 0, 0], dtype=torch.int32, device="cuda")
    with pytest.raises(cd.CDError) as e:
        cd.Graph(off, bad_cols)
    assert e.value.status == cd.CD_EBOUNDS
    with pytest.raises(cd.CDError) as e:
        cd.Graph(off, cols, torch.tensor([1, 0, 1, 1], dtype=torch.int32, device="cuda"))
    assert e.value.status == cd.CD_EINVAL
    with pytest.raises(cd.CDError) as e:
        cd.Graph(torch.tensor([0, 3, 2, 4], dtype=torch.int64, device="cuda"), cols)
    assert e.value.status == cd.CD_ENOTSYM
    G = cd.Graph(off, cols)
    with pytest.raises(cd.CDError) as e:
        G.modularity(torch.tensor([0, 1, 5], dtype=torch.int32, device="cuda"))
    assert e.value.status == cd.CD_EINVAL
    # the handle and the context still work after the errors
    lab, _ = G.lpa()
    assert lab.shape == (3,)


def test_device_generator_matches_host():
    kh = synth.rmat_keys_host(10, 8, "0.57", "0.19", "0.19", seed=3)
    kd = synth.rmat_keys_device(10, 8, "0.57", "0.19", "0.19", seed=3).cpu().numpy()
    np.testing.assert_array_equal(kh, kd)
    gh = synth.rmat(11, 16, seed=5)
    gd = synth.rmat(11, 16, seed=5, device="cuda")
    assert torch.equal(gh.off, gd.off.cpu()) and torch.equal(gh.cols, gd.cols.cpu())


def test_wide_hub_histograms():
    # A hub whose weighted degree exceeds 2^32 makes the library keep hub
    # histograms in two-word slots (label, count); results must not change.
    rng = np.random.default_rng(12)
    n = 4000
    base = synth.sbm(n, 40, "0.05", "0.001", seed=13)
    bu = np.repeat(np.arange(n), np.diff(base.off.numpy()))
    bv = base.cols.numpy().astype(np.int64)
    keep = bu < bv
    edges = list(zip(bu[keep].tolist(), bv[keep].tolist()))
    ws = rng.integers(1, 5, len(edges)).tolist()
    leaves = rng.choice(np.arange(1, n), 1500, replace=False)
    have = set(edges)
    for x in leaves.tolist():
        if (0, x) not in have:
            edges.append((0, x))
            ws.append(int(rng.integers(2**30, 2**31 - 1)))
    g = synth.from_edge_list(n, edges, ws)
    off, cols, w = g.numpy()
    d, vol = oracle.degw(off, cols, w)
    assert d.max() >= 2**32
    G = upload(g)
    lab, rounds = G.lpa()
    olab, otr = oracle.lpa(off, cols, w)
    assert rounds == otr.rounds and np.array_equal(lab.cpu().numpy(), olab)
    lab, levels, q = G.louvain()
    olab, olv, oq, _ = oracle.louvain(off, cols, w)
    assert levels == olv and np.array_equal(lab.cpu().numpy(), olab)
    assert abs(q - oq) <= 1e-12 * max(1.0, abs(oq))


@pytest.mark.parametrize("bins", [(32, 32), (64, 256), (128, 512), (256, 1024), (256, 2048), (64, 4096)])
def test_bins_do_not_change_results(bins):
    # degree bins (and the hub threshold) only change how vertices are scanned
    g = graph("bins_w")
    off, cols, w = g.numpy()
    G = upload(g)
    cd.cd_graph_set_bins(G.h, *bins)
    lab, rounds = G.lpa()
    olab, otr = oracle.lpa(off, cols, w)
    assert rounds == otr.rounds and np.array_equal(lab.cpu().numpy(), olab)
    lab, levels, q = G.louvain()
    olab, olv, oq, _ = oracle.louvain(off, cols, w)
    assert levels == olv and np.array_equal(lab.cpu().numpy(), olab)


def test_hub_tables_shrink_and_keep_results():
    # a low hub threshold makes hubs of many vertices whose neighbourhoods end in
    # few communities, so their tables are compacted below their allocation
    # (the preparation then reads and writes slots); every trace field still
    # equals the oracle's
    g = graph("rmat16")
    off, cols, w = g.numpy()
    nh = int((np.diff(off) > 64).sum())
    G = upload(g)
    cd.cd_graph_set_bins(G.h, 32, 64)
    compacted = 0.0
    lab, rounds = G.lpa(timing=1)
    olab, otr = oracle.lpa(off, cols, w)
    assert rounds == otr.rounds and np.array_equal(lab.cpu().numpy(), olab)
    same_trace(G.trace(), otr)
    p = {x["name"]: x for x in G.profile()}["hub_prepare"]
    compacted += p["alg_bytes"] - 8.0 * nh * p["launches"]
    lab, moves, rounds = G.local_move(timing=1)
    olab, omoves, otr = oracle.local_move(off, cols, w)
    assert (moves, rounds) == (omoves, otr.rounds)
    np.testing.assert_array_equal(lab.cpu().numpy(), olab)
    same_trace(G.trace(), otr)
    p = {x["name"]: x for x in G.profile()}["hub_prepare"]
    compacted += p["alg_bytes"] - 8.0 * nh * p["launches"]
    assert compacted > 0  # slots were compacted (no hub here is large enough for a cleared global build)


def test_autotune_keeps_results():
    g = graph("rmat16")
    off, cols, w = g.numpy()
    G = upload(g)
    tw, th = cd.cd_autotune(G.h, cd.cd_params_default(), 2)
    assert tw in (64, 128, 256) and th in (512, 1024, 2048, 4096) and th >= tw
    lab, levels, q = G.louvain()
    olab, olv, oq, _ = oracle.louvain(off, cols, w)
    assert levels == olv and np.array_equal(lab.cpu().numpy(), olab)


@pytest.mark.parametrize("name", ["lfr50k_w", "rmat16", "bins_w", "sbm10k"])
def test_aggregation_modes_agree(name):
    # hash-combining per community and the radix sort of all arcs build
    # coarse graphs with the same rows, so Louvain ends identically
    g = graph(name)
    G = upload(g)
    a = G.louvain(aggregation=0)
    b = G.louvain(aggregation=1)
    np.testing.assert_array_equal(a[0].cpu().numpy(), b[0].cpu().numpy())
    assert a[1] == b[1] and a[2] == b[2]


def test_aggregate_segment_classes():
    # one community holding every arc (chunked, global table), a few medium
    # ones, many small ones, and empty rows
    g = graph("lfr50k_w")
    off, cols, w = g.numpy()
    G = upload(g)
    deg = np.diff(off)
    big = np.zeros(g.n, dtype=np.int32)
    medium = (np.cumsum(deg) // 3000).astype(np.int32)
    mixed = np.where(np.arange(g.n) < g.n // 2, 0, np.arange(g.n)).astype(np.int32)
    for labels in [big, medium, mixed]:
        k, newid, coff, ccols, cw = oracle.aggregate(off, cols, w, labels)
        C, kg = G.aggregate(torch.from_numpy(labels).cuda())
        goff, gcols, gw = C.download()
        assert kg == k
        np.testing.assert_array_equal(goff, coff)
        gc, gwt = rows_sorted(goff, gcols, gw)
        oc, owt = rows_sorted(coff, ccols, cw)
        np.testing.assert_array_equal(gc, oc)
        np.testing.assert_array_equal(gwt, owt)
        C.close()


@pytest.mark.parametrize("target", [2**31 - 4096, 2**31 + 4096])
def test_key_width_boundary(target):
    # Louvain keys are 64-bit when vol(V) < 2^31 and 128-bit otherwise; a graph
    # on either side of the boundary must give the oracle's result
    rng = np.random.default_rng(21)
    base = synth.sbm(3000, 30, "0.05", "0.002", seed=22)
    bu = np.repeat(np.arange(base.n), np.diff(base.off.numpy()))
    bv = base.cols.numpy().astype(np.int64)
    keep = bu < bv
    edges = list(zip(bu[keep].tolist(), bv[keep].tolist()))
    m = len(edges)
    half = target // 2  # vol = 2 * sum of edge weights
    ws = np.full(m, half // m, dtype=np.int64)
    ws[:half % m] += 1
    idx = rng.permutation(m)
    a, b = idx[: m // 2], idx[m // 2: 2 * (m // 2)]
    delta = rng.integers(0, ws[a] - 1)
    ws[a] -= delta
    ws[b] += delta
    assert ws.min() >= 1 and int(ws.sum()) == half
    g = synth.from_edge_list(base.n, edges, ws.tolist())
    off, cols, w = g.numpy()
    vol = oracle.degw(off, cols, w)[1]
    assert (vol < 2**31) == (target < 2**31)
    G = upload(g)
    lab, levels, q = G.louvain()
    olab, olv, oq, _ = oracle.louvain(off, cols, w)
    assert levels == olv and np.array_equal(lab.cpu().numpy(), olab)
    assert abs(q - oq) <= 1e-12 * max(1.0, abs(oq))


@pytest.mark.parametrize("name", ["sbm10k", "rmat16", "bins_w", "lfr50k_w", "loops_w"])
def test_device_loop_equals_host_loop(name):
    """Rounds after the first run as one captured graph with a device-side
    loop (device_loop = 2) or one host read-back per round (device_loop = 0):
    labels, round counts and every trace field agree."""
    g = graph(name)
    G = upload(g)
    keys = ("level", "round", "active", "arcs", "moved", "deferred", "cands", "moved_arcs")

    def runs(dl):
        lab1, r1 = G.lpa(device_loop=dl)
        t1 = [{k: t[k] for k in keys} for t in G.trace()]
        lab2, lv, q = G.louvain(device_loop=dl)
        t2 = [{k: t[k] for k in keys} for t in G.trace()]
        return lab1.cpu().numpy(), r1, t1, lab2.cpu().numpy(), lv, q, t2

    a, b = runs(2), runs(0)
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[3], b[3])
    assert a[1] == b[1] and a[2] == b[2] and a[4] == b[4] and a[5] == b[5] and a[6] == b[6]


def test_device_loop_batched_rounds_per_graph():
    graphs = [synth.sbm(n, k, "0.2", "0.002", seed=90 + i, wmax=3)
              for i, (n, k) in enumerate([(300, 5), (1200, 12), (80, 2), (2000, 30), (50, 3)])]
    packed, vstart = synth.pack_batch(graphs)
    G = cd.Graph(packed.off.cuda(), packed.cols.cuda(), packed.w.cuda())
    G.set_batches(vstart)
    out = []
    for dl in (1, 0):
        lab, rounds = G.batch_lpa(device_loop=dl, threshold=3)
        lab2, levels, q = G.batch_louvain(device_loop=dl)
        out.append((lab.cpu().numpy(), list(rounds), lab2.cpu().numpy(), list(levels), list(q)))
    np.testing.assert_array_equal(out[0][0], out[1][0])
    np.testing.assert_array_equal(out[0][2], out[1][2])
    assert out[0][1] == out[1][1] and out[0][3] == out[1][3] and out[0][4] == out[1][4]
