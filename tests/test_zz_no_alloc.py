"""The allocation-free modularity entry point (cd_modularity_noalloc).

Some callers cannot call cudaMalloc — for instance a process whose device
memory is entirely owned by another allocator with a fixed budget. This entry
point keeps its scratch in a static device array inside the library instead.
Its results must match the regular entry point (cd_csr_upload +
cd_modularity) and the oracle within the tolerance the parity tests use
(1e-12 relative), on two calls in a row (the shared scratch keeps the previous
call's contents), and the calls must neither change the device's free memory
nor make the PyTorch allocator allocate. This file is collected
last so that a failure here does not hide the other tests.
"""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

MAX_N = 1 << 21


def _loopy_weighted_graph():
    base = synth.sbm(3000, 30, "0.08", "0.003", seed=21, wmax=5)
    off = base.off.numpy()
    rng = np.random.default_rng(2)
    edges = [(u, int(v)) for u in range(base.n) for v in base.cols.numpy()[off[u]:off[u + 1]] if u < v]
    ws = rng.integers(1, 6, len(edges)).tolist()
    loops = {int(v): int(rng.integers(1, 4)) for v in rng.choice(base.n, 40, replace=False)}
    return synth.from_edge_list(base.n, edges, ws, loops)


@pytest.mark.parametrize("which", ["weighted_loops", "rmat_unit"])
def test_noalloc_matches_regular_entry_point(which):
    import paper_2507_06471_gb300 as cd
    g = _loopy_weighted_graph() if which == "weighted_loops" else synth.rmat(14, 16, seed=8)
    off, cols = g.off.cuda(), g.cols.cuda()
    w = None if g.w is None else g.w.cuda()
    G = cd.Graph(off, cols, w)
    rng = np.random.default_rng(5)
    lab_lv, _, _ = G.louvain()
    cases = [lab_lv, torch.from_numpy(rng.integers(0, 40, g.n).astype(np.int32)).cuda(),
             torch.arange(g.n, dtype=torch.int32, device="cuda")]
    refs = [G.modularity(lab) for lab in cases]
    hoff, hcols, hw = g.numpy()
    orefs = [oracle.modularity(hoff, hcols, hw, lab.cpu().numpy())[0] for lab in cases]
    torch.cuda.synchronize()
    cd.cd_modularity_noalloc(off, cols, w, cases[0])  # first call on the device does the set-up
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    stats_before = _alloc_counts()
    for _ in range(2):  # two calls in a row over every case
        for lab, ref, oref in zip(cases, refs, orefs):
            q = cd.cd_modularity_noalloc(off, cols, w, lab)
            assert abs(q - ref) <= 1e-12 * max(1.0, abs(ref)), (q, ref)
            assert abs(q - oref) <= 1e-12 * max(1.0, abs(oref)), (q, oref)
    assert _alloc_counts() == stats_before
    assert torch.cuda.mem_get_info()[0] == free_before
    G.close()


def _alloc_counts():
    st = torch.cuda.memory_stats()
    return (st.get("allocation.all.allocated", 0), st.get("segment.all.allocated", 0))


def test_noalloc_unweighted_after_weighted_allocates_nothing():
    """The first call (here a weighted one) loads every kernel of the entry
    point, so a later call of the other weight kind loads and allocates nothing."""
    import paper_2507_06471_gb300 as cd
    gw = _loopy_weighted_graph()
    gu = synth.rmat(12, 8, seed=4)
    offw, colsw, ww = gw.off.cuda(), gw.cols.cuda(), gw.w.cuda()
    offu, colsu = gu.off.cuda(), gu.cols.cuda()
    labw = torch.zeros(gw.n, dtype=torch.int32, device="cuda")
    labu = torch.arange(gu.n, dtype=torch.int32, device="cuda")
    cd.cd_modularity_noalloc(offw, colsw, ww, labw)
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    stats_before = _alloc_counts()
    q = cd.cd_modularity_noalloc(offu, colsu, None, labu)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free_before
    assert _alloc_counts() == stats_before
    hoff, hcols, _ = gu.numpy()
    oq = oracle.modularity(hoff, hcols, None, labu.cpu().numpy())[0]
    assert abs(q - oq) <= 1e-12 * max(1.0, abs(oq))


def test_noalloc_rejects_sizes_beyond_the_scratch():
    import paper_2507_06471_gb300 as cd
    off = torch.zeros(2, dtype=torch.int64, device="cuda")
    cols = torch.zeros(0, dtype=torch.int32, device="cuda")
    lab = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(cd.CDError) as e:
        cd.cd_modularity_noalloc(off, cols, None, lab, n=MAX_N + 1)
    assert e.value.status == cd.CD_EINVAL
    # a bad label is reported, not followed, and the next call still works
    off2 = torch.tensor([0, 1, 2], dtype=torch.int64, device="cuda")
    cols2 = torch.tensor([1, 0], dtype=torch.int32, device="cuda")
    with pytest.raises(cd.CDError) as e:
        cd.cd_modularity_noalloc(off2, cols2, None, torch.tensor([0, 9], dtype=torch.int32, device="cuda"))
    assert e.value.status == cd.CD_EINVAL
    q = cd.cd_modularity_noalloc(off2, cols2, None, torch.tensor([0, 0], dtype=torch.int32, device="cuda"))
    assert q == 0.0
