"""Global consolidation (Sec. 5.2) on a snapshot, merged back with the rows and
reverse edges of the inserts made meanwhile (Sec. 5.3), against the oracle."""
import numpy as np
import pytest

import synth
from tests import _parity as P

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def svf():
    import paper_2601_08528_b300 as svf
    svf.load()
    return svf


def gpu_graph(ix, n):
    return P.as_u32(ix.graph[:n].cpu().numpy()).astype(np.uint32)


def ids_t(a):
    return torch.from_numpy(np.asarray(a, dtype=np.int32)).cuda()


def test_consolidation_u8_bit_exact_across_a_version_window(svf, orc):
    n0, m, R, L_ins, T_ins = 4000, 200, 32, 64, 32
    X = synth.sample("u8", n0 + 2 * m, 801)
    st = orc.Store.from_vectors(X, "l2")
    g0, _ = orc.build_graph(orc.Store.from_vectors(X[:n0], "l2"), R)
    ix = svf.Index(128, n0 + 2 * m, dtype="u8", metric="l2", R=R, max_batch=1000)
    ix.attach(torch.from_numpy(X[:n0]).cuda(), torch.from_numpy(g0.view(np.int32)))
    seed = ix.params.seed
    g = np.full((n0 + 2 * m, R), orc.EMPTY, dtype=np.uint32)
    g[:n0] = g0
    bits = orc.bitset(n0 + 2 * m)
    # 20 % deletes with the localized repair, on both sides
    rng = np.random.default_rng(802)
    dele = rng.choice(n0, n0 // 5, replace=False)
    ix.delete(ids_t(dele))
    orc.delete(st, n0, g, bits, dele)
    np.testing.assert_array_equal(gpu_graph(ix, n0), g[:n0])
    # snapshot
    ix.consolidate_begin(log_rows=1000)
    snap, snap_bits = g[:n0].copy(), bits.copy()
    # an insert batch and a delete on the active graph, then the run, then another insert
    ix.insert(torch.from_numpy(X[n0:n0 + m]).cuda(), L_ins=L_ins, T_ins=T_ins)
    orc.insert(st, n0, m, g, bits, L_ins, T_ins, seed)
    rows_b = g[n0:n0 + m].copy()
    live = np.setdiff1d(np.arange(n0 + m), dele)
    dele2 = rng.choice(live, 50, replace=False)
    ix.delete(ids_t(dele2))
    orc.delete(st, n0 + m, g, bits, dele2)
    nrows = ix.consolidate_run(cap=512)
    ix.insert(torch.from_numpy(X[n0 + m:]).cuda(), L_ins=L_ins, T_ins=T_ins)
    orc.insert(st, n0 + m, m, g, bits, L_ins, T_ins, seed)
    rows_c = g[n0 + m:].copy()
    ix.consolidate_commit()
    # oracle merge: consolidated snapshot rows, the rows inserted since, and
    # the logged reverse edges replayed onto the snapshot's targets
    cons = snap.copy()
    nrep, _ = orc.consolidate(st, n0, cons, snap_bits)
    merged = g.copy()
    merged[:n0] = cons
    orc.reverse_patch(st, merged, bits, n0, rows_b, n0)
    orc.reverse_patch(st, merged, bits, n0 + m, rows_c, n0)
    assert nrows == nrep and nrep > n0 // 2
    got = gpu_graph(ix, n0 + 2 * m)
    bad = np.where((got != merged).any(1))[0]
    assert len(bad) == 0, f"{len(bad)} rows differ, e.g. {bad[:5]}"


def test_consolidation_restores_connectivity_and_recall(svf, orc):
    # fp32 inner product: after 20 % deletes the consolidated graph names no
    # deleted vertex in rows that had enough live candidates, and the search
    # finds at least as many true neighbours among the live vectors
    n, R = 6000, 32
    X = synth.sample("unit96", n, 811)
    st = orc.Store.from_vectors(X, "ip")
    g0, _ = orc.build_graph(st, R)
    ix = svf.Index(96, n, dtype="f32", metric="ip", R=R, max_batch=1000)
    ix.attach(torch.from_numpy(X).cuda(), torch.from_numpy(g0.view(np.int32)))
    dele = np.random.default_rng(812).choice(n, n // 5, replace=False)
    ix.delete(ids_t(dele))
    isdel = np.zeros(n, bool)
    isdel[dele] = True
    Q = synth.sample("unit96", 300, 813)
    ti, td, _ = orc.knn(st, Q, 10, deleted=orc.bitset(n, dele))
    cfg = svf.SearchConfig(k=10, L=64, T=24, seed=3)

    def recall():
        ids, _ = ix.search(torch.from_numpy(Q).cuda(), cfg)
        ids = P.as_u32(ids.cpu().numpy())
        return P.recall(ids, ti, td, orc.dist_ids(st, Q, ids.astype(np.uint32)))

    before = recall()
    g_before = gpu_graph(ix, n)
    named = np.array([not isdel[u] and isdel[g_before[u][g_before[u] != orc.EMPTY]].any() for u in range(n)])
    rows = ix.consolidate()
    assert rows == named.sum()
    g_after = gpu_graph(ix, n)
    np.testing.assert_array_equal(g_after[~named], g_before[~named])
    left = np.array([isdel[g_after[u][g_after[u] != orc.EMPTY]].any() for u in range(n)])
    assert left[named].mean() < 0.01
    after = recall()
    assert after >= before - 0.002, (before, after)
    assert ix.stats()["repaired_rows"] >= rows


def test_consolidation_errors_and_discard(svf, orc):
    n, R = 3000, 32
    X = synth.sample("u8", n + 300, 821)
    st = orc.Store.from_vectors(X[:n], "l2")
    g0, _ = orc.build_graph(st, R)
    ix = svf.Index(128, n + 300, dtype="u8", metric="l2", R=R, max_batch=1000)
    ix.attach(torch.from_numpy(X[:n]).cuda(), torch.from_numpy(g0.view(np.int32)))
    ix.delete(ids_t(np.arange(0, n, 4)))
    with pytest.raises(svf.SvfError):
        ix.consolidate_run()
    with pytest.raises(svf.SvfError):
        ix.consolidate_commit()
    # a log too small for the inserts made meanwhile: commit refuses, the
    # active graph is left as the updates made it
    ix.consolidate_begin(log_rows=10)
    with pytest.raises(svf.SvfError):
        ix.consolidate_begin(log_rows=10)
    ix.insert(torch.from_numpy(X[n:n + 100]).cuda(), L_ins=64, T_ins=16)
    with pytest.raises(svf.SvfError):
        ix.consolidate_run(cap=R - 1)
    ix.consolidate_run()
    active = gpu_graph(ix, n + 100)
    with pytest.raises(svf.SvfError):
        ix.consolidate_commit()
    np.testing.assert_array_equal(gpu_graph(ix, n + 100), active)
    # abort, and a rebuild, drop a consolidation in progress
    ix.consolidate_begin(log_rows=10)
    ix.consolidate_abort()
    with pytest.raises(svf.SvfError):
        ix.consolidate_run()
    ix.consolidate_begin(log_rows=10)
    ix.attach(torch.from_numpy(X[:n]).cuda(), torch.from_numpy(g0.view(np.int32)))
    with pytest.raises(svf.SvfError):
        ix.consolidate_run()
