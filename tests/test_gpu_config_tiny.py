"""The plain method's tiny configuration exactly as stated, end to end against
the FP64 oracle: n = 10,000 fp32 vectors, d = 128, from the 16-component
Gaussian mixture; graph out-degree 32 built as exact 64-NN then RNG-pruned to
32 (Sec. 3 Build, Sec. 5.1 reordering); 1,000 queries, squared L2, k = 10,
beam L = 64, a fixed 32 iterations (Alg. 1); then 100 inserts (Sec. 5.1,
L_ins = 64, T_ins = 32) and 100 deletes with the localized repair (Sec. 5.2),
and the 1,000 queries again on the updated index.

Each step starts from the GPU's own state (graph, deletion bits), so the
oracle repeats exactly that step: the FP32 rule allows a row or a query to
differ only where the oracle met a near tie (relative gap <= 1e-5).
"""
import numpy as np
import pytest

import synth
from tests import _parity as P

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

N, D, R, NQ, M_INS, M_DEL = 10_000, 128, 32, 1_000, 100, 100
L, T, SEED = 64, 32, 105


@pytest.fixture(scope="module")
def tiny(orc):
    import paper_2601_08528_b300 as svf
    svf.load()
    X = synth.sample("tiny", N + M_INS, 101)
    X[N:] = synth.sample("tiny", M_INS, 103)
    Q = synth.sample("tiny", NQ, 102)
    st = orc.Store.from_vectors(X, "l2")
    ix = svf.Index(D, N + M_INS, dtype="f32", metric="l2", R=R, max_batch=N)
    return svf, X, Q, st, ix


def _search_parity(svf, orc, ix, st, X, Q, n, g, bits):
    ids, dist = ix.search(torch.from_numpy(Q).cuda(), svf.SearchConfig(k=10, L=L, T=T, seed=SEED))
    ids, dist = ids.cpu().numpy(), dist.cpu().numpy()
    o = orc.search(st, n, g, bits, Q, 10, L, T, SEED)
    stats = P.check_fp32_all(ids, dist, o, X, Q, "l2", max_diverged=0.01)
    # recall@10 against exact kNN over the live vectors equals the oracle's within 0.2 points
    dele = None if bits is None else orc.deleted_ids(bits, n)
    ti, td, _ = orc.knn(st, Q, 10, n=n, deleted=bits)
    r_gpu = P.recall(ids, ti, td, orc.dist_ids(st, Q, P.as_u32(ids)))
    r_orc = P.recall(o["ids"], ti, td, orc.dist_ids(st, Q, o["ids"]))
    assert abs(r_gpu - r_orc) <= 0.002, (r_gpu, r_orc)
    if dele is not None:
        assert not np.isin(P.as_u32(ids), dele).any()
    return stats, r_gpu


def test_tiny_config_build_search_insert_delete(orc, tiny):
    svf, X, Q, st, ix = tiny
    # ---- build: exact 64-NN + RNG prune to 32
    ix.build(torch.from_numpy(X[:N]).cuda())
    g_orc, gap = orc.build_graph(orc.Store.from_vectors(X[:N], "l2"), R)
    g = P.as_u32(ix.graph[:N].cpu().numpy()).astype(np.uint32)
    diff = (g != g_orc).any(1)
    assert not (diff & (gap > P.TOL)).any(), f"{(diff & (gap > P.TOL)).sum()} unambiguous rows differ"
    assert diff.mean() < 0.05
    # ---- search, fixed 32 iterations
    stats, r0 = _search_parity(svf, orc, ix, st, X, Q, N, g, None)
    assert r0 >= 0.9
    # ---- 100 inserts on the GPU's graph
    want = np.full((N + M_INS, R), orc.EMPTY, dtype=np.uint32)
    want[:N] = g
    ix.insert(torch.from_numpy(X[N:]).cuda(), L_ins=64, T_ins=32)
    new_gap, tail_gap = orc.insert(st, N, M_INS, want, None, 64, 32, ix.params.seed)
    gi = P.as_u32(ix.graph[:N + M_INS].cpu().numpy()).astype(np.uint32)
    diff = (gi != want).any(1)
    ok = np.zeros(N + M_INS, bool)
    amb_new = np.where(new_gap <= P.TOL)[0] + N
    ok[amb_new] = True
    ok[np.where(tail_gap <= P.TOL)[0]] = True
    for v in amb_new:   # old rows reached by an ambiguous new row (either side's choice)
        for u in set(want[v].tolist()) | set(gi[v].tolist()):
            if u < N:
                ok[u] = True
    assert not (diff & ~ok).any(), f"{(diff & ~ok).sum()} unexplained row differences after the inserts"
    # ---- 100 deletes + localized repair, on the GPU's graph
    n = N + M_INS
    dels = synth.pick_live_ids(n, None, M_DEL, 104)
    assert ix.delete(torch.from_numpy(dels.view(np.int32)).cuda()) == M_DEL
    bits = orc.bitset(n)
    g_del = gi.copy()
    newly, _, gap = orc.delete(st, n, g_del, bits, dels)
    assert newly == M_DEL
    gd = P.as_u32(ix.graph[:n].cpu().numpy()).astype(np.uint32)
    diff = (gd != g_del).any(1)
    assert not (diff & (gap > P.TOL)).any(), f"{(diff & (gap > P.TOL)).sum()} unambiguous repaired rows differ"
    np.testing.assert_array_equal(P.as_u32(ix.del_bits.cpu().numpy())[:len(bits)], bits)
    # ---- the queries again on the updated index
    stats2, r1 = _search_parity(svf, orc, ix, st, X, Q, n, gd, bits)
    print(f"\n[tiny] search {stats} recall {r0:.4f}; after updates {stats2} recall {r1:.4f}")
