"""The measured configurations at full size, every output checked against the
FP64 oracle run on the same inputs.

* unit96, 10M x 96 inner product, R = 32, built as the benchmark builds it
  (every row's exact 64-NN by inner product on the tensor cores, pruned to
  32); all 10,000 queries searched in the benchmark's launch configuration
  (L = 64, T = 40) in every form -- plain FP32, BF16 / FP8 traversal + exact
  FP32 re-rank, and the small-batch form (8 warps per query, T = 8) -- and
  the same 10,000 queries searched by the oracle on the same graph: the FP32
  parity rule on every query, the queries whose trajectories diverged after
  a near tie counted and bounded, and recall@10 against exact kNN equal to
  the oracle's within 0.2 points (exact kNN by the oracle's FP64 brute force
  on 500 sampled queries, and by the tensor-core scan on all 10,000).
* u8, 1M x 128 uint8 squared L2, R = 64: the GPU's exact build (the exact
  tensor-core scan of uint8 rows) checked row by row on 2,000 sampled
  vertices (exact 128-NN + prune by the oracle); all
  10,000 queries bit-exact at L = 64 and L = 128; the 10 % insert stream (ten
  batches of 10,000) compared over the whole graph with the oracle's inserts
  after every batch, and all queries again on the grown graph; a global
  consolidation after 20 % deletes checked bit-exact on sampled rows.
"""
import numpy as np
import pytest

import synth
from tests import _parity as P

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

N96, NQ, SEED = 10_000_000, 10_000, 4
L96, T96 = 64, 40
NGT = 500          # queries given FP64 brute-force ground truth
MAX_DIVERGED = 0.02


@pytest.fixture(scope="module")
def svf():
    import paper_2601_08528_b300 as svf
    svf.load()
    return svf


@pytest.fixture(scope="module")
def unit96(svf):
    X = synth.sample_chunked("unit96", N96, 300)
    ix = svf.Index(96, N96, dtype="f32", metric="ip", R=32, lowp=("bf16", "fp8"), max_batch=N96)
    ix.build(torch.from_numpy(X).cuda())
    torch.cuda.synchronize()
    g = P.as_u32(ix.graph[:N96].cpu().numpy())
    Q = synth.sample_chunked("unit96", NQ, 302)
    return X, ix, g, Q


@pytest.fixture(scope="module")
def truth96(svf, orc, unit96):
    """Exact top-10 by inner product: the oracle's FP64 brute force on NGT
    sampled queries, and the tensor-core scan (checked against the oracle at
    smaller sizes) on all queries, its distances recomputed in FP64."""
    X, ix, g, Q = unit96
    st = orc.Store.from_vectors(X, "ip")
    qs = sample(NQ, NGT, 9)
    oi, od, _ = orc.knn(st, Q[qs], 10)
    ti, _, _ = svf.knn_tc(ix.vectors()[:N96], torch.from_numpy(Q).cuda(), 10, "ip")
    ti = P.as_u32(ti.cpu().numpy())
    td = orc.dist_ids(st, Q, ti)
    # the scan and the brute force agree on the sample's k-th distances
    np.testing.assert_allclose(td[qs, -1], od[:, -1], rtol=1e-6, atol=1e-6)
    return st, qs, oi, od, ti, td


def graph_invariants(g, n):
    """Fixed degree: every entry is a live id < n or EMPTY; no self loops; no
    id twice in a row."""
    empty = np.uint32(0xFFFFFFFF)
    assert ((g < n) | (g == empty)).all()
    rows = np.arange(len(g), dtype=np.uint32)[:, None]
    assert not (g == rows).any(), "self loop"
    s = np.sort(g, axis=1)
    dup = (s[:, 1:] == s[:, :-1]) & (s[:, 1:] != empty)
    assert not dup.any(), f"{dup.any(1).sum()} rows repeat an id"


def test_unit96_10M_graph_invariants(orc, unit96):
    X, ix, g, Q = unit96
    graph_invariants(g, N96)
    assert (g != 0xFFFFFFFF).all()  # 64 candidates always leave 32 after the prune
    assert ix.stats()["build_fallback"] < N96 // 50
    # sampled rows: the oracle's exact 64-NN + RNG prune (FP32 rule: a row may
    # differ only where the oracle met a near tie)
    vs = sample(N96, 64, 20)
    st = orc.Store.from_vectors(X, "ip")
    ids, d, kgap = orc.knn(st, X[vs], 64, self_ids=vs.astype(np.int64))
    for i, v in enumerate(vs):
        row, pgap = orc.prune(st, ids[i], d[i], 32)
        assert np.array_equal(g[v], row) or min(kgap[i], pgap) <= P.TOL, f"row {v}"


def sample(nq, m, seed):
    return np.sort(np.random.default_rng(seed).choice(nq, m, replace=False))


FORMS = {
    "fp32": dict(L=L96, T=T96, W=1, precision="f32"),
    "bf16": dict(L=L96, T=T96, W=1, precision="bf16"),
    "fp8": dict(L=L96, T=T96, W=1, precision="fp8"),
    # the benchmark's small-batch configuration: 8 warps per query (8 parents
    # per iteration), fp8 traversal + exact re-rank
    "fp8-w8": dict(L=64, T=8, W=8, precision="fp8"),
}


@pytest.mark.parametrize("form", list(FORMS))
def test_unit96_10M_every_query_and_recall(svf, orc, unit96, truth96, form):
    X, ix, g, Q = unit96
    st, qs, oi, od, ti, td = truth96
    f = FORMS[form]
    low = f["precision"] != "f32"
    ids, dist = ix.search(torch.from_numpy(Q).cuda(),
                          svf.SearchConfig(k=10, L=f["L"], T=f["T"], precision=f["precision"] if low else None,
                                           rerank=low, seed=SEED, W=f["W"]))
    ids, dist = ids.cpu().numpy(), dist.cpu().numpy()
    if low:
        # oracle: FP64 search over the same low-precision codes, then the
        # exact FP64 distances of its final pool re-sorted by (dist, id)
        lst = orc.Store.from_vectors(X, "ip", dtype=f["precision"])
        o = orc.search(lst, N96, g, None, Q, 10, f["L"], f["T"], SEED, want_pool=True, W=f["W"])
        ref = P.rerank_ref(orc, st, Q, o, 10)
    else:
        ref = orc.search(st, N96, g, None, Q, 10, f["L"], f["T"], SEED, W=f["W"])
    stats = P.check_fp32_all(ids, dist, ref, X, Q, "ip", max_diverged=MAX_DIVERGED)
    # recall@10 equal to the oracle's within 0.2 points, against the FP64
    # brute force (sample) and against the tensor-core scan (every query)
    gi, ri = P.as_u32(ids), ref["ids"].astype(np.int64)
    r_gpu = P.recall(gi[qs], oi, od, orc.dist_ids(st, Q[qs], gi[qs]))
    r_orc = P.recall(ri[qs], oi, od, orc.dist_ids(st, Q[qs], ri[qs]))
    assert abs(r_gpu - r_orc) <= 0.002, (r_gpu, r_orc)
    R_gpu = P.recall(gi, ti, td, orc.dist_ids(st, Q, gi))
    R_orc = P.recall(ri, ti, td, orc.dist_ids(st, Q, ri))
    assert abs(R_gpu - R_orc) <= 0.002, (R_gpu, R_orc)
    print(f"\n[{form}] {stats} recall@10 gpu {R_gpu:.4f} oracle {R_orc:.4f} (sample {r_gpu:.4f} / {r_orc:.4f})")


# ---------------------------------------------------------------- uint8, 1M x 128, R = 64
N8, R8, B8, NB8 = 1_000_000, 64, 10_000, 10


@pytest.fixture(scope="module")
def u8(svf):
    X = synth.sample_chunked("u8", N8 + NB8 * B8, 201)
    ix = svf.Index(128, N8 + NB8 * B8, dtype="u8", metric="l2", R=R8, max_batch=N8)
    ix.build(torch.from_numpy(X[:N8]).cuda())
    torch.cuda.synchronize()
    g = P.as_u32(ix.graph[:N8].cpu().numpy())
    Q = synth.sample_chunked("u8", NQ, 202)
    return X, ix, g, Q


def test_u8_1M_build_rows_sampled(orc, u8):
    X, ix, g, Q = u8
    assert ix.stats()["build_tensor_core"] == 1  # the exact 128-NN came from the tensor-core scan
    graph_invariants(g, N8)
    vs = sample(N8, 2000, 21)
    st = orc.Store.from_vectors(X[:N8], "l2")
    ids, d, _ = orc.knn(st, X[vs], 2 * R8, self_ids=vs.astype(np.int64))
    for i, v in enumerate(vs):
        row, _ = orc.prune(st, ids[i], d[i], R8)
        np.testing.assert_array_equal(g[v], row, err_msg=f"row {v}")


def _u8_search_all(svf, orc, ix, X, g, Q, n, L):
    ids, dist = ix.search(torch.from_numpy(Q).cuda(), svf.SearchConfig(k=10, L=L, T=L // 2, seed=SEED))
    st = orc.Store.from_vectors(X[:n], "l2")
    o = orc.search(st, n, g, None, Q, 10, L, L // 2, SEED)
    P.check_exact(ids.cpu().numpy(), dist.cpu().numpy(), o)


@pytest.mark.parametrize("L", [64, 128])
def test_u8_1M_search_every_query_bit_exact(svf, orc, u8, L):
    X, ix, g, Q = u8
    _u8_search_all(svf, orc, ix, X, g, Q, N8, L)


def test_u8_1M_insert_stream_whole_graph(svf, orc, u8):
    """The 10 % insert stream: ten batches of 10,000; after every batch every
    row of the graph equals the oracle's."""
    X, ix, g, Q = u8
    st = orc.Store.from_vectors(X, "l2")
    want = np.full((N8 + NB8 * B8, R8), orc.EMPTY, dtype=np.uint32)
    want[:N8] = g
    for b in range(NB8):
        n0 = N8 + b * B8
        new = ix.insert(torch.from_numpy(X[n0:n0 + B8]).cuda(), L_ins=128, T_ins=64)
        assert new.cpu().numpy().tolist() == list(range(n0, n0 + B8))
        orc.insert(st, n0, B8, want, None, 128, 64, ix.params.seed)
        got = P.as_u32(ix.graph[:n0 + B8].cpu().numpy())
        bad = np.where((got != want[:n0 + B8]).any(1))[0]
        assert len(bad) == 0, f"batch {b}: {len(bad)} rows differ, e.g. {bad[:5]}"
    graph_invariants(got, N8 + NB8 * B8)
    # every query again, on the grown graph
    _u8_search_all(svf, orc, ix, X, want, Q, N8 + NB8 * B8, 64)


def test_u8_1M_consolidation_rows_sampled(svf, orc, u8):
    # 20 % deletes (with the localized repair), then a global consolidation of
    # the whole graph on the GPU; sampled rows bit-exact against the oracle's
    # consolidation of the same snapshot
    X, ix, _, _ = u8
    n = ix.n_used
    dele = synth.pick_live_ids(n, None, n // 5, 41)
    ix.delete(torch.from_numpy(dele.view(np.int32)).cuda())
    snap = P.as_u32(ix.graph[:n].cpu().numpy()).astype(np.uint32)
    bits = orc.bitset(n, dele)
    isdel = np.zeros(n + 1, bool)
    isdel[dele.astype(np.int64)] = True
    named = ~isdel[:n] & isdel[np.where(snap == orc.EMPTY, n, snap)].any(1)
    rows = ix.consolidate()
    assert rows == named.sum()
    got = P.as_u32(ix.graph[:n].cpu().numpy()).astype(np.uint32)
    rng = np.random.default_rng(42)
    vs = np.concatenate([rng.choice(np.where(named)[0], 24, replace=False),
                         rng.choice(np.where(~named)[0], 8, replace=False)]).astype(np.uint32)
    st = orc.Store.from_vectors(X[:n], "l2")
    want, _ = orc.consolidate_rows(st, n, snap, bits, vs)
    np.testing.assert_array_equal(got[vs], want)
    graph_invariants(got, n)
