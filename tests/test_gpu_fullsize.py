"""The measured configurations at full size, checked on outputs the oracle can
compute one at a time, and by properties that hold at any size.

* unit96, 10M x 96 inner product, R = 32, built as the benchmark builds it
  (exact build of 200,000 rows, then inserts of the rest); 10,000 queries
  searched in the benchmark's launch configuration (L = 64, T = 72: its
  cheapest point at recall@10 >= 0.95 for every form), plain FP32, and BF16 /
  FP8 traversal + exact FP32 re-rank, and the benchmark's small-batch
  configuration (8 warps per query, T = 12); a sample of the queries is
  searched by the FP64 oracle on the same graph.
* u8, 1M x 128 uint8 squared L2, R = 64: the GPU's exact build checked row
  by row on sampled vertices (exact 128-NN + prune by the oracle), sampled
  searches bit-exact, one insert batch of 10,000 vectors compared over the
  whole graph with the oracle's insert of the same batch, and a global
  consolidation after 20 % deletes checked bit-exact on sampled rows.
"""
import numpy as np
import pytest

import synth
from tests import _parity as P

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

N96, NQ, SEED = 10_000_000, 10_000, 4
L96, T96 = 64, 72


@pytest.fixture(scope="module")
def svf():
    import paper_2601_08528_b300 as svf
    svf.load()
    return svf


@pytest.fixture(scope="module")
def unit96(svf):
    X = synth.sample_chunked("unit96", N96, 300)
    ix = svf.Index(96, N96, dtype="f32", metric="ip", R=32, lowp=("bf16", "fp8"), max_batch=1_000_000)
    ix.build(torch.from_numpy(X[:200_000]).cuda())
    while ix.n_used < N96:
        b = min(ix.n_used, 1_000_000, N96 - ix.n_used)
        ix.insert(torch.from_numpy(X[ix.n_used:ix.n_used + b]).cuda(), L_ins=64, T_ins=48)
    torch.cuda.synchronize()
    g = P.as_u32(ix.graph[:N96].cpu().numpy())
    Q = synth.sample_chunked("unit96", NQ, 302)
    return X, ix, g, Q


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


def test_unit96_10M_graph_invariants(unit96):
    X, ix, g, Q = unit96
    graph_invariants(g, N96)
    # the insert path fills every row of a connected build
    assert (g != 0xFFFFFFFF).sum(1).min() > 0


def sample(nq, m, seed):
    return np.sort(np.random.default_rng(seed).choice(nq, m, replace=False))


def test_unit96_10M_fp32_search_sampled(svf, orc, unit96):
    X, ix, g, Q = unit96
    ids, dist = ix.search(torch.from_numpy(Q).cuda(), svf.SearchConfig(k=10, L=L96, T=T96, seed=SEED))
    qs = sample(NQ, 48, 11)
    st = orc.Store.from_vectors(X, "ip")
    o = orc.search(st, N96, g, None, Q[qs], 10, L96, T96, SEED)
    P.check_fp32(ids.cpu().numpy()[qs], dist.cpu().numpy()[qs], o, X, Q[qs], "ip")


@pytest.mark.parametrize("prec", ["fp8", "bf16"])
def test_unit96_10M_lowp_rerank_search_sampled(svf, orc, unit96, prec):
    X, ix, g, Q = unit96
    ids, dist = ix.search(torch.from_numpy(Q).cuda(),
                          svf.SearchConfig(k=10, L=L96, T=T96, precision=prec, rerank=True, seed=SEED))
    qs = sample(NQ, 48, 12)
    lst = orc.Store.from_vectors(X, "ip", dtype=prec)
    o = orc.search(lst, N96, g, None, Q[qs], 10, L96, T96, SEED, want_pool=True)
    # oracle: exact FP64 distances of the final low-precision-traversal pool, re-sorted by (dist, id)
    st = orc.Store.from_vectors(X, "ip")
    ref = P.rerank_ref(orc, st, Q[qs], o, 10)
    P.check_fp32(ids.cpu().numpy()[qs], dist.cpu().numpy()[qs], ref, X, Q[qs], "ip")


def test_unit96_10M_multi_warp_sampled(svf, orc, unit96):
    # the benchmark's small-batch configuration: 8 warps per query (8 parents
    # per iteration), fp8 traversal + exact re-rank, T = 12
    X, ix, g, Q = unit96
    L, T, W = 64, 12, 8
    ids, dist = ix.search(torch.from_numpy(Q).cuda(),
                          svf.SearchConfig(k=10, L=L, T=T, precision="fp8", rerank=True, seed=SEED, W=W))
    qs = sample(NQ, 48, 14)
    lst = orc.Store.from_vectors(X, "ip", dtype="fp8")
    o = orc.search(lst, N96, g, None, Q[qs], 10, L, T, SEED, want_pool=True, W=W)
    st = orc.Store.from_vectors(X, "ip")
    P.check_fp32(ids.cpu().numpy()[qs], dist.cpu().numpy()[qs], P.rerank_ref(orc, st, Q[qs], o, 10), X, Q[qs], "ip")


# ---------------------------------------------------------------- uint8, 1M x 128, R = 64
N8, R8, B8 = 1_000_000, 64, 10_000


@pytest.fixture(scope="module")
def u8(svf):
    X = synth.sample_chunked("u8", N8 + B8, 201)
    ix = svf.Index(128, N8 + B8, dtype="u8", metric="l2", R=R8, max_batch=N8)
    ix.build(torch.from_numpy(X[:N8]).cuda())
    torch.cuda.synchronize()
    g = P.as_u32(ix.graph[:N8].cpu().numpy())
    return X, ix, g


def test_u8_1M_build_rows_sampled(orc, u8):
    X, ix, g = u8
    graph_invariants(g, N8)
    vs = sample(N8, 24, 21)
    st = orc.Store.from_vectors(X[:N8], "l2")
    ids, d, _ = orc.knn(st, X[vs], 2 * R8, self_ids=vs.astype(np.int64))
    for i, v in enumerate(vs):
        row, _ = orc.prune(st, ids[i], d[i], R8)
        np.testing.assert_array_equal(g[v], row, err_msg=f"row {v}")


def test_u8_1M_search_sampled_bit_exact(svf, orc, u8):
    X, ix, g = u8
    Q = synth.sample_chunked("u8", NQ, 202)
    for L in (64, 128):
        ids, dist = ix.search(torch.from_numpy(Q).cuda(), svf.SearchConfig(k=10, L=L, T=L // 2, seed=SEED))
        qs = sample(NQ, 48, 30 + L)
        st = orc.Store.from_vectors(X[:N8], "l2")
        o = orc.search(st, N8, g, None, Q[qs], 10, L, L // 2, SEED)
        P.check_exact(ids.cpu().numpy()[qs], dist.cpu().numpy()[qs], o)


def test_u8_1M_insert_batch_whole_graph(svf, orc, u8):
    X, ix, g = u8
    st = orc.Store.from_vectors(X, "l2")
    want = np.zeros((N8 + B8, R8), dtype=np.uint32)
    want[:N8] = g
    new = ix.insert(torch.from_numpy(X[N8:N8 + B8]).cuda(), L_ins=128, T_ins=64)
    assert new.cpu().numpy().tolist() == list(range(N8, N8 + B8))
    orc.insert(st, N8, B8, want, None, 128, 64, ix.params.seed)
    got = P.as_u32(ix.graph[:N8 + B8].cpu().numpy())
    bad = np.where((got != want).any(1))[0]
    assert len(bad) == 0, f"{len(bad)} rows differ, e.g. {bad[:5]}"
    graph_invariants(got, N8 + B8)


def test_u8_1M_consolidation_rows_sampled(svf, orc, u8):
    # 20 % deletes (with the localized repair), then a global consolidation of
    # the whole graph on the GPU; sampled rows bit-exact against the oracle's
    # consolidation of the same snapshot
    X, ix, _ = u8
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
