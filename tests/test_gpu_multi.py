"""Search with W warps per query (W parents per iteration, Sec. 4.4 intra-query
parallelism over Alg. 1) against the FP64 oracle's W-parent search."""
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


_cache = {}


def setup(orc, mix, n, R, metric, seed):
    key = (mix, n, R, metric, seed)
    if key not in _cache:
        X = synth.sample(mix, n, seed)
        st = orc.Store.from_vectors(X, metric)
        g, _ = orc.build_graph(st, R)
        _cache[key] = (X, st, g)
    return _cache[key]


def make_index(svf, X, g, metric, R, lowp=(), deleted=None, n_cap=None):
    n, d = X.shape
    ix = svf.Index(d, n_cap or n, dtype="u8" if X.dtype == np.uint8 else "f32", metric=metric, R=R, lowp=lowp,
                   max_batch=1000)
    ix.attach(torch.from_numpy(X).cuda(), torch.from_numpy(g.view(np.int32)), deleted=deleted)
    return ix


@pytest.mark.parametrize("W,L,T", [(2, 64, 16), (4, 64, 8), (8, 128, 6), (4, 256, 10), (8, 32, 3)])
def test_multi_fp32_l2_parity(svf, orc, W, L, T):
    X, st, g = setup(orc, "tiny", 3000, 32, "l2", 701)
    Q = synth.sample("tiny", 200, 702)
    ix = make_index(svf, X, g, "l2", 32)
    ids, dist = ix.search(torch.from_numpy(Q).cuda(), svf.SearchConfig(k=10, L=L, T=T, seed=7, W=W))
    o = orc.search(st, 3000, g, None, Q, 10, L, T, 7, W=W)
    P.check_fp32(ids.cpu().numpy(), dist.cpu().numpy(), o, X, Q, "l2")
    s = ix.stats()
    assert s["search_queries"] == 200
    assert s["search_iters"] == o["iters"].sum()


@pytest.mark.parametrize("R,W,L", [(64, 2, 64), (64, 4, 128), (32, 8, 64), (64, 8, 256)])
def test_multi_u8_bit_exact(svf, orc, R, W, L):
    X, st, g = setup(orc, "u8", 4000, R, "l2", 711)
    Q = synth.sample("u8", 200, 712)
    ix = make_index(svf, X, g, "l2", R)
    T = max(4, L // (2 * W))
    ids, dist = ix.search(torch.from_numpy(Q).cuda(), svf.SearchConfig(k=10, L=L, T=T, seed=5, W=W))
    o = orc.search(st, 4000, g, None, Q, 10, L, T, 5, W=W)
    P.check_exact(ids.cpu().numpy(), dist.cpu().numpy(), o)
    s = ix.stats()
    assert s["search_iters"] == o["iters"].sum()
    if s["hash_resets"] == 0:
        assert s["search_evals"] == o["evals"].sum()


def test_multi_w1_is_the_one_warp_search(svf, orc):
    X, st, g = setup(orc, "u8", 4000, 64, "l2", 711)
    Q = torch.from_numpy(synth.sample("u8", 100, 713)).cuda()
    ix = make_index(svf, X, g, "l2", 64)
    a = ix.search(Q, svf.SearchConfig(k=10, L=64, T=24, seed=3))
    b = ix.search(Q, svf.SearchConfig(k=10, L=64, T=24, seed=3, W=1))
    for x, y in zip(a, b):
        assert torch.equal(x, y)


@pytest.mark.parametrize("prec,W", [("fp8", 4), ("bf16", 2)])
def test_multi_lowp_rerank_parity(svf, orc, prec, W):
    X, st, g = setup(orc, "unit96", 3000, 32, "ip", 721)
    Q = synth.sample("unit96", 200, 722)
    ix = make_index(svf, X, g, "ip", 32, lowp=(prec,))
    L, T = 64, 8
    ids, dist = ix.search(torch.from_numpy(Q).cuda(),
                          svf.SearchConfig(k=10, L=L, T=T, precision=prec, rerank=True, seed=4, W=W))
    lst = orc.Store.from_vectors(X, "ip", dtype=prec)
    o = orc.search(lst, 3000, g, None, Q, 10, L, T, 4, want_pool=True, W=W)
    P.check_fp32(ids.cpu().numpy(), dist.cpu().numpy(), P.rerank_ref(orc, st, Q, o, 10), X, Q, "ip")


def test_multi_deletions_small_hash_and_padding(svf, orc):
    # deleted ids never come back; a small visited table forces resets; n < L pads
    X, st, g = setup(orc, "u8", 4000, 64, "l2", 711)
    n = 4000
    dele = np.arange(0, n, 5, dtype=np.int64)
    bits = orc.bitset(n, dele)
    ix = make_index(svf, X, g, "l2", 64, deleted=dele)
    Q = synth.sample("u8", 100, 731)
    cfg = svf.SearchConfig(k=10, L=64, T=20, seed=2, W=4, hash_log2=10)
    ids, dist = ix.search(torch.from_numpy(Q).cuda(), cfg)
    o = orc.search(st, n, g, bits, Q, 10, 64, 20, 2, W=4)
    P.check_exact(ids.cpu().numpy(), dist.cpu().numpy(), o)
    assert not np.isin(P.as_u32(ids.cpu().numpy()), dele).any()
    assert ix.stats()["hash_resets"] > 0

    Xs = synth.sample("u8", 20, 741)
    sts = orc.Store.from_vectors(Xs, "l2")
    gs, _ = orc.build_graph(sts, 32)
    ixs = make_index(svf, Xs, gs, "l2", 32, n_cap=64)
    Qs = synth.sample("u8", 5, 742)
    ids, dist = ixs.search(torch.from_numpy(Qs).cuda(), svf.SearchConfig(k=32, L=64, T=50, seed=1, W=8))
    o = orc.search(sts, 20, gs, None, Qs, 32, 64, 50, 1, W=8)
    P.check_exact(ids.cpu().numpy(), dist.cpu().numpy(), o)
    assert (P.as_u32(ids.cpu().numpy())[:, 20:] == 0xFFFFFFFF).all()


def test_multi_single_query_and_t0(svf, orc):
    X, st, g = setup(orc, "tiny", 3000, 32, "l2", 701)
    Q = synth.sample("tiny", 1, 751)
    ix = make_index(svf, X, g, "l2", 32)
    for T in (0, 1, 40):
        ids, dist = ix.search(torch.from_numpy(Q).cuda(), svf.SearchConfig(k=10, L=64, T=T, seed=8, W=8))
        o = orc.search(st, 3000, g, None, Q, 10, 64, T, 8, W=8)
        P.check_fp32(ids.cpu().numpy(), dist.cpu().numpy(), o, X, Q, "l2", min_identical=0.0)


def test_multi_large_rows_stage_in_rounds(svf, orc):
    # fp32 d=128, R=64, L=256, W=8: W full staging buffers exceed the shared
    # memory of a CTA, so each warp stages its rows in several rounds
    X, st, g = setup(orc, "tiny", 2500, 64, "l2", 761)
    Q = synth.sample("tiny", 64, 762)
    ix = make_index(svf, X, g, "l2", 64)
    ids, dist = ix.search(torch.from_numpy(Q).cuda(), svf.SearchConfig(k=10, L=256, T=6, seed=6, W=8))
    o = orc.search(st, 2500, g, None, Q, 10, 256, 6, 6, W=8)
    P.check_fp32(ids.cpu().numpy(), dist.cpu().numpy(), o, X, Q, "l2")


def test_multi_rejects_bad_arguments(svf, orc):
    X, st, g = setup(orc, "unit96", 3000, 32, "ip", 721)
    ix = make_index(svf, X, g, "ip", 32)
    Q = torch.from_numpy(synth.sample("unit96", 4, 1)).cuda()
    for W in (3, 16, -1):
        with pytest.raises(svf.SvfError):
            ix.search(Q, svf.SearchConfig(k=10, L=64, W=W))
    net = torch.zeros(1160, dtype=torch.int16, device="cuda")
    with pytest.raises(svf.SvfError):
        ix.search(Q, svf.SearchConfig(k=10, L=64, W=2, mlp=net))

