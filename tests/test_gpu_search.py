"""GPU search / build / kNN / codec parity against the FP64 oracle (C ABI)."""
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
    assert torch.cuda.is_available()
    return svf


_cache = {}


def orc_graph(orc, mix, n, R, seed, metric, mode=0):
    key = (mix, n, R, seed, metric, mode)
    if key not in _cache:
        X = synth.sample(mix, n, seed)
        st = orc.Store.from_vectors(X, metric)
        g, gap = orc.build_graph(st, R, mode)
        _cache[key] = (X, st, g, gap)
    return _cache[key]


def gpu_index(svf, X, g, metric, R, n_cap=None, lowp=(), deleted=None, prune="rng", max_batch=1000):
    n, d = X.shape
    ix = svf.Index(d, n_cap or n, dtype="u8" if X.dtype == np.uint8 else "f32", metric=metric, R=R, lowp=lowp,
                   prune=prune, max_batch=max_batch)
    ix.attach(torch.from_numpy(X).cuda(), torch.from_numpy(g.view(np.int32)), deleted=deleted)
    return ix


@pytest.mark.parametrize("L,T", [(32, 16), (64, 32), (128, 64), (256, 40)])
def test_search_fp32_l2_parity(svf, orc, L, T):
    X, st, g, _ = orc_graph(orc, "tiny", 3000, 32, 201, "l2")
    Q = synth.sample("tiny", 300, 202)
    ix = gpu_index(svf, X, g, "l2", 32)
    ids, dist = ix.search(torch.from_numpy(Q).cuda(), svf.SearchConfig(k=10, L=L, T=T, seed=77))
    o = orc.search(st, 3000, g, None, Q, 10, L, T, 77)
    P.check_fp32(ids.cpu().numpy(), dist.cpu().numpy(), o, X, Q, "l2")
    ti, td, _ = orc.knn(st, Q, 10)
    r_gpu = P.recall(ids.cpu().numpy(), ti, td, orc.dist_ids(st, Q, P.as_u32(ids.cpu().numpy())))
    r_orc = P.recall(o["ids"], ti, td, orc.dist_ids(st, Q, o["ids"]))
    assert abs(r_gpu - r_orc) <= 0.002
    assert ix.stats()["search_queries"] == 300


@pytest.mark.parametrize("R,L", [(64, 64), (64, 128), (32, 64)])
def test_search_u8_bit_exact(svf, orc, R, L):
    X, st, g, _ = orc_graph(orc, "u8", 4000, R, 211, "l2")
    Q = synth.sample("u8", 300, 212)
    ix = gpu_index(svf, X, g, "l2", R)
    ids, dist = ix.search(torch.from_numpy(Q).cuda(), svf.SearchConfig(k=10, L=L, T=L // 2, seed=5))
    o = orc.search(st, 4000, g, None, Q, 10, L, L // 2, 5)
    P.check_exact(ids.cpu().numpy(), dist.cpu().numpy(), o)
    s = ix.stats()
    assert s["search_iters"] == o["iters"].sum()
    if s["hash_resets"] == 0:
        assert s["search_evals"] == o["evals"].sum()


def test_search_ip_parity(svf, orc):
    X, st, g, _ = orc_graph(orc, "unit96", 3000, 32, 221, "ip")
    Q = synth.sample("unit96", 300, 222)
    ix = gpu_index(svf, X, g, "ip", 32)
    ids, dist = ix.search(torch.from_numpy(Q).cuda(), svf.SearchConfig(k=10, L=128, T=64, seed=9))
    o = orc.search(st, 3000, g, None, Q, 10, 128, 64, 9)
    P.check_fp32(ids.cpu().numpy(), dist.cpu().numpy(), o, X, Q, "ip")


def test_search_with_deletions_and_small_hash(svf, orc):
    # a tiny visited table forces resets: the result must not change
    X, st, g, _ = orc_graph(orc, "u8", 4000, 64, 211, "l2")
    dels = synth.pick_live_ids(4000, None, 800, 231)
    bits = orc.bitset(4000, dels)
    Q = synth.sample("u8", 200, 232)
    ix = gpu_index(svf, X, g, "l2", 64, deleted=dels)
    o = orc.search(st, 4000, g, bits, Q, 10, 64, 64, 3)
    for hb in (0, 9):
        ids, dist = ix.search(torch.from_numpy(Q).cuda(), svf.SearchConfig(k=10, L=64, T=64, seed=3, hash_log2=hb))
        P.check_exact(ids.cpu().numpy(), dist.cpu().numpy(), o)
    assert ix.stats()["hash_resets"] > 0
    assert not np.isin(P.as_u32(ids.cpu().numpy()), dels).any()


def test_search_edge_cases(svf, orc):
    # n_used < L and k: results padded; empty batch; caller-provided keys
    X = synth.sample("u8", 20, 241)
    st = orc.Store.from_vectors(X, "l2")
    g, _ = orc.build_graph(st, 32)
    ix = gpu_index(svf, X, g, "l2", 32, n_cap=64)
    Q = synth.sample("u8", 7, 242)
    ids, dist = ix.search(torch.from_numpy(Q).cuda(), svf.SearchConfig(k=32, L=64, T=100, seed=1))
    o = orc.search(st, 20, g, None, Q, 32, 64, 100, 1)
    P.check_exact(ids.cpu().numpy(), dist.cpu().numpy(), o)
    assert (P.as_u32(ids.cpu().numpy())[:, 20:] == 0xFFFFFFFF).all()
    e_ids, _ = ix.search(torch.empty((0, X.shape[1]), dtype=torch.uint8, device="cuda"), svf.SearchConfig(k=5))
    assert e_ids.shape == (0, 5)
    keys = np.arange(7, dtype=np.uint64) * np.uint64(0x9E3779B97F4A7C15)
    ids, dist = ix.search(torch.from_numpy(Q).cuda(), svf.SearchConfig(k=10, L=32, T=8, seed=1),
                          qkeys=torch.from_numpy(keys.view(np.int64)).cuda())
    o = orc.search(st, 20, g, None, Q, 10, 32, 8, 1, qkeys=keys)
    P.check_exact(ids.cpu().numpy(), dist.cpu().numpy(), o)


def test_search_rejects_bad_arguments(svf, orc):
    X, st, g, _ = orc_graph(orc, "u8", 4000, 64, 211, "l2")
    ix = gpu_index(svf, X, g, "l2", 64)
    Q = torch.from_numpy(synth.sample("u8", 4, 1)).cuda()
    for cfg in (svf.SearchConfig(k=10, L=48), svf.SearchConfig(k=40, L=64), svf.SearchConfig(k=0),
                svf.SearchConfig(k=10, L=64, precision="bf16")):
        with pytest.raises(svf.SvfError):
            ix.search(Q, cfg)


# ---------------------------------------------------------------- build (exact 2R-NN + prune)
@pytest.mark.parametrize("mix,metric,R,mode", [("u8", "l2", 64, 0), ("u8", "l2", 32, 1), ("tiny", "l2", 32, 0),
                                               ("unit96", "ip", 32, 0)])
def test_build_parity(svf, orc, mix, metric, R, mode):
    n = 2500
    X, st, g, gap = orc_graph(orc, mix, n, R, 251, metric, mode)
    ix = svf.Index(X.shape[1], n, dtype="u8" if mix == "u8" else "f32", metric=metric, R=R,
                   prune="rank" if mode else "rng", max_batch=n)
    ix.build(torch.from_numpy(X).cuda())
    gg = P.as_u32(ix.graph[:n].cpu().numpy())
    diff = (gg != g).any(1)
    if mix == "u8":
        assert not diff.any(), f"{diff.sum()} rows differ"
    else:
        assert not (diff & (gap > P.TOL)).any(), f"{(diff & (gap > P.TOL)).sum()} unambiguous rows differ"
        assert diff.mean() < 0.05


def test_build_tiny_n(svf, orc):
    for n in (1, 2, 5, 40):
        X = synth.sample("u8", n, 261 + n)
        st = orc.Store.from_vectors(X, "l2")
        g, _ = orc.build_graph(st, 32)
        ix = svf.Index(128, 64, dtype="u8", R=32, max_batch=64)
        ix.build(torch.from_numpy(X).cuda())
        np.testing.assert_array_equal(P.as_u32(ix.graph[:n].cpu().numpy()), g)


# ---------------------------------------------------------------- kNN / codecs
@pytest.mark.parametrize("mix,metric,k", [("u8", "l2", 10), ("tiny", "l2", 100), ("unit96", "ip", 10)])
def test_knn_parity(svf, orc, mix, metric, k):
    X = synth.sample(mix, 5000, 271)
    Q = synth.sample(mix, 97, 272)
    st = orc.Store.from_vectors(X, metric)
    oi, od, og = orc.knn(st, Q, k)
    ids, dist = svf.knn(torch.from_numpy(X).cuda(), torch.from_numpy(Q).cuda(), k, metric)
    gi = P.as_u32(ids.cpu().numpy())
    if mix == "u8":
        np.testing.assert_array_equal(gi, oi)
        np.testing.assert_array_equal(dist.cpu().numpy(), od.astype(np.int64))
    else:
        same = (gi == oi).all(1)
        assert not (~same & (og > P.TOL)).any()
        sc = P.dist_scale(X, Q, oi.astype(np.int64), metric)
        assert (np.abs(dist.cpu().numpy()[same] - od[same]) <= P.TOL * sc[same]).all()


def test_codecs_bit_exact(svf, orc):
    X = synth.sample("unit96", 3000, 281)
    X[0] = 0.0
    X[1, :5] = [1e-9, -3e-5, 500.0, -1e4, 2.0 ** -10]
    Xt = torch.from_numpy(X).cuda()
    lib = svf.load()
    import ctypes as C
    bf = torch.empty((3000, 96), dtype=torch.int16, device="cuda")
    f8 = torch.empty((3000, 128), dtype=torch.uint8, device="cuda")
    s = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.svf_encode_bf16(C.c_void_p(Xt.data_ptr()), 3000, 96, C.c_void_p(bf.data_ptr()), s) == 0
    assert lib.svf_encode_fp8(C.c_void_p(Xt.data_ptr()), 3000, 96, C.c_void_p(f8.data_ptr()), 128, s) == 0
    np.testing.assert_array_equal(bf.cpu().numpy().view(np.uint16), orc.bf16_encode_rows(X))
    got = f8.cpu().numpy()
    want = orc.fp8_encode_rows(X)
    np.testing.assert_array_equal(got[:, :100], want[:, :100])


@pytest.mark.parametrize("mix,metric", [("unit96", "ip"), ("tiny", "l2")])
def test_build_on_tensor_cores_rows_sampled(svf, orc, mix, metric):
    """At n >= 65,536 fp32 inner-product rows the build's exact 2R-NN come
    from the tensor cores (certified bf16 scan + exact fp32 band re-scoring,
    SIMT scan for the rows that fail the certificate); squared L2 keeps the
    SIMT scan.  Sampled rows equal the oracle's exact 64-NN + RNG prune,
    except where the oracle met a near tie."""
    n, R = 70_000, 32
    X = synth.sample(mix, n, 281)
    ix = svf.Index(X.shape[1], n, dtype="f32", metric=metric, R=R, max_batch=n)
    ix.build(torch.from_numpy(X).cuda())
    g = P.as_u32(ix.graph[:n].cpu().numpy())
    s = ix.stats()
    assert s["build_fallback"] < (n // 10 if metric == "ip" else 1)
    assert s["build_tensor_core"] == (1 if metric == "ip" else 0)
    vs = np.sort(np.random.default_rng(282).choice(n, 400, replace=False))
    st = orc.Store.from_vectors(X, metric)
    ids, d, kgap = orc.knn(st, X[vs], 2 * R, self_ids=vs.astype(np.int64))
    differ = 0
    for i, v in enumerate(vs):
        row, pgap = orc.prune(st, ids[i], d[i], R)
        if not np.array_equal(g[v], row):
            differ += 1
            assert min(kgap[i], pgap) <= P.TOL, f"row {v} differs without a near tie"
    assert differ <= len(vs) // 20
    # no self loops or repeats, every row full
    assert not (g == np.arange(n)[:, None]).any()
    srt = np.sort(g, 1)
    assert not ((srt[:, 1:] == srt[:, :-1]) & (srt[:, 1:] != 0xFFFFFFFF)).any()
    assert (g != 0xFFFFFFFF).all()


@pytest.mark.parametrize("R,metric", [(64, "l2"), (32, "l2"), (64, "ip")])
def test_build_u8_on_tensor_cores_bit_exact(svf, orc, R, metric):
    """uint8 stores of n >= 65,536 rows take the tensor-core scan too: values
    0..255 are exact in bf16 and every partial sum of products is an integer
    below 2^24, so the scan's distances are exact, the certificate needs no
    error band, and sampled graph rows equal the oracle's exact 2R-NN + RNG
    prune bit for bit (K = 128 runs the 512-candidate re-score)."""
    n = 70_000
    X = synth.sample("u8", n, 283)
    ix = svf.Index(X.shape[1], n, dtype="u8", metric=metric, R=R, max_batch=n)
    ix.build(torch.from_numpy(X).cuda())
    s = ix.stats()
    assert s["build_tensor_core"] == 1
    assert s["build_fallback"] < n // 10
    g = P.as_u32(ix.graph[:n].cpu().numpy())
    vs = np.sort(np.random.default_rng(284).choice(n, 300, replace=False))
    st = orc.Store.from_vectors(X, metric)
    ids, d, _ = orc.knn(st, X[vs], 2 * R, self_ids=vs.astype(np.int64))
    for i, v in enumerate(vs):
        row, _ = orc.prune(st, ids[i], d[i], R)
        np.testing.assert_array_equal(g[v], row, err_msg=f"row {v}")
    assert not (g == np.arange(n)[:, None]).any()


@pytest.mark.parametrize("R", [32, 64])
def test_build_rows_past_both_certificates_bit_exact(svf, orc, R):
    """Rows whose neighbourhoods are exact ties (100 copies of each of 20
    uint8 vectors: every list's bound equals the 2R-th distance, 0) fail the
    certificate of the first scan and of the second (R = 32; R = 64 has
    none), so the exact SIMT scan recomputes them, their batch split into
    row slices whose lists are merged.  Those rows and sampled others equal
    the oracle's exact 2R-NN + prune bit for bit."""
    n = 70_000
    X = synth.sample("u8", n, 285)
    X[:2000] = np.repeat(X[:20], 100, axis=0)
    ix = svf.Index(X.shape[1], n, dtype="u8", metric="l2", R=R, max_batch=n)
    ix.build(torch.from_numpy(X).cuda())
    s = ix.stats()
    assert s["build_tensor_core"] == 1
    assert s["build_fallback"] >= 2000
    g = P.as_u32(ix.graph[:n].cpu().numpy())
    rng = np.random.default_rng(286)
    vs = np.sort(np.concatenate([rng.choice(2000, 120, replace=False), 2000 + rng.choice(n - 2000, 80, replace=False)]))
    st = orc.Store.from_vectors(X, "l2")
    ids, d, _ = orc.knn(st, X[vs], 2 * R, self_ids=vs.astype(np.int64))
    for i, v in enumerate(vs):
        row, _ = orc.prune(st, ids[i], d[i], R)
        np.testing.assert_array_equal(g[v], row, err_msg=f"row {v}")


def test_gather_probe_measures_random_rows(svf):
    """The random-row fetch ceiling probe copies at least the rows asked for
    (whole batches of every warp), reports a plausible device time, and
    rejects a bad layout on the device path too."""
    import torch
    n, pitch = 2_000_000, 128  # 256 MB: above the L2
    table = torch.zeros(n * pitch, dtype=torch.uint8, device="cuda")
    for wps in (16, 24, 32):
        rows, ms = svf.gather_probe(table, n, pitch, 112, 1_000_000, warps_per_sm=wps)
        assert rows >= 1_000_000 and rows % 32 == 0
        rate = rows / (ms / 1e3)
        assert 1e8 < rate < 1e12, (wps, rate)
    rows, ms = svf.gather_probe(table, 1, pitch, 128, 5000)  # every copy reads the same row
    assert rows >= 5000 and ms > 0
    with pytest.raises(svf.SvfError):
        svf.gather_probe(table, n, pitch, 120, 1000)
