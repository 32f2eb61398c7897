"""Pins of the FP64 oracle to things other than itself (CPU only).

Each test ties one oracle function to a closed form, a library routine, a
hand-worked case or an invariant, chosen so that a dropped term, a wrong sign
or index or a swapped operand fails at least one of them.
"""
import json
import math
import os

import numpy as np
import pytest

import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _np_knn(X, Q, k, metric, exclude=None):
    """Brute force with numpy in float64 and lexsort on (dist, id)."""
    Xd = X.astype(np.float64)
    Qd = Q.astype(np.float64)
    out_i, out_d = [], []
    for i, q in enumerate(Qd):
        if metric == "l2":
            dist = ((Xd - q) ** 2).sum(1)
        else:
            dist = -(Xd @ q)
        ids = np.arange(len(Xd))
        if exclude is not None:
            keep = ids != exclude[i]
            ids, dist = ids[keep], dist[keep]
        o = np.lexsort((ids, dist))[:k]
        out_i.append(ids[o])
        out_d.append(dist[o])
    return np.array(out_i), np.array(out_d)


# ---------------------------------------------------------------- kNN (Sec. 2.1)
@pytest.mark.parametrize("mix,metric", [("tiny", "l2"), ("u8", "l2"), ("unit96", "ip")])
def test_knn_matches_numpy_bruteforce(orc, mix, metric):
    X = synth.sample(mix, 600, 11)
    Q = synth.sample(mix, 40, 12)
    st = orc.Store.from_vectors(X, metric)
    ids, dist, _ = orc.knn(st, Q, 10)
    ni, nd = _np_knn(X, Q, 10, metric)
    np.testing.assert_array_equal(ids, ni)
    np.testing.assert_allclose(dist, nd, rtol=1e-12, atol=1e-12)


def test_knn_u8_distances_are_exact_integers(orc):
    X = synth.sample("u8", 300, 13)
    Q = synth.sample("u8", 10, 14)
    _, dist, _ = orc.knn(orc.Store.from_vectors(X, "l2"), Q, 5)
    assert np.all(dist == np.round(dist))
    q0 = Q[0].astype(np.int64)
    best = min(int(((X[j].astype(np.int64) - q0) ** 2).sum()) for j in range(300))
    assert dist[0, 0] == best


def test_knn_self_exclusion_and_ties(orc):
    # four identical points: distance ties are broken by id, self excluded
    X = np.zeros((4, 16), dtype=np.float32)
    st = orc.Store.from_vectors(X, "l2")
    ids, dist, gap = orc.knn(st, X, 3, self_ids=np.arange(4))
    np.testing.assert_array_equal(ids, [[1, 2, 3], [0, 2, 3], [0, 1, 3], [0, 1, 2]])
    assert np.all(dist == 0) and np.all(gap == 0)


def test_knn_skips_deleted(orc):
    X = synth.sample("tiny", 200, 15)
    st = orc.Store.from_vectors(X, "l2")
    ids0, _, _ = orc.knn(st, X[:5], 3)
    bits = orc.bitset(200, ids0[:, 0])
    ids1, _, _ = orc.knn(st, X[:5], 3, deleted=bits)
    assert not np.isin(ids1, ids0[:, 0]).any()


# ---------------------------------------------------------------- generators
def test_splitmix64_published_vector(orc):
    # splitmix64 seeded with 0: its first output is 0xE220A8397B1DCDAF
    assert orc.splitmix64(0) == 0xE220A8397B1DCDAF


def test_query_key_definition(orc):
    q = np.arange(8, dtype=np.float32)
    words = q.view(np.uint32)
    want = 0
    for i, w in enumerate(words):
        want = (want + orc.splitmix64((i << 32) | int(w))) & 0xFFFFFFFFFFFFFFFF
    assert orc.query_key(q) == want
    q2 = q.copy()
    q2[3] = 3.0000002
    assert orc.query_key(q2) != want


# ---------------------------------------------------------------- codecs
def test_bf16_matches_torch_rne(orc):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(5)
    x = np.concatenate([rng.standard_normal(20000).astype(np.float32) * 10.0 ** rng.integers(-30, 30, 20000),
                        np.array([0.0, -0.0, 1.0, 3.0e38, -3.0e38, 1e-40, np.inf, -np.inf], dtype=np.float32)])
    # midpoints: exact ties between two bf16 values must go to the even one
    base = rng.integers(0, 1 << 15, 2000).astype(np.uint32) << 16
    x = np.concatenate([x, (base | 0x8000).view(np.float32)]).astype(np.float32)
    x = x[np.isfinite(x) | np.isinf(x)]
    ref = torch.from_numpy(x).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    ours = np.array([orc.bf16_encode(float(v)) for v in x], dtype=np.uint16)
    np.testing.assert_array_equal(ours, ref)


def test_e4m3_table_definition(orc):
    vals = [orc.e4m3_decode(c) for c in range(256)]
    assert vals[0x7E] == 448.0 and vals[0xFE] == -448.0
    assert vals[0x01] == 2.0 ** -9 and vals[0x08] == 2.0 ** -6 and vals[0x38] == 1.0
    assert math.isnan(vals[0x7F]) and math.isnan(vals[0xFF])
    finite = [v for v in vals if not math.isnan(v)]
    assert max(finite) == 448.0 and len(finite) == 254
    for c in range(256):
        if not math.isnan(vals[c]) and not (c == 0x80):  # -0 encodes back to 0x80 too
            assert orc.e4m3_encode(vals[c]) == c
    assert orc.e4m3_encode(-0.0) == 0x80


def test_e4m3_matches_torch_in_range_and_saturates(orc):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(6)
    x = (rng.standard_normal(20000) * 10.0 ** rng.uniform(-4, 2.6, 20000)).astype(np.float32)
    x = x[np.abs(x) <= 448.0]
    # exact midpoints between adjacent codes
    vals = np.array([orc.e4m3_decode(c) for c in range(0x7E)])
    mids = ((vals[1:] + vals[:-1]) / 2).astype(np.float32)
    x = np.concatenate([x, mids, -mids])
    ref = torch.from_numpy(x).to(torch.float8_e4m3fn).view(torch.uint8).numpy()
    ours = np.array([orc.e4m3_encode(float(v)) for v in x], dtype=np.uint8)
    np.testing.assert_array_equal(ours, ref)
    assert orc.e4m3_encode(1e6) == 0x7E and orc.e4m3_encode(-470.0) == 0xFE


def test_fp8_rows_scale_and_error_bound(orc):
    X = synth.sample("unit96", 50, 7)
    rows = orc.fp8_encode_rows(X)
    assert rows.shape[1] == orc.fp8_pitch(96) == 128
    s = rows[:, 96:100].copy().view(np.float32)[:, 0]
    np.testing.assert_array_equal(s, (np.abs(X).max(1) / np.float32(448.0)).astype(np.float32))
    dec = np.array([[orc.e4m3_decode(c) for c in r[:96]] for r in rows]) * s[:, None]
    # E4M3 normals carry 3 fraction bits: relative error <= 2^-4 (half ulp)
    big = np.abs(X) >= s[:, None] * 2.0 ** -6
    assert np.all(np.abs(dec - X)[big] <= np.abs(X)[big] * 2.0 ** -4 + 1e-12)


# ---------------------------------------------------------------- prune (Sec. 5.1)
def _golden(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


def test_prune_rng_hand_worked_case(orc):
    g = _golden("prune_rng_2d.json")
    pts = np.array(g["points"], dtype=np.float32)  # row 0 is v
    st = orc.Store.from_vectors(np.pad(pts, ((0, 0), (0, 2))), "l2")
    ids = np.array(g["candidates_sorted"], dtype=np.uint32)
    d = ((pts[ids] - pts[0]) ** 2).sum(1).astype(np.float64)
    out, _ = orc.prune(st, ids, d, g["R"], orc.PRUNE_RNG)
    assert out.tolist() == g["expected_row"]


def test_prune_rank_hand_worked_case(orc):
    g = _golden("prune_rank.json")
    X = np.zeros((g["n"], 4), dtype=np.float32)
    st = orc.Store.from_vectors(X, "l2")
    nbr = np.array(g["neighbour_lists"], dtype=np.uint32)
    ids = np.array(g["candidates_sorted"], dtype=np.uint32)
    out, _ = orc.prune(st, ids, np.zeros(len(ids)), g["R"], orc.PRUNE_RANK, nbr=nbr)
    assert out.tolist() == g["expected_row"]


def test_prune_collinear_keeps_only_nearest(orc):
    # points on a line on one side of v: every farther point has a detour
    # through each nearer one, so the counts are 0,1,2,...: order kept
    X = np.zeros((6, 4), dtype=np.float32)
    X[:, 0] = np.arange(6)
    st = orc.Store.from_vectors(X, "l2")
    ids = np.arange(1, 6, dtype=np.uint32)
    out, _ = orc.prune(st, ids, (ids.astype(np.float64)) ** 2, 3)
    assert out.tolist() == [1, 2, 3]
    # v in the middle: the two nearest on opposite sides both survive first
    X[:, 0] = [0, -1, 1.5, -2.5, 3.5, -4.5]
    st = orc.Store.from_vectors(X, "l2")
    ids = np.array([1, 2, 3, 4, 5], dtype=np.uint32)
    out, _ = orc.prune(st, ids, X[ids, 0].astype(np.float64) ** 2, 3)
    assert out.tolist() == [1, 2, 3]
    out, _ = orc.prune(st, ids, X[ids, 0].astype(np.float64) ** 2, 5)
    assert out[:2].tolist() == [1, 2]


def test_prune_identity_when_no_detours(orc):
    # RANK with empty neighbour lists: all counts are 0 -> input order
    X = np.zeros((10, 4), dtype=np.float32)
    st = orc.Store.from_vectors(X, "l2")
    nbr = np.full((10, 4), orc.EMPTY, dtype=np.uint32)
    ids = np.array([5, 2, 9, 1], dtype=np.uint32)
    out, _ = orc.prune(st, ids, np.arange(4.0), 6, orc.PRUNE_RANK, nbr=nbr)
    assert out.tolist() == [5, 2, 9, 1, orc.EMPTY, orc.EMPTY]


# ---------------------------------------------------------------- build
def test_build_rows_are_pruned_exact_knn(orc):
    X = synth.sample("tiny", 400, 21)
    st = orc.Store.from_vectors(X, "l2")
    R = 8
    g, gap = orc.build_graph(st, R)
    knn_i, knn_d = _np_knn(X, X, 2 * R, "l2", exclude=np.arange(400))
    for v in range(0, 400, 37):
        row, _ = orc.prune(st, knn_i[v], knn_d[v], R)
        np.testing.assert_array_equal(g[v], row)
    assert np.all(g != np.arange(400)[:, None])
    assert all(len(set(r)) == R for r in g)


# ---------------------------------------------------------------- search (Alg. 1)
def _ring_graph(n, R, seed):
    """Random rows that always contain i+1 (mod n): strongly connected."""
    rng = np.random.default_rng(seed)
    g = np.empty((n, R), dtype=np.uint32)
    for i in range(n):
        others = rng.choice(np.setdiff1d(np.arange(n), [i, (i + 1) % n]), R - 1, replace=False)
        g[i] = np.concatenate([[(i + 1) % n], others])
    return g


@pytest.mark.parametrize("mix,metric", [("tiny", "l2"), ("u8", "l2"), ("unit96", "ip")])
def test_search_with_beam_ge_n_is_exact_knn(orc, mix, metric):
    n = 150
    X = synth.sample(mix, n, 31)
    Q = synth.sample(mix, 20, 32)
    st = orc.Store.from_vectors(X, metric)
    g = _ring_graph(n, 4, 33)
    r = orc.search(st, n, g, None, Q, 10, 256, 256, 1)
    ni, nd = _np_knn(X, Q, 10, metric)
    np.testing.assert_array_equal(r["ids"], ni)
    np.testing.assert_allclose(r["dist"], nd, rtol=1e-12, atol=1e-9)


def test_search_init_is_the_draw_sequence(orc):
    # T=0: the pool is exactly the first L distinct draws, sorted
    n, L = 1000, 16
    X = synth.sample("tiny", n, 41)
    st = orc.Store.from_vectors(X, "l2")
    g = _ring_graph(n, 4, 42)
    q = X[:1]
    key = orc.query_key(q[0])
    base = orc.splitmix64(7 ^ orc.splitmix64(key))
    draws = []
    for j in range(4 * L):
        i = ((orc.splitmix64(base ^ j) >> 32) * n) >> 32
        if i not in draws:
            draws.append(i)
        if len(draws) == L:
            break
    r = orc.search(st, n, g, None, q, L, L, 0, 7, want_pool=True)
    d = ((X[draws].astype(np.float64) - q[0].astype(np.float64)) ** 2).sum(1)
    want = np.array(draws)[np.lexsort((draws, d))]
    np.testing.assert_array_equal(r["pool_ids"][0], want)


def test_search_deleted_never_returned_and_deterministic(orc):
    n = 2000
    X = synth.sample("tiny", n, 51)
    st = orc.Store.from_vectors(X, "l2")
    g, _ = orc.build_graph(st, 16)
    Q = synth.sample("tiny", 30, 52)
    bits = orc.bitset(n, np.arange(0, n, 3))
    r1 = orc.search(st, n, g, bits, Q, 10, 64, 32, 3)
    r2 = orc.search(st, n, g, bits, Q, 10, 64, 32, 3)
    np.testing.assert_array_equal(r1["ids"], r2["ids"])
    assert not np.any(r1["ids"] % 3 == 0)
    # evaluations are bounded by L + T*R
    assert np.all(r1["evals"] <= 64 + 32 * 16)


def test_search_tiny_n_pads(orc):
    X = synth.sample("tiny", 5, 61)
    st = orc.Store.from_vectors(X, "l2")
    g = _ring_graph(5, 2, 62)
    r = orc.search(st, 5, g, None, X[:2], 10, 32, 8, 1)
    assert np.all(r["ids"][:, 5:] == orc.EMPTY) and np.all(np.isinf(r["dist"][:, 5:]))
    assert sorted(r["ids"][0, :5].tolist()) == [0, 1, 2, 3, 4]


def test_search_w_parents_hand_worked(orc):
    # W nearest unexpanded entries per iteration (Sec. 4.4 intra-query
    # parallelism over Alg. 1): a hand-worked 12-point line graph
    g = _golden("search_wparents_hand.json")
    n, L = g["n"], g["L"]
    X = np.zeros((n, 4), dtype=np.float32)
    X[:, 0] = np.arange(n)
    st = orc.Store.from_vectors(X, "l2")
    graph = np.array(g["graph"], dtype=np.uint32)
    q = np.array([g["query"]], dtype=np.float32)
    r0 = orc.search(st, n, graph, None, q, L, L, 0, g["seed"], want_pool=True)
    assert r0["pool_ids"][0].tolist() == g["init_pool"]
    for c in g["cases"]:
        r = orc.search(st, n, graph, None, q, L, L, c["T"], g["seed"], want_pool=True, W=c["W"])
        assert r["pool_ids"][0].tolist() == c["pool"], c
        assert (r["iters"][0], r["evals"][0]) == (c["parents"], c["evals"]), c
        assert r["ids"][0].tolist() == c["pool"]
    bits = orc.bitset(n, g["deleted"])
    for c in g["cases_deleted"]:
        r = orc.search(st, n, graph, bits, q, L, L, c["T"], g["seed"], want_pool=True, W=c["W"])
        assert r["pool_ids"][0].tolist() == c["pool"], c
        assert (r["iters"][0], r["evals"][0]) == (c["parents"], c["evals"]), c


@pytest.mark.parametrize("W", [2, 4, 8])
def test_search_w_parents_beam_ge_n_is_exact_knn(orc, W):
    n = 150
    X = synth.sample("tiny", n, 31)
    Q = synth.sample("tiny", 20, 32)
    st = orc.Store.from_vectors(X, "l2")
    g = _ring_graph(n, 4, 33)
    r = orc.search(st, n, g, None, Q, 10, 256, 256, 1, W=W)
    ni, nd = _np_knn(X, Q, 10, "l2")
    np.testing.assert_array_equal(r["ids"], ni)
    np.testing.assert_allclose(r["dist"], nd, rtol=1e-12, atol=1e-9)


def test_search_w_parents_counts_and_range(orc):
    # every iteration expands exactly W parents while the pool has that many
    # unexpanded entries (a large graph and few iterations); W = 1 is Alg. 1
    n = 3000
    X = synth.sample("tiny", n, 81)
    st = orc.Store.from_vectors(X, "l2")
    g, _ = orc.build_graph(st, 16)
    Q = synth.sample("tiny", 16, 82)
    for W in (1, 2, 4):
        r = orc.search(st, n, g, None, Q, 10, 64, 6, 5, W=W)
        assert np.all(r["iters"] == 6 * W)
        assert np.all(r["evals"] <= 64 + 6 * W * 16)
    a = orc.search(st, n, g, None, Q, 10, 64, 20, 5)
    b = orc.search(st, n, g, None, Q, 10, 64, 20, 5, W=1)
    np.testing.assert_array_equal(a["ids"], b["ids"])
    for W in (0, 33):
        with pytest.raises(ValueError):
            orc.search(st, n, g, None, Q, 10, 64, 4, 5, W=W)


# ---------------------------------------------------------------- global consolidation (Sec. 5.2, 5.3)
def _consolidate_case(orc):
    g = _golden("consolidate_hand.json")
    pts = np.array(g["points"], dtype=np.float32)
    st = orc.Store.from_vectors(np.pad(pts, ((0, 0), (0, 2))), "l2")
    n0 = g["n0"]
    bits = orc.bitset(len(pts), g["delete"])
    return g, st, n0, bits


def test_consolidate_hand_worked(orc):
    g, st, n0, bits = _consolidate_case(orc)
    graph = np.array(g["graph"], dtype=np.uint32)
    nrep, _ = orc.consolidate(st, n0, graph, bits)
    assert graph.tolist() == g["consolidated"] and nrep == g["rewritten"]
    capped = np.array(g["graph"], dtype=np.uint32)
    orc.consolidate(st, n0, capped, bits, cap=g["R"])
    assert capped.tolist() == g["consolidated_cap3"]
    with pytest.raises(ValueError):
        orc.consolidate(st, n0, capped, bits, cap=g["R"] - 1)
    # the localized repair leaves rows with at most R/2 deleted entries alone
    loc = np.array(g["graph"], dtype=np.uint32)
    newly, rep, _ = orc.delete(st, n0, loc, orc.bitset(len(g["points"])), g["delete"])
    assert (newly, rep) == (1, 0) and loc.tolist() == g["graph"]


def test_consolidate_rows_equals_the_whole_graph_pass(orc):
    # the sampled form gives the rows of the whole pass, from the unchanged graph
    n, R = 1500, 16
    X = synth.sample("u8", n, 97)
    st = orc.Store.from_vectors(X, "l2")
    g, _ = orc.build_graph(st, R)
    bits = orc.bitset(n, np.random.default_rng(98).choice(n, n // 4, replace=False))
    only = np.random.default_rng(99).choice(n, 60, replace=False).astype(np.uint32)
    before = g.copy()
    rows, _ = orc.consolidate_rows(st, n, g, bits, only, cap=200)
    np.testing.assert_array_equal(g, before)
    orc.consolidate(st, n, g, bits, cap=200)
    np.testing.assert_array_equal(rows, g[only])


def test_reverse_edge_replay_hand_worked(orc):
    g, st, n0, bits = _consolidate_case(orc)
    rows = np.array([g["new_row"]], dtype=np.uint32)
    for tmax, want in ((n0, g["replayed"]), (1, g["replayed_tmax1"])):
        graph = np.array(g["consolidated"], dtype=np.uint32)
        orc.reverse_patch(st, graph, bits, n0, rows, tmax)
        assert graph.tolist() == want


def test_reverse_edge_replay_equals_the_insert_patch(orc):
    # replaying an insert batch's rows onto the graph the insert started from
    # gives the rows the insert itself wrote (the same requests, distances
    # recomputed)
    n0, m, R = 1500, 120, 16
    X = synth.sample("u8", n0 + m, 91)
    st = orc.Store.from_vectors(X, "l2")
    g0, _ = orc.build_graph(orc.Store.from_vectors(X[:n0], "l2"), R)
    g = np.full((n0 + m, R), orc.EMPTY, dtype=np.uint32)
    g[:n0] = g0
    orc.insert(st, n0, m, g, None, 32, 16, 9)
    r = np.full((n0 + m, R), orc.EMPTY, dtype=np.uint32)
    r[:n0] = g0
    orc.reverse_patch(st, r, None, n0, g[n0:], n0)
    np.testing.assert_array_equal(r[:n0], g[:n0])


def test_consolidation_of_every_affected_row(orc):
    # invariants on a larger graph: after 20 % deletes every live row that
    # named a deleted vertex names none (when enough live candidates exist),
    # rows without deleted entries are unchanged, deleted rows are untouched
    n, R = 2000, 16
    X = synth.sample("u8", n, 95)
    st = orc.Store.from_vectors(X, "l2")
    g, _ = orc.build_graph(st, R)
    dele = np.random.default_rng(96).choice(n, n // 5, replace=False)
    bits = orc.bitset(n, dele)
    isdel = np.zeros(n, bool)
    isdel[dele] = True
    before = g.copy()
    nrep, _ = orc.consolidate(st, n, g, bits, cap=R * R + R)
    named = np.array([(~isdel[u]) and isdel[before[u]].any() for u in range(n)])
    assert nrep == named.sum()
    np.testing.assert_array_equal(g[~named], before[~named])
    left = np.array([isdel[g[u][g[u] != orc.EMPTY]].any() for u in range(n)])
    assert left[named].mean() < 0.01
    assert (g != np.arange(n)[:, None]).all()


# ---------------------------------------------------------------- insert (Sec. 5.1)
def test_insert_invariants_and_read_after_write(orc):
    n0, m, R = 1500, 200, 16
    X = synth.sample("tiny", n0 + m, 71)
    st = orc.Store.from_vectors(X, "l2")
    g0, _ = orc.build_graph(orc.Store.from_vectors(X[:n0], "l2"), R)
    g = np.full((n0 + m, R), orc.EMPTY, dtype=np.uint32)
    g[:n0] = g0
    orc.insert(st, n0, m, g, None, 32, 16, 9)
    H = R // 2
    np.testing.assert_array_equal(g[:n0, :H], g0[:, :H])  # head halves untouched
    for v in range(n0 + m):
        live = g[v][g[v] != orc.EMPTY]
        assert len(set(live.tolist())) == len(live) and v not in live
        assert np.all(live < n0 + m)
    assert np.all(g[n0:] < n0)  # new rows point at old vertices only
    # read-after-write (the paper's consistency test searches for the vector
    # just inserted): most new vectors are found at rank 1 once linked in
    r = orc.search(st, n0 + m, g, None, X[n0:], 1, 64, 32, 5)
    assert np.mean(r["ids"][:, 0] == np.arange(n0, n0 + m)) >= 0.8


def test_insert_reverse_tail_is_sorted_best(orc):
    n0, m, R = 800, 50, 8
    X = synth.sample("tiny", n0 + m, 81)
    st = orc.Store.from_vectors(X, "l2")
    g0, _ = orc.build_graph(orc.Store.from_vectors(X[:n0], "l2"), R)
    g = np.full((n0 + m, R), orc.EMPTY, dtype=np.uint32)
    g[:n0] = g0
    orc.insert(st, n0, m, g, None, 16, 8, 2)
    H = R // 2
    changed = np.where((g[:n0] != g0).any(1))[0]
    assert len(changed) > 0
    for u in changed:
        chosen = [v for v in range(n0, n0 + m) if u in g[v]]
        pool = [t for t in g0[u, H:] if t != orc.EMPTY] + chosen
        d = ((X[pool].astype(np.float64) - X[u]) ** 2).sum(1)
        best = np.array(pool)[np.lexsort((pool, d))][:R - H]
        np.testing.assert_array_equal(g[u, H:H + len(best)], best)


# ---------------------------------------------------------------- delete (Sec. 5.2)
def test_delete_validation_and_counting(orc):
    X = synth.sample("tiny", 300, 91)
    st = orc.Store.from_vectors(X, "l2")
    g, _ = orc.build_graph(st, 8)
    bits = orc.bitset(300)
    g_before, b_before = g.copy(), bits.copy()
    newly, _, _ = orc.delete(st, 300, g, bits, [5, 300])
    assert newly == -1
    np.testing.assert_array_equal(g, g_before)
    np.testing.assert_array_equal(bits, b_before)
    newly, _, _ = orc.delete(st, 300, g, bits, [5, 6, 5])
    assert newly == 2
    newly, _, _ = orc.delete(st, 300, g, bits, [6, 7])
    assert newly == 1
    assert orc.deleted_ids(bits, 300).tolist() == [5, 6, 7]


def test_delete_repair_hand_worked(orc):
    g = _golden("repair_hand.json")
    X = np.array(g["points"], dtype=np.float32)
    X = np.pad(X, ((0, 0), (0, 2)))
    st = orc.Store.from_vectors(X, "l2")
    graph = np.array(g["graph"], dtype=np.uint32)
    bits = orc.bitset(len(X))
    newly, rep, _ = orc.delete(st, len(X), graph, bits, g["delete"], c=g["c"])
    assert newly == len(g["delete"]) and rep == g["repaired"]
    assert graph[g["vertex"]].tolist() == g["expected_row"]


def test_delete_repair_threshold_and_search(orc):
    n, R = 3000, 16
    X = synth.sample("tiny", n, 101)
    st = orc.Store.from_vectors(X, "l2")
    g, _ = orc.build_graph(st, R)
    bits = orc.bitset(n)
    dels = synth.pick_live_ids(n, None, 900, 102)
    before = g.copy()
    newly, rep, _ = orc.delete(st, n, g, bits, dels)
    assert newly == 900
    isdel = np.zeros(n, bool)
    isdel[dels] = True
    nd_before = isdel[before].sum(1)
    hit = (~isdel) & (2 * nd_before > R)
    assert rep == hit.sum() > 0
    np.testing.assert_array_equal(g[~hit], before[~hit])  # only V^L rows change
    nd_after = isdel[g[hit]].sum(1)
    assert np.all(nd_after <= R // 2)
    r = orc.search(st, n, g, bits, synth.sample("tiny", 50, 103), 10, 64, 32, 4)
    assert not np.isin(r["ids"], dels).any()


# ---------------------------------------------------------------- learned stop
def _net(rng, scale=0.3):
    return orc_mod().MLP(rng.standard_normal((64, 16)) * scale, rng.standard_normal(64) * 0.1,
                         rng.standard_normal(64) * scale, 0.05)


def orc_mod():
    import oracle
    return oracle


def test_mlp_gradient_finite_differences(orc):
    rng = np.random.default_rng(3)
    net = _net(rng)
    F = rng.standard_normal((64, 16))
    y = (rng.random(64) < 0.5).astype(np.float64)
    loss, grad = orc.mlp_backward(net, F, y)
    z, p = orc.mlp_forward(net, F)
    want = np.mean(np.logaddexp(0, z) - y * z)
    assert abs(loss - want) < 1e-12
    eps = 1e-6
    for name, shape in [("W1", (64, 16)), ("b1", (64,)), ("w2", (64,))]:
        arr = getattr(net, name)
        for idx in [tuple(rng.integers(0, s) for s in shape) for _ in range(12)]:
            old = arr[idx]
            arr[idx] = old + eps
            lp, _ = orc.mlp_backward(net, F, y)
            arr[idx] = old - eps
            lm, _ = orc.mlp_backward(net, F, y)
            arr[idx] = old
            assert abs((lp - lm) / (2 * eps) - grad[name][idx]) < 1e-6
    old = net.b2
    net.b2 = old + eps
    lp, _ = orc.mlp_backward(net, F, y)
    net.b2 = old - eps
    lm, _ = orc.mlp_backward(net, F, y)
    net.b2 = old
    assert abs((lp - lm) / (2 * eps) - grad["b2"]) < 1e-6


def test_mlp_learns_separable_toy(orc):
    rng = np.random.default_rng(4)
    net = _net(rng, 0.1)
    F = rng.standard_normal((512, 16))
    y = (F[:, 3] + 0.5 * F[:, 7] > 0).astype(np.float64)
    loss0, _ = orc.mlp_backward(net, F, y)
    for _ in range(400):
        loss, g = orc.mlp_backward(net, F, y)
        net.W1 -= 0.5 * g["W1"]
        net.b1 -= 0.5 * g["b1"]
        net.w2 -= 0.5 * g["w2"]
        net.b2 -= 0.5 * g["b2"]
    assert loss < 0.1 < loss0


def test_stop_extremes_reduce_to_fixed_T(orc):
    n = 2000
    X = synth.sample("tiny", n, 111)
    st = orc.Store.from_vectors(X, "l2")
    g, _ = orc.build_graph(st, 16)
    Q = synth.sample("tiny", 40, 112)
    never = orc.MLP(np.zeros((64, 16)), np.zeros(64), np.zeros(64), -50.0)
    always = orc.MLP(np.zeros((64, 16)), np.zeros(64), np.zeros(64), 50.0)
    plain = orc.search(st, n, g, None, Q, 10, 64, 32, 1)
    r = orc.search_ex(st, n, g, None, Q, 10, 64, 32, 1, net=never, tau=0.5, t_min=4)
    np.testing.assert_array_equal(r["ids"], plain["ids"])
    assert np.all(r["stop_iter"] == -1)
    short = orc.search(st, n, g, None, Q, 10, 64, 6, 1)
    r = orc.search_ex(st, n, g, None, Q, 10, 64, 32, 1, net=always, tau=0.5, t_min=6)
    np.testing.assert_array_equal(r["ids"], short["ids"])
    assert np.all(r["stop_iter"] == 6)
    # evaluated every 4 iterations from t_min = 5: first chance after 5
    r = orc.search_ex(st, n, g, None, Q, 10, 64, 32, 1, net=always, tau=0.5, t_min=5, t_every=4)
    assert np.all(r["stop_iter"] == 5)
    # a network that says "stop" only from t+1 >= 7 (b2 + 10 f0 with T=10),
    # evaluated at 4, 7, 10: stops at 7
    W1 = np.zeros((64, 16))
    W1[0, 0] = 10.0
    w2 = np.zeros(64)
    w2[0] = 1.0
    ramp = orc.MLP(W1, np.zeros(64), w2, -6.5)
    r = orc.search_ex(st, n, g, None, Q, 10, 64, 10, 1, net=ramp, tau=0.5, t_min=4, t_every=3)
    assert np.all(r["stop_iter"] == 7)


def test_trace_features_and_labels(orc):
    n = 2000
    X = synth.sample("tiny", n, 121)
    st = orc.Store.from_vectors(X, "l2")
    g, _ = orc.build_graph(st, 16)
    Q = synth.sample("tiny", 20, 122)
    T = 32
    r = orc.search_ex(st, n, g, None, Q, 10, 64, T, 1, trace=True)
    plain = orc.search(st, n, g, None, Q, 10, 64, T, 1)
    np.testing.assert_array_equal(r["ids"], plain["ids"])
    for qi in range(20):
        nf = r["n_feat"][qi]
        f = r["feat"][qi, :nf]
        np.testing.assert_allclose(f[:, 0], np.arange(1, nf + 1) / T)
        assert np.all(f[:, 1] >= 0) and np.all(np.diff(f[:, 1]) >= -1e-12)   # best only improves
        assert np.all(f[:, 2] >= 0) and np.all(f[:, 3] >= f[:, 2])
        assert np.all(f[:, 12] >= -1e-12)                                    # d_k never rises
        np.testing.assert_allclose(f[:, 7] + f[:, 10], np.minimum(64, f[:, 7] * 64 + f[:, 10] * 64) / 64)
        # the top-k at the last change equals the final one: a search cut at
        # t_last + 1 iterations returns the same ids
        tl = r["t_last"][qi]
        cut = orc.search(st, n, g, None, Q[qi:qi + 1], 10, 64, tl + 1, 1)
        assert set(cut["ids"][0]) == set(plain["ids"][qi])
        if tl >= 1:
            cut = orc.search(st, n, g, None, Q[qi:qi + 1], 10, 64, tl, 1)
            assert set(cut["ids"][0]) != set(plain["ids"][qi])


def test_trace_features_hand_worked(orc):
    """All 16 learned-stop features of a hand-worked trace on the 12-point
    line graph (f5 population std, f6 admitted over R, f8 new top-k ids, f9
    iterations since the last top-k change, f11 parent rank, f13 drop of d1,
    f14 next parent against dk, f15 the running average of f6)."""
    line = _golden("search_wparents_hand.json")
    g = _golden("search_trace_hand.json")
    n = line["n"]
    X = np.zeros((n, 4), dtype=np.float32)
    X[:, 0] = np.arange(n)
    st = orc.Store.from_vectors(X, "l2")
    graph = np.array(line["graph"], dtype=np.uint32)
    q = np.array([line["query"]], dtype=np.float32)
    r = orc.search_ex(st, n, graph, None, q, g["k"], g["L"], g["T"], g["seed"], trace=True)
    assert r["n_feat"][0] == g["n_feat"] and r["t_last"][0] == g["t_last"]
    want = np.array(g["feat"])
    np.testing.assert_allclose(r["feat"][0, :g["n_feat"]], want, rtol=1e-12, atol=1e-14)
    assert not r["feat"][0, g["n_feat"]:].any()
    # the pools the features were read from
    for t, pool in enumerate(g["pool_after"]):
        p = orc.search(st, n, graph, None, q, g["L"], g["L"], t + 1, g["seed"], want_pool=True)
        assert p["pool_ids"][0].tolist() == pool
    # label y_t = (t >= t_last): a search cut after t_last + 1 iterations has the final top k
    full = orc.search(st, n, graph, None, q, g["k"], g["L"], g["T"], g["seed"])
    cut = orc.search(st, n, graph, None, q, g["k"], g["L"], g["t_last"] + 1, g["seed"])
    assert cut["ids"].tolist() == full["ids"].tolist()


# ---------------------------------------------------------------- WAVP (Sec. 4.3, Eq. 2, Alg. 2)
@pytest.mark.parametrize("case", [0, 1])
def test_wavp_round_hand_worked(orc, case):
    """One maintenance round worked by hand: candidate order by descending
    F_lambda with an id tie, an empty slot taken first, referenced slots
    passed over and cleared, a victim tie decided by slot, and (case 1) the
    second sweep when too few slots were unreferenced."""
    g = _golden("wavp_round_hand.json")
    c = g["cases"][case]
    n, M = c["n"], c["M"]
    owner = np.array(c["owner"], dtype=np.int32)
    ref = np.array(c["ref"], dtype=np.uint8)
    map_ = np.full(n, -1, dtype=np.int32)
    for s, o in enumerate(owner):
        if o >= 0:
            map_[o] = s
    freq = np.zeros(n, dtype=np.uint32)
    for x, f in c["freq"].items():
        freq[int(x)] = f
    ein = np.zeros(n, dtype=np.uint32)
    for x, e in c["ein"].items():
        ein[int(x)] = e
    p, e = orc.wavp_round(map_, owner, ref, freq, ein, c["queue"], c["B"], c["hand"], c["W"], g["alpha"], g["beta"])
    assert (p, e) == (c["promoted"], c["evicted"])
    assert owner.tolist() == c["owner_after"]
    assert ref.tolist() == c["ref_after"]
    want = np.full(n, -1, dtype=np.int32)
    for x, s in c["mapped_after"].items():
        want[int(x)] = s
    np.testing.assert_array_equal(map_, want)
