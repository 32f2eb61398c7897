"""Serving form: tiered store (device cache over pinned host rows with WAVP
placement) and the continuous-batching request loop (C ABI)."""
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


def built(svf, mix, n, n_cap, R=32, metric="l2", seed=701, max_batch=None, lowp=()):
    X = synth.sample(mix, n_cap, seed)
    ix = svf.Index(X.shape[1], n_cap, dtype="u8" if X.dtype == np.uint8 else "f32", metric=metric, R=R,
                   max_batch=max_batch or n, lowp=lowp)
    ix.build(torch.from_numpy(X[:n]).cuda())
    return X, ix


def test_tiered_search_equals_device_search(svf):
    X, ix = built(svf, "u8", 6000, 6000, R=64)
    Q = torch.from_numpy(synth.sample("u8", 500, 702)).cuda()
    cfg = svf.SearchConfig(k=10, L=64, T=48, seed=3)
    ids0, d0 = ix.search(Q, cfg)
    ix.enable_tier(M=600, theta0=0.5, promote_batch=256, sweep=4, qcap=4096)
    ix.release_device_store()
    ix.stats_reset()
    ids1, d1 = ix.search(Q, cfg)
    assert torch.equal(ids0, ids1) and torch.equal(d0, d1)
    s = ix.stats()
    assert s["cache_hits"] > 0 and s["cache_misses"] > 0
    promoted = ix.maintain()
    assert promoted > 0
    assert int((ix.tier_map()[:6000] >= 0).sum().item()) == 600
    ids2, d2 = ix.search(Q, cfg)
    assert torch.equal(ids0, ids2) and torch.equal(d0, d2)


def test_tiered_multi_warp_and_rerank_equal_device_search(svf):
    # several warps per query over the tiered store: traversal rows (fp32) and
    # re-rank rows (fp8 traversal resident) read through the cache give the
    # results of the device-resident store, and the cache counters see them
    X, ix = built(svf, "unit96", 6000, 6000, R=32, metric="ip", lowp=("fp8",))
    Q = torch.from_numpy(synth.sample("unit96", 300, 703)).cuda()
    cfgs = [svf.SearchConfig(k=10, L=64, T=10, seed=3, W=4),
            svf.SearchConfig(k=10, L=64, T=8, seed=3, W=8, precision="fp8", rerank=True)]
    want = [ix.search(Q, c) for c in cfgs]
    ix.enable_tier(M=600, theta0=0.5, promote_batch=256, sweep=4, qcap=4096)
    ix.release_device_store()
    for c, (i0, d0) in zip(cfgs, want):
        ix.stats_reset()
        i1, d1 = ix.search(Q, c)
        assert torch.equal(i0, i1) and torch.equal(d0, d1)
        s = ix.stats()
        assert s["cache_hits"] > 0 and s["cache_misses"] > 0


def test_promotion_follows_a_skewed_workload(svf):
    """Queries from one mixture component: the rows they touch get promoted
    and the hit rate of the same workload rises (Eq. 2 / Alg. 2 at work)."""
    lab = []
    X = synth.sample("tiny", 8000, 741, labels_out=lab)
    ix = svf.Index(128, 8000, dtype="f32", metric="l2", R=32, max_batch=8000)
    ix.build(torch.from_numpy(X).cuda())
    ql = []
    Qall = synth.sample("tiny", 4000, 742, labels_out=ql)
    Q = torch.from_numpy(Qall[ql[0] == 3]).cuda()
    cfg = svf.SearchConfig(k=10, L=64, T=32)
    ids0, d0 = ix.search(Q, cfg)
    ix.enable_tier(M=1200, theta0=1.0, promote_batch=512, sweep=4, qcap=8192)
    ix.release_device_store()

    def hit_rate():
        ix.stats_reset()
        ids, d = ix.search(Q, cfg)
        assert torch.equal(ids, ids0) and torch.equal(d, d0)
        s = ix.stats()
        return s["cache_hits"] / (s["cache_hits"] + s["cache_misses"])

    r0 = hit_rate()
    for _ in range(4):
        ix.maintain()
        r = hit_rate()
    assert r > r0 + 0.2, (r0, r)


def test_tiered_updates_equal_device_updates(svf):
    X, a = built(svf, "u8", 3000, 3600, R=32, max_batch=3000)
    _, b = built(svf, "u8", 3000, 3600, R=32, max_batch=3000)
    b.enable_tier(M=300, theta0=0.5, promote_batch=128, qcap=2048)
    b.release_device_store()
    Q = torch.from_numpy(synth.sample("u8", 200, 711)).cuda()
    cfg = svf.SearchConfig(k=10, L=64, T=32)
    for step in range(3):
        xi = torch.from_numpy(X[3000 + 200 * step:3200 + 200 * step]).cuda()
        a.insert(xi, L_ins=64, T_ins=32)
        b.insert(xi, L_ins=64, T_ins=32)
        dels = torch.from_numpy(synth.pick_live_ids(a.n_used, None, 150, 712 + step).view(np.int32)).cuda()
        assert a.delete(dels) == b.delete(dels)
        b.maintain()
        assert torch.equal(a.graph[:a.n_used], b.graph[:b.n_used])
        ia, da = a.search(Q, cfg)
        ib, db = b.search(Q, cfg)
        assert torch.equal(ia, ib) and torch.equal(da, db)


@pytest.mark.parametrize("ein_mode", ["freq", "indegree"])
def test_wavp_round_matches_oracle(svf, orc, ein_mode):
    n, M = 4000, 256
    X, ix = built(svf, "u8", n, n, R=32)
    ix.enable_tier(M=M, theta0=1e9, promote_batch=64, sweep=4, qcap=1024)
    rng = np.random.default_rng(721)
    # a crafted state: 200 cached ids, some referenced slots, a queue of 150
    owner = np.full(M, -1, np.int32)
    cached = rng.choice(n, 200, replace=False)
    slots = rng.choice(M, 200, replace=False)
    owner[slots] = cached
    map_ = np.full(n, -1, np.int32)
    map_[cached] = slots
    ref = (rng.random(M) < 0.3).astype(np.uint8)
    if ein_mode == "freq":
        freq = rng.permutation(n).astype(np.uint32)   # distinct F, exact in fp32 and fp64
        ein = np.zeros(n, np.uint32)
    else:
        freq = np.zeros(n, np.uint32)
        ein = rng.integers(0, 60, n).astype(np.uint32)
    queue = rng.choice(np.setdiff1d(np.arange(n), cached), 150, replace=False).astype(np.uint32)
    tb = ix.tier_bufs
    tb["owner"][:M * 4].view(torch.int32).copy_(torch.from_numpy(owner))
    tb["map"][:n * 4].view(torch.int32).copy_(torch.from_numpy(map_))
    tb["ref"][:M].copy_(torch.from_numpy(ref))
    fq = freq.copy()
    fq[queue] |= np.uint32(1 << 31)  # queued ids carry the queued flag
    tb["freq"][:n * 4].view(torch.int32).copy_(torch.from_numpy(fq.view(np.int32)))
    tb["ein"][:n * 4].view(torch.int32).copy_(torch.from_numpy(ein.view(np.int32)))
    tb["queue"][:150 * 4].view(torch.int32).copy_(torch.from_numpy(queue.view(np.int32)))
    ix.status.view(torch.int64)[11] = 150
    torch.cuda.synchronize()
    got = ix.maintain()
    p, e = orc.wavp_round(map_, owner, ref, freq, ein, queue, 64, 0, 256, 0.6, 0.4)
    assert got == p
    np.testing.assert_array_equal(tb["owner"][:M * 4].view(torch.int32).cpu().numpy(), owner)
    np.testing.assert_array_equal(tb["map"][:n * 4].view(torch.int32).cpu().numpy(), map_)
    np.testing.assert_array_equal(tb["ref"][:M].cpu().numpy(), ref)
    # queued flags cleared, counts kept; the cache holds the host rows
    f = tb["freq"][:n * 4].view(torch.int32).cpu().numpy().view(np.uint32)
    np.testing.assert_array_equal(f, freq)
    cache = tb["cache"][:M * 128].view(M, 128).cpu().numpy()
    promoted_slots = np.where(np.isin(owner, queue))[0]
    assert len(promoted_slots) == p
    for s in promoted_slots:
        np.testing.assert_array_equal(cache[s], X[owner[s]])


def _trace(rng, n_req, n_start, X, n_base):
    """A mixed request stream: search batches log-uniform in [1, 256],
    inserts and deletes (roughly 90:9:1)."""
    reqs, n_used, nxt = [], n_base, n_base
    for i in range(n_req):
        u = rng.random()
        if u < 0.09 and nxt + 100 <= len(X):
            reqs.append(("insert", nxt, 100))
            nxt += 100
        elif u < 0.10:
            reqs.append(("delete", int(rng.integers(0, 1 << 30)), 40))
        else:
            reqs.append(("search", int(rng.integers(0, 1 << 30)), int(np.exp(rng.uniform(0, np.log(256))))))
    return reqs


def _serve_trace(svf, ix, X, n0, reqs, cfg, consistency, **kw):
    """Submit the trace at once (so searches and updates overlap), drain, and
    return the completions, the search outputs and the update inputs."""
    srv = svf.Server(ix, max_inflight=6, n_streams=4, maintain_every=4, consistency=consistency, **kw)
    outs, dev_inputs = {}, []
    deleted = set()
    n_used = n0
    for tag, (op, a, b) in enumerate(reqs):
        if op == "search":
            Q = torch.from_numpy(synth.sample("u8", b, 10_000 + tag)).cuda()
            oi = torch.empty((b, 10), dtype=torch.int32, device="cuda")
            od = torch.empty((b, 10), dtype=torch.int32, device="cuda")
            srv.search(tag, Q, cfg, oi, od)
            outs[tag] = (Q, oi, od)
        elif op == "insert":
            xi = torch.from_numpy(X[a:a + b]).cuda()
            srv.insert(tag, xi, L_ins=64, T_ins=32)
            dev_inputs.append((tag, "insert", xi))
            n_used += b
        else:
            ids = synth.pick_live_ids(n_used, np.array(sorted(deleted), np.int64), b, a)
            deleted.update(ids.tolist())
            di = torch.from_numpy(ids.view(np.int32)).cuda()
            srv.delete(tag, di)
            dev_inputs.append((tag, "delete", di))
    srv.drain(300)
    comps = {c["tag"]: c for c in srv.poll(10000)}
    srv.stop()
    assert len(comps) == len(reqs) and all(c["status"] == 0 for c in comps.values())
    return comps, outs, {t: (k, v) for t, k, v in dev_inputs}, n_used


def _check_epochs(reqs, comps, consistency):
    """Update E completes with epoch E (submission order).  A search's epoch
    is every update submitted before it (barrier, read-after-write) or, in the
    snapshot mode, at most that.  Returns {epoch: [search tags]}."""
    by_epoch, submitted = {}, 0
    for tag, (op, a, b) in enumerate(reqs):
        c = comps[tag]
        assert c["t_done"] >= c["t_start"] > 0
        if op == "search":
            if consistency == "snapshot":
                assert c["epoch"] <= submitted
            else:
                assert c["epoch"] == submitted, (tag, c["epoch"], submitted)
            by_epoch.setdefault(c["epoch"], []).append(tag)
        else:
            submitted += 1
            assert c["epoch"] == submitted
    return by_epoch


def _overlaps(reqs, comps):
    """Searches of an older epoch whose host interval overlapped an update."""
    n = 0
    ups = [comps[t] for t, r in enumerate(reqs) if r[0] != "search"]
    for t, r in enumerate(reqs):
        if r[0] != "search":
            continue
        c = comps[t]
        n += any(u["epoch"] > c["epoch"] and u["t_start"] < c["t_done"] and c["t_start"] < u["t_done"] for u in ups)
    return n


@pytest.mark.parametrize("consistency,tiered", [("barrier", False), ("barrier", True), ("read-after-write", False),
                                                 ("snapshot", False), ("snapshot", True)])
def test_server_results_equal_alone(svf, consistency, tiered):
    """Each search served in the mix equals the same search run alone on the
    index state of its epoch; updates advance the epoch in submission order.
    In the versioned modes updates overlap searches of older epochs, which
    read the rows the update rewrites from their shadows."""
    n0, ncap = 8000, 12000
    X, ix = built(svf, "u8", n0, ncap, R=32, max_batch=8000)
    _, ref_ix = built(svf, "u8", n0, ncap, R=32, max_batch=8000)
    if tiered:
        ix.enable_tier(M=1500, theta0=0.5, promote_batch=256, qcap=4096)
        ix.release_device_store()
    rng = np.random.default_rng(731)
    reqs = _trace(rng, 120, n0, X, n0)
    cfg = svf.SearchConfig(k=10, L=64, T=32)
    comps, outs, upd, n_used = _serve_trace(svf, ix, X, n0, reqs, cfg, consistency)
    by_epoch = _check_epochs(reqs, comps, consistency)
    # replay alone, in order, each search at its epoch
    epoch = 0
    for tag, (op, a, b) in enumerate(reqs + [("end", 0, 0)]):
        if op == "search":
            continue
        for t in by_epoch.pop(epoch, []):
            Q, oi, od = outs[t]
            ri, rd = ref_ix.search(Q, cfg)
            assert torch.equal(ri, oi) and torch.equal(rd, od), f"request {t} at epoch {epoch}"
        if op == "end":
            break
        kind, v = upd[tag]
        if kind == "insert":
            ref_ix.insert(v, L_ins=64, T_ins=32)
        else:
            ref_ix.delete(v)
        epoch += 1
    assert not by_epoch
    torch.cuda.synchronize()
    assert torch.equal(ix.graph[:n_used], ref_ix.graph[:n_used])
    if consistency != "barrier":
        assert _overlaps(reqs, comps) > 0, "no update overlapped an older search"


@pytest.mark.parametrize("consistency", ["read-after-write", "snapshot"])
def test_served_searches_match_oracle_at_their_epochs(svf, orc, consistency):
    """Oracle replay of the served stream: the FP64 oracle applies the same
    inserts and deletes in submission order (Sec. 5.1, 5.2) and searches
    every served batch on the index state of its epoch; uint8 data, so ids
    and distances agree bit for bit."""
    n0, ncap = 6000, 9000
    X, ix = built(svf, "u8", n0, ncap, R=32, max_batch=6000)
    g = np.full((ncap, 32), orc.EMPTY, dtype=np.uint32)
    g[:n0] = P.as_u32(ix.graph[:n0].cpu().numpy())
    st = orc.Store.from_vectors(X, "l2")
    bits = orc.bitset(ncap)
    rng = np.random.default_rng(741)
    reqs = _trace(rng, 100, n0, X, n0)
    cfg = svf.SearchConfig(k=10, L=64, T=32)
    comps, outs, upd, n_used = _serve_trace(svf, ix, X, n0, reqs, cfg, consistency)
    by_epoch = _check_epochs(reqs, comps, consistency)
    seed = ix.params.seed
    n, epoch, checked = n0, 0, 0
    for tag, (op, a, b) in enumerate(reqs + [("end", 0, 0)]):
        if op == "search":
            continue
        for t in by_epoch.pop(epoch, []):
            Q, oi, od = outs[t]
            o = orc.search(st, n, g, bits, Q.cpu().numpy(), 10, 64, 32, seed)
            P.check_exact(oi.cpu().numpy(), od.cpu().numpy(), o)
            checked += 1
        if op == "end":
            break
        kind, v = upd[tag]
        if kind == "insert":
            orc.insert(st, n, b, g, bits, 64, 32, seed)
            n += b
        else:
            orc.delete(st, n, g, bits, v.cpu().numpy().view(np.uint32))
        epoch += 1
    assert not by_epoch and checked > 50
    np.testing.assert_array_equal(P.as_u32(ix.graph[:n].cpu().numpy()), g[:n])


def test_tiered_lowp_rerank_equals_device(svf):
    """BF16/FP8 copies stay whole in device memory; the exact re-rank reads
    the fp32 rows through the tier: results equal the untiered index, before
    and after inserts (their low-precision rows are encoded from the input)."""
    X = synth.sample("unit96", 5000, 751)
    a = svf.Index(96, 5000, dtype="f32", metric="ip", R=32, lowp=("fp8",), max_batch=4000)
    b = svf.Index(96, 5000, dtype="f32", metric="ip", R=32, lowp=("fp8",), max_batch=4000)
    for ix in (a, b):
        ix.build(torch.from_numpy(X[:4000]).cuda())
    b.enable_tier(M=400, theta0=0.5, promote_batch=128, qcap=2048)
    b.release_device_store()
    Q = torch.from_numpy(synth.sample("unit96", 300, 752)).cuda()
    cfg = svf.SearchConfig(k=10, L=64, T=48, precision="fp8", rerank=True)
    for step in range(2):
        ia, da = a.search(Q, cfg)
        ib, db = b.search(Q, cfg)
        assert torch.equal(ia, ib) and torch.equal(da, db)
        xi = torch.from_numpy(X[4000 + 500 * step:4500 + 500 * step]).cuda()
        a.insert(xi)
        b.insert(xi)
        b.maintain()
    assert torch.equal(a.vecs_fp8[:5000 * 128], b.vecs_fp8[:5000 * 128])


# ---------------------------------------------------------------- placement-policy ablations
def _clock_round(map_, owner, ref, queue, B, hand, W):
    """CLOCK (recency only): the first B queued ids in queue order go into
    the unreferenced slots the clock meets first (empty slots before owned
    ones); referenced slots lose their bit; a second pass over the window
    when too few were unreferenced."""
    M = len(owner)
    B, W = min(B, len(queue)), min(W, M)

    def collect():
        keys = []
        for i in range(W):
            s = (hand + i) % M
            if ref[s]:
                ref[s] = 0
                continue
            keys.append((0 if owner[s] < 0 else i + 1, s))
        return keys

    keys = collect()
    if len(keys) < B:
        keys = collect()
    victims = [s for _, s in sorted(keys)][:B]
    for x, s in zip(queue[:B], victims):
        if owner[s] >= 0:
            map_[owner[s]] = -1
        owner[s], map_[x], ref[s] = x, s, 1
    return min(B, len(victims))


@pytest.mark.parametrize("policy", ["clock", "lfu", "static"])
def test_policy_round(svf, orc, policy):
    n, M, B = 4000, 256, 64
    X, ix = built(svf, "u8", n, n, R=32)
    ix.enable_tier(M=M, theta0=1e9, promote_batch=B, sweep=4, qcap=1024)
    ix.reset_tier(M=M, theta0=1e9, promote_batch=B, sweep=4, qcap=1024, policy=policy)  # re-tier under the policy
    rng = np.random.default_rng(731)
    owner = np.full(M, -1, np.int32)
    cached = rng.choice(n, 220, replace=False)
    slots = rng.choice(M, 220, replace=False)
    owner[slots] = cached
    map_ = np.full(n, -1, np.int32)
    map_[cached] = slots
    ref = (rng.random(M) < 0.4).astype(np.uint8)
    freq = rng.permutation(n).astype(np.uint32)
    ein = rng.integers(0, 60, n).astype(np.uint32)  # ignored by clock and lfu
    queue = rng.choice(np.setdiff1d(np.arange(n), cached), 150, replace=False).astype(np.uint32)
    tb = ix.tier_bufs
    tb["owner"][:M * 4].view(torch.int32).copy_(torch.from_numpy(owner))
    tb["map"][:n * 4].view(torch.int32).copy_(torch.from_numpy(map_))
    tb["ref"][:M].copy_(torch.from_numpy(ref))
    fq = freq.copy()
    fq[queue] |= np.uint32(1 << 31)
    tb["freq"][:n * 4].view(torch.int32).copy_(torch.from_numpy(fq.view(np.int32)))
    tb["ein"][:n * 4].view(torch.int32).copy_(torch.from_numpy(ein.view(np.int32)))
    tb["queue"][:150 * 4].view(torch.int32).copy_(torch.from_numpy(queue.view(np.int32)))
    ix.status.view(torch.int64)[11] = 150
    torch.cuda.synchronize()
    got = ix.maintain()
    if policy == "static":
        want = 0
    elif policy == "lfu":
        want, _ = orc.wavp_round(map_, owner, ref, freq, ein, queue, B, 0, 4 * B, 1.0, 0.0)  # F_recent alone
    else:
        want = _clock_round(map_, owner, ref, queue, B, 0, 4 * B)
    assert got == want
    np.testing.assert_array_equal(tb["owner"][:M * 4].view(torch.int32).cpu().numpy(), owner)
    np.testing.assert_array_equal(tb["map"][:n * 4].view(torch.int32).cpu().numpy(), map_)
    np.testing.assert_array_equal(tb["ref"][:M].cpu().numpy(), ref)
    cache = tb["cache"][:M * 128].view(M, 128).cpu().numpy()
    for s in np.where(np.isin(owner, queue))[0]:
        np.testing.assert_array_equal(cache[s], X[owner[s]])


@pytest.mark.parametrize("policy,queued", [("clock", True), ("static", False), ("wavp", False)])
def test_policy_admission_on_misses(svf, policy, queued):
    """With a threshold no miss reaches, WAVP queues nothing; CLOCK queues every
    missed row regardless; STATIC never queues.  Results stay those of the
    untiered store."""
    X, ix = built(svf, "u8", 6000, 6000, R=32)
    Q = torch.from_numpy(synth.sample("u8", 300, 741)).cuda()
    cfg = svf.SearchConfig(k=10, L=64, T=32, seed=3)
    ia, da = ix.search(Q, cfg)
    ix.enable_tier(M=500, theta0=1e9, promote_batch=256, sweep=4, qcap=4096, policy=policy)
    ib, db = ix.search(Q, cfg)
    torch.cuda.synchronize()
    assert torch.equal(ia, ib) and torch.equal(da, db)
    assert ix.stats()["cache_misses"] > 0
    assert (int(ix.status.view(torch.int64)[11]) > 0) == queued


@pytest.mark.parametrize("policy", ["lru", "lrfu"])
def test_recency_policy_round(svf, policy):
    """LRU / LRFU (the paper's Sec. 6.3 baselines): every queued miss is a
    candidate, in miss order; the victims are the window's slots with the
    oldest last hit (LRU) or the lowest C after folding the round's hits,
    C <- C / 2 + hits with lambda = 1 (LRFU); an empty slot first, ties by
    slot.  Checked against a plain host reference of the round."""
    n, M, B = 4000, 256, 64
    X, ix = built(svf, "u8", n, n, R=32)
    ix.enable_tier(M=M, promote_batch=B, sweep=4, qcap=1024)
    ix.reset_tier(M=M, promote_batch=B, sweep=4, qcap=1024, policy=policy, lrfu_lambda=1.0)
    rng = np.random.default_rng(733)
    owner = np.full(M, -1, np.int32)
    cached = rng.choice(n, 230, replace=False)
    slots = rng.choice(M, 230, replace=False)
    owner[slots] = cached
    map_ = np.full(n, -1, np.int32)
    map_[cached] = slots
    stat = np.zeros((M, 2), np.uint32)
    if policy == "lru":
        stat[:, 0] = rng.permutation(M).astype(np.uint32) + 1       # distinct last-hit stamps
        stat[slots[:20], 0] = 7                                      # a tie, decided by slot
    else:
        stat[:, 0] = rng.integers(0, 4, M).astype(np.uint32)        # hits of the round
        stat[:, 1] = (rng.integers(0, 16, M) * 0.25).astype(np.float32).view(np.uint32)  # C, exact halves
    queue = rng.choice(np.setdiff1d(np.arange(n), cached), 150, replace=False).astype(np.uint32)
    tb = ix.tier_bufs
    tb["owner"][:M * 4].view(torch.int32).copy_(torch.from_numpy(owner))
    tb["map"][:n * 4].view(torch.int32).copy_(torch.from_numpy(map_))
    tb["slot_stat"][:M * 8].view(torch.int32).copy_(torch.from_numpy(stat.view(np.int32).reshape(-1)))
    fq = np.zeros(n, np.uint32)
    fq[queue] = np.uint32(1 << 31) | np.uint32(1)
    tb["freq"][:n * 4].view(torch.int32).copy_(torch.from_numpy(fq.view(np.int32)))
    tb["queue"][:150 * 4].view(torch.int32).copy_(torch.from_numpy(queue.view(np.int32)))
    ix.status.view(torch.int64)[11] = 150
    torch.cuda.synchronize()
    got = ix.maintain()
    # host reference of the round (window = 4 * B slots from hand 0)
    if policy == "lrfu":
        c = stat[:, 1].view(np.float32) * np.float32(0.5) + stat[:, 0].astype(np.float32)
        stat[:, 1] = c.astype(np.float32).view(np.uint32)
        stat[:, 0] = 0
    keys = []
    for s in range(4 * B):
        if owner[s] < 0:
            k = -1.0
        else:
            k = float(stat[s, 0]) if policy == "lru" else float(stat[s, 1:2].view(np.float32)[0])
        keys.append((k, s))
    victims = [s for _, s in sorted(keys)][:B]
    for x, s in zip(queue[:B], victims):
        if owner[s] >= 0:
            map_[owner[s]] = -1
        owner[s], map_[x] = x, s
        if policy == "lru":
            stat[s, 0] = 0  # this round's tick: no call has read the tier since the reset
        else:
            stat[s] = (0, np.float32(1.0).view(np.uint32))
    assert got == B
    np.testing.assert_array_equal(tb["owner"][:M * 4].view(torch.int32).cpu().numpy(), owner)
    np.testing.assert_array_equal(tb["map"][:n * 4].view(torch.int32).cpu().numpy(), map_)
    np.testing.assert_array_equal(tb["slot_stat"][:M * 8].view(torch.int32).cpu().numpy().view(np.uint32).reshape(M, 2),
                                  stat)
    cache = tb["cache"][:M * 128].view(M, 128).cpu().numpy()
    for s in victims:
        np.testing.assert_array_equal(cache[s], X[owner[s]])


@pytest.mark.parametrize("policy", ["lru", "lrfu"])
def test_recency_policies_keep_results(svf, policy):
    """Whatever the placement, results equal the device-resident search; hits
    stamp (LRU) or count (LRFU) the slot state, and a smaller cache after a
    reset still serves every row."""
    X, ix = built(svf, "u8", 5000, 5000, R=32)
    Q = torch.from_numpy(synth.sample("u8", 400, 734)).cuda()
    cfg = svf.SearchConfig(k=10, L=64, T=32, seed=5)
    want = ix.search(Q, cfg)
    ix.enable_tier(M=1000, theta0=0.5, promote_batch=256, qcap=4096)
    ix.release_device_store()
    for M in (1000, 300):
        ix.reset_tier(M=M, promote_batch=256, qcap=4096, policy=policy)
        for _ in range(3):
            got = ix.search(Q, cfg)
            assert torch.equal(got[0], want[0]) and torch.equal(got[1], want[1])
            assert ix.maintain() > 0
        st = ix.tier_bufs["slot_stat"][:M * 8].view(torch.int32).view(M, 2).cpu().numpy()
        assert (st[:, 0] != 0).any() or (st[:, 1] != 0).any()
        assert int((ix.tier_map()[:5000] >= 0).sum().item()) == M


def test_server_updates_beyond_the_shadow_capacity(svf):
    """An insert that would rewrite more rows than the version buffer holds
    (here 100 vectors x R = 32 rows > 1,000 shadow rows) runs as a barrier;
    the results still equal the same searches run alone at their epochs, and
    the graph equals the one built alone."""
    n0, ncap = 6000, 9000
    X, ix = built(svf, "u8", n0, ncap, R=32, max_batch=6000)
    _, ref_ix = built(svf, "u8", n0, ncap, R=32, max_batch=6000)
    rng = np.random.default_rng(751)
    reqs = _trace(rng, 90, n0, X, n0)
    cfg = svf.SearchConfig(k=10, L=64, T=32)
    comps, outs, upd, n_used = _serve_trace(svf, ix, X, n0, reqs, cfg, "snapshot", shadow_rows=1000)
    by_epoch = _check_epochs(reqs, comps, "snapshot")
    epoch = 0
    for tag, (op, a, b) in enumerate(reqs + [("end", 0, 0)]):
        if op == "search":
            continue
        for t in by_epoch.pop(epoch, []):
            Q, oi, od = outs[t]
            ri, rd = ref_ix.search(Q, cfg)
            assert torch.equal(ri, oi) and torch.equal(rd, od), f"request {t} at epoch {epoch}"
        if op == "end":
            break
        kind, v = upd[tag]
        if kind == "insert":
            ref_ix.insert(v, L_ins=64, T_ins=32)
        else:
            ref_ix.delete(v)
        epoch += 1
    torch.cuda.synchronize()
    assert torch.equal(ix.graph[:n_used], ref_ix.graph[:n_used])


def test_server_rejects_bad_consistency_setup(svf):
    from paper_2601_08528_b300 import _lib as L
    X, ix = built(svf, "u8", 2000, 2000, R=32)
    with pytest.raises(KeyError):
        svf.Server(ix, consistency="eventual")
    import ctypes as C
    h = C.c_void_p()
    cfg = L.ServeCfg(4, 2, 64, 2, None, 0, 1000)  # snapshot mode without a version buffer
    assert L.load().svf_serve_start(ix._h, C.byref(cfg), C.byref(h)) == L.SVF_EINVAL
    cfg = L.ServeCfg(4, 2, 64, 7, None, 0, 0)
    assert L.load().svf_serve_start(ix._h, C.byref(cfg), C.byref(h)) == L.SVF_EINVAL
