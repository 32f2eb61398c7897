"""GPU insert / delete+repair parity against the FP64 oracle (C ABI).

uint8 data: every graph row after every batch is compared bit for bit.
fp32 data: rows may differ only where the oracle met a near tie, or where
they received reverse edges from a new row that itself differed.
"""
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


def _index(svf, orc, mix, n0, n_cap, R, metric, prune, seed, max_batch=2000):
    X = synth.sample(mix, n_cap, seed)
    st = orc.Store.from_vectors(X, metric)
    g0, _ = orc.build_graph(orc.Store.from_vectors(X[:n0], metric), R, 1 if prune == "rank" else 0)
    g = np.full((n_cap, R), orc.EMPTY, dtype=np.uint32)
    g[:n0] = g0
    ix = svf.Index(X.shape[1], n_cap, dtype="u8" if X.dtype == np.uint8 else "f32", metric=metric, R=R,
                   prune=prune, max_batch=max_batch)
    ix.attach(torch.from_numpy(X[:n0]).cuda(), torch.from_numpy(g0.view(np.int32)))
    return X, st, g, ix


@pytest.mark.parametrize("R,prune,L_ins", [(64, "rng", 128), (32, "rank", 64), (32, "rng", 32)])
def test_insert_u8_bit_exact_batches(svf, orc, R, prune, L_ins):
    n0, m, nb = 2000, 300, 3
    X, st, g, ix = _index(svf, orc, "u8", n0, n0 + m * nb, R, "l2", prune, 301)
    mode = 1 if prune == "rank" else 0
    n = n0
    for b in range(nb):
        ids = ix.insert(torch.from_numpy(X[n:n + m]).cuda(), L_ins=L_ins, T_ins=L_ins // 2)
        assert ids.cpu().numpy().tolist() == list(range(n, n + m))
        orc.insert(st, n, m, g, None, L_ins, L_ins // 2, ix.params.seed, mode)
        n += m
        gg = P.as_u32(ix.graph[:n].cpu().numpy())
        bad = np.where((gg != g[:n]).any(1))[0]
        assert len(bad) == 0, f"batch {b}: {len(bad)} rows differ, e.g. {bad[:5]}"
    s = ix.stats()
    assert s["n_used"] == n and s["reverse_targets"] > 0


def test_insert_fp32_parity(svf, orc):
    n0, m = 2000, 400
    X, st, g, ix = _index(svf, orc, "tiny", n0, n0 + m, 32, "l2", "rng", 311)
    ix.insert(torch.from_numpy(X[n0:]).cuda(), L_ins=64, T_ins=32)
    new_gap, tail_gap = orc.insert(st, n0, m, g, None, 64, 32, ix.params.seed, 0)
    gg = P.as_u32(ix.graph[:n0 + m].cpu().numpy())
    diff = (gg != g).any(1)
    amb_new = np.where(new_gap <= P.TOL)[0] + n0
    # old rows touched by an ambiguous new row (either side's choice)
    touched = set()
    for v in amb_new:
        touched.update(g[v].tolist())
        touched.update(gg[v].tolist())
    ok = np.zeros(n0 + m, bool)
    ok[amb_new] = True
    ok[np.where(tail_gap <= P.TOL)[0]] = True
    for u in touched:
        if u < n0:
            ok[u] = True
    assert not (diff & ~ok).any(), f"{(diff & ~ok).sum()} unexplained row differences"
    assert diff.mean() < 0.1


def test_insert_capacity_and_empty(svf, orc):
    X, st, g, ix = _index(svf, orc, "u8", 500, 600, 32, "l2", "rng", 321)
    with pytest.raises(svf.SvfError) as e:
        ix.insert(torch.from_numpy(X[:101]).cuda())
    assert e.value.code == -2
    assert ix.insert(torch.from_numpy(X[:0]).cuda()).numel() == 0
    assert ix.stats()["n_used"] == 500


@pytest.mark.parametrize("R,prune", [(32, "rng"), (64, "rng"), (32, "rank")])
def test_delete_repair_u8_bit_exact(svf, orc, R, prune):
    n = 3000
    X, st, g, ix = _index(svf, orc, "u8", n, n, R, "l2", prune, 331)
    bits = orc.bitset(n)
    mode = 1 if prune == "rank" else 0
    for b, cnt in enumerate((300, 600, 900)):
        dels = synth.pick_live_ids(n, orc.deleted_ids(bits, n), cnt, 332 + b)
        dup = np.concatenate([dels, dels[:5]])
        newly = ix.delete(torch.from_numpy(dup.view(np.int32)).cuda())
        on, rep, _ = orc.delete(st, n, g, bits, dup, c=8, mode=mode)
        assert newly == on == cnt
        gg = P.as_u32(ix.graph[:n].cpu().numpy())
        bad = np.where((gg != g).any(1))[0]
        assert len(bad) == 0, f"round {b}: {len(bad)} rows differ, e.g. {bad[:5]}"
        np.testing.assert_array_equal(P.as_u32(ix.del_bits.cpu().numpy()), bits)
    s = ix.stats()
    assert s["n_deleted"] == 1800 and s["repaired_rows"] > 0


def test_delete_invalid_id_changes_nothing(svf, orc):
    X, st, g, ix = _index(svf, orc, "u8", 1000, 1000, 32, "l2", "rng", 341)
    before = ix.graph.clone()
    with pytest.raises(svf.SvfError) as e:
        ix.delete(torch.tensor([3, 1000], dtype=torch.int32))
    assert e.value.code == -1
    assert torch.equal(before, ix.graph)
    assert int(ix.del_bits.sum().item()) == 0
    assert ix.delete(torch.tensor([3, 3], dtype=torch.int32)) == 1
    assert ix.delete(torch.tensor([3], dtype=torch.int32)) == 0


def test_delete_fp32_parity_and_search_after(svf, orc):
    n = 3000
    X, st, g, ix = _index(svf, orc, "tiny", n, n, 32, "l2", "rng", 351)
    bits = orc.bitset(n)
    dels = synth.pick_live_ids(n, None, 900, 352)
    ix.delete(torch.from_numpy(dels.view(np.int32)).cuda())
    _, rep, gap = orc.delete(st, n, g, bits, dels)
    gg = P.as_u32(ix.graph[:n].cpu().numpy())
    diff = (gg != g).any(1)
    assert not (diff & (gap > P.TOL)).any()
    Q = synth.sample("tiny", 100, 353)
    ids, _ = ix.search(torch.from_numpy(Q).cuda(), __import__("paper_2601_08528_b300").SearchConfig(k=10, L=64, T=32))
    assert not np.isin(P.as_u32(ids.cpu().numpy()), dels).any()
