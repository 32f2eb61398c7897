"""Shared helpers of the GPU-vs-oracle parity tests.

Rule (FP32 path vs the FP64 oracle): distances agree within 1e-5 relative
(for the inner product relative to sum |q_i x_i|); ids may differ only for
queries whose oracle run met a decisive comparison with a relative gap at or
below 1e-5 (a near tie); recall@10 against exact kNN agrees within 0.2
points.  Integer (uint8) paths must agree bit for bit.
"""
import numpy as np

TOL = 1e-5


def dist_scale(X, Q, ids, metric):
    """Per-entry magnitude: |d| for L2, sum |q_i x_i| for IP."""
    ids = np.asarray(ids, dtype=np.int64)
    ok = ids >= 0
    Xd = X.astype(np.float64)
    Qd = Q.astype(np.float64)
    out = np.ones(ids.shape)
    for qi in range(ids.shape[0]):
        sel = ids[qi][ok[qi]]
        if metric == "ip":
            out[qi, ok[qi]] = np.abs(Xd[sel] * Qd[qi]).sum(1)
        else:
            out[qi, ok[qi]] = ((Xd[sel] - Qd[qi]) ** 2).sum(1)
    return out


def as_u32(a):
    return np.asarray(a).astype(np.int64) & 0xFFFFFFFF


def check_fp32(gpu_ids, gpu_d, orc, X, Q, metric, tol=TOL, min_identical=0.9):
    """Compare a GPU FP32 search with oracle output dict (ids, dist, gap)."""
    gi = as_u32(gpu_ids)
    oi = orc["ids"].astype(np.int64)
    same = (gi == oi).all(1)
    amb = orc["gap"] <= tol
    bad = ~same & ~amb
    assert not bad.any(), f"{bad.sum()} unambiguous queries differ, e.g. q={np.where(bad)[0][:5]}"
    # distances on agreeing queries
    sc = dist_scale(X, Q, np.where(oi == 0xFFFFFFFF, -1, oi)[same], metric)
    od = orc["dist"][same]
    gd = np.asarray(gpu_d, dtype=np.float64)[same]
    fin = np.isfinite(od)
    err = np.abs(gd[fin] - od[fin]) / np.maximum(sc[fin], 1e-30)
    assert (err <= tol).all(), f"max relative distance error {err.max():.3g}"
    assert np.isinf(gd[~fin]).all()
    # near ties are common in these mixtures; still, most queries must agree
    # exactly or the ambiguity rule would be vacuous
    assert same.mean() >= min_identical, f"only {same.mean():.2%} of queries identical ({amb.mean():.2%} ambiguous)"
    return same.mean(), amb.mean()


def check_fp32_all(gpu_ids, gpu_d, orc, X, Q, metric, tol=TOL, min_identical=0.9, max_diverged=None):
    """check_fp32 over a whole batch, also for the ambiguous queries whose ids
    differ: where the two sides returned different ids, the k distances are
    still compared position by position; a query whose distances differ by
    more than the tolerance there has taken another trajectory after its near
    tie ("diverged").  Returns a dict of counts; `max_diverged` (a fraction of
    the batch) bounds the diverged queries."""
    frac_same, frac_amb = check_fp32(gpu_ids, gpu_d, orc, X, Q, metric, tol, min_identical)
    gi = as_u32(gpu_ids)
    oi = orc["ids"].astype(np.int64)
    differ = np.where(~(gi == oi).all(1))[0]
    diverged = 0
    if len(differ):
        gd = np.asarray(gpu_d, dtype=np.float64)[differ]
        od = orc["dist"][differ]
        sc = np.maximum(dist_scale(X, Q[differ], np.where(oi[differ] == 0xFFFFFFFF, -1, oi[differ]), metric),
                        dist_scale(X, Q[differ], np.where(gi[differ] == 0xFFFFFFFF, -1, gi[differ]), metric))
        fin = np.isfinite(od) & np.isfinite(gd)
        err = np.where(fin, np.abs(gd - od) / np.maximum(sc, 1e-30), 0.0)
        both_inf = np.isfinite(od) == np.isfinite(gd)
        diverged = int(((err > tol).any(1) | ~both_inf.all(1)).sum())
    n = len(gi)
    if max_diverged is not None:
        assert diverged <= max_diverged * n, f"{diverged} of {n} queries diverged after a near tie"
    return {"n": n, "identical": int(round(frac_same * n)), "ambiguous": int(round(frac_amb * n)),
            "ids_differ": int(len(differ)), "diverged": diverged}


def check_exact(gpu_ids, gpu_d, orc):
    gi = as_u32(gpu_ids)
    oi = orc["ids"].astype(np.int64)
    np.testing.assert_array_equal(gi, oi)
    od = orc["dist"]
    gd = np.asarray(gpu_d).astype(np.int64)
    fin = np.isfinite(od)
    np.testing.assert_array_equal(gd[fin], od[fin].astype(np.int64))
    assert (gd[~fin] == 2**31 - 1).all()


def recall(ids, true_ids, true_d, found_d_exact):
    k = true_ids.shape[1]
    kth = true_d[:, k - 1:k]
    # a relative slack of 1e-12 on either sign of distance (inner-product
    # distances are negative, so scaling kth would tighten the test instead)
    ok = (as_u32(ids) != 0xFFFFFFFF) & (found_d_exact <= kth + 1e-12 * np.abs(kth) + 1e-300)
    return float(ok.sum()) / (ids.shape[0] * k)


def rerank_ref(orc, st, Q, o, k):
    """Oracle of the exact re-rank: FP64 distances (store `st`) of the final
    low-precision-traversal pool o["pool_ids"], re-sorted by (dist, id); the
    gap also covers the re-sorted k-boundary."""
    pd = orc.dist_ids(st, Q, o["pool_ids"])
    nq = len(Q)
    want_i = np.empty((nq, k), np.int64)
    want_d = np.empty((nq, k))
    gaps = np.empty(nq)
    for q in range(nq):
        order = np.lexsort((o["pool_ids"][q], pd[q]))
        want_i[q] = o["pool_ids"][q][order[:k]]
        want_d[q] = pd[q][order[:k]]
        s = pd[q][order[:k + 1]]
        gaps[q] = np.min(np.abs(np.diff(s))) if len(s) > 1 else np.inf
    return {"ids": want_i, "dist": want_d, "gap": np.minimum(gaps, o["gap"])}
