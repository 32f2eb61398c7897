#!/usr/bin/env python
"""Search throughput at recall@10 >= 0.95 on the 10M x 96 inner-product workload.

Workload ("unit96-10M"): n = 10,000,000 unit-normalised fp32 vectors, d = 96,
a 4,096-component Gaussian mixture of low intrinsic dimension (synth), inner
product; out-degree R = 32; 10,000 queries per step, k = 10.  The index
keeps fp32, bfloat16 and FP8-E4M3 (+ per-vector scale) copies of the vectors.
Its graph is built on the GPU: an exact 2R-NN + prune build of the first
200,000 vectors, then batched inserts of the rest (Sec. 5.1 insert path).

Forms compared (each at the cheapest swept (L, T) reaching recall@10 >= 0.95
against exact ground truth on held-out queries): plain FP32 traversal; BF16 / FP8 traversal with
an exact FP32 re-rank of the final pool; the same with the learned early stop
(trained here on traces of 200,000 training queries).  `value` is the QPS of
the fastest form; one step = one search launch over the 10,000-query batch.

Every form's (L, T) is chosen on 20,000 held-out calibration queries and
then measured on the 10,000 timed queries.  `--impl reference` times the CPU
oracle (FP64, all host cores) on the same batch, same graph, same (L, T):
one pass over all 10,000 queries per step.
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

K = 10
R = 32
N_BOOT = 200_000
MAX_BATCH = 1_000_000
ROW_BYTES = {"f32": 384, "bf16": 192, "fp8": 100}  # bytes of one row's values (+ FP8 scale)


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=10_000_000)
    ap.add_argument("--nq", type=int, default=10_000)
    ap.add_argument("--ntrain", type=int, default=200_000)
    ap.add_argument("--target", type=float, default=0.95)
    ap.add_argument("--serve-rate", type=float, default=500.0, help="requests/s of the serving stream (0: skip)")
    ap.add_argument("--serve-seconds", type=float, default=6.0)
    ap.add_argument("--workload", default="unit96-10M", choices=["unit96-10M", "serve128-50M"])
    ap.add_argument("--serve-rates", default="25,50,100,200")
    ap.add_argument("--serve-form", default="fp32", choices=["fp32", "fp8"],
                    help="serving traversal: fp32 rows through the tier, or a resident fp8 copy + exact re-rank")
    ap.add_argument("--graph", default="exact", choices=["exact", "bootstrap"],
                    help="unit96-10M graph: exact 2R-NN + prune of every row, or 200K exact + inserts")
    ap.add_argument("--u8", type=int, default=1, help="also measure the 1M x 128 uint8 configuration (0: skip)")
    ap.add_argument("--fixed-point", default="",
                    help="form,L,T: time that form at that point only, without the stop networks (profiling)")
    ap.add_argument("--cache-ratios", default="0.1",
                    help="cache sizes (fractions of n) of the placement ablation on a moving hot set (empty: skip)")
    ap.add_argument("--cache-policies", default="wavp,lru,lrfu",
                    help="placement policies of that ablation (wavp,clock,lfu,static,lru,lrfu)")
    ap.add_argument("--cache-seconds", type=float, default=6.0)
    ap.add_argument("--cache-rate", type=float, default=50.0)
    ap.add_argument("--serve-policies", default="",
                    help="comma list of extra cache placement policies (clock,lfu,static,lru,lrfu) run on the same serving "
                         "stream after WAVP, for the ablation")
    ap.add_argument("--serve-window", default="",
                    help="W,speed: queries from a sliding window of W components moving `speed` components/s "
                         "(default: Zipf(1.1) over all components)")
    ap.add_argument("--serve-cache-frac", type=float, default=0.3125, help="device cache rows / n (unit96-10M)")
    ap.add_argument("--serve-maintain-every", type=int, default=128, help="search batches between maintenance")
    ap.add_argument("--serve-trav", default="fp8", choices=["fp8", "fp32"],
                    help="unit96-10M serving stream: the measured fp8 form (traversal resident, re-rank rows "
                         "through the tier), or plain fp32 (every traversal row through the tier)")
    ap.add_argument("--consolidate", type=int, default=1,
                    help="unit96-10M: delete 20%% of the index and consolidate it (before the serving stream, "
                         "which then runs on the consolidated index); 0 skips")
    ap.add_argument("--serve-small", type=int, default=1,
                    help="serve128-50M: latency-bound search batches run with several warps per query, W by "
                         "batch size from a measurement before tiering (0: one warp per query throughout)")
    ap.add_argument("--serve-barrier", action="store_true",
                    help="serve128-50M: also run each rate's stream in the barrier consistency mode")
    ap.add_argument("--serve-compare", action="store_true",
                    help="serve128-50M: also run each rate's stream with one warp per query throughout")
    ap.add_argument("--raw-rates", default="500,2000,5000,10000",
                    help="request rates of the read-after-write consistency stream (empty: skip)")
    ap.add_argument("--raw-seconds", type=float, default=1.0)
    ap.add_argument("--serve-lins", type=int, default=128, help="insert search pool of the 50M build")
    ap.add_argument("--serve-tins", type=int, default=96, help="insert search iterations of the 50M build")
    return ap.parse_args()


# ---------------------------------------------------------------- setup
def build_index(svf, torch, X, log_t, streams=1, graph="exact"):
    """The unit96 index: graph "exact" = every row's exact 2R nearest
    neighbours by inner product pruned to R (svf_build; the tensor-core scan
    of the rows against themselves); "bootstrap" = the exact build of the
    first 200,000 rows, then the rest inserted in batches of up to 1M."""
    n = X.shape[0]
    cap = n + 300_000 * streams
    if graph == "exact":
        ix = svf.Index(96, cap, dtype="f32", metric="ip", R=R, lowp=("bf16", "fp8"), max_batch=n)
        Xd = torch.from_numpy(X).cuda()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        ix.build(Xd)
        e1.record()
        e1.synchronize()
        del Xd
        ix.build_s = e0.elapsed_time(e1) / 1e3
        ix.build_fallback = ix.stats()["build_fallback"]
        log_t("exact build", n, f"{ix.build_s:.1f} s", "rows by the exact scan:", ix.build_fallback)
        ix.graph_desc = "exact 2R-NN by inner product (tensor cores, certified) pruned to R = 32 by RNG"
        return ix
    ix = svf.Index(96, cap, dtype="f32", metric="ip", R=R, lowp=("bf16", "fp8"), max_batch=MAX_BATCH)
    n0 = min(N_BOOT, n)
    t = time.time()
    ix.build(torch.from_numpy(X[:n0]).cuda())
    torch.cuda.synchronize()
    log_t("bootstrap build", n0, time.time() - t)
    while ix.n_used < n:
        b = min(ix.n_used, MAX_BATCH, n - ix.n_used)
        ix.insert(torch.from_numpy(X[ix.n_used:ix.n_used + b]).cuda(), L_ins=64, T_ins=48)
    torch.cuda.synchronize()
    ix.build_s, ix.build_fallback = None, None
    ix.graph_desc = f"exact 2R-NN+prune of {N_BOOT} then inserts (L_ins=64, T_ins=48)"
    return ix


def insert_rate(svf, torch, ix, X_new, batch=MAX_BATCH):
    """Insert throughput (Sec. 5.1 path) of batches of `batch` new vectors,
    CUDA events around each svf_insert (host->device copies outside)."""
    secs, done = 0.0, 0
    for i in range(0, X_new.shape[0], batch):
        xb = torch.from_numpy(X_new[i:i + batch]).cuda()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        ix.insert(xb, L_ins=64, T_ins=48)
        e1.record()
        e1.synchronize()
        secs += e0.elapsed_time(e1) / 1e3
        done += xb.shape[0]
    return done / secs


def time_search(torch, ix, Q, cfg, reps=3):
    ix.search(Q, cfg)
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        ix.search(Q, cfg)
        b.record()
        b.synchronize()
        ts.append(a.elapsed_time(b) / 1e3)
    return min(ts)


def sweep(torch, ix, Q, gt, forms, grid, target, learned):
    from paper_2601_08528_b300.learned import recall_at_k
    pts = []
    for name, base in forms:
        for L, T in grid:
            cfg = dataclasses.replace(base, L=L, T=T)
            if name.endswith("+stop"):
                net = learned.get((cfg.precision, L, T))
                if net is None or net.tau >= 1.0:
                    continue
                cfg = dataclasses.replace(cfg, mlp=net.packed, tau=net.tau, t_min=net.t_min, t_every=net.t_every)
            ix.stats_reset()
            ids, _ = ix.search(Q, cfg)
            its = ix.stats()["search_iters"] / Q.shape[0]
            rec = recall_at_k(ids, gt)
            sec = time_search(torch, ix, Q, cfg)
            pts.append({"form": name, "L": L, "T": T, "recall": rec, "qps": Q.shape[0] / sec, "cfg": cfg,
                        "iters": its})
            log(f"  {name:16s} L={L:3d} T={T:3d} recall={rec:.4f} qps={Q.shape[0] / sec:,.0f} iters={its:.1f}")
    best = {}
    for p in pts:
        if p["recall"] >= target and (p["form"] not in best or p["qps"] > best[p["form"]]["qps"]):
            best[p["form"]] = p
    return pts, best


STOP_POINTS = [(64, 40), (64, 44), (64, 48), (64, 56), (64, 64)]
STOP_EVERY = 4


METRIC = "search QPS at recall@10>=0.95 (plain FP32 vs BF16/FP8 + learned stop)"


def small_batch(svf, torch, ix, Q, gt, cfg, target, Ws=(1, 2, 4, 8), sizes=(1, 16), reps=200):
    """Several warps per query (W parents per iteration) for latency-bound
    batches: for each W the cheapest swept T whose recall@10 over all queries
    reaches `target`, then the latency of batches of 1 and 16 queries through
    the public API (CUDA events around the call, host overhead included)."""
    out = {}
    for W in Ws:
        Ts = sorted({max(2, int(np.ceil(cfg.T * f / W))) for f in (0.8, 1.0, 1.25, 1.5, 2.0)})
        pick = None
        for T in Ts:
            c = dataclasses.replace(cfg, T=T, W=W, mlp=None)
            ids, _ = ix.search(Q, c)
            r = (ids.long().unsqueeze(2) == gt.long().unsqueeze(1)).any(2).float().mean().item()
            if r >= target:
                pick = (c, r)
                break
        if pick is None:
            continue
        c, r = pick
        row = {"T": c.T, "recall@10": r}
        for b in sizes:
            ts = []
            for i in range(reps):
                q = Q[(i * b) % (Q.shape[0] - b):][:b]
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                ix.search(q, c)
                e1.record()
                e1.synchronize()
                ts.append(e0.elapsed_time(e1))
            row[f"b{b}_p50_ms"] = float(np.percentile(ts, 50))
            row[f"b{b}_p99_ms"] = float(np.percentile(ts, 99))
        row["cfg"] = c
        out[W] = row
    return out


def consolidation(svf, torch, ix, Q, cfg, frac=0.2, frac2=0.05, seed=307, probes=400):
    """Global consolidation (Sec. 5.2 under the multi-version mechanism of
    Sec. 5.3) on the device-resident index.  Deletes `frac` of it (with the
    localized repair), reports recall@10 of `cfg` against exact kNN over the
    live vectors before and after a consolidation run alone, then deletes
    `frac2` more and consolidates on a low-priority stream while searches of
    the same batch run back to back on a high-priority stream.  Returns the
    report and the deleted ids."""
    n = ix.n_used
    out = {"deleted_frac": frac}
    dele = synth.pick_live_ids(n, None, int(n * frac), seed)
    ix.delete(torch.from_numpy(dele.view(np.int32)).cuda())
    isdel = torch.zeros(n, dtype=torch.bool, device="cuda")
    isdel[torch.from_numpy(dele.astype(np.int64)).cuda()] = True
    g32, _, _ = svf.knn_tc(ix.vectors()[:n], Q, 32, "ip")
    g = g32.long()
    live = ~isdel[g]
    keep = live & (torch.cumsum(live.int(), 1) <= K)
    gt = torch.where(keep, g, torch.full_like(g, -1))

    def recall():
        ids, _ = ix.search(Q, cfg)
        hit = (ids.long().unsqueeze(2) == gt.unsqueeze(1)).any(2)
        return hit.float().sum().item() / (Q.shape[0] * K)

    def t_search(stream):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ix.search(Q, cfg, stream=stream)
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1)

    out["recall_before"] = recall()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    out["rows_rewritten"] = ix.consolidate()
    e1.record()
    e1.synchronize()
    out["seconds"] = e0.elapsed_time(e1) / 1e3
    out["recall_after"] = recall()
    # in the background: a second consolidation after more deletes
    dele2 = synth.pick_live_ids(n, dele, int(n * frac2), seed + 1)
    ix.delete(torch.from_numpy(dele2.view(np.int32)).cuda())
    lo, hi = torch.cuda.Stream.priority_range()
    bg, fg = torch.cuda.Stream(priority=lo), torch.cuda.Stream(priority=hi)
    base = float(np.median([t_search(fg) for _ in range(5)]))
    torch.cuda.synchronize()
    b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ix.consolidate_begin(0, stream=bg)
    b0.record(bg)
    rows2 = ix.consolidate_run(stream=bg)
    b1.record(bg)
    during = []
    while not b1.query() and len(during) < probes:
        during.append(t_search(fg))
    b1.synchronize()
    ix.consolidate_commit(stream=bg)
    torch.cuda.synchronize()
    out["background"] = {"deleted_frac_more": frac2, "rows_rewritten": rows2,
                         "seconds": b0.elapsed_time(b1) / 1e3, "search_ms_alone": base,
                         "search_ms_during_p50": float(np.median(during)) if during else None,
                         "searches_during": len(during),
                         "note": "consolidation on a low-priority stream, searches of the same 10K batch on a "
                                 "high-priority stream back to back until it ends"}
    return out, np.union1d(dele, dele2)


def pick_cfg(small, sz, cfg):
    """The search config of a batch of sz queries: that of the first (b, cfg_b)
    in `small` (ascending b) with sz <= b, else cfg."""
    return next((cb for b, cb in small if sz <= b), cfg) if small else cfg


def w_policy(sb, sizes=(16, 256, 1024)):
    """Serving policy from small_batch's measurement: a batch of up to b
    queries (b in `sizes`) takes the W with the lowest one-call latency at b;
    larger batches keep one warp per query.  Returns [(b, cfg), ...]."""
    out = []
    for b in sizes:
        key = f"b{b}_p50_ms"
        cand = [(r[key], W) for W, r in sb.items() if key in r]
        if not cand:
            continue
        _, W = min(cand)
        if W == 1:
            continue
        if out and out[-1][1].W == W:
            out[-1] = (b, out[-1][1])  # the same W over a wider range
        else:
            out.append((b, sb[W]["cfg"]))
    return out


def max_over_ranks(x, dist):
    """Max over ranks of a host float: every rank's timed region ends when the
    slowest does (NCCL reduces a device tensor, gloo a host one)."""
    if dist is None:
        return float(x)
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], device=dev, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, world, seconds):
    """Whole-job throughput: the units all ranks processed over the max-over-
    ranks time (weak scaling: every rank has its own batch)."""
    return world * units_per_rank / seconds


def u8_leg(svf, torch, log_t, n=1_000_000, nq=10_000, R8=64, batches=10, batch=10_000):
    """The integer-exact configuration: n uint8 vectors, d = 128, squared L2
    exact in int32, out-degree 64 (exact 128-NN + RNG prune), 10,000 queries
    at L = 64 and 128 (T = L / 2), then a 10 % insert stream in batches of
    10,000 (L_ins = 128, T_ins = 64).  Search QPS with the HBM roofline of
    its launch, inserts/s, and the oracle timed on the same queries."""
    X = synth.sample_chunked("u8", n + batches * batch, 201)
    Q_np = synth.sample_chunked("u8", nq, 202)
    ix = svf.Index(128, n + batches * batch, dtype="u8", metric="l2", R=R8, max_batch=n)
    torch.cuda.synchronize()
    t = time.time()
    ix.build(torch.from_numpy(X[:n]).cuda())
    torch.cuda.synchronize()
    out = {"workload": f"u8-1M: {n} x 128 uint8 (1,024-centre mixture), squared L2 exact in int32, R = {R8}",
           "build_s": time.time() - t}
    Q = torch.from_numpy(Q_np).cuda()
    gt = svf.knn(ix.vectors()[:n], Q, K, "l2")[0]
    from paper_2601_08528_b300.learned import recall_at_k
    peaks, _ = measured_peaks()
    for L in (64, 128):
        cfg = svf.SearchConfig(k=K, L=L, T=L // 2)
        ix.stats_reset()
        ids, _ = ix.search(Q, cfg)
        s = ix.stats()
        sec = time_search(torch, ix, Q, cfg, reps=5)
        alg = s["search_iters"] * R8 * 4 + s["search_evals"] * 128 + nq * (128 + K * 8)
        out[f"L{L}"] = {"T": L // 2, "recall@10": recall_at_k(ids, gt), "qps": nq / sec, "ms": 1e3 * sec,
                        "iters_per_query": s["search_iters"] / nq, "evals_per_query": s["search_evals"] / nq,
                        "roofline": {"achieved_gbs": alg / sec / 1e9, "frac": alg / sec / 1e9 / peaks["hbm_gbs"]}}
        log_t("u8", L, json.dumps(out[f"L{L}"]))
    secs = 0.0
    for b in range(batches):
        xb = torch.from_numpy(X[n + b * batch:n + (b + 1) * batch]).cuda()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        ix.insert(xb, L_ins=128, T_ins=64)
        e1.record()
        e1.synchronize()
        secs += e0.elapsed_time(e1) / 1e3
    out["inserts_per_s"] = batches * batch / secs
    out["insert_stream"] = f"{batches} batches of {batch}, L_ins = 128, T_ins = 64"
    # the oracle on the host cores, the same queries at L = 64 on the built graph
    import oracle as orc
    g_np = ix.graph[:n].cpu().numpy().view(np.uint32)
    st = orc.Store.from_vectors(X[:n], "l2")
    t = time.time()
    orc.search(st, n, g_np, None, Q_np, K, 64, 32, 0x5F0C)
    out["cpu_baseline"] = {"value": nq / (time.time() - t), "unit": "queries/s", "cores": orc.threads(),
                           "kind": "oracle", "sample": f"all {nq} queries at L = 64, T = 32"}
    ix.close()
    return out


def unit96_name(n):
    return f"unit96-{n // 1_000_000}M" if n % 1_000_000 == 0 else f"unit96-{n}"


def exact_knn(svf, X, Q, k, metric):
    """Ground-truth ids: the tensor-core scan (bf16 products, exact fp32
    rescoring, certificate with SIMT fallback) where it applies, else the
    SIMT scan."""
    if X.dtype.is_floating_point and X.shape[1] % 16 == 0 and X.shape[1] <= 128 and k <= 32:
        ids, _, fb = svf.knn_tc(X, Q, k, metric)
        if fb:
            print(f"  ground truth: {fb} of {Q.shape[0]} queries by the SIMT fallback", file=sys.stderr, flush=True)
        return ids
    return svf.knn(X, Q, k, metric)[0]


def train_stops(torch, svf, ix, Qtr, gt_cal, ncal, precisions):
    """One stop network per (precision, L, T_max), trained on traces of the
    plain search of the training queries and calibrated (tau) on held-out
    training queries for <= 0.2 pt recall@10 loss against fixed T_max."""
    from paper_2601_08528_b300 import learned
    nets = {}
    for prec in precisions:
        for L, T in STOP_POINTS:
            cfg = svf.SearchConfig(k=K, L=L, T=T, precision=prec, rerank=prec is not None)
            feat, meta = learned.capture_traces(ix, Qtr[ncal:], cfg)
            ids = learned.sample_ids(meta, T)
            net = learned.train(feat, meta, T, ids, epochs=3, batch=8192, lr=5e-3, seed=11)
            net.t_min, net.t_every = T // 4, STOP_EVERY
            del feat
            tau, r0, r1 = learned.calibrate(ix, net, Qtr[:ncal], gt_cal, cfg)
            net.tau = tau
            nets[(prec, L, T)] = net
            log(f"  stop net {prec} L={L} T={T}: loss={net.loss:.4f} samples={ids.numel()} tau={tau} "
                f"recall fixed={r0:.4f} stop={r1:.4f}")
    return nets


# ---------------------------------------------------------------- serving
def serve_stream(svf, torch, ix, mix, X_ins, rate, duration, warm, seed, cfg, zipf_s=1.1, max_inflight=8,
                 n_streams=4, maintain_every=128, L_ins=64, T_ins=32, max_batch=2048, window=None, small=None,
                 consistency="snapshot"):
    """Open-loop Poisson stream at `rate` requests/s for `duration` s through
    the continuous-batching server: 90:9:1 search:insert:delete requests,
    batch sizes floor(exp(U[0, ln max_batch])), query components ~ Zipf(s).
    small = [(b, cfg_b), ...] in ascending b: a search batch of sz queries
    runs with the cfg of the first b >= sz (several warps per query), else
    with cfg.  consistency: the server's mode ("snapshot": searches read the
    last completed update's state and never wait; "read-after-write";
    "barrier").  Returns latency percentiles (ms) per op over the requests
    that arrived after `warm` s, query and insert throughput, and cache
    counters."""
    rng = np.random.default_rng(seed)
    m = synth.MIXTURES[mix]
    arr, ops, sizes = [], [], []
    t = 0.0
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= duration:
            break
        arr.append(t)
        u = rng.random()
        ops.append(0 if u < 0.90 else (1 if u < 0.99 else 2))
        sizes.append(max(1, min(max_batch, int(np.exp(rng.uniform(0, np.log(max_batch)))))))
    nq = sum(sz for o, sz in zip(ops, sizes) if o == 0)
    if window:
        # query components from a sliding window (width, components/s): the hot set moves
        wdraw = synth.window_components(m.n_centres, window[0], window[1], seed + 2)
        wrng = np.random.default_rng(seed + 3)
        labels = np.concatenate([wdraw(wrng, ta, sz) for ta, o, sz in zip(arr, ops, sizes) if o == 0] or
                                [np.zeros(1, np.int64)])
        Qall = torch.from_numpy(synth.sample_chunked(m, max(nq, 1), seed + 1,
                                                     component_sampler=synth.given_components(labels),
                                                     workers=1)).cuda()
    else:
        Qall = torch.from_numpy(synth.sample_chunked(m, max(nq, 1), seed + 1,
                                                     component_sampler=synth.zipf_components(m.n_centres, zipf_s,
                                                                                              seed + 2))).cuda()
    k = cfg.k
    ids_out = torch.empty((max(nq, 1), k), dtype=torch.int32, device="cuda")
    d_out = torch.empty((max(nq, 1), k), dtype=torch.int32 if m.dtype == "u8" else torch.float32, device="cuda")
    srv = svf.Server(ix, max_inflight=max_inflight, n_streams=n_streams, maintain_every=maintain_every,
                     consistency=consistency, shadow_rows=max_batch * ix.R)
    ix.stats_reset()
    qo, io = 0, 0
    n_used = ix.n_used
    deleted = 0
    t0 = svf.Server.now() + 0.5
    for tag, (ta, op, sz) in enumerate(zip(arr, ops, sizes)):
        if op == 0:
            c = pick_cfg(small, sz, cfg)
            srv.search(tag, Qall[qo:qo + sz], c, ids_out[qo:qo + sz], d_out[qo:qo + sz], t_arrival=t0 + ta)
            qo += sz
        elif op == 1:
            sz = min(sz, X_ins.shape[0] - io, ix.n_cap - n_used)
            if sz <= 0:
                continue
            srv.insert(tag, torch.from_numpy(X_ins[io:io + sz]).cuda(), L_ins=L_ins, T_ins=T_ins, t_arrival=t0 + ta)
            io += sz
            n_used += sz
        else:
            ids = torch.from_numpy(rng.integers(0, n_used, sz).astype(np.int32)).cuda()
            srv.delete(tag, ids, t_arrival=t0 + ta)
            deleted += sz
    srv.drain(duration + 600)
    comps = srv.poll(1 << 20)
    srv.stop()
    st = ix.stats()
    lat = {0: [], 1: [], 2: []}
    by_size = {"1-16": [], "17-256": [], "257-2048": []}  # search latency by batch size
    done_q = done_i = 0
    t_first, t_last = None, None
    for c in comps:
        if c["t_arrival"] - t0 < warm:
            continue
        lat[c["op"]].append(1e3 * (c["t_done"] - c["t_arrival"]))
        if c["op"] == 0:
            by_size["1-16" if c["count"] <= 16 else "17-256" if c["count"] <= 256 else "257-2048"].append(lat[0][-1])
        if c["op"] == 0:
            done_q += c["count"]
        elif c["op"] == 1:
            done_i += c["count"]
        t_first = c["t_arrival"] if t_first is None else min(t_first, c["t_arrival"])
        t_last = c["t_done"] if t_last is None else max(t_last, c["t_done"])
    span = max(t_last - t_first, 1e-9) if t_first is not None else 1.0

    def pct(v, q):
        return float(np.percentile(v, q)) if v else None
    names = {0: "search", 1: "insert", 2: "delete"}
    out = {"rate_req_per_s": rate, "duration_s": duration, "warmup_s": warm, "requests": len(comps),
           "qps": done_q / span, "inserts_per_s": done_i / span,
           "latency_ms": {names[o]: {"p50": pct(v, 50), "p99": pct(v, 99), "n": len(v)} for o, v in lat.items()},
           "search_latency_ms_by_batch": {k: {"p50": pct(v, 50), "p99": pct(v, 99), "n": len(v)}
                                          for k, v in by_size.items()},
           "cache_hit_rate": (st["cache_hits"] / max(1, st["cache_hits"] + st["cache_misses"]))
           if st["cache_hits"] + st["cache_misses"] else None,
           "promoted": st["promoted"], "evicted": st["evicted"], "consistency": consistency}
    return out


def read_after_write(svf, torch, ix, X_new, rates, cfg, seconds=2.0, batch=10, seed=320):
    """The consistency experiment of Table 3 (Sec. 6): an open-loop Poisson
    stream of requests, half inserts of `batch` new vectors and half searches
    for the vectors the previous insert added, under each consistency mode.
    Recall@1 = fraction of those searches whose nearest result is the vector
    itself; p99 over all requests.  Returns {mode: {rate: {...}}}."""
    out = {}
    used = 0
    for mode in ("read-after-write", "snapshot"):
        out[mode] = {}
        for rate in rates:
            rng = np.random.default_rng(seed)
            arr = np.cumsum(rng.exponential(1.0 / rate, int(rate * seconds)))
            n_pairs = min(len(arr) // 2, (X_new.shape[0] - used) // batch, (ix.n_cap - ix.n_used) // batch)
            if n_pairs <= 0:
                continue
            xs = torch.from_numpy(X_new[used:used + n_pairs * batch]).cuda()
            used += n_pairs * batch
            ids = torch.empty((n_pairs * batch, cfg.k), dtype=torch.int32, device="cuda")
            dd = torch.empty((n_pairs * batch, cfg.k), dtype=torch.float32, device="cuda")
            srv = svf.Server(ix, max_inflight=8, n_streams=4, consistency=mode, shadow_rows=batch * ix.R)
            base = ix.n_used
            t0 = svf.Server.now() + 0.2
            for i in range(n_pairs):
                sl = slice(i * batch, (i + 1) * batch)
                srv.insert(2 * i, xs[sl], L_ins=64, T_ins=32, t_arrival=t0 + arr[2 * i])
                srv.search(2 * i + 1, xs[sl], cfg, ids[sl], dd[sl], t_arrival=t0 + arr[2 * i + 1])
            srv.drain(600)
            comps = srv.poll(1 << 20)
            srv.stop()
            want = torch.arange(base, base + n_pairs * batch, device="cuda", dtype=torch.int64)
            r1 = (ids[:, 0].long() == want).float().mean().item()
            lat = [1e3 * (c["t_done"] - c["t_arrival"]) for c in comps]
            slat = [1e3 * (c["t_done"] - c["t_arrival"]) for c in comps if c["op"] == 0]
            out[mode][str(rate)] = {"recall@1": r1, "p99_ms": float(np.percentile(lat, 99)),
                                    "search_p50_ms": float(np.percentile(slat, 50)),
                                    "search_p99_ms": float(np.percentile(slat, 99)), "pairs": n_pairs}
            log(f"  read-after-write stream {mode} rate {rate}: {out[mode][str(rate)]}")
    return out


# ---------------------------------------------------------------- clocks
class Clocks:
    def __init__(self):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                       "-lms", "100"], stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self, dev_index=0):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        self.p.wait()
        self.f.seek(0)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            c = [x.strip() for x in line.split(",")]
            if len(c) < 9 or c[0] != str(dev_index):
                continue
            try:
                sm.append(float(c[1]))
                mx = float(c[2])
            except ValueError:
                continue
            for nm, v in zip(names, c[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.f.name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def csrc_hash(root=None):
    """Hash of the library's code: every source under csrc/ with comments and
    blank lines removed, so that a comment edit does not mark a profile of
    unchanged kernels as stale."""
    import glob
    import hashlib
    import re
    h = hashlib.sha256()
    for f in sorted(glob.glob(os.path.join(root or ROOT, "paper_2601_08528_b300", "csrc", "*"))):
        with open(f, encoding="utf-8") as fh:
            txt = re.sub(r"/\*.*?\*/", "", fh.read(), flags=re.S)
        lines = [re.sub(r"//.*$", "", ln).rstrip() for ln in txt.splitlines()]
        h.update("\n".join(ln for ln in lines if ln.strip()).encode())
    return h.hexdigest()[:16]


def profiled_traffic(form, L, T):
    """DRAM bytes per launch from the committed ncu summary of the timed
    configuration, if the kernel sources are unchanged since the capture."""
    path = os.path.join(ROOT, "profiles", "search_kernel_unit96_10M.md")
    try:
        txt = open(path).read()
    except OSError:
        return None
    vals = dict(line.split(": ", 1) for line in txt.splitlines() if line.startswith(("traffic_bytes", "source_sha")))
    head = txt.splitlines()[0]
    if vals.get("source_sha", "").strip() != csrc_hash() or f"L={L}, T={T}" not in head or form.split("+")[0] not in head:
        return None
    return float(vals["traffic_bytes_per_launch"])


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0}, "fallback"


# ---------------------------------------------------------------- CPU oracle timing
class OracleTimer:
    """The oracle timed on the host cores in `form`: fixed-T FP64 search over
    the fp32 rows, or over the bf16 / fp8 copy followed by the exact FP64
    re-rank of the final pool (the same steps as the GPU form).  The stores
    are laid out once; `rate(Q)` times one pass over the queries Q and returns
    (queries/s, threads)."""

    def __init__(self, X, graph_np, L, T, form="fp32"):
        import oracle as orc
        self.orc = orc
        self.prec = form.split("+")[0]
        self.st = orc.Store.from_vectors(X, "ip")
        self.trav = self.st if self.prec == "fp32" else orc.Store.from_vectors(X, "ip", dtype=self.prec)
        self.n, self.g, self.L, self.T = X.shape[0], graph_np, L, T

    def run(self, q):
        o = self.orc.search(self.trav, self.n, self.g, None, q, K, self.L, self.T, 0x5F0C,
                            want_pool=self.prec != "fp32")
        if self.prec != "fp32":  # exact re-rank of the final pool
            pd = self.orc.dist_ids(self.st, q, o["pool_ids"])
            for i in range(len(q)):
                np.lexsort((o["pool_ids"][i], pd[i]))[:K]
        return o

    def rate(self, Q):
        t = time.time()
        self.run(Q)
        return Q.shape[0] / (time.time() - t), self.orc.threads()


def select_points(torch, ix, forms, grid, target, learned, Qcal, gt_cal, Qe, gt):
    """Operating points chosen on held-out calibration queries, measured on the
    evaluation queries: for each form the cheapest swept (L, T) whose recall@10
    over Qcal reaches `target`, then its recall and QPS over Qe (queries the
    choice never saw)."""
    from paper_2601_08528_b300.learned import recall_at_k
    pts, chosen = sweep(torch, ix, Qcal, gt_cal, forms, grid, target, learned)
    best = {}
    for name, p in chosen.items():
        cfg = p["cfg"]
        ix.stats_reset()
        ids, _ = ix.search(Qe, cfg)
        its = ix.stats()["search_iters"] / Qe.shape[0]
        sec = time_search(torch, ix, Qe, cfg)
        best[name] = {"form": name, "L": p["L"], "T": p["T"], "recall": recall_at_k(ids, gt), "qps": Qe.shape[0] / sec,
                      "cfg": cfg, "iters": its, "recall_cal": p["recall"]}
        log(f"  chosen {name:16s} L={p['L']:3d} T={p['T']:3d} recall cal {p['recall']:.4f} eval "
            f"{best[name]['recall']:.4f} qps={best[name]['qps']:,.0f}")
    return pts, best


# ---------------------------------------------------------------- serving workload (50M)
def serve_main(a, svf, torch, log_t):
    """The serving form at full size: n = 50M fp32 d=128 (squared L2), R = 32,
    built on the GPU (exact build of 200K + inserts), then tiered: all rows in
    pinned host memory behind an 8 GB device cache (15.6M rows) with WAVP
    placement; an open-loop Poisson stream per offered rate."""
    n = 50_000_000
    X = synth.sample_chunked("serve128", n, 500)
    log_t("data", X.shape)
    lowp = ("fp8",) if a.serve_form == "fp8" else ()
    ix = svf.Index(128, n + 2_000_000, dtype="f32", metric="l2", R=R, lowp=lowp, max_batch=MAX_BATCH)
    ix.build(torch.from_numpy(X[:N_BOOT]).cuda())
    while ix.n_used < n:
        b = min(ix.n_used, MAX_BATCH, n - ix.n_used)
        ix.insert(torch.from_numpy(X[ix.n_used:ix.n_used + b]).cuda(), L_ins=a.serve_lins, T_ins=a.serve_tins)
    torch.cuda.synchronize()
    log_t("built")
    Qe = torch.from_numpy(synth.sample_chunked("serve128", 2000, 502)).cuda()
    gt = exact_knn(svf, ix.vectors()[:n], Qe, K, "l2")
    from paper_2601_08528_b300.learned import recall_at_k
    op = None
    for L, T in [(64, 64), (64, 96), (128, 64), (128, 96), (256, 128), (256, 192), (256, 256), (256, 384)]:
        cfg = svf.SearchConfig(k=K, L=L, T=T, precision=a.serve_form if lowp else None, rerank=bool(lowp))
        r = recall_at_k(ix.search(Qe, cfg)[0], gt)
        log_t(f"  L={L} T={T} recall={r:.4f}")
        if r >= a.target:
            op = (cfg, r)
            break
    cfg, rec = op if op else (cfg, r)
    # latency-bound batches: W by batch size from one-call latencies measured before tiering
    sb = small_batch(svf, torch, ix, Qe, gt, cfg, a.target, sizes=(1, 16, 256, 1024)) if a.serve_small else {}
    log_t("small batches", {W: {k: v for k, v in r.items() if k != "cfg"} for W, r in sb.items()})
    small = w_policy(sb) or None
    slots = int(8e9 // (128 * 4))
    ix.enable_tier(M=slots, theta0=2.0, promote_batch=2048, sweep=4, qcap=16384)
    ix.release_device_store()
    del X
    log_t("tiered", slots)
    X_ins = synth.sample_chunked("serve128", 1_500_000, 503)
    res, res1, resb = [], [], []
    for i, rate in enumerate(float(x) for x in a.serve_rates.split(",")):
        r = serve_stream(svf, torch, ix, "serve128", X_ins[i * 300_000:(i + 1) * 300_000], rate, a.serve_seconds,
                         2.0, 510 + i, cfg, small=small)
        res.append(r)
        log_t("rate", rate, json.dumps(r))
        if small and a.serve_compare:
            # the same stream with one warp per query throughout
            r = serve_stream(svf, torch, ix, "serve128", X_ins[i * 300_000:(i + 1) * 300_000], rate,
                             a.serve_seconds, 2.0, 510 + i, cfg)
            res1.append(r)
            log_t("rate one warp", rate, json.dumps(r))
        if a.serve_barrier:
            # the same stream with every update a barrier
            r = serve_stream(svf, torch, ix, "serve128", X_ins[i * 300_000:(i + 1) * 300_000], rate,
                             a.serve_seconds, 2.0, 510 + i, cfg, small=small, consistency="barrier")
            resb.append(r)
            log_t("rate barrier", rate, json.dumps(r))
    p99 = [x["latency_ms"]["search"]["p99"] for x in res if x["latency_ms"]["search"]["p99"] is not None]
    out = {"metric": "serving p99 search latency (ms) at offered load", "value": min(p99) if p99 else None,
           "unit": "ms", "n_gpus": 1, "higher_is_better": False, "data": "synthetic", "dtype": "f32",
           "config": {"workload": "serve128-50M", "form": a.serve_form, "n": n, "d": 128, "R": R,
                      "build": f"exact 2R-NN+prune of {N_BOOT} then inserts (L_ins={a.serve_lins}, T_ins={a.serve_tins})",
                      "cache_rows": slots, "L": cfg.L,
                      "T": cfg.T, "recall@10": rec, "mix": "90:9:1", "batch": "log-uniform 1..2048",
                      "queries": "Zipf(1.1) over components",
                      "small_batches": (", ".join(f"W = {c.W} (T = {c.T}) up to {b} queries" for b, c in small)
                                        + ", else W = 1" if small else None)},
           "small_batch": {str(W): {k: v for k, v in r.items() if k != "cfg"} for W, r in sb.items()},
           "rates": res}
    if res1:
        out["rates_one_warp"] = res1
    if resb:
        out["rates_barrier"] = resb
    print(json.dumps(out), flush=True)
    return 0


# ---------------------------------------------------------------- main
def main():
    a = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    import torch
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group("nccl")
    if a.impl == "reference" and rank != 0:
        return 0
    import paper_2601_08528_b300 as svf
    from paper_2601_08528_b300 import learned as lrn

    t0 = time.time()

    def log_t(*x):
        log(f"[{time.time() - t0:7.1f}s]", *x)

    if a.workload == "serve128-50M":
        return serve_main(a, svf, torch, log_t)
    X = synth.sample_chunked("unit96", a.n, 300)
    Qe_np = synth.sample_chunked("unit96", a.nq, 302 + rank)
    log_t("data", X.shape)
    policies = [p for p in a.serve_policies.split(",") if p]
    # capacity for the inserts of every serving stream: the main one, the
    # one-warp-per-query rerun and the placement ablation
    ratios = [float(x) for x in a.cache_ratios.split(",") if x]
    cpols = [p for p in a.cache_policies.split(",") if p]
    # insert headroom: 300K rows per serving stream, 100K per ablation stream
    ix = build_index(svf, torch, X, log_t, streams=6 + len(policies) + (len(ratios) * len(cpols) + 2) // 3,
                     graph=a.graph)
    Xd = ix.vectors()[:a.n]
    Qe = torch.from_numpy(Qe_np).cuda()
    gt = exact_knn(svf, Xd, Qe, K, "ip")
    torch.cuda.synchronize()
    log_t("ground truth")

    grid = [(32, 40), (32, 48), (64, 32), (64, 36), (64, 38), (64, 40), (64, 44), (64, 48), (64, 56), (64, 64),
            (64, 72), (64, 96), (128, 32), (128, 40), (128, 48), (128, 64), (128, 96), (256, 96), (256, 128)]
    # held-out calibration queries (the first tenth of the training queries):
    # every operating point is chosen on them, never on the timed batch
    ncal = a.ntrain // 10
    Qtr_np = synth.sample_chunked("unit96", a.ntrain, 401)
    Qcal = torch.from_numpy(Qtr_np[:ncal]).cuda()
    gt_cal = exact_knn(svf, Xd, Qcal, K, "ip")
    if a.impl == "reference":
        # the oracle on the headline form (fp8 traversal + exact re-rank) at its
        # cheapest operating point with recall@10 >= target on the calibration
        # queries; each step is one pass over the whole timed batch
        form = "fp8+rerank"
        base = [(form, svf.SearchConfig(k=K, precision="fp8", rerank=True))]
        _, best = select_points(torch, ix, base, grid, a.target, {}, Qcal, gt_cal, Qe, gt)
        op = best.get(form) or {"L": 256, "T": 192}
        g_np = ix.graph[:a.n].cpu().numpy().view(np.uint32)
        timer = OracleTimer(X, g_np, op["L"], op["T"], form)
        steps, cores = [], 0
        for s in range(a.warmup + a.steps):
            q, cores = timer.rate(Qe_np)
            if s >= a.warmup:
                steps.append(q)
        v = statistics.median(steps)
        sample = (f"all {a.nq} queries of the batch per step (median of {a.steps} steps), FP64 fixed-T search over "
                  f"the fp8 copy + exact re-rank at L={op['L']} T={op['T']} on the GPU-built graph")
        out = {"impl": "reference", "metric": METRIC, "value": v, "unit": "queries/s",
               "n_gpus": 1, "steps": a.steps, "warmup": a.warmup, "higher_is_better": True, "scaling": "weak",
               "vs_baseline": None, "dtype": "f64", "data": "synthetic",
               "config": {"workload": unit96_name(a.n), "n": a.n, "d": 96, "R": R, "nq": a.nq, "k": K, "L": op["L"],
                          "T": op["T"], "form": form, "l2": "inputs larger than L2"},
               "cpu_baseline": {"value": v, "unit": "queries/s", "cores": cores, "kind": "oracle", "sample": sample},
               "e2e": {"value": v, "unit": "queries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(out), flush=True)
        return 0

    forms = [("fp32", svf.SearchConfig(k=K)),
             ("bf16+rerank", svf.SearchConfig(k=K, precision="bf16", rerank=True)),
             ("fp8+rerank", svf.SearchConfig(k=K, precision="fp8", rerank=True)),
             ("bf16+rerank+stop", svf.SearchConfig(k=K, precision="bf16", rerank=True)),
             ("fp8+rerank+stop", svf.SearchConfig(k=K, precision="fp8", rerank=True))]
    if a.fixed_point:
        # one form at a given (L, T), no stop networks (profiling runs)
        fname, fl, ft = a.fixed_point.split(",")
        forms, grid, nets = [f for f in forms if f[0] == fname], [(int(fl), int(ft))], {}
    else:
        # learned stop: traces of the plain search of training queries
        Qtr = torch.from_numpy(Qtr_np).cuda()
        nets = train_stops(torch, svf, ix, Qtr, gt_cal, ncal, ["bf16", "fp8"])
        del Qtr
        log_t("stop networks")
    del Qtr_np
    pts, best = select_points(torch, ix, forms, grid, a.target, nets, Qcal, gt_cal, Qe, gt)
    log_t("sweep")
    if not best and a.fixed_point:
        best = {p["form"]: dict(p, recall_cal=p["recall"]) for p in pts}
    if not best:
        raise SystemExit("no form reached the recall target")
    lowp = {k: v for k, v in best.items() if k != "fp32"}
    win = max(lowp.values() if lowp else best.values(), key=lambda p: p["qps"])
    cfg = win["cfg"]
    # what any stop rule could save at the headline point: a stop after the
    # last iteration that changed each query's top 10 (traces of the timed
    # queries) against the iterations the fixed-T search runs
    _, meta = lrn.capture_traces(ix, Qe, dataclasses.replace(cfg, mlp=None))
    ran, last = meta[:, 0].double(), meta[:, 1].double()
    stop_bound = {"L": cfg.L, "T": cfg.T, "form": win["form"], "iters_fixed_T": ran.mean().item(),
                  "iters_perfect_stop": (last + 1).clamp(min=1).mean().item(),
                  "last_change_p50": last.median().item(), "last_change_p90": last.quantile(0.9).item()}
    stop_bound["saving_bound"] = 1.0 - stop_bound["iters_perfect_stop"] / stop_bound["iters_fixed_T"]
    log_t("stop bound", json.dumps(stop_bound))

    # ---- timed region: `steps` launches of the winning form
    st = torch.cuda.current_stream()
    for _ in range(a.warmup):
        ix.search(Qe, cfg)
    torch.cuda.synchronize()
    ix.stats_reset()
    clocks = Clocks()
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(a.steps)]
    ids_out = torch.empty((a.nq, K), dtype=torch.int32, device="cuda")
    d_out = torch.empty((a.nq, K), dtype=torch.float32, device="cuda")
    torch.cuda.nvtx.range_push("timed")
    for e0, e1 in evs:
        e0.record(st)
        ix.search(Qe, cfg, out_ids=ids_out, out_dist=d_out)
        e1.record(st)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    if dist:
        dist.barrier()
    per = [e0.elapsed_time(e1) / 1e3 for e0, e1 in evs]
    total = max_over_ranks(sum(per), dist)
    s = ix.stats()
    # ---- end to end: pinned host queries in, results out, every step
    Qh = torch.from_numpy(Qe_np).pin_memory()
    ids_h = torch.empty((a.nq, K), dtype=torch.int32).pin_memory()
    d_h = torch.empty((a.nq, K), dtype=torch.float32).pin_memory()
    # Double-buffered pipeline through the public API: step k's search runs on
    # the compute stream while a copy stream uploads step k+1's queries and
    # downloads step k-1's results (every step still moves its full batch).
    Qd = [torch.empty_like(Qe), torch.empty_like(Qe)]
    io = [torch.empty_like(ids_out), torch.empty_like(ids_out)]
    do = [torch.empty_like(d_out), torch.empty_like(d_out)]
    cs = torch.cuda.Stream()
    ev = lambda: torch.cuda.Event()
    up, srch = [ev(), ev()], [ev(), ev()]
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    cs.wait_event(e0)
    with torch.cuda.stream(cs):
        Qd[0].copy_(Qh, non_blocking=True)
        up[0].record(cs)
    for k in range(a.steps):
        b = k & 1
        st.wait_event(up[b])
        ix.search(Qd[b], cfg, out_ids=io[b], out_dist=do[b], stream=st)
        srch[b].record(st)
        with torch.cuda.stream(cs):
            if k + 1 < a.steps:
                if k >= 1:
                    cs.wait_event(srch[b ^ 1])  # step k-1's search has read its buffer
                Qd[b ^ 1].copy_(Qh, non_blocking=True)
                up[b ^ 1].record(cs)
            cs.wait_event(srch[b])
            ids_h.copy_(io[b], non_blocking=True)
            d_h.copy_(do[b], non_blocking=True)
    st.wait_stream(cs)
    e1.record(st)
    e1.synchronize()
    e2e_t = max_over_ranks(e0.elapsed_time(e1) / 1e3, dist)
    clk = clocks.stop(torch.cuda.current_device())
    # ---- latency-bound batches: several warps per query (not timed above)
    sb = small_batch(svf, torch, ix, Qe, gt, cfg, a.target, sizes=(1, 16, 256, 1024))
    log_t("small batches", {W: {k: v for k, v in r.items() if k != "cfg"} for W, r in sb.items()})
    # insert throughput: 1M new vectors in one batch (the later legs run on
    # the grown index)
    ins_rate = insert_rate(svf, torch, ix, synth.sample_chunked("unit96", MAX_BATCH, 303))
    log_t("inserts/s", ins_rate)

    # ---- roofline of the search kernel (the only launch of a step)
    nq = a.nq
    form = win["form"]
    row_b = ROW_BYTES["bf16" if form.startswith("bf16") else "fp8" if form.startswith("fp8") else "f32"]
    iters, evals = s["search_iters"] / a.steps, s["search_evals"] / a.steps
    alg = iters * R * 4 + evals * row_b + nq * (96 * 4 + K * 8)
    if cfg.rerank:
        alg += nq * cfg.L * 384
    mean_launch = total / a.steps
    peaks, src = measured_peaks()
    achieved = alg / mean_launch / 1e9
    # the random-row fetch ceiling: the kernel's own copy pattern over uniform
    # random rows of the traversal store, nothing computed (svf_gather_probe)
    tstore, tpitch, trow = ((ix.vecs_fp8, 128, 112) if form.startswith("fp8") else
                            (ix.vecs_bf16, 192, 192) if form.startswith("bf16") else (ix.vecs, 384, 384))
    fetched = iters + evals + (nq * cfg.L if cfg.rerank else 0)
    by_w = {}
    for wps in (16, 24, 32):
        got, ms = svf.gather_probe(tstore, ix.n_used, tpitch, trow, int(evals), warps_per_sm=wps, seed=11 + wps)
        by_w[wps] = got / (ms / 1e3)
    best_w = max(by_w, key=by_w.get)
    gather = {"rows_per_s": by_w[best_w], "row_bytes": trow, "warps_per_sm": best_w,
              "rows_per_s_by_warps_per_sm": {str(w): v for w, v in by_w.items()},
              "kernel_rows_per_s": fetched / mean_launch, "frac": fetched / mean_launch / by_w[best_w],
              "note": "kernel rows = graph rows + traversal rows + re-rank rows per launch, each one random fetch"}
    log_t("gather ceiling", gather)
    out = {
        "metric": METRIC,
        "value": job_rate(nq * a.steps, world, total),
        "unit": "queries/s",
        "n_gpus": world, "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * total / a.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": form.split("+")[0],
        "data": "synthetic",
        "config": {"workload": unit96_name(a.n), "n": a.n, "d": 96, "R": R, "nq": nq, "k": K, "form": form,
                   "L": cfg.L, "T": cfg.T, "tau": getattr(cfg, "tau", None) if cfg.mlp is not None else None,
                   "recall@10": win["recall"], "l2": f"inputs larger than L2 ({a.n * 96 * 4 / 1e9:.1f} GB store, {a.n * R * 4 / 1e9:.1f} GB graph)",
                   "graph": ix.graph_desc, "build_s": ix.build_s, "build_rows_by_exact_scan": ix.build_fallback},
        "forms": {k: {"qps": v["qps"], "recall@10": v["recall"], "recall@10_calibration": v["recall_cal"],
                      "L": v["L"], "T": v["T"], "iters": v["iters"]} for k, v in best.items()},
        "stop_bound": stop_bound,
        "operating_point": "each form's cheapest swept (L, T) with recall@10 >= target on 20,000 held-out "
                           "calibration queries; recall and QPS measured on the 10,000 timed queries",
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                     "frac": achieved / peaks["hbm_gbs"], "traffic": profiled_traffic(form, cfg.L, cfg.T),
                     "peak_source": src,
                     "alg_bytes_per_launch": alg, "iters_per_launch": iters, "evals_per_launch": evals,
                     "hash_resets_per_launch": s["hash_resets"] / a.steps, "gather_ceiling": gather},
        "e2e": {"value": job_rate(nq * a.steps, world, e2e_t), "unit": "queries/s",
                "h2d_bytes_per_step": Qh.numel() * 4, "d2h_bytes_per_step": ids_h.numel() * 4 + d_h.numel() * 4},
        "gpu_launches": a.steps,
        "clocks": clk,
        "small_batch": {"form": form, "L": cfg.L,
                        "note": "W warps per query expand W parents per iteration; latency of one call of the "
                                "public API on a batch of b queries (CUDA events, host overhead included)",
                        "by_W": {str(W): {k: v for k, v in r.items() if k != "cfg"} for W, r in sb.items()}},
    }
    # global consolidation after 20 % deletes (before the store is tiered)
    gone = None
    if a.consolidate:
        out["consolidation"], gone = consolidation(svf, torch, ix, Qe, cfg)
        log_t("consolidation", json.dumps(out["consolidation"]))
    # serving: the same index with its fp32 rows tiered behind a device cache
    # of 31 % of them (the 8 GB : 25.6 GB ratio of the 50M serving workload),
    # fp8 traversal resident, exact re-rank through the tier; an open-loop
    # Poisson stream of uneven batches with inserts and deletes
    if a.serve_rate > 0:
        tier = dict(M=int(a.n * a.serve_cache_frac), theta0=2.0, promote_batch=2048, sweep=4, qcap=16384)
        win_arg = tuple(float(x) for x in a.serve_window.split(",")) if a.serve_window else None
        if win_arg:
            win_arg = (int(win_arg[0]), win_arg[1])
        sopt = dict(maintain_every=a.serve_maintain_every, window=win_arg)
        # the buffers hold the largest cache any run below uses; runs reset it smaller
        m_alloc = int(a.n * max([a.serve_cache_frac] + ratios))
        ix.enable_tier(**dict(tier, M=m_alloc))
        if m_alloc != tier["M"]:
            ix.reset_tier(**tier)
        X_ins = synth.sample_chunked("unit96", 200_000, 305)
        if a.serve_trav == "fp32":
            fp = best.get("fp32", {"L": 64, "T": 96})
            cfg = svf.SearchConfig(k=K, L=fp["L"], T=fp["T"])
            trav = "fp32 traversal through the tier"
        else:
            trav = "fp8 traversal + exact re-rank"
        # latency-bound batches take the several-warps-per-query path, W by
        # batch size from the one-call latencies measured above
        if a.serve_trav != "fp32":
            sopt["small"] = w_policy(sb)
        out["serving"] = serve_stream(svf, torch, ix, "unit96", X_ins, a.serve_rate, a.serve_seconds, 1.0, 306, cfg,
                                      **sopt)
        qmix = (f"queries from a window of {win_arg[0]} components moving {win_arg[1]:g}/s" if win_arg
                else "Zipf(1.1) queries")
        out["serving"]["workload"] = (f"unit96-10M tiered: fp32 rows in pinned host memory behind a "
                                      f"{tier['M'] / 1e6:.1f}M-row device cache, {trav}, {qmix}, 90:9:1 mix, "
                                      "batches log-uniform 1..2048")
        out["serving"]["policy"] = "wavp"
        if sopt.get("small"):
            out["serving"]["small_batches"] = ", ".join(f"W = {c.W} (T = {c.T}) up to {b} queries"
                                                        for b, c in sopt["small"]) + ", else W = 1"
        log_t("serving", json.dumps(out["serving"]))
        # the same stream (same seed, re-tiered cache) under the other two
        # consistency modes: a search waits for every update submitted before
        # it, or every update waits for the searches and runs alone
        for mode in ("read-after-write", "barrier"):
            ix.reset_tier(policy="wavp", **tier)
            r = serve_stream(svf, torch, ix, "unit96", X_ins, a.serve_rate, a.serve_seconds, 1.0, 306, cfg,
                             **dict(sopt, consistency=mode))
            out["serving_" + mode.replace("-", "_")] = r
            log_t("serving", mode, json.dumps(r))
        if a.raw_rates:
            # Table 3's experiment: half inserts of 10 vectors, half searches for them
            ix.reset_tier(policy="wavp", **tier)
            X_raw = synth.sample_chunked("unit96", 200_000, 308)
            out["read_after_write"] = read_after_write(svf, torch, ix, X_raw,
                                                       [float(x) for x in a.raw_rates.split(",")], cfg,
                                                       seconds=a.raw_seconds)
            out["read_after_write"]["note"] = ("requests alternate an insert of 10 new vectors and a search for "
                                               "them (Poisson arrivals); recall@1 = the vector itself returned first")
        if sopt.get("small"):
            # the same stream (same seed, re-tiered cache) with one warp per query throughout
            ix.reset_tier(policy="wavp", **tier)
            one = dict(sopt, small=None)
            out["serving_one_warp"] = serve_stream(svf, torch, ix, "unit96", X_ins, a.serve_rate, a.serve_seconds,
                                                   1.0, 306, cfg, **one)
            log_t("serving one warp per query", json.dumps(out["serving_one_warp"]))
        # placement ablation: the same stream (same seed) after re-tiering the
        # same index under each other policy
        if policies:
            out["serving_policies"] = {"wavp": out["serving"]}
            for p in policies:
                ix.reset_tier(policy=p, **tier)
                r = serve_stream(svf, torch, ix, "unit96", X_ins, a.serve_rate, a.serve_seconds, 1.0, 306, cfg,
                                 **sopt)
                r["policy"] = p
                out["serving_policies"][p] = r
                log_t("serving", p, json.dumps(r))
        if ratios:
            # placement ablation (Sec. 6.3) on a moving hot set: queries from a
            # window of 64 components advancing 4 per second, every traversal
            # row (fp32) read through the tier, maintenance every 16 search
            # batches; each policy at each cache size, from a cold start
            fp = best.get("fp32", {"L": 64, "T": 96})
            c32 = svf.SearchConfig(k=K, L=fp["L"], T=fp["T"])
            wopt = dict(maintain_every=16, window=(64, 4.0))
            sweep_out = {"workload": (f"unit96-10M tiered, fp32 traversal through the tier (L={fp['L']}, T={fp['T']}), "
                                      f"queries from a window of 64 components moving 4/s, {a.cache_rate:g} req/s "
                                      f"for {a.cache_seconds:g} s, 90:9:1 mix, maintenance every 16 search batches"),
                         "by_ratio": {}}
            for r in ratios:
                row = {}
                for p in cpols:
                    ix.reset_tier(**dict(tier, M=int(a.n * r), policy=p))
                    res = serve_stream(svf, torch, ix, "unit96", X_ins, a.cache_rate, a.cache_seconds, 1.0, 309, c32,
                                       **wopt)
                    row[p] = {"cache_hit_rate": res["cache_hit_rate"], "qps": res["qps"], "promoted": res["promoted"],
                              "search_p50_ms": res["latency_ms"]["search"]["p50"],
                              "search_p99_ms": res["latency_ms"]["search"]["p99"]}
                    log_t("cache ablation", r, p, json.dumps(row[p]))
                sweep_out["by_ratio"][f"{r:g}"] = row
            out["cache_ablation"] = sweep_out
    # deletes (1% of the index, uniformly drawn live ids) with localized repair
    dels = torch.from_numpy(synth.pick_live_ids(a.n, gone, a.n // 100, 304).view(np.int32)).cuda()
    torch.cuda.synchronize()
    t_del = time.time()
    ix.delete(dels)
    torch.cuda.synchronize()
    t_del = time.time() - t_del
    out["updates"] = {"inserts_per_s": ins_rate, "insert_batch": MAX_BATCH, "L_ins": 64, "T_ins": 48,
                      "deletes_per_s": dels.numel() / t_del, "delete_batch": dels.numel(),
                      "repaired_rows": ix.stats()["repaired_rows"]}
    if a.u8 and rank == 0:
        out["u8_1M"] = u8_leg(svf, torch, log_t)
    if rank == 0:
        # oracle timed on host cores: the headline form at the headline (L, T)
        # (a stop form is timed without its network, i.e. for the full T)
        hf, hc = win["form"].replace("+stop", ""), win["cfg"]
        g_np = ix.graph[:a.n].cpu().numpy().view(np.uint32)
        qps, cores = OracleTimer(X, g_np, hc.L, hc.T, hf).rate(Qe_np)
        out["cpu_baseline"] = {"value": qps, "unit": "queries/s", "cores": cores, "kind": "oracle",
                               "sample": f"all {a.nq} queries of the batch, FP64 fixed-T search in the {hf} form at "
                                         f"L={hc.L} T={hc.T} on the same graph"}
        print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
