"""A graph index on one GPU: torch allocates the device buffers, libsvf runs.

``Index`` owns torch tensors for every buffer the C ABI borrows and forwards
Build / Search / Insert / Delete (SVFusion Sec. 2.2) to the library.  Nothing
here computes: inputs are checked for dtype/shape/device and passed by
pointer on the current CUDA stream.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import torch

from . import _lib as L


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


@dataclass
class SearchConfig:
    k: int = 10
    L: int = 64
    T: int = 32
    precision: str | None = None   # None: primary; "bf16" / "fp8"
    rerank: bool = False
    seed: int = 0
    hash_log2: int = 0
    mlp: torch.Tensor | None = None  # packed bf16 stop network (device)
    tau: float = 0.5
    t_min: int = 4
    t_every: int = 1
    W: int = 1     # parents per iteration = warps per query (1, 2, 4, 8)


class Index:
    def __init__(self, d: int, n_cap: int, dtype: str = "f32", metric: str = "l2", R: int = 32,
                 prune: str = "rng", repair_c: int = 8, lowp: tuple[str, ...] = (), seed: int = 0x5F0C,
                 max_batch: int = 100_000, device: str | torch.device = "cuda"):
        lib = L.load()
        dev = torch.device(device)
        if dev.type == "cuda" and dev.index is None:
            dev = torch.device("cuda", torch.cuda.current_device())
        self.device = dev
        self.d, self.n_cap, self.R = d, n_cap, R
        self.dtype, self.metric = dtype, metric
        self.params = L.Params(d, L.U8 if dtype == "u8" else L.F32, L.IP if metric == "ip" else L.L2, R, n_cap,
                               L.PRUNE_RANK if prune == "rank" else L.PRUNE_RNG, repair_c,
                               (1 if "bf16" in lowp else 0) | (2 if "fp8" in lowp else 0), 0, seed)
        sz = L.Sizes()
        L.check(lib.svf_buffer_sizes(C.byref(self.params), max(1, max_batch), C.byref(sz)))
        u8 = torch.uint8

        def buf(nbytes):
            return torch.empty(max(int(nbytes), 256), dtype=u8, device=self.device) if nbytes else None

        self.vecs = buf(sz.vecs)
        self.vecs_bf16 = buf(sz.vecs_bf16)
        self.vecs_fp8 = buf(sz.vecs_fp8)
        self.graph_buf = buf(sz.graph)
        self.del_buf = buf(sz.del_bits)
        self.workspace = buf(sz.workspace)
        self.status = buf(sz.status)
        b = L.Buffers(self.vecs.data_ptr(), _ptr(self.vecs_bf16) and self.vecs_bf16.data_ptr(),
                      _ptr(self.vecs_fp8) and self.vecs_fp8.data_ptr(), self.graph_buf.data_ptr(),
                      self.del_buf.data_ptr(), self.workspace.data_ptr(), self.workspace.numel(),
                      self.status.data_ptr(), self.status.numel())
        h = C.c_void_p()
        with torch.cuda.device(self.device):
            L.check(lib.svf_create(C.byref(self.params), C.byref(b), C.byref(h)))
        self._h = h
        self.n_used = 0

    # ------------------------------------------------------------ views
    @property
    def graph(self) -> torch.Tensor:
        """[n_cap, R] int32 view of the graph (0xFFFFFFFF reads as -1)."""
        return self.graph_buf[: self.n_cap * self.R * 4].view(torch.int32).view(self.n_cap, self.R)

    @property
    def del_bits(self) -> torch.Tensor:
        return self.del_buf[: (self.n_cap + 31) // 32 * 4].view(torch.int32)

    def vectors(self) -> torch.Tensor:
        esz = 1 if self.dtype == "u8" else 4
        t = self.vecs[: self.n_cap * self.d * esz]
        return t.view(self.n_cap, self.d) if self.dtype == "u8" else t.view(torch.float32).view(self.n_cap, self.d)

    def _qcheck(self, X: torch.Tensor):
        want = torch.uint8 if self.dtype == "u8" else torch.float32
        if X.dtype != want or X.dim() != 2 or X.shape[1] != self.d or X.device != self.device:
            raise ValueError(f"expected a {want} [m, {self.d}] tensor on {self.device}")
        return X.contiguous()

    # ------------------------------------------------------------ operations
    def build(self, X: torch.Tensor, stream=None) -> None:
        X = self._qcheck(X)
        L.check(L.load().svf_build(self._h, _ptr(X), X.shape[0], _stream(stream)))
        self.n_used = X.shape[0]

    def attach(self, X: torch.Tensor, graph: torch.Tensor, deleted=None) -> None:
        """Load an index built elsewhere (vectors, graph rows, deleted ids)."""
        X = self._qcheck(X)
        n = X.shape[0]
        self.vectors()[:n].copy_(X)
        g = graph.to(self.device, torch.int32) if graph.dtype != torch.int32 else graph.to(self.device)
        self.graph[:n].copy_(g)
        self.del_bits.zero_()
        if deleted is not None and len(deleted):
            import numpy as np
            bits = np.zeros((self.n_cap + 31) // 32, dtype=np.uint32)
            for i in np.asarray(deleted, dtype=np.int64):
                bits[i >> 5] |= np.uint32(1 << (int(i) & 31))
            self.del_bits.copy_(torch.from_numpy(bits.view(np.int32)))
        lib = L.load()
        if self.params.lowp & 1:
            L.check(lib.svf_encode_bf16(_ptr(X), n, self.d, _ptr(self.vecs_bf16), _stream()))
        if self.params.lowp & 2:
            L.check(lib.svf_encode_fp8(_ptr(X), n, self.d, _ptr(self.vecs_fp8), (self.d + 4 + 31) // 32 * 32,
                                       _stream()))
        torch.cuda.synchronize(self.device)
        L.check(lib.svf_attach(self._h, n))
        self.n_used = n

    def search(self, Q: torch.Tensor, cfg: SearchConfig, out_ids=None, out_dist=None, stream=None, qkeys=None,
               trace_feat=None, trace_meta=None, pool_out=None):
        Q = self._qcheck(Q)
        nq = Q.shape[0]
        if out_ids is None:
            out_ids = torch.empty((nq, cfg.k), dtype=torch.int32, device=self.device)
        if out_dist is None:
            out_dist = torch.empty((nq, cfg.k), dtype=torch.int32 if self.dtype == "u8" else torch.float32,
                                   device=self.device)
        prec = {None: L.U8 if self.dtype == "u8" else L.F32, "bf16": L.BF16, "fp8": L.FP8}[cfg.precision]
        import math
        z_tau = math.log(cfg.tau / (1.0 - cfg.tau)) if cfg.mlp is not None else 0.0
        sp = L.SearchParams(cfg.k, cfg.L, cfg.T, prec, int(cfg.rerank), cfg.t_min, _ptr(cfg.mlp), z_tau,
                            cfg.hash_log2, _ptr(qkeys), cfg.seed, _ptr(trace_feat), _ptr(trace_meta), _ptr(pool_out),
                            cfg.t_every, cfg.W)
        L.check(L.load().svf_search(self._h, _ptr(Q), nq, C.byref(sp), _ptr(out_ids), _ptr(out_dist),
                                    _stream(stream)))
        return out_ids, out_dist

    def insert(self, X: torch.Tensor, L_ins: int = 64, T_ins: int = 32, stream=None) -> torch.Tensor:
        X = self._qcheck(X)
        ids = torch.empty(X.shape[0], dtype=torch.int32, device=self.device)
        L.check(L.load().svf_insert(self._h, _ptr(X), X.shape[0], L_ins, T_ins, _ptr(ids), _stream(stream)))
        self.n_used += X.shape[0]
        return ids

    def delete(self, ids: torch.Tensor, stream=None) -> int:
        ids = ids.to(self.device, torch.int32).contiguous()
        newly = torch.zeros(1, dtype=torch.int64, device=self.device)
        L.check(L.load().svf_delete(self._h, _ptr(ids), ids.numel(), _ptr(newly), _stream(stream)))
        return int(newly.item())

    # ------------------------------------------------------------ global consolidation
    def consolidate_begin(self, log_rows: int = 1_000_000, stream=None) -> None:
        """Snapshot the graph for a global consolidation (svf_consolidate_begin);
        up to log_rows inserted rows may be logged until the commit."""
        lib = L.load()
        nbytes = C.c_size_t(0)
        L.check(lib.svf_consolidate_sizes(C.byref(self.params), log_rows, C.byref(nbytes)))
        buf = torch.empty(max(int(nbytes.value), 256), dtype=torch.uint8, device=self.device)
        L.check(lib.svf_consolidate_begin(self._h, _ptr(buf), nbytes.value, log_rows, _stream(stream)))
        self._cons_buf = buf  # borrowed by the library until commit / abort

    def consolidate_run(self, cap: int = 0, stream=None) -> int:
        """Consolidate the snapshot (may run on its own stream; cap: most
        candidates per row, 0 = automatic); returns the number of rows it
        rewrites."""
        rows = C.c_int64(0)
        L.check(L.load().svf_consolidate_run(self._h, cap, C.byref(rows), _stream(stream)))
        return int(rows.value)

    def consolidate_commit(self, stream=None) -> None:
        """Merge the consolidated snapshot into the active graph."""
        try:
            L.check(L.load().svf_consolidate_commit(self._h, _stream(stream)))
        finally:
            self._cons_buf = None

    def consolidate_abort(self) -> None:
        L.check(L.load().svf_consolidate_abort(self._h))
        self._cons_buf = None

    def consolidate(self, cap: int = 0, stream=None) -> int:
        """begin + run + commit on one stream; returns the rewritten rows."""
        self.consolidate_begin(0, stream)
        rows = self.consolidate_run(cap, stream)
        self.consolidate_commit(stream)
        return rows

    # ------------------------------------------------------------ tiered store
    def enable_tier(self, M: int, qcap: int = 16384, promote_batch: int = 2048, sweep: int = 4, alpha: float = 0.6,
                    beta: float = 0.4, theta0: float = 2.0, decay_every: int = 1 << 16, policy: str = "wavp",
                    lrfu_lambda: float = 0.5) -> None:
        """Move the primary rows to pinned host memory behind a device cache of
        M rows with workload-aware placement (see svf_tier_enable; policy:
        wavp, clock, lfu, static, lru or lrfu)."""
        lib = L.load()
        tp = L.TierParams(M, qcap, promote_batch, sweep, alpha, beta, theta0, decay_every, L.TIER_POLICIES[policy],
                          lrfu_lambda)
        sz = L.TierSizes()
        L.check(lib.svf_tier_buffer_sizes(C.byref(self.params), C.byref(tp), C.byref(sz)))
        u8 = torch.uint8
        dev = ("cache", "map", "owner", "ref", "freq", "ein", "queue", "scratch")
        self.tier_bufs = {f: torch.empty(max(int(getattr(sz, f)), 256), dtype=u8, device=self.device)
                          for f in dev + ("slot_stat",)}
        self.host_store = torch.empty(int(sz.host), dtype=u8).pin_memory()
        tb = L.TierBuffers(*[self.tier_bufs[f].data_ptr() for f in dev], self.host_store.data_ptr(),
                           self.tier_bufs["slot_stat"].data_ptr())
        L.check(lib.svf_tier_enable(self._h, C.byref(tp), C.byref(tb), _stream()))
        torch.cuda.synchronize(self.device)

    def reset_tier(self, M: int, qcap: int = 16384, promote_batch: int = 2048, sweep: int = 4, alpha: float = 0.6,
                   beta: float = 0.4, theta0: float = 2.0, decay_every: int = 1 << 16, policy: str = "wavp",
                   lrfu_lambda: float = 0.5) -> None:
        """Re-initialise the tiered store with new placement parameters (see
        svf_tier_reset); M may shrink to any size up to the enabled one."""
        tp = L.TierParams(M, qcap, promote_batch, sweep, alpha, beta, theta0, decay_every, L.TIER_POLICIES[policy],
                          lrfu_lambda)
        L.check(L.load().svf_tier_reset(self._h, C.byref(tp), _stream()))
        torch.cuda.synchronize(self.device)

    def release_device_store(self) -> None:
        """After enable_tier the device copy of the primary rows is not read;
        free it (vectors() is unavailable afterwards)."""
        self.vecs = None
        torch.cuda.empty_cache()

    def tier_map(self) -> torch.Tensor:
        return self.tier_bufs["map"][: self.n_cap * 4].view(torch.int32)

    def maintain(self, stream=None) -> int:
        n = C.c_int64(0)
        L.check(L.load().svf_tier_maintain(self._h, C.byref(n), _stream(stream)))
        return int(n.value)

    def theta(self) -> float:
        return float(L.load().svf_tier_theta(self._h))

    def sync(self) -> None:
        L.check(L.load().svf_sync(self._h))

    def stats(self) -> dict:
        c = L.Counters()
        L.check(L.load().svf_stats(self._h, C.byref(c)))
        return {f: getattr(c, f) for f, _ in L.Counters._fields_}

    def stats_reset(self) -> None:
        L.check(L.load().svf_stats_reset(self._h))

    def close(self) -> None:
        if getattr(self, "_h", None):
            L.load().svf_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def knn(X: torch.Tensor, Q: torch.Tensor, k: int, metric: str = "l2", self_ids: torch.Tensor | None = None,
        stream=None):
    """Exact brute-force kNN on the GPU (ground truth)."""
    lib = L.load()
    dt = L.U8 if X.dtype == torch.uint8 else L.F32
    X = X.contiguous()
    Q = Q.contiguous()
    nq = Q.shape[0]
    work = torch.empty((nq, k), dtype=torch.int64, device=X.device)
    ids = torch.empty((nq, k), dtype=torch.int32, device=X.device)
    dist = torch.empty((nq, k), dtype=torch.int32 if dt == L.U8 else torch.float32, device=X.device)
    L.check(lib.svf_knn(_ptr(X), X.shape[0], X.shape[1], dt, L.IP if metric == "ip" else L.L2, _ptr(Q), nq,
                        _ptr(self_ids), k, _ptr(work), _ptr(ids), _ptr(dist), _stream(stream)))
    return ids, dist


class Server:
    """Continuous-batching request loop (svf_serve_*): submit searches,
    inserts and deletes; poll completions with host timestamps."""

    CONSISTENCY = {"barrier": 0, "read-after-write": 1, "snapshot": 2}

    def __init__(self, ix: Index, max_inflight: int = 8, n_streams: int = 4, maintain_every: int = 64,
                 consistency: str = "barrier", shadow_rows: int | None = None):
        """consistency: "barrier" (an update drains the searches and runs
        alone), "read-after-write" (updates overlap earlier searches; a search
        sees every update submitted before it) or "snapshot" (a search sees
        the updates completed when it is admitted and never waits).  The two
        versioned modes keep a device version buffer for up to `shadow_rows`
        rewritten rows per update (default 2,048 inserted vectors' worth)."""
        self.ix = ix
        self.lib = L.load()
        h = C.c_void_p()
        mode = self.CONSISTENCY[consistency]
        self.versions = None
        vb, rows = 0, 0
        if mode:
            rows = shadow_rows or 2048 * ix.R
            vb = int(self.lib.svf_serve_version_bytes(ix._h, rows))
            self.versions = torch.empty(vb, dtype=torch.uint8, device=ix.device)
        cfg = L.ServeCfg(max_inflight, n_streams, maintain_every, mode, _ptr(self.versions), vb, rows)
        with torch.cuda.device(ix.device):
            L.check(self.lib.svf_serve_start(ix._h, C.byref(cfg), C.byref(h)))
        self._s = h
        self._keep = {}

    @staticmethod
    def now() -> float:
        return float(L.load().svf_serve_now())

    def _submit(self, r, keep):
        self._keep[r.tag] = keep
        L.check(self.lib.svf_serve_submit(self._s, C.byref(r)))

    def search(self, tag: int, Q: torch.Tensor, cfg: SearchConfig, out_ids: torch.Tensor, out_dist: torch.Tensor,
               t_arrival: float = 0.0):
        prec = {None: L.U8 if self.ix.dtype == "u8" else L.F32, "bf16": L.BF16, "fp8": L.FP8}[cfg.precision]
        import math
        z_tau = math.log(cfg.tau / (1.0 - cfg.tau)) if cfg.mlp is not None else 0.0
        sp = L.SearchParams(cfg.k, cfg.L, cfg.T, prec, int(cfg.rerank), cfg.t_min, _ptr(cfg.mlp), z_tau,
                            cfg.hash_log2, None, cfg.seed, None, None, None, cfg.t_every, cfg.W)
        r = L.Request(L.OP_SEARCH, Q.shape[0], Q.data_ptr(), sp, out_ids.data_ptr(), out_dist.data_ptr(), None, 0, 0,
                      tag, t_arrival)
        self._submit(r, (Q, out_ids, out_dist, cfg))

    def insert(self, tag: int, X: torch.Tensor, L_ins: int = 64, T_ins: int = 32, out_ids=None, t_arrival: float = 0.0):
        r = L.Request(L.OP_INSERT, X.shape[0], X.data_ptr(), L.SearchParams(), None, None, _ptr(out_ids), L_ins,
                      T_ins, tag, t_arrival)
        self._submit(r, (X, out_ids))
        self.ix.n_used += X.shape[0]

    def delete(self, tag: int, ids: torch.Tensor, t_arrival: float = 0.0):
        r = L.Request(L.OP_DELETE, ids.numel(), ids.data_ptr(), L.SearchParams(), None, None, None, 0, 0, tag,
                      t_arrival)
        self._submit(r, (ids,))

    def poll(self, max_n: int = 4096) -> list[dict]:
        buf = (L.Completion * max_n)()
        n = C.c_int32(0)
        L.check(self.lib.svf_serve_poll(self._s, buf, max_n, C.byref(n)))
        out = []
        for i in range(n.value):
            c = buf[i]
            self._keep.pop(c.tag, None)
            out.append({f: getattr(c, f) for f, _ in L.Completion._fields_})
        return out

    def drain(self, timeout: float = 600.0) -> None:
        L.check(self.lib.svf_serve_drain(self._s, timeout))

    def stop(self) -> None:
        if self._s:
            L.check(self.lib.svf_serve_stop(self._s))
            self._s = None


def knn_tc(X: torch.Tensor, Q: torch.Tensor, k: int, metric: str = "l2", stream=None):
    """Exact kNN on the tensor cores (fp32, d <= 128, k <= 32).  Returns
    (ids, dists, number of queries recomputed by the SIMT fallback)."""
    lib = L.load()
    X = X.contiguous()
    Q = Q.contiguous()
    n, d = X.shape
    nq = Q.shape[0]
    nbytes = int(lib.svf_knn_tc_scratch_bytes(n, nq, d, k))
    scratch = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=X.device)
    ids = torch.empty((nq, k), dtype=torch.int32, device=X.device)
    dist = torch.empty((nq, k), dtype=torch.float32, device=X.device)
    fb = C.c_int64(0)
    L.check(lib.svf_knn_tc(_ptr(X), n, d, L.IP if metric == "ip" else L.L2, _ptr(Q), nq, k, _ptr(scratch), nbytes,
                           _ptr(ids), _ptr(dist), C.byref(fb), _stream(stream)))
    return ids, dist, int(fb.value)


def gather_probe(table: torch.Tensor, n: int, pitch: int, row_bytes: int, rows: int, warps_per_sm: int = 24,
                 seed: int = 1, stream=None):
    """Random-row fetch ceiling (svf_gather_probe): about `rows` rows of
    `row_bytes` bytes at uniform random ids of the first n rows of `table`
    (device, rows `pitch` bytes apart), copied by the search kernel's copy
    pattern with no arithmetic.  Returns (rows copied, device milliseconds)."""
    lib = L.load()
    status = torch.zeros(2, dtype=torch.int64, device=table.device)
    nrows = C.c_int64(0)
    ms = C.c_float(0.0)
    L.check(lib.svf_gather_probe(_ptr(table), n, pitch, row_bytes, rows, warps_per_sm, seed, _ptr(status),
                                 C.byref(nrows), C.byref(ms), _stream(stream)))
    return int(nrows.value), float(ms.value)
