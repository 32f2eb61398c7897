"""Python face of the FP64 CPU oracle (``svf_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, the package's smoke check and the
benchmark's CPU-baseline leg are the only callers.  Nothing here imports the
CUDA package, and the CUDA package never imports this.

Every function takes and returns numpy arrays.  Stores are described by
(rows, dtype, metric); the helpers here lay rows out exactly as the C code
expects (fp32 / uint8 / bf16 codes / FP8 codes + fp32 scale at byte d).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "svf_oracle.c")
_LIB = os.path.join(_HERE, "liborc.so")

EMPTY = 0xFFFFFFFF
F32, U8, BF16, FP8 = 0, 1, 2, 3
L2, IP = 0, 1
PRUNE_RNG, PRUNE_RANK = 0, 1
_DT = {"f32": F32, "u8": U8, "bf16": BF16, "fp8": FP8}
_MT = {"l2": L2, "ip": IP}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, FP64, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
                               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


class _Store(C.Structure):
    _fields_ = [("data", C.c_void_p), ("n", C.c_int64), ("d", C.c_int32), ("dtype", C.c_int32),
                ("pitch", C.c_int64), ("metric", C.c_int32), ("pad_", C.c_int32)]


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        P, I64, I32, U64, D = C.c_void_p, C.c_int64, C.c_int32, C.c_uint64, C.c_double
        S = C.POINTER(_Store)
        sig = {
            "orc_splitmix64": (U64, [U64]),
            "orc_query_key": (U64, [P, I64]),
            "orc_bf16_encode": (C.c_uint16, [C.c_float]),
            "orc_bf16_decode": (D, [C.c_uint16]),
            "orc_e4m3_encode": (C.c_uint8, [C.c_float]),
            "orc_e4m3_decode": (D, [C.c_uint8]),
            "orc_fp8_encode_rows": (None, [P, I64, I32, P, I64]),
            "orc_bf16_encode_rows": (None, [P, I64, I32, P, I64]),
            "orc_knn": (None, [S, P, P, I64, P, I32, P, P, P]),
            "orc_prune": (D, [S, P, P, P, I32, I32, P, I32, I32, P]),
            "orc_build": (None, [S, I32, I32, P, P]),
            "orc_search": (I32, [S, I64, P, I32, P, P, I64, P, I32, I32, I32, U64, I32, P, P, P, P, P, P, P]),
            "orc_insert": (None, [S, I64, I64, P, I32, P, I32, I32, U64, I32, P, P]),
            "orc_delete": (I64, [S, I64, P, I32, P, P, I64, I32, I32, P, P]),
            "orc_consolidate": (I64, [S, I64, P, I32, P, I32, I32, P]),
            "orc_consolidate_rows": (I64, [S, I64, P, I32, P, I32, I32, P, I64, P, P]),
            "orc_reverse_patch": (None, [S, P, I32, P, I64, I64, P, I64, P]),
            "orc_threads": (I32, []),
            "orc_set_threads": (None, [I32]),
            "orc_mlp_forward": (None, [P, P, P, D, P, I64, P, P]),
            "orc_mlp_backward": (D, [P, P, P, D, P, P, I64, P, P, P, P]),
            "orc_search_ex": (None, [S, I64, P, I32, P, P, I64, P, I32, I32, I32, U64, P, P, P, P, P, P,
                                     P, P, P, D, D, I32, I32, P, P]),
            "orc_dist_ids": (None, [S, P, I64, P, I32, P]),
            "orc_wavp_round": (None, [I64, P, P, P, P, P, P, I64, I64, I64, I64, D, D, P, P]),
        }
        for name, (res, args) in sig.items():
            if not hasattr(_lib, name):
                continue
            f = getattr(_lib, name)
            f.restype = res
            f.argtypes = args
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


class Store:
    """A row store in the oracle's layout.  ``rows`` keeps the raw bytes."""

    def __init__(self, rows: np.ndarray, dtype: str, metric: str, d: int):
        self.rows = np.ascontiguousarray(rows)
        self.dtype = dtype
        self.metric = metric
        self.d = d
        self.pitch = self.rows.strides[0] if self.rows.ndim == 2 else self.rows.itemsize * d
        self.n = self.rows.shape[0]

    def c(self, n: int | None = None) -> _Store:
        return _Store(self.rows.ctypes.data, self.n if n is None else n, self.d, _DT[self.dtype],
                      self.pitch, _MT[self.metric], 0)

    @staticmethod
    def from_vectors(x: np.ndarray, metric: str, dtype: str | None = None) -> "Store":
        """Primary store from fp32 or uint8 vectors, or an encoded bf16/fp8 copy."""
        n, d = x.shape
        if dtype is None:
            dtype = "u8" if x.dtype == np.uint8 else "f32"
        if dtype in ("u8", "f32"):
            return Store(x, dtype, metric, d)
        if dtype == "bf16":
            return Store(bf16_encode_rows(x), "bf16", metric, d)
        return Store(fp8_encode_rows(x), "fp8", metric, d)


def fp8_pitch(d: int) -> int:
    return (d + 4 + 31) // 32 * 32


def bf16_encode_rows(x: np.ndarray) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float32)
    n, d = x.shape
    out = np.zeros((n, d), dtype=np.uint16)
    lib().orc_bf16_encode_rows(_p(x), n, d, _p(out), 2 * d)
    return out


def fp8_encode_rows(x: np.ndarray) -> np.ndarray:
    """FP8 E4M3 codes with the fp32 scale at byte d; rows fp8_pitch(d) bytes."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    n, d = x.shape
    out = np.zeros((n, fp8_pitch(d)), dtype=np.uint8)
    lib().orc_fp8_encode_rows(_p(x), n, d, _p(out), out.shape[1])
    return out


def bf16_encode(x: float) -> int:
    return int(lib().orc_bf16_encode(x))


def bf16_decode(h: int) -> float:
    return float(lib().orc_bf16_decode(h))


def e4m3_encode(x: float) -> int:
    return int(lib().orc_e4m3_encode(x))


def e4m3_decode(c: int) -> float:
    return float(lib().orc_e4m3_decode(c))


def splitmix64(x: int) -> int:
    return int(lib().orc_splitmix64(x & 0xFFFFFFFFFFFFFFFF))


def query_key(q: np.ndarray) -> int:
    q = np.ascontiguousarray(q)
    return int(lib().orc_query_key(_p(q), q.nbytes))


def bitset(n_cap: int, deleted=None) -> np.ndarray:
    b = np.zeros((n_cap + 31) // 32, dtype=np.uint32)
    if deleted is not None:
        for i in np.asarray(deleted, dtype=np.int64):
            b[i >> 5] |= np.uint32(1 << (int(i) & 31))
    return b


def deleted_ids(bits: np.ndarray, n_used: int) -> np.ndarray:
    ids = np.arange(n_used, dtype=np.int64)
    return ids[((bits[ids >> 5] >> (ids & 31).astype(np.uint32)) & 1).astype(bool)]


def knn(store: Store, Q: np.ndarray, k: int, n: int | None = None, deleted: np.ndarray | None = None,
        self_ids: np.ndarray | None = None):
    """Exact k-NN by (dist, id): returns ids [nq,k] u32, dist [nq,k] f64, gap [nq]."""
    Q = np.ascontiguousarray(Q)
    nq = Q.shape[0]
    ids = np.zeros((nq, k), dtype=np.uint32)
    dist = np.zeros((nq, k), dtype=np.float64)
    gap = np.zeros(nq, dtype=np.float64)
    si = None if self_ids is None else np.ascontiguousarray(self_ids, dtype=np.int64)
    st = store.c(n)
    lib().orc_knn(C.byref(st), _p(deleted), _p(Q), nq, _p(si), k, _p(ids), _p(dist), _p(gap))
    return ids, dist, gap


def prune(store: Store, cand_ids, cand_d, R: int, mode: int = PRUNE_RNG, nbr: np.ndarray | None = None,
          cand_s=None):
    cand_ids = np.ascontiguousarray(cand_ids, dtype=np.uint32)
    cand_d = np.ascontiguousarray(cand_d, dtype=np.float64)
    cs = None if cand_s is None else np.ascontiguousarray(cand_s, dtype=np.float64)
    out = np.zeros(R, dtype=np.uint32)
    nw = 0 if nbr is None else nbr.shape[1]
    nb = None if nbr is None else np.ascontiguousarray(nbr, dtype=np.uint32)
    st = store.c()
    g = lib().orc_prune(C.byref(st), _p(cand_ids), _p(cand_d), _p(cs), len(cand_ids), mode, _p(nb), nw, R,
                        _p(out))
    return out, g


def build_graph(store: Store, R: int, mode: int = PRUNE_RNG):
    """Exact 2R-NN graph pruned to R: returns graph [n,R] u32 and row gaps [n]."""
    g = np.zeros((store.n, R), dtype=np.uint32)
    gap = np.zeros(store.n, dtype=np.float64)
    st = store.c()
    lib().orc_build(C.byref(st), R, mode, _p(g), _p(gap))
    return g, gap


def search(store: Store, n_used: int, graph: np.ndarray, delbits: np.ndarray | None, Q: np.ndarray, k: int,
           L: int, T: int, seed: int, qkeys: np.ndarray | None = None, want_pool: bool = False, W: int = 1):
    """Algorithm 1 with fixed T; W > 1 expands the W nearest unexpanded pool
    entries per iteration (iters counts parents).  Returns a dict of numpy
    arrays."""
    Q = np.ascontiguousarray(Q)
    nq = Q.shape[0]
    R = graph.shape[1]
    graph = np.ascontiguousarray(graph, dtype=np.uint32)
    out = {
        "ids": np.zeros((nq, k), dtype=np.uint32),
        "dist": np.zeros((nq, k), dtype=np.float64),
        "gap": np.zeros(nq, dtype=np.float64),
        "iters": np.zeros(nq, dtype=np.int32),
        "evals": np.zeros(nq, dtype=np.int64),
    }
    if want_pool:
        out["pool_ids"] = np.zeros((nq, L), dtype=np.uint32)
        out["pool_dist"] = np.zeros((nq, L), dtype=np.float64)
    qk = None if qkeys is None else np.ascontiguousarray(qkeys, dtype=np.uint64)
    st = store.c()
    rc = lib().orc_search(C.byref(st), n_used, _p(graph), R, _p(delbits), _p(Q), nq, _p(qk), k, L, T, seed, W,
                          _p(out["ids"]), _p(out["dist"]), _p(out["gap"]), _p(out["iters"]), _p(out["evals"]),
                          _p(out.get("pool_ids")), _p(out.get("pool_dist")))
    if rc != 0:
        raise ValueError(f"W = {W} out of range")
    return out


def insert(store: Store, n0: int, m: int, graph: np.ndarray, delbits: np.ndarray | None, L_ins: int, T_ins: int,
           seed: int, mode: int = PRUNE_RNG):
    """Insert store rows [n0, n0+m) into ``graph`` (modified in place; it needs
    >= n0+m rows).  Returns (new_gap [m], tail_gap [n0])."""
    assert graph.flags.c_contiguous and graph.dtype == np.uint32
    R = graph.shape[1]
    new_gap = np.zeros(max(m, 1), dtype=np.float64)
    tail_gap = np.zeros(max(n0, 1), dtype=np.float64)
    st = store.c()
    lib().orc_insert(C.byref(st), n0, m, _p(graph), R, _p(delbits), L_ins, T_ins, seed, mode, _p(new_gap),
                     _p(tail_gap))
    return new_gap[:m], tail_gap[:n0]


def delete(store: Store, n_used: int, graph: np.ndarray, delbits: np.ndarray, ids, c: int = 8,
           mode: int = PRUNE_RNG):
    """Logical delete + localized repair (in place).  Returns
    (newly_deleted or -1, repaired_rows, rows_gap [n_used])."""
    assert graph.flags.c_contiguous and graph.dtype == np.uint32
    ids = np.ascontiguousarray(ids, dtype=np.uint32)
    R = graph.shape[1]
    rep = np.zeros(1, dtype=np.int64)
    gap = np.zeros(max(n_used, 1), dtype=np.float64)
    st = store.c()
    newly = lib().orc_delete(C.byref(st), n_used, _p(graph), R, _p(delbits), _p(ids), len(ids), c, mode,
                             _p(rep), _p(gap))
    return int(newly), int(rep[0]), gap[:n_used]


def consolidate(store: Store, n0: int, graph: np.ndarray, delbits: np.ndarray, cap: int = 512,
                mode: int = PRUNE_RNG):
    """Global consolidation of graph rows [0, n0) (in place) under the
    deletion bits `delbits`.  Returns (rewritten_rows, rows_gap [n0])."""
    assert graph.flags.c_contiguous and graph.dtype == np.uint32
    R = graph.shape[1]
    gap = np.zeros(max(n0, 1), dtype=np.float64)
    st = store.c()
    nrep = lib().orc_consolidate(C.byref(st), n0, _p(graph), R, _p(delbits), cap, mode, _p(gap))
    if nrep < 0:
        raise ValueError("cap must be >= R")
    return int(nrep), gap[:n0]


def consolidate_rows(store: Store, n0: int, graph: np.ndarray, delbits: np.ndarray, only, cap: int = 512,
                     mode: int = PRUNE_RNG):
    """The consolidated rows of the vertices `only` (graph unchanged).
    Returns (rows [len(only)][R], rows_gap [len(only)])."""
    graph = np.ascontiguousarray(graph, dtype=np.uint32)
    only = np.ascontiguousarray(only, dtype=np.uint32)
    R = graph.shape[1]
    out = np.zeros((len(only), R), dtype=np.uint32)
    gap = np.zeros(max(len(only), 1), dtype=np.float64)
    st = store.c()
    rc = lib().orc_consolidate_rows(C.byref(st), n0, _p(graph), R, _p(delbits), cap, mode, _p(only), len(only),
                                    _p(out), _p(gap))
    if rc < 0:
        raise ValueError("cap must be >= R")
    return out, gap[:len(only)]


def reverse_patch(store: Store, graph: np.ndarray, delbits: np.ndarray | None, n0: int, rows: np.ndarray, tmax: int):
    """The reverse edges of new vertices n0 .. n0+m-1 (graph rows `rows`)
    applied to the tails of their targets < tmax (in place).  Returns the
    per-target gap [tmax]."""
    assert graph.flags.c_contiguous and graph.dtype == np.uint32
    rows = np.ascontiguousarray(rows, dtype=np.uint32)
    R = graph.shape[1]
    gap = np.zeros(max(tmax, 1), dtype=np.float64)
    st = store.c()
    lib().orc_reverse_patch(C.byref(st), _p(graph), R, _p(delbits), n0, rows.shape[0], _p(rows), tmax, _p(gap))
    return gap[:tmax]


def recall_at_k(found: np.ndarray, true_ids: np.ndarray, true_d: np.ndarray, found_d_exact: np.ndarray) -> float:
    """Recall@k with ties at the k-th exact distance counted as hits: a
    returned id is correct if its exact distance is <= the k-th exact
    distance (the paper leaves Recall@k undefined; this is the usual
    |returned cap true| / k made tie-robust)."""
    k = true_ids.shape[1]
    kth = true_d[:, k - 1:k]
    ok = (found != EMPTY) & (found_d_exact <= kth)
    return float(ok.sum()) / (found.shape[0] * k)


def dist_ids(store: Store, Q: np.ndarray, ids: np.ndarray) -> np.ndarray:
    """Exact FP64 distances from each query to the given ids (+inf for EMPTY)."""
    Q = np.ascontiguousarray(Q)
    ids = np.ascontiguousarray(ids, dtype=np.uint32)
    out = np.zeros(ids.shape, dtype=np.float64)
    st = store.c()
    lib().orc_dist_ids(C.byref(st), _p(Q), Q.shape[0], _p(ids), ids.shape[1], _p(out))
    return out


NFEAT, NHID = 16, 64


class MLP:
    """Stop-network weights as float64 arrays (W1 [64,16], b1 [64], w2 [64], b2)."""

    def __init__(self, W1, b1, w2, b2):
        self.W1 = np.ascontiguousarray(W1, dtype=np.float64).reshape(NHID, NFEAT)
        self.b1 = np.ascontiguousarray(b1, dtype=np.float64).reshape(NHID)
        self.w2 = np.ascontiguousarray(w2, dtype=np.float64).reshape(NHID)
        self.b2 = float(b2)

    def rounded_bf16(self) -> "MLP":
        """The same network with every weight rounded to bfloat16 (RNE)."""
        r = np.vectorize(lambda v: bf16_decode(bf16_encode(float(np.float32(v)))))
        return MLP(r(self.W1), r(self.b1), r(self.w2), float(r(np.float64(self.b2))))


def mlp_forward(net: MLP, F: np.ndarray):
    F = np.ascontiguousarray(F, dtype=np.float64)
    nb = F.shape[0]
    z = np.zeros(nb)
    p = np.zeros(nb)
    lib().orc_mlp_forward(_p(net.W1), _p(net.b1), _p(net.w2), net.b2, _p(F), nb, _p(z), _p(p))
    return z, p


def mlp_backward(net: MLP, F: np.ndarray, y: np.ndarray):
    F = np.ascontiguousarray(F, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    gW1 = np.zeros((NHID, NFEAT))
    gb1 = np.zeros(NHID)
    gw2 = np.zeros(NHID)
    gb2 = np.zeros(1)
    loss = lib().orc_mlp_backward(_p(net.W1), _p(net.b1), _p(net.w2), net.b2, _p(F), _p(y), F.shape[0],
                                  _p(gW1), _p(gb1), _p(gw2), _p(gb2))
    return float(loss), {"W1": gW1, "b1": gb1, "w2": gw2, "b2": float(gb2[0])}


def search_ex(store: Store, n_used: int, graph: np.ndarray, delbits, Q: np.ndarray, k: int, L: int, T: int,
              seed: int, trace: bool = False, net: MLP | None = None, tau: float = 0.5, t_min: int = 4,
              qkeys=None, t_every: int = 1):
    """Search with the per-iteration trace and/or the learned stop."""
    Q = np.ascontiguousarray(Q)
    nq = Q.shape[0]
    R = graph.shape[1]
    graph = np.ascontiguousarray(graph, dtype=np.uint32)
    out = {
        "ids": np.zeros((nq, k), dtype=np.uint32),
        "dist": np.zeros((nq, k), dtype=np.float64),
        "gap": np.zeros(nq),
        "n_feat": np.zeros(nq, dtype=np.int32),
        "t_last": np.zeros(nq, dtype=np.int32),
        "stop_iter": np.zeros(nq, dtype=np.int32),
        "margin": np.zeros(nq),
    }
    if trace:
        out["feat"] = np.zeros((nq, T, NFEAT))
    z_tau = float(np.log(tau / (1.0 - tau)))
    qk = None if qkeys is None else np.ascontiguousarray(qkeys, dtype=np.uint64)
    st = store.c()
    args = (None, None, None, 0.0) if net is None else (_p(net.W1), _p(net.b1), _p(net.w2), net.b2)
    lib().orc_search_ex(C.byref(st), n_used, _p(graph), R, _p(delbits), _p(Q), nq, _p(qk), k, L, T, seed,
                        _p(out["ids"]), _p(out["dist"]), _p(out["gap"]), _p(out.get("feat")), _p(out["n_feat"]),
                        _p(out["t_last"]), *args, z_tau, t_min, t_every, _p(out["stop_iter"]), _p(out["margin"]))
    return out


def wavp_round(map_, owner, ref, freq, ein, queue, B, hand, W, alpha, beta):
    """One batched round of Alg. 2 (in place on map_, owner, ref)."""
    M = owner.shape[0]
    p, e = np.zeros(1, np.int64), np.zeros(1, np.int64)
    q = np.ascontiguousarray(queue, dtype=np.uint32)
    lib().orc_wavp_round(M, _p(map_), _p(owner), _p(ref), _p(freq), _p(ein), _p(q), len(q), B, hand, W, alpha, beta,
                         _p(p), _p(e))
    return int(p[0]), int(e[0])


def threads() -> int:
    return int(lib().orc_threads())


def set_threads(t: int) -> None:
    lib().orc_set_threads(t)
