"""Learned early stop for the graph search: trace capture, training, calibration.

The search of Alg. 1 runs a fixed number of iterations T.  A small network
(16 per-iteration features -> 64 ReLU -> 1 logit, bf16 weights at inference)
predicts, after every iteration, whether the top-k set has already reached
its final value; the search stops once the logit reaches logit(tau) and at
least t_min iterations ran.  Fixed-T search stays the fallback (tau -> 1).

Training data are traces of the plain search (features of every iteration
and the last iteration that changed the top-k); every arithmetic step runs
in libsvf's kernels (trace-mode search, svf_mlp_grad / svf_mlp_adam /
svf_mlp_pack); this module only orders the calls and shuffles sample ids.
"""
from __future__ import annotations

import ctypes as C
import dataclasses

import numpy as np
import torch

from . import _lib as L
from .index import Index, SearchConfig, _ptr, _stream


@dataclasses.dataclass
class StopNet:
    params: torch.Tensor   # fp32 [1153] master weights
    packed: torch.Tensor   # bf16 [1160] as int16 (what the search reads)
    tau: float = 0.5
    t_min: int = 4
    t_every: int = 1
    loss: float = float("nan")


def capture_traces(ix: Index, Q: torch.Tensor, cfg: SearchConfig, chunk: int = 50_000):
    """Plain search with the per-iteration trace: features [nq, T, 16] and
    meta [nq, 2] = (iterations run, last iteration that changed the top-k)."""
    nq, T = Q.shape[0], cfg.T
    feat = torch.empty((nq, T, 16), dtype=torch.float32, device=ix.device)
    meta = torch.empty((nq, 2), dtype=torch.int32, device=ix.device)
    for s in range(0, nq, chunk):
        e = min(nq, s + chunk)
        ix.search(Q[s:e], dataclasses.replace(cfg, mlp=None), trace_feat=feat[s:e], trace_meta=meta[s:e])
    return feat, meta


def sample_ids(meta: torch.Tensor, T: int) -> torch.Tensor:
    """Ids q*T + t of every traced iteration (t < iterations run)."""
    ran = meta[:, 0].to(torch.int64)
    t = torch.arange(T, device=meta.device)
    mask = t[None, :] < ran[:, None]
    ids = (torch.arange(meta.shape[0], device=meta.device)[:, None] * T + t[None, :])[mask]
    return ids.to(torch.int32)


def init_params(seed: int, device) -> torch.Tensor:
    rng = np.random.default_rng(seed)
    W1 = rng.standard_normal((64, 16)) * np.sqrt(2.0 / 16)
    w2 = rng.standard_normal(64) * np.sqrt(1.0 / 64)
    p = np.concatenate([W1.ravel(), np.zeros(64), w2, [0.0]]).astype(np.float32)
    return torch.from_numpy(p).to(device)


def train(feat: torch.Tensor, meta: torch.Tensor, T: int, ids: torch.Tensor, epochs: int = 3, batch: int = 4096,
          lr: float = 3e-3, seed: int = 7, params: torch.Tensor | None = None, stream=None) -> StopNet:
    lib = L.load()
    dev = feat.device
    prm = init_params(seed, dev) if params is None else params.clone()
    m = torch.zeros_like(prm)
    v = torch.zeros_like(prm)
    grad = torch.empty_like(prm)
    partial = torch.empty(int(lib.svf_mlp_partial_floats(batch)), dtype=torch.float32, device=dev)
    loss = torch.zeros(1, dtype=torch.float32, device=dev)
    gen = torch.Generator(device="cpu").manual_seed(seed)
    n = ids.numel()
    step = 0
    st = _stream(stream)
    for _ in range(epochs):
        perm = ids[torch.randperm(n, generator=gen).to(dev)]
        for s in range(0, n - batch + 1, batch):
            b = perm[s:s + batch].contiguous()
            L.check(lib.svf_mlp_grad(_ptr(feat), _ptr(meta), T, _ptr(b), batch, _ptr(prm), _ptr(grad),
                                     _ptr(partial), _ptr(loss), st))
            step += 1
            L.check(lib.svf_mlp_adam(_ptr(prm), _ptr(grad), _ptr(m), _ptr(v), step, C.c_float(lr), C.c_float(0.9),
                                     C.c_float(0.999), C.c_float(1e-8), st))
    packed = torch.empty(L.MLP_PACKED, dtype=torch.int16, device=dev)
    L.check(lib.svf_mlp_pack(_ptr(prm), _ptr(packed), st))
    return StopNet(prm, packed, loss=float(loss.item()))


def recall_at_k(ids: torch.Tensor, gt: torch.Tensor) -> float:
    """|returned cap true| / k, averaged (evaluation only)."""
    k = gt.shape[1]
    hit = (ids[:, :k, None] == gt[:, None, :]).any(-1)
    return float(hit.float().mean().item())


def calibrate(ix: Index, net: StopNet, Q: torch.Tensor, gt: torch.Tensor, cfg: SearchConfig,
              max_loss: float = 0.002, taus=(0.5, 0.6, 0.7, 0.8, 0.85, 0.9, 0.93, 0.95, 0.97, 0.98, 0.99, 0.995,
                                           0.998, 0.999)) -> tuple[float, float, float]:
    """Smallest tau whose recall@k is within max_loss of fixed-T search on
    calibration queries.  Returns (tau, recall_fixed, recall_stop); tau = 1
    means no tau qualified and the fixed-T fallback is used."""
    base_ids, _ = ix.search(Q, dataclasses.replace(cfg, mlp=None))
    r0 = recall_at_k(base_ids, gt)
    for tau in taus:
        ids, _ = ix.search(Q, dataclasses.replace(cfg, mlp=net.packed, tau=tau, t_min=net.t_min,
                                                  t_every=net.t_every))
        r = recall_at_k(ids, gt)
        if r >= r0 - max_loss:
            return tau, r0, r
    return 1.0, r0, r0
