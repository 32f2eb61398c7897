"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module only draws random numbers (numpy PCG64); it contains none of the
search/insert/delete arithmetic.  The paper evaluates on public datasets
(Table 2: Wikipedia, MSMARCO, MSTuring, Deep1B, Text2Image) that are not
available here; the Gaussian mixtures below stand in for them with the
shapes and value ranges of the workloads:

* ``tiny``      n=10,000 fp32, d=128, 16 centres U[-5,5]^d, sigma=1 (L2).
* ``u8``        n=1,000,000 uint8, d=128, 1,024 centres U[32,224]^d,
                sigma=20, rounded half-to-even and clipped to [0,255] (L2).
* ``unit96``    n=10,000,000 fp32, d=96 (Deep1B's dimension), 4,096
                components with a low intrinsic dimension, unit-normalised
                (inner product): a fixed random orthonormal basis A (96 x 16),
                component means z_c ~ N(0, I_16), x = normalize(A (z_c + u)
                + 0.02 e) with u ~ N(0, I_16), e ~ N(0, I_96).  Real
                descriptors such as Deep1B's have a low intrinsic dimension;
                a mixture of 4,096 isotropic 96-d blobs would instead split
                into thousands of disconnected neighbourhoods.
* ``serve128``  n=50,000,000 fp32, d=128, 16,384 components built like
                ``unit96`` (16-dimensional latent structure, 0.02 isotropic
                noise) but not normalised (squared L2).

Every draw is keyed by an explicit seed so a test, the oracle and a GPU run
see byte-identical inputs.
"""
from __future__ import annotations

import concurrent.futures
import dataclasses
import os

import numpy as np

__all__ = ["Mixture", "MIXTURES", "centres", "latent_basis", "sample", "sample_chunked", "pick_live_ids", "zipf_components"]


@dataclasses.dataclass(frozen=True)
class Mixture:
    name: str
    d: int
    n_centres: int
    dtype: str            # "f32" or "u8"
    centre_kind: str      # "uniform" or "unit"
    centre_lo: float
    centre_hi: float
    sigma: float
    centre_seed: int
    normalize: bool = False
    latent_dim: int = 0       # "latent": component means and noise live in span(A)
    iso_sigma: float = 0.0    # "latent": isotropic noise added in the full space


MIXTURES = {
    "tiny": Mixture("tiny", 128, 16, "f32", "uniform", -5.0, 5.0, 1.0, 101),
    "u8": Mixture("u8", 128, 1024, "u8", "uniform", 32.0, 224.0, 20.0, 201),
    "unit96": Mixture("unit96", 96, 4096, "f32", "latent", 0.0, 0.0, 1.0, 301, normalize=True,
                      latent_dim=16, iso_sigma=0.02),
    "serve128": Mixture("serve128", 128, 16384, "f32", "latent", 0.0, 0.0, 1.0, 501, latent_dim=16, iso_sigma=0.02),
}


def centres(mix: Mixture) -> np.ndarray:
    """The mixture's centres, float64 [n_centres, d] ([n_centres, r] latent
    means for a "latent" mixture)."""
    rng = np.random.default_rng(mix.centre_seed)
    if mix.centre_kind == "uniform":
        return rng.uniform(mix.centre_lo, mix.centre_hi, size=(mix.n_centres, mix.d))
    if mix.centre_kind == "latent":
        return rng.standard_normal(size=(mix.n_centres, mix.latent_dim))
    c = rng.standard_normal(size=(mix.n_centres, mix.d))
    return c / np.linalg.norm(c, axis=1, keepdims=True)


def latent_basis(mix: Mixture) -> np.ndarray:
    """Orthonormal [d, r] basis of a "latent" mixture."""
    rng = np.random.default_rng(mix.centre_seed + 1_000_003)
    return np.linalg.qr(rng.standard_normal(size=(mix.d, mix.latent_dim)))[0]


def _finish(mix: Mixture, x: np.ndarray) -> np.ndarray:
    if mix.normalize:
        x = x / np.linalg.norm(x, axis=1, keepdims=True)
    if mix.dtype == "u8":
        # numpy's rint rounds half to even
        return np.clip(np.rint(x), 0, 255).astype(np.uint8)
    return x.astype(np.float32)


def sample(mix: Mixture | str, n: int, seed: int, labels_out: list | None = None) -> np.ndarray:
    """Draw n points: a uniformly chosen centre plus isotropic Gaussian noise."""
    if isinstance(mix, str):
        mix = MIXTURES[mix]
    c = centres(mix)
    rng = np.random.default_rng(seed)
    lab = rng.integers(0, mix.n_centres, size=n)
    if mix.centre_kind == "latent":
        A = latent_basis(mix)
        z = c[lab] + mix.sigma * rng.standard_normal(size=(n, mix.latent_dim))
        x = z @ A.T + mix.iso_sigma * rng.standard_normal(size=(n, mix.d))
    else:
        x = c[lab] + mix.sigma * rng.standard_normal(size=(n, mix.d))
    if labels_out is not None:
        labels_out.append(lab)
    return _finish(mix, x)


def sample_chunked(mix: Mixture | str, n: int, seed: int, chunk: int = 1 << 20,
                   component_sampler=None, workers: int | None = None) -> np.ndarray:
    """Like :func:`sample` for large n: float32 arithmetic, drawn in chunks.

    Chunk j uses the generator seeded by (seed, j), so the result depends
    only on (mix, n, seed, chunk).  ``component_sampler(rng, m)`` may replace
    the uniform choice of centre (the serving stream draws Zipf components).
    """
    if isinstance(mix, str):
        mix = MIXTURES[mix]
    c = centres(mix).astype(np.float32)
    out = np.empty((n, mix.d), dtype=np.uint8 if mix.dtype == "u8" else np.float32)
    A = latent_basis(mix).astype(np.float32) if mix.centre_kind == "latent" else None

    def one(j):
        s = j * chunk
        m = min(chunk, n - s)
        rng = np.random.default_rng([seed, j])
        if component_sampler is None:
            lab = rng.integers(0, mix.n_centres, size=m)
        else:
            lab = component_sampler(rng, m)
        if mix.centre_kind == "latent":
            z = rng.standard_normal(size=(m, mix.latent_dim), dtype=np.float32)
            z *= np.float32(mix.sigma)
            z += c[lab]
            x = z @ A.T
            x += np.float32(mix.iso_sigma) * rng.standard_normal(size=(m, mix.d), dtype=np.float32)
        else:
            x = rng.standard_normal(size=(m, mix.d), dtype=np.float32)
            x *= np.float32(mix.sigma)
            x += c[lab]
        if mix.normalize:
            x /= np.linalg.norm(x, axis=1, keepdims=True)
        if mix.dtype == "u8":
            out[s:s + m] = np.clip(np.rint(x), 0, 255).astype(np.uint8)
        else:
            out[s:s + m] = x

    nchunk = (n + chunk - 1) // chunk
    if workers is None:
        workers = min(16, os.cpu_count() or 1)
    if workers <= 1 or nchunk == 1:
        for j in range(nchunk):
            one(j)
    else:
        with concurrent.futures.ThreadPoolExecutor(workers) as ex:
            list(ex.map(one, range(nchunk)))
    return out


def pick_live_ids(n_used: int, deleted: np.ndarray | None, m: int, seed: int) -> np.ndarray:
    """m distinct ids drawn uniformly from the live ids in [0, n_used)."""
    rng = np.random.default_rng(seed)
    live = np.arange(n_used, dtype=np.int64)
    if deleted is not None and deleted.size:
        live = np.setdiff1d(live, deleted.astype(np.int64))
    return np.sort(rng.choice(live, size=min(m, live.size), replace=False)).astype(np.uint32)


def given_components(labels: np.ndarray):
    """Sampler that hands out the given component labels in order (use with
    workers=1 so chunks are drawn in order)."""
    pos = [0]

    def draw(rng, m):
        out = labels[pos[0]:pos[0] + m]
        pos[0] += m
        return out
    return draw


def window_components(n_components: int, width: int, speed: float, seed: int):
    """Components of a sliding window: a query arriving at time t (s) draws
    uniformly from `width` consecutive components (of a seeded permutation)
    starting at floor(t * speed).  Returns f(rng, t, m)."""
    perm = np.random.default_rng(seed).permutation(n_components)

    def draw(rng, t, m):
        start = int(np.floor(t * speed))
        return perm[(start + rng.integers(0, width, m)) % n_components]
    return draw


def zipf_components(n_components: int, s: float, seed: int):
    """Sampler of mixture components ~ Zipf(s) over a seeded permutation."""
    perm = np.random.default_rng(seed).permutation(n_components)
    w = 1.0 / np.arange(1, n_components + 1, dtype=np.float64) ** s
    cdf = np.cumsum(w / w.sum())

    def draw(rng, m):
        r = np.searchsorted(cdf, rng.random(m), side="right")
        return perm[np.minimum(r, n_components - 1)]
    return draw
