"""Seeded synthetic inputs: binary code databases, queries and per-query k.

This module only draws inputs; it holds none of the search arithmetic.  Both
the tests (which feed the same codes to the GPU library and to the CPU
oracle) and the benchmark use it.

The paper's datasets (SIFT 1B, Gist 80M) and its learned hash functions are
not available, so two generators stand in for them (Sec. 5):

- uniform codes: every bit i.i.d. Bernoulli(0.5);
- LSH-style codes: 128-d vectors from a mixture of 1000 isotropic Gaussians
  (centres U[0,255], sigma 20, clipped to [0,255]), mean-centred, then
  binarised by the sign of q random N(0,1) projections (Sec. 5: LSH codes are
  signs of random projections of mean-centred features).  The projections
  themselves (``lsh_projections``) are the real-valued queries of the
  asymmetric re-ranking.

Codes are packed little-endian into W = q/64 uint64 words: bit b of a code is
bit (b % 64) of word (b // 64).  Small databases are drawn with numpy on the
host; large ones with torch on the GPU in fixed chunks (chunk c is seeded
with (seed << 20) + c), so a given (n, q, seed) always gives the same codes
on the same device kind.
"""
from __future__ import annotations

import numpy as np

DIM = 128            # feature dimension of the LSH-style vectors
N_CENTRES = 1000     # mixture components
SIGMA = 20.0         # per-dimension noise
N_TRAIN = 1_000_000  # vectors used for the centring mean
_mu_cache: dict = {}


def words(q: int) -> int:
    if q % 64:
        raise ValueError("q must be a multiple of 64")
    return q // 64


# --------------------------------------------------------------------- uniform
def uniform_codes(n: int, q: int, seed: int) -> np.ndarray:
    """(n, q/64) uint64, each bit Bernoulli(0.5), numpy PCG64 seeded `seed`."""
    rng = np.random.default_rng(seed)
    return rng.integers(0, 2**64, size=(n, words(q)), dtype=np.uint64, endpoint=False)


def uniform_codes_torch(n: int, q: int, seed: int, device="cuda", chunk: int = 100_000_000):
    """(n, q/64) int64 tensor (bit pattern of uint64 codes) drawn on `device`."""
    import torch

    W = words(q)
    out = torch.empty((n, W), dtype=torch.int64, device=device)
    for c, s in enumerate(range(0, n, chunk)):
        e = min(n, s + chunk)
        g = torch.Generator(device=device)
        g.manual_seed((seed << 20) + c)
        raw = torch.randint(0, 256, ((e - s) * W * 8,), dtype=torch.uint8, device=device, generator=g)
        out[s:e] = raw.view(torch.int64).view(e - s, W)
        del raw
    return out


# ------------------------------------------------------------------ LSH-style
def _centres() -> np.ndarray:
    return np.random.default_rng(1000).uniform(0, 255, (N_CENTRES, DIM)).astype(np.float32)


def _projection(q: int) -> np.ndarray:
    return np.random.default_rng(1000 + q).standard_normal((q, DIM)).astype(np.float32)


def _draw_vectors(rng: np.random.Generator, n: int, centres: np.ndarray) -> np.ndarray:
    idx = rng.integers(0, N_CENTRES, size=n)
    x = centres[idx] + rng.normal(0.0, SIGMA, size=(n, DIM)).astype(np.float32)
    return np.clip(x, 0.0, 255.0, out=x)


def training_mean() -> np.ndarray:
    """float64 mean of N_TRAIN vectors drawn with seed 2 (fixed centring)."""
    if "mu" not in _mu_cache:
        rng = np.random.default_rng(2)
        centres = _centres()
        acc = np.zeros(DIM, dtype=np.float64)
        step = 200_000
        for s in range(0, N_TRAIN, step):
            acc += _draw_vectors(rng, min(step, N_TRAIN - s), centres).sum(axis=0, dtype=np.float64)
        _mu_cache["mu"] = acc / N_TRAIN
    return _mu_cache["mu"]


def _pack_bits(bits: np.ndarray) -> np.ndarray:
    """(n, q) bool -> (n, q/64) uint64, bit b -> word b//64, bit b%64."""
    n, q = bits.shape
    b = bits.reshape(n, q // 64, 64).astype(np.uint64)
    return (b << np.arange(64, dtype=np.uint64)).sum(axis=2, dtype=np.uint64)


def lsh_codes(n: int, q: int, seed: int, chunk: int = 200_000) -> np.ndarray:
    """(n, q/64) uint64 LSH-style codes drawn with numpy (host; n up to ~1e7)."""
    return lsh_projections(n, q, seed, chunk, keep_proj=False)[0]


def lsh_projections(n: int, q: int, seed: int, chunk: int = 200_000, keep_proj: bool = True):
    """(codes, proj): the codes of lsh_codes(n, q, seed) and the float32
    projections (n, q) whose signs they are (bit b set where proj[:, b] > 0),
    the real-valued form of the same vectors."""
    words(q)
    rng = np.random.default_rng(seed)
    centres, P = _centres(), _projection(q)
    mu = training_mean().astype(np.float32)
    out = np.empty((n, q // 64), dtype=np.uint64)
    proj = np.empty((n, q), dtype=np.float32) if keep_proj else None
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        x = _draw_vectors(rng, e - s, centres) - mu
        y = x @ P.T
        out[s:e] = _pack_bits(y > 0)
        if keep_proj:
            proj[s:e] = y
    return out, proj


def lsh_codes_torch(n: int, q: int, seed: int, device="cuda", chunk: int = 10_000_000):
    """(n, q/64) int64 tensor of LSH-style codes drawn with torch on `device`."""
    return _lsh_torch(n, q, seed, device, chunk, False, False)[0]


def lsh_projections_torch(n: int, q: int, seed: int, device="cuda", chunk: int = 10_000_000):
    """(codes, proj): the codes of lsh_codes_torch(n, q, seed) and the float32
    projections (n, q) on `device` whose signs they are."""
    return _lsh_torch(n, q, seed, device, chunk, True, False)[:2]


def lsh_vectors_torch(n: int, q: int, seed: int, device="cuda", chunk: int = 10_000_000):
    """(codes, proj, x): as lsh_projections_torch, plus the mean-centred
    128-d float32 vectors x the projections were taken of."""
    return _lsh_torch(n, q, seed, device, chunk, True, True)


def _lsh_torch(n, q, seed, device, chunk, keep_proj, keep_x):
    import torch

    W = words(q)
    centres = torch.from_numpy(_centres()).to(device)
    P = torch.from_numpy(_projection(q)).to(device)
    mu = torch.from_numpy(training_mean().astype(np.float32)).to(device)
    shifts = torch.arange(64, device=device, dtype=torch.int64)
    out = torch.empty((n, W), dtype=torch.int64, device=device)
    proj = torch.empty((n, q), dtype=torch.float32, device=device) if keep_proj else None
    xs = torch.empty((n, DIM), dtype=torch.float32, device=device) if keep_x else None
    for c, s in enumerate(range(0, n, chunk)):
        e = min(n, s + chunk)
        g = torch.Generator(device=device)
        g.manual_seed((seed << 20) + c)
        idx = torch.randint(0, N_CENTRES, (e - s,), device=device, generator=g)
        x = torch.randn((e - s, DIM), device=device, generator=g)
        x.mul_(SIGMA).add_(centres[idx]).clamp_(0.0, 255.0).sub_(mu)
        y = x @ P.T
        if keep_x:
            xs[s:e] = x
        del x
        bits = y > 0
        if keep_proj:
            proj[s:e] = y
        del y
        b = bits.view(e - s, W, 64).to(torch.int64)
        out[s:e] = (b << shifts).sum(dim=2)
        del bits, b
    return out, proj, xs


# ------------------------------------------------------------------ queries
def per_query_k(nq: int, seed: int = 3, kmax: int = 1000) -> np.ndarray:
    """k = floor(exp(U ln(kmax+1))) clipped to [1, kmax], log-uniform."""
    u = np.random.default_rng(seed).random(nq)
    k = np.floor(np.exp(u * np.log(kmax + 1.0))).astype(np.int64)
    return np.clip(k, 1, kmax).astype(np.uint32)


def poisson_arrivals(n: int, rate_qps: float, seed: int = 4) -> np.ndarray:
    """Arrival times (s) of a Poisson stream with the given rate."""
    gaps = np.random.default_rng(seed).exponential(1.0 / rate_qps, size=n)
    return np.cumsum(gaps)


def as_uint64(t) -> np.ndarray:
    """Host copy of a code tensor/array as uint64 (same bits)."""
    if isinstance(t, np.ndarray):
        return np.ascontiguousarray(t.view(np.uint64) if t.dtype == np.int64 else t, dtype=np.uint64)
    return t.detach().cpu().numpy().view(np.uint64)
