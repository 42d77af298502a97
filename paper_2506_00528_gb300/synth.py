"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle side.

This module only draws numbers: Gaussian-mixture embeddings shaped like the
paper's workloads (l2-normalised rows, Sec. 1.1), uniform points on the
hypersphere (the "Uniform" rows of the paper's data-set table, Sec. 5.1),
and Poisson arrival times.  It holds none of the method's arithmetic
(no encoding, no distance, no selection).

Recipe (all float32):
  centres c_j ~ N(0, I_d), j < n_centres
  row     = c_j + sigma * z,  j uniform, z ~ N(0, I_d)
  optional anisotropy: row_i *= s_i with s_i ~ logU[0.1, 1] shared by
  database and queries (one draw per dimension)
  then each row is divided by its l2 norm.
Separate seed streams are used for centres, scales, database rows, query
rows and arrivals, so the query set is disjoint from the database draw.
"""
from __future__ import annotations

import numpy as np

BASE_SEED = 20250531
STREAM_CENTRES, STREAM_SCALES, STREAM_DB, STREAM_QUERIES, STREAM_ARRIVALS = range(5)


def _rng(seed: int, stream: int) -> np.random.Generator:
    return np.random.default_rng([int(seed), int(stream)])


def mixture_params(d: int, n_centres: int, anisotropic: bool, seed: int = BASE_SEED):
    """Centres [n_centres, d] and per-dimension scales [d] (ones if isotropic)."""
    centres = _rng(seed, STREAM_CENTRES).standard_normal((n_centres, d)).astype(np.float32)
    if anisotropic:
        lo, hi = np.log(0.1), np.log(1.0)
        scales = np.exp(_rng(seed, STREAM_SCALES).uniform(lo, hi, size=d)).astype(np.float32)
    else:
        scales = np.ones(d, dtype=np.float32)
    return centres, scales


def mixture_numpy(n: int, d: int, n_centres: int = 64, sigma: float = 0.5,
                  anisotropic: bool = False, stream: int = STREAM_DB,
                  seed: int = BASE_SEED) -> np.ndarray:
    """n rows of the Gaussian mixture, l2-normalised, float32 [n, d] (host)."""
    centres, scales = mixture_params(d, n_centres, anisotropic, seed)
    g = _rng(seed, stream)
    j = g.integers(0, n_centres, size=n)
    rows = centres[j] + np.float32(sigma) * g.standard_normal((n, d)).astype(np.float32)
    rows *= scales[None, :]
    norms = np.sqrt(np.sum(rows.astype(np.float64) ** 2, axis=1, keepdims=True))
    return (rows / norms).astype(np.float32)


def mixture_torch(n: int, d: int, n_centres: int = 1024, sigma: float = 0.5,
                  anisotropic: bool = True, stream: int = STREAM_DB,
                  seed: int = BASE_SEED, device="cuda", out=None, chunk: int = 1 << 20):
    """Same recipe drawn on a torch device in chunks (for multi-GB databases).

    Centres and scales come from numpy (identical to ``mixture_numpy``); the
    per-row draws use a torch generator seeded from (seed, stream), so rows are
    reproducible on the same device and torch version.
    """
    import torch
    centres_np, scales_np = mixture_params(d, n_centres, anisotropic, seed)
    centres = torch.from_numpy(centres_np).to(device)
    scales = torch.from_numpy(scales_np).to(device)
    if out is None:
        out = torch.empty((n, d), dtype=torch.float32, device=device)
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed) * 1000003 + int(stream))
    for r0 in range(0, n, chunk):
        m = min(chunk, n - r0)
        j = torch.randint(0, n_centres, (m,), generator=gen, device=device)
        z = torch.randn((m, d), generator=gen, device=device, dtype=torch.float32)
        rows = centres.index_select(0, j).add_(z, alpha=float(sigma)).mul_(scales)
        rows.div_(torch.linalg.vector_norm(rows, dim=1, keepdim=True))
        out[r0:r0 + m].copy_(rows)
        del j, z, rows
    return out


def uniform_sphere(n: int, d: int, seed: int = BASE_SEED, stream: int = STREAM_DB) -> np.ndarray:
    """n points uniform on the unit hypersphere in R^d, float32 [n, d]."""
    g = _rng(seed, stream)
    z = g.standard_normal((n, d))
    return (z / np.linalg.norm(z, axis=1, keepdims=True)).astype(np.float32)


def ternary_random(n: int, d: int, x: int, seed: int = BASE_SEED, stream: int = STREAM_DB) -> np.ndarray:
    """n random ternary vectors with exactly x non-zeros (uniform over the vertex set)."""
    g = _rng(seed, stream)
    V = np.zeros((n, d), dtype=np.int8)
    for r in range(n):
        pos = g.choice(d, size=x, replace=False)
        V[r, pos] = np.where(g.integers(0, 2, size=x) == 1, 1, -1)
    return V


def poisson_arrivals(n: int, rate_per_s: float, seed: int = BASE_SEED) -> np.ndarray:
    """Arrival times (seconds) of a Poisson process with the given rate."""
    g = _rng(seed, STREAM_ARRIVALS)
    return np.cumsum(g.exponential(1.0 / rate_per_s, size=n))


def log_uniform_ints(n: int, lo: int, hi: int, seed: int = BASE_SEED, stream: int = STREAM_ARRIVALS + 1) -> np.ndarray:
    """n integers round(exp(U[log lo, log hi])) clipped to [lo, hi]."""
    g = _rng(seed, stream)
    v = np.rint(np.exp(g.uniform(np.log(lo), np.log(hi), size=n))).astype(np.int64)
    return np.clip(v, lo, hi)
