"""Seeded synthetic inputs for batched RMQ.

This module only draws random inputs; it contains none of the method's
arithmetic.  Tests, the benchmark and the CPU oracle all take their arrays
and queries from here, so both sides of every comparison see identical data.

Generators (numpy ``Generator(PCG64(seed))``, identical on x86 and Arm):

* ``uniform_array``        -- int32 values uniform in [lo, hi)
* ``paper_permutation``    -- the paper's array (Sec. 4): the identity
  permutation of 1..n after n/2 random swaps of pairs of cells
* ``uniform_queries``      -- l, r uniform over [0, n), swapped so l <= r
  (Sec. 4 draws them the same way, 1-based)
* ``log_width_queries``    -- width w log-uniform in [wmin, wmax], l uniform
  in [0, n - w], r = l + w - 1 (tie-heavy short-range workload)
* ``uneven_batch``         -- many arrays, n and q log-uniform (multi-array
  workload)
* ``served_array_sizes``   -- array sizes log-uniform, rescaled to a total
"""
from __future__ import annotations

import math

import numpy as np

INT32_SPAN = 2 ** 31


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def uniform_array(n: int, seed: int, lo: int = 0, hi: int = INT32_SPAN) -> np.ndarray:
    """int32[n] uniform in [lo, hi)."""
    return rng(seed).integers(lo, hi, size=int(n), dtype=np.int32)


def paper_permutation(n: int, seed: int) -> np.ndarray:
    """Identity permutation of 1..n after n/2 sequential random pair swaps.

    Swaps are applied in the order drawn.  Batches whose cells are all
    distinct commute and are applied at once; a batch with a repeated cell is
    applied one swap at a time, so the result equals the sequential process.
    """
    g = rng(seed)
    a = np.arange(1, n + 1, dtype=np.int32)
    nswaps = n // 2
    batch = 1024
    done = 0
    while done < nswaps:
        b = min(batch, nswaps - done)
        i = g.integers(0, n, size=b)
        j = g.integers(0, n, size=b)
        cells = np.concatenate([i, j])
        if len(np.unique(cells)) == 2 * b:
            a[i], a[j] = a[j].copy(), a[i].copy()
        else:
            for s in range(b):
                x, y = i[s], j[s]
                a[x], a[y] = a[y], a[x]
        done += b
    return a


def uniform_queries(n: int, q: int, seed: int):
    """(l, r) int32[q] with l, r uniform over [0, n) and swapped so l <= r."""
    g = rng(seed)
    a = g.integers(0, n, size=int(q), dtype=np.int64)
    b = g.integers(0, n, size=int(q), dtype=np.int64)
    l = np.minimum(a, b).astype(np.int32)
    r = np.maximum(a, b).astype(np.int32)
    return l, r


def log_width_queries(n: int, q: int, seed: int, wmin: int = 1, wmax: int = 10_000):
    """Width w = floor(exp(U * ln wmax)) clamped to [wmin, min(wmax, n)],
    l uniform in [0, n - w], r = l + w - 1 (never clipped)."""
    g = rng(seed)
    wmax = min(wmax, n)
    u = g.random(int(q))
    w = np.floor(np.exp(u * math.log(wmax))).astype(np.int64)
    w = np.clip(w, wmin, wmax)
    l = (g.random(int(q)) * (n - w + 1)).astype(np.int64)
    l = np.minimum(l, n - w)
    r = l + w - 1
    return l.astype(np.int32), r.astype(np.int32)


def log_uniform_ints(g: np.random.Generator, count: int, lo: float, hi: float) -> np.ndarray:
    """int64[count] drawn log-uniform in [lo, hi]."""
    u = g.random(int(count))
    v = np.exp(math.log(lo) + u * (math.log(hi) - math.log(lo)))
    return np.clip(np.floor(v).astype(np.int64), int(lo), int(hi))


def uneven_batch(num_arrays: int, seed: int, n_lo: float = 1e4, n_hi: float = 1e7,
                 q_lo: float = 10, q_hi: float = 1e5):
    """Sizes for the multi-array workload: (n_i, q_i) log-uniform, int64 arrays."""
    g = rng(seed)
    ns = log_uniform_ints(g, num_arrays, n_lo, n_hi)
    qs = log_uniform_ints(g, num_arrays, q_lo, q_hi)
    return ns, qs


def served_array_sizes(num_arrays: int, total: int, seed: int, n_lo: float = 1e6,
                       n_hi: float = 2e8) -> np.ndarray:
    """Log-uniform sizes rescaled to sum to `total`, each clamped to n_hi with
    the excess spread over the unclamped arrays."""
    g = rng(seed)
    s = log_uniform_ints(g, num_arrays, n_lo, n_hi).astype(np.float64)
    s *= total / s.sum()
    for _ in range(64):
        over = s > n_hi
        if not over.any():
            break
        excess = (s[over] - n_hi).sum()
        s[over] = n_hi
        free = ~over & (s < n_hi)
        s[free] += excess * s[free] / s[free].sum()
    out = np.floor(s).astype(np.int64)
    out[np.argmin(out)] += total - out.sum()
    return out
