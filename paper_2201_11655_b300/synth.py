"""Seeded synthetic directed graphs shaped like the paper's workloads.

This module only draws arc lists.  It holds none of the counting method's
arithmetic (no ordering, no enumeration, no classification), so both the CUDA
path and the CPU oracle may take their inputs from it.

Every generator returns ``(n, src, dst)`` with ``src``/``dst`` int32 numpy
arrays.  Unless stated otherwise the arc list is simple: no self-loops and no
repeated ordered pair.  Generators are deterministic functions of their seed
(numpy PCG64).

Workload shapes:

* ``gnp``       -- directed G(n, p): every ordered pair (i, j), i != j, is an
                   arc independently with probability p (the random-graph
                   model of the section comparing VDMC to theory in G(n,p)).
* ``gnp_undirected`` -- undirected G(n, p): every unordered pair is an edge
                   with probability p, given as one arc i -> j, i < j.
* ``chung_lu``  -- directed Chung-Lu graph with Pareto out- and in-weights
                   (fat-tailed degree, the shape of the real networks of
                   Table 1), optional reciprocity.
* ``er_uniform``-- m arcs with uniform random endpoints (the G(n,p) scaling
                   runs of Fig. 3/4 at fixed mean degree).
* ``batch``     -- many small graphs of uneven size, half G(n,p), half
                   Chung-Lu, for the batched launch.
* ``serve_requests`` -- a Poisson request stream of Chung-Lu graphs of
                   log-uniform size, for the serving loop.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "gnp",
    "gnp_undirected",
    "chung_lu",
    "er_uniform",
    "batch",
    "serve_requests",
    "simple_arcs",
    "WORKLOADS",
    "workload",
]


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def simple_arcs(src, dst):
    """Drop self-loops and repeated ordered pairs; sort by (src, dst)."""
    src = np.asarray(src, dtype=np.int64)
    dst = np.asarray(dst, dtype=np.int64)
    keep = src != dst
    src, dst = src[keep], dst[keep]
    if src.size == 0:
        return np.zeros(0, np.int32), np.zeros(0, np.int32)
    n = int(max(src.max(), dst.max())) + 1
    key = np.unique(src * n + dst)
    return (key // n).astype(np.int32), (key % n).astype(np.int32)


def gnp(n: int, p: float, seed: int):
    """Directed G(n, p): each ordered pair i != j is an arc with probability p."""
    rng = _rng(seed)
    if n <= 4096:
        a = rng.random((n, n)) < p
        np.fill_diagonal(a, False)
        src, dst = np.nonzero(a)
        return n, src.astype(np.int32), dst.astype(np.int32)
    # Large n: draw the arc count, then distinct off-diagonal pairs.
    npairs = n * (n - 1)
    m = int(rng.binomial(npairs, p))
    got = np.zeros(0, np.int64)
    while got.size < m:
        need = int((m - got.size) * 1.1) + 16
        idx = rng.integers(0, npairs, size=need, dtype=np.int64)
        got = np.unique(np.concatenate([got, idx]))
    got = rng.permutation(got)[:m]
    i = got // (n - 1)
    j = got % (n - 1)
    j = j + (j >= i)
    src, dst = simple_arcs(i, j)
    return n, src, dst


def gnp_undirected(n: int, p: float, seed: int):
    """Undirected G(n, p): each unordered pair {i, j} is an edge with probability p (one arc i -> j, i < j)."""
    rng = _rng(seed)
    a = np.triu(rng.random((n, n)) < p, k=1)
    src, dst = np.nonzero(a)
    return n, src.astype(np.int32), dst.astype(np.int32)


def _draw_weighted(rng, w, size):
    """Indices drawn with probability proportional to w (with replacement)."""
    cdf = np.cumsum(w, dtype=np.float64)
    cdf /= cdf[-1]
    u = rng.random(size)
    return np.minimum(np.searchsorted(cdf, u, side="right"), w.size - 1)


def chung_lu(n: int, mean_out_degree: float, exponent: float, seed: int,
             reciprocity: float = 0.0, max_degree: float | None = None):
    """Directed Chung-Lu graph with Pareto weights.

    Out- and in-weights are drawn independently from a Pareto law whose
    density decays as w^-exponent (x_min = 1).  ``mean_out_degree`` is the
    target mean out-degree *before* reciprocal arcs are added, so the final
    mean out-degree is about mean_out_degree * (1 + reciprocity).  Weights
    are capped so that no vertex's expected out- or in-degree exceeds
    ``max_degree`` (default sqrt(n * mean_out_degree), the Chung-Lu
    validity bound).  ``m0 = round(n * mean_out_degree)`` arcs are drawn
    with the tail proportional to the out-weight and the head proportional
    to the in-weight; then each arc independently also gets its reverse with
    probability ``reciprocity``.  Self-loops and repeated arcs are removed.
    """
    rng = _rng(seed)
    a = exponent - 1.0
    w_out = rng.pareto(a, n) + 1.0
    w_in = rng.pareto(a, n) + 1.0
    m0 = int(round(n * mean_out_degree))
    if max_degree is None:
        max_degree = math.sqrt(n * mean_out_degree)
    for w in (w_out, w_in):
        # Expected degree of v is m0 * w[v] / sum(w); clip iteratively.
        for _ in range(50):
            cap = max_degree * w.sum() / m0
            if w.max() <= cap * (1 + 1e-9):
                break
            np.minimum(w, cap, out=w)
    src = _draw_weighted(rng, w_out, m0)
    dst = _draw_weighted(rng, w_in, m0)
    if reciprocity > 0:
        back = rng.random(m0) < reciprocity
        src, dst = (np.concatenate([src, dst[back]]),
                    np.concatenate([dst, src[back]]))
    s, d = simple_arcs(src, dst)
    return n, s, d


def er_uniform(n: int, m: int, seed: int):
    """m distinct arcs with uniform random endpoints (self-loops and repeats redrawn)."""
    rng = _rng(seed)
    got = np.zeros(0, np.int64)
    while got.size < m:
        need = int((m - got.size) * 1.05) + 16
        s = rng.integers(0, n, size=need, dtype=np.int64)
        d = rng.integers(0, n, size=need, dtype=np.int64)
        k = s * n + d
        k = k[s != d]
        # keep first occurrences in draw order so the result is seed-stable
        k = np.concatenate([got, k])
        _, first = np.unique(k, return_index=True)
        got = k[np.sort(first)]
    got = got[:m]
    src, dst = simple_arcs(got // n, got % n)
    return n, src, dst


def batch(num_graphs: int, seed: int, n_lo: int = 10, n_hi: int = 500):
    """Many small independent graphs of uneven size.

    n is log-uniform in [n_lo, n_hi]; p is uniform in [0.02, 0.2].  Half of
    the graphs (by a fair coin) are G(n, p); the other half are Chung-Lu with
    weight exponent 2.5 and mean out-degree p * (n - 1).  Returns a list of
    ``(n, src, dst)``.
    """
    rng = _rng(seed)
    out = []
    for g in range(num_graphs):
        n = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        p = float(rng.uniform(0.02, 0.2))
        sub = int(rng.integers(0, 2**62))
        if rng.random() < 0.5:
            out.append(gnp(n, p, sub))
        else:
            out.append(chung_lu(n, max(p * (n - 1), 0.5), 2.5, sub))
    return out


def serve_requests(num: int, seed: int, rate_hz: float,
                   n_lo: int = 1000, n_hi: int = 2_000_000):
    """Poisson stream of count requests over Chung-Lu graphs.

    Returns a list of dicts ``{"t": arrival seconds, "k": 3|4, "n": ...,
    "mean_out_degree": ..., "exponent": ..., "seed": ...}``; the graph itself
    is drawn lazily with :func:`chung_lu` from those parameters so that a long
    stream costs no memory up front.  n is log-uniform in [n_lo, n_hi], mean
    out-degree uniform in [4, 16], exponent uniform in [2.1, 2.8], k is 3 or
    4 with equal probability.
    """
    rng = _rng(seed)
    t = 0.0
    reqs = []
    for i in range(num):
        t += float(rng.exponential(1.0 / rate_hz))
        reqs.append({
            "t": t,
            "k": int(3 + rng.integers(0, 2)),
            "n": int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi))))),
            "mean_out_degree": float(rng.uniform(4.0, 16.0)),
            "exponent": float(rng.uniform(2.1, 2.8)),
            "seed": int(rng.integers(0, 2**62)),
        })
    return reqs


# Named single-graph workloads (the plain, one-graph-per-launch configs).
WORKLOADS = {
    # Directed G(100, 0.08).
    "gnp_n100_p0.08": lambda seed=0: gnp(100, 0.08, seed),
    # Directed Chung-Lu, 1M vertices, ~10M arcs, Pareto exponent 2.3, max
    # expected degree 20k, reciprocity 0.2.
    "chunglu_n1M_m10M_a2.3_r0.2": lambda seed=2: chung_lu(
        1_000_000, 10.0 / 1.2, 2.3, seed, reciprocity=0.2, max_degree=20_000),
    # The same power-law shape at 1/10 and 3/10 scale (profiling captures;
    # the cap on the expected degree scales with sqrt(n)).
    "chunglu_n100k_m1M_a2.3_r0.2": lambda seed=2: chung_lu(
        100_000, 10.0 / 1.2, 2.3, seed, reciprocity=0.2, max_degree=6_000),
    "chunglu_n300k_m3M_a2.3_r0.2": lambda seed=2: chung_lu(
        300_000, 10.0 / 1.2, 2.3, seed, reciprocity=0.2, max_degree=11_000),
    # Directed uniform-endpoint ER, 4M vertices, 32M arcs, and the same
    # shape at 1/4 scale (profiling captures).
    "er_n4M_m32M": lambda seed=3: er_uniform(4_000_000, 32_000_000, seed),
    "er_n1M_m8M": lambda seed=3: er_uniform(1_000_000, 8_000_000, seed),
}


def workload(name: str, seed: int | None = None):
    f = WORKLOADS[name]
    return f() if seed is None else f(seed)
