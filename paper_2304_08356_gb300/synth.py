"""Seeded synthetic temporal graphs.

This module only draws inputs: edge lists (u, v, t) as uint32 numpy arrays.
It holds none of the sampler's arithmetic (no Philox, no path counting) and
is shared by the CPU oracle's tests and by the CUDA path's tests and bench.
Randomness comes from numpy's PCG64 (`numpy.random.default_rng`).

The paper's data sets (the temporal graphs of its Table 1) are not available;
these generators stand in for them with matched shape: power-law degrees,
|T| close to |E|, bursty contacts.

Workloads (sizes of the paper's experimental regime, Section 5 / Table 1):

* ``uniform_small``   n=100, 2,000 draws of (u,v) uniform with u != v,
                      t uniform in [1,200]; duplicates allowed.
* ``chung_lu_bursty`` Chung-Lu static skeleton (weights (i+1)^(-1/(gamma-1)),
                      random id permutation, u and v drawn independently by
                      weight, u == v redrawn); each static edge gets
                      K ~ Geometric(p) contacts forming a burst: first contact
                      at a centre c ~ U[0, t_max], later ones at c plus
                      cumulative Exp(mean mu) gaps, rounded and clipped to
                      [0, t_max]; static edges are drawn until m contacts exist
                      (the last burst is truncated).
* ``chung_lu_uniform_t`` Chung-Lu pairs drawn per temporal edge, t uniform in
                      [0, t_max).
"""
from __future__ import annotations

import numpy as np


def _as_u32(u, v, t):
    return (np.ascontiguousarray(u, dtype=np.uint32),
            np.ascontiguousarray(v, dtype=np.uint32),
            np.ascontiguousarray(t, dtype=np.uint32))


def uniform_small(n: int = 100, m: int = 2000, t_lo: int = 1, t_hi: int = 200,
                  seed: int = 1):
    """u, v uniform with u != v, t uniform in [t_lo, t_hi]; duplicates kept."""
    rng = np.random.default_rng(seed)
    u = rng.integers(0, n, size=m)
    # v uniform over the n-1 ids other than u
    v = rng.integers(0, n - 1, size=m)
    v = v + (v >= u)
    t = rng.integers(t_lo, t_hi + 1, size=m)
    return _as_u32(u, v, t)


def _chung_lu_weights(n: int, gamma: float, rng):
    w = (np.arange(n, dtype=np.float64) + 1.0) ** (-1.0 / (gamma - 1.0))
    perm = rng.permutation(n)
    p = np.empty(n, dtype=np.float64)
    p[perm] = w / w.sum()
    return p


def _draw_pairs(n: int, p, k: int, rng):
    """k directed pairs (u, v), u and v drawn independently with weights p,
    pairs with u == v redrawn."""
    cdf = np.cumsum(p)
    cdf[-1] = 1.0
    u = np.searchsorted(cdf, rng.random(k), side="right")
    v = np.searchsorted(cdf, rng.random(k), side="right")
    bad = np.nonzero(u == v)[0]
    while bad.size:
        v[bad] = np.searchsorted(cdf, rng.random(bad.size), side="right")
        bad = bad[u[bad] == v[bad]]
    return np.minimum(u, n - 1), np.minimum(v, n - 1)


def chung_lu_bursty(n: int = 20000, m: int = 500000, gamma: float = 2.3,
                    p_contacts: float = 0.3, mu: float = 1000.0,
                    t_max: int = 1_000_000, seed: int = 1):
    """Chung-Lu skeleton with Poisson-burst contacts (see module docstring)."""
    rng = np.random.default_rng(seed)
    p = _chung_lu_weights(n, gamma, rng)
    us, vs, ts = [], [], []
    have = 0
    while have < m:
        k = max(1024, int((m - have) * p_contacts * 1.2))
        u, v = _draw_pairs(n, p, k, rng)
        K = rng.geometric(p_contacts, size=k)
        csum = np.cumsum(K)
        last = int(np.searchsorted(csum, m - have, side="left"))
        if last < k:
            # keep edges 0..last, truncate the burst of edge `last`
            u, v, K = u[:last + 1], v[:last + 1], K[:last + 1].copy()
            K[-1] -= int(csum[last] - (m - have))
        centre = rng.random(u.size) * t_max
        tot = int(K.sum())
        owner = np.repeat(np.arange(u.size), K)
        gaps = rng.exponential(mu, size=tot)
        # the first contact of each burst sits at the centre
        first = np.zeros(u.size, dtype=np.int64)
        first[1:] = np.cumsum(K)[:-1]
        gaps[first] = 0.0
        cg = np.cumsum(gaps)
        base = cg[first]
        tt = centre[owner] + (cg - base[owner])
        tt = np.clip(np.rint(tt), 0, t_max)
        us.append(u[owner]); vs.append(v[owner]); ts.append(tt)
        have += tot
    return _as_u32(np.concatenate(us), np.concatenate(vs), np.concatenate(ts))


def chung_lu_uniform_t(n: int = 1_000_000, m: int = 20_000_000, gamma: float = 2.1,
                       t_max: int = 1 << 24, seed: int = 1):
    """Chung-Lu pairs drawn independently per temporal edge, t uniform in
    [0, t_max)."""
    rng = np.random.default_rng(seed)
    p = _chung_lu_weights(n, gamma, rng)
    u, v = _draw_pairs(n, p, m, rng)
    t = rng.integers(0, t_max, size=m)
    return _as_u32(u, v, t)


def random_tiny(n: int, m: int, t_hi: int, seed: int, self_loops: bool = False):
    """Small random multigraph for brute-force checks: u, v uniform (self
    loops optional), t uniform in [1, t_hi] (ties are frequent)."""
    rng = np.random.default_rng(seed)
    u = rng.integers(0, n, size=m)
    if self_loops:
        v = rng.integers(0, n, size=m)
    else:
        v = rng.integers(0, n - 1, size=m)
        v = v + (v >= u)
    t = rng.integers(1, t_hi + 1, size=m)
    return _as_u32(u, v, t)


def batch_instances(count: int = 256, n_lo: int = 500, n_hi: int = 50000,
                    edges_per_node: int = 20, gamma: float = 2.3, seed0: int = 1000):
    """Uneven instances: n log-uniform in [n_lo, n_hi], m = edges_per_node*n,
    bursty Chung-Lu, instance g seeded with seed0 + g."""
    out = []
    for g in range(count):
        rng = np.random.default_rng(seed0 + g)
        ng = int(np.floor(np.exp(rng.uniform(np.log(n_lo), np.log(n_hi)))))
        out.append(chung_lu_bursty(n=ng, m=edges_per_node * ng, gamma=gamma,
                                   seed=seed0 + g))
    return out
