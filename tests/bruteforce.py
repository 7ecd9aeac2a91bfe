"""Brute-force enumeration of temporal walks on tiny graphs (test helper).

Independent of the oracle: every time-respecting walk from (s, -inf) is
listed explicitly and the optimal sets of Def. 1 (paper Sec. 3) are picked
from the full list by their definitions:

* sh  -- walks s -> z with the minimum number of hops;
* sfm -- among the sh walks, those with the earliest arrival at z;
* pfm -- walks whose every prefix is foremost: each visited vertex is reached
         at its earliest arrival time fa (the minimum arrival over all walks);
* fsfm -- the foremost walks (arrival fa(z)) with the minimum number of hops.

A walk is a sequence of vertex appearances with strictly increasing times
(Sec. 3); vertices may repeat in a walk, so nothing here assumes that
optimal walks are simple.  Inputs must be tiny (times bound the walk length).
"""
from __future__ import annotations

from collections import defaultdict
from fractions import Fraction

NEG = -1  # time of the source appearance (s, -inf)


def dedupe(u, v, t):
    """Distinct (u, v, t) triples with u != v."""
    return sorted({(int(a), int(b), int(c)) for a, b, c in zip(u, v, t) if a != b})


def walks_from(edges, s):
    """All walks from (s, -inf) as (vertices, times) tuples, one edge or more."""
    adj = defaultdict(list)
    for a, b, c in edges:
        adj[a].append((b, c))
    out = []
    stack = [((s,), (NEG,))]
    while stack:
        vs, ts = stack.pop()
        for b, c in adj[vs[-1]]:
            if c > ts[-1]:
                w = (vs + (b,), ts + (c,))
                out.append(w)
                stack.append(w)
    return out


def optimal_sets(edges, n, s):
    """{z: {opt: [walks]}} for every z != s reachable from s."""
    ws = walks_from(edges, s)
    by_end = defaultdict(list)
    for w in ws:
        if w[0][-1] != s:
            by_end[w[0][-1]].append(w)
    fa = {}
    for vs, ts in ws:
        z = vs[-1]
        if z != s:
            fa[z] = min(fa.get(z, ts[-1]), ts[-1])
    res = {}
    for z, lst in by_end.items():
        h = min(len(w[0]) - 1 for w in lst)
        sh = [w for w in lst if len(w[0]) - 1 == h]
        arr = min(w[1][-1] for w in sh)
        sfm = [w for w in sh if w[1][-1] == arr]
        pfm = [w for w in lst if all(w[1][i] == fa.get(w[0][i]) for i in range(1, len(w[0])))]
        fore = [w for w in lst if w[1][-1] == fa[z]]
        hf = min(len(w[0]) - 1 for w in fore)
        fsfm = [w for w in fore if len(w[0]) - 1 == hf]
        res[z] = {0: sh, 1: sfm, 2: pfm, 3: fsfm}
    return res


def sigma_table(edges, n):
    """sigma[(opt, s, z)] = number of optimal walks (0 if unreachable)."""
    sig = {}
    for s in range(n):
        sets = optimal_sets(edges, n, s)
        for z in range(n):
            if z == s:
                continue
            for opt in (0, 1, 2):
                sig[(opt, s, z)] = len(sets[z][opt]) if z in sets else 0
    return sig


def exact_bc(edges, n, opt):
    """b_v = 1/(n(n-1)) sum_{s != z} #(optimal walks through v) / sigma_sz, as Fractions."""
    acc = [Fraction(0)] * n
    for s in range(n):
        sets = optimal_sets(edges, n, s)
        for z, d in sets.items():
            lst = d[opt]
            if not lst:
                continue
            through = defaultdict(int)
            for vs, _ in lst:
                for v in set(vs[1:-1]):
                    if v != s and v != z:
                        through[v] += 1
            for v, k in through.items():
                acc[v] += Fraction(k, len(lst))
    return [a / (n * (n - 1)) for a in acc]


def mean_internal(edges, n, opt):
    """rho = 1/(n(n-1)) sum_{s != z} mean over optimal walks of |Int(tp)|."""
    acc = Fraction(0)
    for s in range(n):
        for z, d in optimal_sets(edges, n, s).items():
            lst = d[opt]
            if lst:
                acc += Fraction(sum(len(vs) - 2 for vs, _ in lst), len(lst))
    return acc / (n * (n - 1))


def distances(edges, n, opt):
    """d[(u, v)] for reachable v != u: minimum hops among optimal walks
    (sh and sfm: minimum hops over all walks; pfm: minimum hops among pfm walks;
    fsfm: minimum hops among the foremost walks)."""
    d = {}
    for u in range(n):
        for z, sets in optimal_sets(edges, n, u).items():
            lst = sets[opt] if opt in (2, 3) else sets[0]
            if lst:
                d[(u, z)] = min(len(vs) - 1 for vs, _ in lst)
    return d


def exact_edge_bc(edges, n, opt, temporal):
    """Temporal edge betweenness (paper App. A), as Fractions: with
    temporal=True, b_(u,v,t) for every temporal edge; otherwise b_(u,v) for
    every underlying edge: 1/(n(n-1)) sum_{s != z} #(optimal walks using the
    edge) / sigma_sz.  Every edge of a walk counts, the first and last too."""
    acc = defaultdict(Fraction)
    for s in range(n):
        for z, d in optimal_sets(edges, n, s).items():
            lst = d[opt]
            if not lst:
                continue
            through = defaultdict(int)
            for vs, ts in lst:
                keys = {(vs[k], vs[k + 1], ts[k + 1]) if temporal else (vs[k], vs[k + 1]) for k in range(len(vs) - 1)}
                for key in keys:
                    through[key] += 1
            for key, k in through.items():
                acc[key] += Fraction(k, len(lst))
    return {key: a / (n * (n - 1)) for key, a in acc.items()}


def mean_edges(edges, n, opt):
    """1/(n(n-1)) sum_{s != z} mean over optimal walks of the number of
    distinct underlying edges they use (App. A's Psi)."""
    acc = Fraction(0)
    for s in range(n):
        for z, d in optimal_sets(edges, n, s).items():
            lst = d[opt]
            if lst:
                acc += Fraction(sum(len({(vs[k], vs[k + 1]) for k in range(len(vs) - 1)}) for vs, _ in lst), len(lst))
    return acc / (n * (n - 1))
