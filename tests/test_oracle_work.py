"""Pins of the oracle's search work counters (E_scan, U, S_new, F: the exact
counters behind the algorithmic-byte model of the measurement) against the
same definitions evaluated on brute-force walk sets.  The levels, the
appearance states and the earliest arrivals come from enumerating every
time-respecting walk (tests/bruteforce.py), not from the oracle's search.
No GPU."""
from collections import defaultdict

import numpy as np
import pytest

import bruteforce as BF
from oracle import oracle as O
from paper_2304_08356_gb300 import synth

NEG = BF.NEG


def bf_work(edges, n, opt, s, z):
    """(escan, eadd, snew, fseg) of one sample by the counters' definitions,
    from brute-force walks (edges deduplicated, no self loops)."""
    out_s = [e for e in edges if e[0] == s]
    in_z = [e for e in edges if e[1] == z]
    if not out_s or not in_z:
        return (0, 0, 0, 0)
    tz = max(c for _, _, c in in_z)
    walks = BF.walks_from(edges, s)
    if opt == 2:
        fa = {s: NEG}
        for vs, ts in walks:
            v = vs[-1]
            if v != s:
                fa[v] = min(fa.get(v, ts[-1]), ts[-1])
        ts_s = min(c for _, _, c in out_s)
        te = fa.get(z, tz)
        inf = float("inf")
        escan = sum(1 for a, b, c in edges if b != s and ts_s <= c <= te)
        eadd = sum(1 for a, b, c in edges
                   if b != s and b in fa and c == fa[b] and c <= te and fa.get(a, inf) < fa[b])
        return (escan, eadd, 0, 0)
    level = {}
    for vs, ts in walks:
        key = (vs[-1], ts[-1])
        level[key] = min(level.get(key, len(vs) - 1), len(vs) - 1)
    fsfm = opt == 3
    keep = (lambda t: t <= tz) if fsfm else (lambda t: t < tz)
    levels = defaultdict(list)
    levels[0].append((s, NEG))
    for (v, t), k in level.items():
        if keep(t):
            levels[k].append((v, t))
    zl = [k for (v, t), k in level.items() if v == z]
    if not fsfm and zl:
        d = min(zl)
        last_searched, last_expanded = d - 1, d - 2
    else:
        K = max(k for k, lst in levels.items() if lst)
        last_searched = last_expanded = K
    escan = eadd = snew = fseg = 0
    for k in range(last_searched + 1):
        first = {}
        for v, t in levels[k]:
            first[v] = min(first.get(v, t), t)
        fseg += len(first)
        if not fsfm:
            escan += len(in_z)
        if k > last_expanded:
            continue
        for u, t0 in first.items():
            for a, b, c in edges:
                if a == u and c > t0 and keep(c):
                    escan += 1
                    if level[(b, c)] == k + 1:
                        eadd += 1
        snew += len(levels[k + 1])
    return (escan, eadd, snew, fseg)


@pytest.mark.parametrize("seed", range(24))
def test_work_counters_against_bruteforce(seed):
    rng = np.random.default_rng(500 + seed)
    n = int(rng.integers(3, 7))
    m = int(rng.integers(4, 18))
    u, v, t = synth.random_tiny(n, m, t_hi=int(rng.integers(2, 7)), seed=3000 + seed, self_loops=(seed % 4 == 0))
    edges = BF.dedupe(u, v, t)
    g = O.Graph(u, v, t, n=n)
    count = 40
    for opt in (0, 1, 2, 3):
        got = g.work(opt, 17 + seed, 0, count)
        for i in range(count):
            s, z = O.draw_pair(n, 17 + seed, i)
            assert tuple(int(x) for x in got[i]) == bf_work(edges, n, opt, s, z), (opt, i, s, z)


def test_work_counter_invariants():
    """sh and sfm run the same search (equal counters); every new state is
    reached by at least one counted edge (eadd >= snew); the pull test makes
    escan >= |in(z)| per searched level."""
    u, v, t = synth.uniform_small(n=60, m=900, t_hi=40, seed=8)
    g = O.Graph(u, v, t, n=60)
    w0, w1 = g.work(0, 3, 0, 300), g.work(1, 3, 0, 300)
    assert np.array_equal(w0, w1)
    assert np.all(w0[:, 1] >= w0[:, 2])
    assert w0[:, 0].sum() > 0 and g.work(2, 3, 0, 300)[:, 1].sum() > 0


@pytest.mark.parametrize("opt", [0, 1, 2, 3])
def test_estimate_sums_the_sample_counters(opt):
    """Algorithm 1's reported counters are the sums over its samples: the r
    estimation samples with fixed r; the s' bootstrap samples and the r
    estimation samples in a progressive run."""
    u, v, t = synth.uniform_small(n=40, m=500, t_hi=60, seed=11)
    g = O.Graph(u, v, t, n=40)
    _, _, info = g.estimate(opt, 0.1, 0.1, 4, fixed_r=200)
    w = g.work(opt, 4, 0, 200).sum(axis=0)
    assert [info["edges_scanned"], info["sigma_adds"], info["states_new"], info["frontier_vertices"]] == \
        [int(x) for x in w]
    _, _, info = g.estimate(opt, 0.1, 0.1, 4)
    w = g.work(opt, 4, 0, info["r"]).sum(axis=0) + \
        g.work(opt, 4, 0, info["bootstrap"], dom_pair=O.D_BOOT_PAIR, dom_path=O.D_BOOT_PATH).sum(axis=0)
    assert [info["edges_scanned"], info["sigma_adds"], info["states_new"], info["frontier_vertices"]] == \
        [int(x) for x in w]
