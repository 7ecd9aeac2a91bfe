"""Pins of the CPU oracle against values fixed by the paper and by the
mathematics (no GPU).  Each test names what it pins."""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import bruteforce as BF
from oracle import oracle as O
from paper_2304_08356_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------
# Philox4x32-10 (Salmon et al., SC'11) against an independent implementation:
# curand's PHILOX4_32_10 host generator (called, not reproduced).  Observed
# layout of its output: block j (4 words) for seed K is Philox4x32-10 with key
# (K_lo, K_hi) and counter (q_lo, q_hi, j mod 65536, 0), q = j div 65536; a
# generator offset of 4j starts at block j.  Counter word 3 is pinned on the
# GPU against curand's device API (tests/test_gpu_philox.py).
# --------------------------------------------------------------------------
def _curand_host():
    import ctypes as C
    import glob
    cands = glob.glob("/usr/local/cuda/lib64/libcurand.so*") + glob.glob("/usr/local/cuda/targets/*/lib/libcurand.so*")
    for c in ["libcurand.so"] + cands:
        try:
            return C.CDLL(c)
        except OSError:
            continue
    return None


def test_philox_matches_curand_host_generator():
    import ctypes as C
    L = _curand_host()
    if L is None:
        pytest.skip("libcurand not available")
    PHILOX4_32_10 = 161                               # curandRngType_t value
    checked = 0
    for seed in (0, 1, 0x123456789ABCDEF0, 0xFFFFFFFFFFFFFFFF, 0x00000000DEADBEEF):
        for q, w2 in ((0, 0), (0, 1), (0, 65535), (1, 3), ((1 << 32) + 5, 777), ((1 << 40) + 12345, 40000)):
            block = q * 65536 + w2
            gen = C.c_void_p()
            assert L.curandCreateGeneratorHost(C.byref(gen), PHILOX4_32_10) == 0
            assert L.curandSetPseudoRandomGeneratorSeed(gen, C.c_ulonglong(seed)) == 0
            assert L.curandSetGeneratorOffset(gen, C.c_ulonglong(4 * block)) == 0
            out = (C.c_uint * 4)()
            assert L.curandGenerate(gen, out, C.c_size_t(4)) == 0
            L.curandDestroyGenerator(gen)
            ctr = [q & 0xFFFFFFFF, q >> 32, w2, 0]
            assert O.philox(ctr, [seed & 0xFFFFFFFF, seed >> 32]) == list(out), (seed, ctr)
            checked += 1
    assert checked == 30


def test_uniform_draw_range_and_frequencies():
    # rejection sampling: values in [0, N) and flat frequencies (chi-square)
    N, K = 12, 12000
    xs = np.array([O.uniform64(N, 99, i, O.D_PAIR) for i in range(K)])
    assert xs.min() >= 0 and xs.max() < N
    f = np.bincount(xs, minlength=N)
    chi2 = ((f - K / N) ** 2 / (K / N)).sum()
    assert chi2 < 40.0          # 11 dof, p ~ 1e-4
    assert O.uniform64(1, 5, 3, 0) == 0


def test_pair_draw_uniform_over_ordered_pairs():
    n, K = 5, 20000
    cnt = np.zeros((n, n))
    for i in range(K):
        s, z = O.draw_pair(n, 7, i)
        assert s != z and 0 <= s < n and 0 <= z < n
        cnt[s, z] += 1
    assert np.all(np.diag(cnt) == 0)
    e = K / (n * (n - 1))
    chi2 = (((cnt - e) ** 2) / e)[~np.eye(n, dtype=bool)].sum()
    assert chi2 < 60.0          # 19 dof


def test_rademacher_is_bit_of_block():
    for i in (0, 1, 77):
        w = O.philox([i & 0xFFFFFFFF, i >> 32, O.D_RADE, 0], [1234, 0])
        for j in range(128):
            bit = (w[j >> 5] >> (j & 31)) & 1
            assert O.rademacher(1234, i, j) == (1 if bit else -1)


# --------------------------------------------------------------------------
# Worked example (paper App. A, figure "example_tp")
# --------------------------------------------------------------------------
def _example():
    edges, expect = [], {0: [], 1: [], 2: []}
    names = {}
    for line in open(os.path.join(GOLDEN, "example_tp.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        if "|" in line:
            opt, p = [x.strip() for x in line.split("|")]
            expect[{"sh": 0, "sfm": 1, "pfm": 2}[opt]].append(
                [(names[tok.split(":")[0]], int(tok.split(":")[1])) for tok in p.split()])
            continue
        a, b, t = line.split()
        for x in (a, b):
            names.setdefault(x, len(names))
        edges.append((names[a], names[b], int(t)))
    return edges, expect, names


def test_worked_example_paths():
    edges, expect, names = _example()
    u, v, t = zip(*edges)
    g = O.Graph(u, v, t)
    s, z = names["s"], names["z"]
    for opt in (0, 1, 2):
        sig, d = g.sigma(opt, s, z)
        assert sig == len(expect[opt])
        got = []
        for x in range(sig):
            p, ts = g.unrank(opt, s, z, x, with_times=True)
            got.append(list(zip(p, ts)))
        assert sorted(got) == sorted(expect[opt])
    assert g.sigma(0, s, z)[1] == 3          # d_sh(s, z) = 3 hops
    assert g.sigma(2, s, z)[1] == 4          # fa(z) = 4


# --------------------------------------------------------------------------
# Brute force on tiny graphs: sigma for every pair, and the path draw is a
# bijection x -> optimal path (Theorem on the path sampler, App. C).
# --------------------------------------------------------------------------
@pytest.mark.parametrize("seed", range(60))
def test_bruteforce_sigma_and_bijection(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(3, 7))
    m = int(rng.integers(4, 16))
    u, v, t = synth.random_tiny(n, m, t_hi=int(rng.integers(2, 7)), seed=1000 + seed, self_loops=(seed % 5 == 0))
    edges = BF.dedupe(u, v, t)
    g = O.Graph(u, v, t, n=n)
    assert g.m == len(edges)
    for s in range(n):
        sets = BF.optimal_sets(edges, n, s)
        for z in range(n):
            if z == s:
                continue
            for opt in (0, 1, 2, 3):
                want = sets[z][opt] if z in sets else []
                sig, _ = g.sigma(opt, s, z)
                assert sig == len(want), (opt, s, z)
                got = sorted(tuple(zip(*g.unrank(opt, s, z, x, with_times=True))) for x in range(sig))
                assert got == sorted(tuple(zip(vs, ts)) for vs, ts in want)


@pytest.mark.parametrize("seed", range(12))
def test_exact_bc_against_bruteforce_and_lemma1(seed):
    u, v, t = synth.random_tiny(6, 14, t_hi=5, seed=2000 + seed)
    edges = BF.dedupe(u, v, t)
    g = O.Graph(u, v, t, n=6)
    for opt in (0, 1, 2, 3):
        want = BF.exact_bc(edges, 6, opt)
        got = g.exact_bc(opt)
        assert np.allclose(got, [float(x) for x in want], rtol=0, atol=1e-15)
        # Lemma 1 (Sec. 3): sum_v b_v = rho
        assert abs(sum(want) - BF.mean_internal(edges, 6, opt)) == 0


def test_layered_dag_reduces_to_static_path_counts():
    # Textbook reduction: in a layered DAG whose edge times equal the head's
    # layer, every static path is time-respecting and every s->z path has the
    # same length, so sh sigma equals the static path count (dynamic program).
    rng = np.random.default_rng(5)
    widths = [1, 3, 4, 3, 1]
    ids, base = [], 0
    for w in widths:
        ids.append(list(range(base, base + w)))
        base += w
    edges = []
    for L in range(len(widths) - 1):
        for a in ids[L]:
            for b in ids[L + 1]:
                if rng.random() < 0.7 or L in (0, len(widths) - 2):
                    edges.append((a, b, L + 1))
    u, v, t = zip(*edges)
    g = O.Graph(u, v, t, n=base)
    s, z = ids[0][0], ids[-1][0]
    cnt = {s: 1}
    for L in range(1, len(widths)):
        for b in ids[L]:
            cnt[b] = sum(cnt.get(a, 0) for (a, bb, _) in edges if bb == b)
    for opt in (0, 1, 2, 3):
        assert g.sigma(opt, s, z)[0] == cnt[z]


def test_equal_timestamps_single_edge_paths():
    # All timestamps equal: every temporal path is one edge (strict increase).
    u, v, _ = synth.uniform_small(n=30, m=200, seed=3)
    t = np.full(u.size, 7, np.uint32)
    g = O.Graph(u, v, t, n=30)
    pairs = {(int(a), int(b)) for a, b in zip(u, v) if a != b}
    for (s, z) in [(0, 1), (2, 9), (5, 4)]:
        for opt in (0, 1, 2, 3):
            assert g.sigma(opt, s, z)[0] == (1 if (s, z) in pairs else 0)
    est, hits, info = g.estimate(0, 0.1, 0.1, 1, fixed_r=300)
    assert hits.sum() == 0 and info["sum_int_len"] == 0
    reach, dlb = g.stats_counts(0, 1, 0, all_sources=True)
    assert dlb == 1 and int(reach[1]) == len(pairs)


# --------------------------------------------------------------------------
# Algorithm 1 pieces
# --------------------------------------------------------------------------
def test_estimate_invariants_and_mcera_recount():
    u, v, t = synth.uniform_small(n=40, m=500, t_hi=60, seed=11)
    g = O.Graph(u, v, t, n=40)
    r, c, seed = 300, 25, 17
    for opt in (0, 1, 2, 3):
        est, hits, info = g.estimate(opt, 0.1, 0.1, seed, c=c, fixed_r=r)
        samples = g.samples(opt, seed, 0, r)
        # hits = number of samples whose drawn path has v internal
        H = np.zeros(40, np.int64)
        S = np.zeros((c, 40), np.int64)
        for i, (_, _, _, p) in enumerate(samples):
            lam = [O.rademacher(seed, i, j) for j in range(c)]
            for x in p[1:-1]:
                H[x] += 1
                S[:, x] += lam
        assert np.array_equal(hits.astype(np.int64), H)
        assert int(H.sum()) == info["sum_int_len"]                # Lemma 1, sample form
        assert info["rade_num"] == int(S.max(axis=1).sum())      # sup over all nodes, no |.|
        assert info["max_hits"] == int(H.max())
        assert np.array_equal(est, hits.astype(np.float64) / r)


def test_sd_bound_special_cases():
    # Theorem 1 with R = 0 reduces to sqrt(2 ln(4/d) v / r) + ln(4/d)/(3r)
    L = math.log(4 / 0.05)
    assert O.xi_from_R(0.0, 0.01, 0.05, 1000) == pytest.approx(math.sqrt(2 * L * 0.01 / 1000) + L / 3000, rel=1e-14)
    # with W = 0 and Rc = 0: R~ = 0, R = 2 ln(4/d)/r
    R = 2 * L / 1000
    assert O.sd_bound(0.0, 0.0, 0.0, 0.05, 1000, 25) == pytest.approx(2 * R + math.sqrt(2 * L * 4 * R / 1000) + L / 3000, rel=1e-14)
    # decreasing in r
    xs = [O.sd_bound(0.01, 0.02, 0.02, 0.05, r, 25) for r in (100, 1000, 10000, 100000)]
    assert all(a > b for a, b in zip(xs, xs[1:]))
    # hand-evaluated closed form of omega: vhat=0.01, rho=2, eps=0.01, delta=0.05
    # ((0.02 + 0.0066667)/1e-4) * (ln 400 + ln 20) = 266.6667 * 8.9872 = 2396.6
    assert O.omega_bound(0.01, 2.0, 0.01, 0.05) == pytest.approx(2396.58, rel=1e-4)


def test_progressive_schedule_properties():
    u, v, t = synth.chung_lu_bursty(n=400, m=6000, seed=3)
    g = O.Graph(u, v, t)
    eps, delta = 0.05, 0.1
    est, hits, info = g.estimate(0, eps, delta, 5)
    assert info["bootstrap"] == O.sample_size_bootstrap(eps, delta) == 47
    assert info["s1"] >= info["bootstrap"] or info["s1"] == info["omega"]
    assert info["r"] <= info["omega"]
    assert info["xi"] <= eps or info["r"] >= info["omega"]
    # schedule: r after k rounds follows s_i = min(omega, ceil(1.2 s_{i-1}))
    s = info["s1"]
    for _ in range(info["rounds"] - 1):
        s = min(info["omega"], math.ceil(1.2 * s))
    assert s == info["r"]
    # s1 is the least s in [s', omega] with xi(R = 0) <= eps
    assert np.isclose(est.sum(), info["sum_int_len"] / info["r"])


# --------------------------------------------------------------------------
# Small-config accuracy: Hoeffding / Theorem 1 against exact betweenness
# --------------------------------------------------------------------------
def test_small_config_within_hoeffding_and_xi():
    u, v, t = synth.uniform_small()
    g = O.Graph(u, v, t, n=100)
    exact = g.exact_bc(0)
    est, hits, info = g.estimate(0, 0.05, 0.1, 1, fixed_r=1000)
    sd = np.abs(est - exact).max()
    assert sd <= math.sqrt(math.log(2 * 100 / 0.1) / (2 * 1000))   # 0.0617 (Hoeffding + union bound)
    assert sd <= info["xi"]                                          # Theorem 1
    # Lemma 1 on the exact side: sum of exact betweenness = rho >= 0
    assert exact.sum() > 0


# --------------------------------------------------------------------------
# Algorithm 2: with every node as a source the estimates are exact
# --------------------------------------------------------------------------
@pytest.mark.parametrize("seed", range(8))
def test_stats_all_sources_against_bruteforce(seed):
    n = 6
    u, v, t = synth.random_tiny(n, 14, t_hi=6, seed=3000 + seed)
    edges = BF.dedupe(u, v, t)
    g = O.Graph(u, v, t, n=n)
    for opt in (0, 1, 2, 3):
        d = BF.distances(edges, n, opt)
        reach, dlb = g.stats_counts(opt, 0, 0, all_sources=True)
        D = max(d.values()) if d else 0
        assert dlb == D
        for h in range(D + 1):
            assert int(reach[h]) == sum(1 for x in d.values() if x <= h)
        st = O.stats_summary(reach, dlb, n, n)
        if d:
            assert st["zeta"] == pytest.approx(len(d) / (n * (n - 1)), rel=1e-14)
            assert st["psi"] == pytest.approx(sum(d.values()) / len(d), rel=1e-14)
    # sfm distances equal sh distances
    assert np.array_equal(g.stats_counts(0, 0, 0, True)[0], g.stats_counts(1, 0, 0, True)[0])


def test_wimpy_variance_bound_covers_the_variance():
    """The appendix's variance bound from the empirical wimpy variance W holds
    with probability >= 1 - delta: for a 0/1 estimator f with E[f^2] = p, the
    bound computed from W = (hits)/r falls below p in at most a delta share
    of independent samples.  A bound without its square-root or ln/r terms
    fails this at these sizes."""
    rng = np.random.default_rng(12)
    for p, r, delta in ((0.02, 500, 0.1), (0.2, 200, 0.05), (0.001, 4000, 0.1)):
        hits = rng.binomial(r, p, size=4000)
        vh = np.array([O.wimpy_variance_bound(h / r, delta, r) for h in hits])
        assert (vh >= hits / r).all()
        miss = float((vh < p).mean())
        assert miss <= delta, (p, r, miss)
        # the same with the square-root term dropped undershoots far more often
        L = math.log(1 / delta)
        bare = hits / r + L / r
        assert float((bare < p).mean()) > miss
    # W = 0: only the confidence terms remain, 2 ln(1/delta) / r
    assert O.wimpy_variance_bound(0.0, 0.1, 1000) == pytest.approx(2 * math.log(10) / 1000, rel=1e-15)


# --------------------------------------------------------------------------
# Temporal edge betweenness (App. A): edge ids, the two lemmas, estimates.
# --------------------------------------------------------------------------
@pytest.mark.parametrize("seed", range(8))
def test_edge_ids_follow_the_drawn_paths(seed):
    u, v, t = synth.random_tiny(6, 16, t_hi=5, seed=3000 + seed)
    g = O.Graph(u, v, t, n=6)
    eu, ev, et, ue, nu = g.edge_ids()
    # ids: temporal edges in (v, t, u) order, underlying edges in (v, u) order
    assert sorted(zip(ev, et, eu)) == list(zip(ev, et, eu))
    und = sorted({(int(b), int(a)) for a, b in zip(eu, ev)})
    assert nu == len(und) and all(und[ue[e]] == (int(ev[e]), int(eu[e])) for e in range(g.m))
    for opt in (0, 1, 2, 3):
        for (s, z, sig, path, pe) in g.samples(opt, 4, 0, 300, cap=8, edges=True):
            assert len(pe) == max(len(path) - 1, 0)
            ts = [int(et[e]) for e in pe]
            assert all(int(eu[e]) == path[k] and int(ev[e]) == path[k + 1] for k, e in enumerate(pe))
            assert all(a < b for a, b in zip(ts, ts[1:]))


@pytest.mark.parametrize("seed", range(8))
def test_edge_betweenness_lemmas_on_bruteforce(seed):
    """App. A: b_e = sum_t b_(e,t) and sum_e b_e = Psi (mean edges of an
    optimal path over all ordered pairs), exactly."""
    u, v, t = synth.random_tiny(6, 14, t_hi=5, seed=4000 + seed)
    edges = BF.dedupe(u, v, t)
    for opt in (0, 1, 2, 3):
        bt = BF.exact_edge_bc(edges, 6, opt, temporal=True)
        bu = BF.exact_edge_bc(edges, 6, opt, temporal=False)
        agg = {}
        for (a, b, _), x in bt.items():
            agg[(a, b)] = agg.get((a, b), 0) + x
        assert agg == bu
        assert sum(bu.values()) == BF.mean_edges(edges, 6, opt)


@pytest.mark.parametrize("target", [1, 2])
def test_edge_estimates_within_hoeffding(target):
    """Fixed-r estimates of edge betweenness against the brute-force values:
    max error within Hoeffding's bound at delta = 1e-3 (one-sided union over
    the family), and the hit totals equal the drawn paths' edge counts."""
    u, v, t = synth.random_tiny(6, 14, t_hi=5, seed=4100)
    edges = BF.dedupe(u, v, t)
    g = O.Graph(u, v, t, n=6)
    eu, ev, et, ue, nu = g.edge_ids()
    r = 20000
    for opt in (0, 2):
        est, hits, info = g.estimate(opt, 0.05, 0.1, 3, fixed_r=r, target=target)
        exact = BF.exact_edge_bc(edges, 6, opt, temporal=(target == 2))
        F = len(est)
        assert F == (g.m if target == 2 else nu)
        want = np.zeros(F)
        for e in range(g.m):
            key = (int(eu[e]), int(ev[e]), int(et[e])) if target == 2 else (int(eu[e]), int(ev[e]))
            want[e if target == 2 else ue[e]] = float(exact.get(key, 0))
        bound = math.sqrt(math.log(2 * F / 1e-3) / (2 * r))
        assert np.abs(est - want).max() <= bound
        rows = g.samples(opt, 3, 0, r, cap=8)
        assert hits.sum() == info["sum_int_len"] == sum(max(len(p) - 1, 0) for (_, _, _, p) in rows)
    # underlying hits are the temporal hits summed per underlying edge
    _, ht, _ = g.estimate(2, 0.05, 0.1, 5, fixed_r=3000, target=2)
    _, hu, _ = g.estimate(2, 0.05, 0.1, 5, fixed_r=3000, target=1)
    assert np.array_equal(np.bincount(ue, weights=ht, minlength=nu).astype(np.uint64), hu)


# --------------------------------------------------------------------------
# The ob estimator (Sec. 4.1): f_v(s,z) = sigma_sz(v) / sigma_sz, carried as
# the nearest multiple of 2^-32 (ties up).
# --------------------------------------------------------------------------
def _round32(a, b):
    """Nearest integer to 2^32 a / b, ties up (Python integers)."""
    return (2 * a * (1 << 32) + b) // (2 * b)


@pytest.mark.parametrize("seed", range(10))
def test_through_counts_against_bruteforce(seed):
    """sigma_sz(v) = the number of optimal walks from s to z with v internal,
    counted on the explicit walk list; their sum over v is the total internal
    length of the optimal walks (every pair, every optimality)."""
    u, v, t = synth.random_tiny(6, 16, t_hi=5, seed=5000 + seed, self_loops=True)
    edges = BF.dedupe(u, v, t)
    g = O.Graph(u, v, t, n=6)
    for s in range(6):
        sets = BF.optimal_sets(edges, 6, s)
        for z in range(6):
            if z == s:
                continue
            for opt in (0, 1, 2, 3):
                walks = sets[z][opt] if z in sets else []
                sig, th = g.through(opt, s, z)
                assert sig == len(walks)
                want = [0] * 6
                for vs, _ in walks:
                    for x in set(vs[1:-1]):
                        want[x] += 1
                assert th == want, (s, z, opt)
                assert sum(th) == sum(len(vs) - 2 for vs, _ in walks)


def test_fixed32_rounding():
    rng = np.random.default_rng(11)
    cases = [(0, 1), (1, 1), (1, 2), (1, 3), (2, 3), (1, 1 << 33), (3, 1 << 34), (1, (1 << 33) + 1),
             ((1 << 64) - 1, (1 << 64) - 1), ((1 << 127), (1 << 128) - 1), ((1 << 128) - 2, (1 << 128) - 1),
             (1, (1 << 128) - 1), ((1 << 96) + 12345, (1 << 97) + 1)]
    for _ in range(3000):
        bits = int(rng.integers(1, 129))
        b = int(rng.integers(1, 1 << 62)) if bits <= 62 else (int(rng.integers(1, 1 << 62)) << (bits - 62)) | 1
        b = min(b, (1 << 128) - 1)
        a = b * int(rng.integers(0, 1 << 30)) // (1 << 30)
        cases.append((a, b))
    for a, b in cases:
        assert O.fixed32(a, b) == _round32(a, b), (a, b)


@pytest.mark.parametrize("opt", [0, 1, 2])
def test_ob_sums_recounted(opt):
    """A fixed-r ob run recounted from the per-pair through counts with
    Python's own rounding: hits, the wimpy maximum, N_R and the total."""
    u, v, t = synth.uniform_small(n=40, m=500, seed=3)
    g = O.Graph(u, v, t, n=40)
    r, c, seed = 300, 7, 9
    est, hits, info = g.estimate(opt, 0.05, 0.1, seed, c=c, fixed_r=r, estimator=1)
    H = np.zeros(40, dtype=object); W = np.zeros(40, dtype=object)
    S = np.zeros((c, 40), dtype=object)
    tot = 0
    for i in range(r):
        s, z = O.draw_pair(40, seed, i)
        sig, th = g.through(opt, s, z)
        for x in range(40):
            if th[x]:
                q = _round32(th[x], sig)
                H[x] += q
                W[x] += (q * q + (1 << 31)) >> 32
                tot += q
                for j in range(c):
                    S[j, x] += O.rademacher(seed, i, j) * q
    assert [int(x) for x in hits] == list(H)
    assert info["max_hits"] == max(W) and info["sum_int_len"] == tot
    assert info["rade_num"] == sum(max(S[j]) for j in range(c))
    assert np.array_equal(est, np.array([float(h) for h in H]) / (r * 4294967296.0))


@pytest.mark.parametrize("opt", [0, 2])
def test_ob_estimates_within_hoeffding(opt):
    """The ob estimate is unbiased for b_v: against brute-force exact values,
    max error within Hoeffding's bound (f in [0,1]) at delta = 1e-3."""
    u, v, t = synth.random_tiny(7, 22, t_hi=6, seed=4200)
    edges = BF.dedupe(u, v, t)
    g = O.Graph(u, v, t, n=7)
    r = 20000
    est, _, _ = g.estimate(opt, 0.05, 0.1, 2, fixed_r=r, estimator=1)
    exact = np.array([float(x) for x in BF.exact_bc(edges, 7, opt)])
    assert np.abs(est - exact).max() <= math.sqrt(math.log(2 * 7 / 1e-3) / (2 * r))


def test_ob_progressive_and_invalid():
    u, v, t = synth.uniform_small(n=60, m=900, seed=6)
    g = O.Graph(u, v, t, n=60)
    est, hits, info = g.estimate(0, 0.05, 0.1, 4, estimator=1)
    assert info["rounds"] >= 1 and info["r"] >= info["s1"] and (info["xi"] <= 0.05 or info["r"] >= info["omega"])
    assert 0.0 <= est.min() and est.max() <= 1.0
    for kw in (dict(target=1), dict(target=2), dict(fixed_r=1 << 30, c=2)):
        with pytest.raises(O.OracleError):
            g.estimate(0, 0.05, 0.1, 4, estimator=1, **kw)


# --------------------------------------------------------------------------
# The RTB estimator (App. C): f_v(s) = 1/(n-1) sum_z sigma_sz(v) / sigma_sz
# from one full search and a backward dependency accumulation; every term
# rounded to 2^-32 units.
# --------------------------------------------------------------------------
def test_muldiv_round():
    rng = np.random.default_rng(5)
    cases = [(0, 5, 1), (1, 1, 2), (1, 3, 2), (3, 1, 6), ((1 << 64) - 1, (1 << 64) - 1, (1 << 64) - 1),
             ((1 << 127), (1 << 64) - 1, (1 << 128) - 1), ((1 << 128) - 2, 12345, (1 << 128) - 1)]
    for _ in range(3000):
        bits = int(rng.integers(1, 129))
        d = (int(rng.integers(1, 1 << 62)) << max(bits - 62, 0)) | 1
        d = min(d, (1 << 128) - 1)
        a = d * int(rng.integers(0, 1 << 30)) // (1 << 30)
        x = int(rng.integers(0, 1 << 63)) >> int(rng.integers(0, 63))
        cases.append((a, x, d))
    for a, x, d in cases:
        assert O.muldiv_round(a, x, d) == (2 * a * x + d) // (2 * d), (a, x, d)


@pytest.mark.parametrize("seed", range(8))
def test_rtb_values_against_bruteforce(seed):
    """Every source of random tiny graphs, every optimality: the oracle's
    2^-32-unit value of f_v(s) is within 64 units (1.5e-8) of the exact
    rational from the brute-force optimal walk sets."""
    n = 6
    u, v, t = synth.random_tiny(n, 18, t_hi=5, seed=6000 + seed, self_loops=True)
    edges = BF.dedupe(u, v, t)
    g = O.Graph(u, v, t, n=n)
    seen = set()
    for i in range(200):
        s = O.uniform64(n, 77, i, 0)
        if s in seen:
            continue
        seen.add(s)
        sets = BF.optimal_sets(edges, n, s)
        for opt in (0, 1, 2, 3):
            want = [Fraction(0)] * n
            for z, d in sets.items():
                lst = d[opt]
                if not lst:
                    continue
                for vs, _ in lst:
                    for x in set(vs[1:-1]):
                        want[x] += Fraction(1, len(lst) * (n - 1))
            q = g.rtb_values(opt, 77, i)
            for x in range(n):
                assert abs(Fraction(int(q[x]), 1 << 32) - want[x]) <= Fraction(64, 1 << 32), (s, opt, x)
        if len(seen) == n:
            break
    assert len(seen) == n


@pytest.mark.parametrize("opt", [0, 1, 2])
def test_rtb_estimates_within_hoeffding(opt):
    """E[f_v(s)] over a uniform source is b_v: fixed-r RTB estimates against
    brute-force exact betweenness, and the hit sums recounted from the
    per-sample values."""
    u, v, t = synth.random_tiny(7, 22, t_hi=6, seed=4300)
    edges = BF.dedupe(u, v, t)
    g = O.Graph(u, v, t, n=7)
    r, seed = 8000, 4
    est, hits, info = g.estimate(opt, 0.05, 0.1, seed, fixed_r=r, estimator=2, c=5)
    exact = np.array([float(x) for x in BF.exact_bc(edges, 7, opt)])
    assert np.abs(est - exact).max() <= math.sqrt(math.log(2 * 7 / 1e-3) / (2 * r))
    tot = np.zeros(7, dtype=object)
    for i in range(r):
        tot += g.rtb_values(opt, seed, i).astype(object)
    assert [int(x) for x in hits] == list(tot) and info["sum_int_len"] == int(sum(tot))


def test_rtb_progressive_and_invalid():
    u, v, t = synth.uniform_small(n=50, m=700, seed=9)
    g = O.Graph(u, v, t, n=50)
    est, hits, info = g.estimate(2, 0.05, 0.1, 4, estimator=2)
    assert info["r"] >= info["s1"] and (info["xi"] <= 0.05 or info["r"] >= info["omega"])
    with pytest.raises(O.OracleError):
        g.estimate(0, 0.05, 0.1, 4, estimator=2, target=1)


# --------------------------------------------------------------------------
# Temporal closeness from Algorithm 2's searches (App. D remark; harmonic
# reading): sum_k round(2^32 / d(u_k, v)) over the sampled sources.
# --------------------------------------------------------------------------
@pytest.mark.parametrize("opt", [0, 1, 2, 3])
def test_closeness_against_bruteforce(opt):
    n = 7
    u, v, t = synth.random_tiny(n, 24, t_hi=6, seed=4400 + opt)
    edges = BF.dedupe(u, v, t)
    g = O.Graph(u, v, t, n=n)
    dist = BF.distances(edges, n, opt)
    r_s, seed = 3000, 12
    sm, cl = g.closeness(opt, seed, r_s)
    want = [0] * n
    for k in range(r_s):
        src = O.uniform64(n, seed, k, 5)
        for x in range(n):
            d = dist.get((src, x))
            if d:
                want[x] += ((1 << 33) + d) // (2 * d)
    assert [int(x) for x in sm] == want
    assert np.array_equal(cl, np.array([(float(w) * n) / (4294967296.0 * r_s * (n - 1)) for w in want]))
    exact = [sum(Fraction(1, dist[(a, x)]) for a in range(n) if (a, x) in dist) / (n - 1) for x in range(n)]
    bound = n / (n - 1) * math.sqrt(math.log(2 * n / 1e-3) / (2 * r_s))
    assert max(abs(cl[x] - float(exact[x])) for x in range(n)) <= bound
