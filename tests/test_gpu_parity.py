"""GPU path (through the C ABI) against the CPU oracle: bit-exact per-sample
results, hit counts, estimates, c-MCERA sums and Algorithm 2 reach counts;
the floating-point stopping bound xi within 1e-12 relative."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2304_08356_gb300 import synth

pytestmark = pytest.mark.gpu
XI_RTOL = 1e-12


@pytest.fixture(scope="module")
def M():
    from paper_2304_08356_gb300 import build as B
    B.build()
    from paper_2304_08356_gb300 import mantra
    return mantra


def _graphs():
    """(name, (u, v, t), n) -- small and medium cases spanning several CTA
    tiles, ragged frontiers, ties, duplicates, self loops and degenerate shapes."""
    out = [("uniform_n100_m2000", synth.uniform_small(), 100),
           ("uniform_ties", synth.uniform_small(n=60, m=900, t_lo=1, t_hi=8, seed=4), 60),
           ("bursty_n700", synth.chung_lu_bursty(n=700, m=12000, seed=9), 0),
           ("tiny_loops_dups", synth.random_tiny(7, 40, t_hi=4, seed=5, self_loops=True), 7)]
    # chain 0 -> 1 -> ... -> 39 with increasing times plus shortcuts (deep levels)
    cu = list(range(39)) + [0, 5, 10, 20]
    cv = list(range(1, 40)) + [7, 12, 30, 35]
    ct = list(range(1, 40)) + [3, 9, 15, 36]
    out.append(("chain_shortcuts", (np.array(cu), np.array(cv), np.array(ct)), 40))
    # hub: vertex 0 linked to/from everyone at many times (long segments)
    rng = np.random.default_rng(2)
    hu = np.concatenate([np.zeros(600, int), rng.integers(1, 80, 600)])
    hv = np.concatenate([rng.integers(1, 80, 600), np.zeros(600, int)])
    ht = rng.integers(1, 300, 1200)
    out.append(("hub", (hu, hv, ht), 80))
    out.append(("two_nodes", (np.array([0, 1, 0]), np.array([1, 0, 1]), np.array([5, 6, 9])), 2))
    return out


def _cmp_samples(gpu, orc):
    assert len(gpu) == len(orc)
    for q, (a, b) in enumerate(zip(gpu, orc)):
        assert a == b, (q, a, b)


@pytest.mark.parametrize("case", range(7))
@pytest.mark.parametrize("opt", [0, 1, 2])
def test_sample_paths_bit_exact(M, case, opt):
    name, (u, v, t), n = _graphs()[case]
    g = M.Graph(u, v, t, n=n)
    o = O.Graph(u, v, t, n=n)
    assert (g.n, g.m, g.slots, g.self_loops, g.duplicates) == (o.n, o.m, o.slots, o.self_loops, o.duplicates)
    count = 600
    for dp, dq, i0 in ((M.D_PAIR, M.D_PATH, 0), (M.D_BOOT_PAIR, M.D_BOOT_PATH, 123)):
        _cmp_samples(g.sample_paths(opt, 31, i0, count, dp, dq, cap=g.n + 1),
                     o.samples(opt, 31, i0, count, dp, dq, cap=o.n + 1))


@pytest.mark.parametrize("opt", [0, 1, 2])
def test_fixed_r_small_config_bit_exact(M, opt):
    # n=100, |E|=2000 uniform, r = 1000 samples, seed 1, c = 25, no stopping
    u, v, t = synth.uniform_small()
    g = M.Graph(u, v, t, n=100)
    o = O.Graph(u, v, t, n=100)
    est, hits, info = g.estimate(opt, 0.05, 0.1, 1, fixed_r=1000)
    oest, ohits, oinfo = o.estimate(opt, 0.05, 0.1, 1, fixed_r=1000)
    assert np.array_equal(hits, ohits)
    assert np.array_equal(est.view(np.uint64), oest.view(np.uint64))
    for k in ("r", "rounds", "sum_int_len", "max_hits", "rade_num"):
        assert info[k] == oinfo[k], k
    assert info["xi"] == pytest.approx(oinfo["xi"], rel=XI_RTOL)
    assert hits.sum() == info["sum_int_len"]


@pytest.mark.parametrize("opt", [0, 1, 2])
@pytest.mark.parametrize("eps", [0.1, 0.05])
def test_progressive_bit_exact(M, opt, eps):
    u, v, t = synth.chung_lu_bursty(n=1500, m=30000, seed=21)
    g = M.Graph(u, v, t)
    o = O.Graph(u, v, t)
    est, hits, info = g.estimate(opt, eps, 0.1, 7)
    oest, ohits, oinfo = o.estimate(opt, eps, 0.1, 7)
    for k in ("r", "rounds", "omega", "s1", "bootstrap", "sum_int_len", "max_hits", "rade_num"):
        assert info[k] == oinfo[k], k
    assert np.array_equal(hits, ohits)
    assert np.array_equal(est.view(np.uint64), oest.view(np.uint64))
    for k in ("xi", "vhat", "rho_hat"):
        assert info[k] == pytest.approx(oinfo[k], rel=XI_RTOL), k


def test_progressive_options(M):
    u, v, t = synth.chung_lu_bursty(n=800, m=15000, seed=4)
    g = M.Graph(u, v, t)
    o = O.Graph(u, v, t)
    for kw in (dict(c=7, growth=1.5, bootstrap=60, delta_sched=1), dict(c=128), dict(c=1)):
        _, hits, info = g.estimate(2, 0.08, 0.2, 3, **kw)
        _, ohits, oinfo = o.estimate(2, 0.08, 0.2, 3, **kw)
        assert np.array_equal(hits, ohits)
        for k in ("r", "rounds", "omega", "s1", "rade_num"):
            assert info[k] == oinfo[k], (kw, k)


@pytest.mark.parametrize("opt", [0, 1, 2])
def test_bursty_20k_full_size(M, opt):
    """Chung-Lu n=20,000, gamma 2.3, 500,000 bursty contacts, eps=0.01,
    delta=0.1, c=25: the launch configuration the benchmark times.  The
    oracle checks sampled samples one by one; the whole run is checked by
    its invariants and by re-deriving the hit counts from per-sample paths."""
    u, v, t = synth.chung_lu_bursty()
    g = M.Graph(u, v, t)
    est, hits, info = g.estimate(opt, 0.01, 0.1, 1)
    r = info["r"]
    assert info["bootstrap"] == 231
    assert r <= info["omega"] and (info["xi"] <= 0.01 or r == info["omega"])
    assert int(hits.sum()) == info["sum_int_len"]
    assert np.array_equal(est.view(np.uint64), (hits.astype(np.float64) / r).view(np.uint64))
    # hits re-derived from the per-sample paths of all r samples (same kernels)
    cap = 64
    sp = g.sample_paths(opt, 1, 0, r, cap=cap)
    H = np.zeros(g.n, np.uint64)
    for (_, _, _, p) in sp:
        assert len(p) <= cap
        for x in p[1:-1]:
            H[x] += 1
    assert np.array_equal(H, hits)
    # oracle on sampled indices
    o = O.Graph(u, v, t)
    rng = np.random.default_rng(opt)
    idx = sorted(rng.choice(r, size=24, replace=False).tolist()) + [0, r - 1]
    for i in idx:
        _cmp_samples(g.sample_paths(opt, 1, i, 1, cap=g.n + 1), o.samples(opt, 1, i, 1, cap=o.n + 1))


def _layered(width, layers):
    """s -> L1 -> ... -> L_layers -> z, complete between consecutive layers,
    edge time = layer index of the head: sigma_sz = width ** layers."""
    ids = [[0]]
    nxt = 1
    for _ in range(layers):
        ids.append(list(range(nxt, nxt + width)))
        nxt += width
    ids.append([nxt])
    n = nxt + 1
    u, v, t = [], [], []
    for L in range(len(ids) - 1):
        for a in ids[L]:
            for b in ids[L + 1]:
                u.append(a); v.append(b); t.append(L + 1)
    return np.array(u), np.array(v), np.array(t), n, 0, nxt


def _index_of_pair(n, s, z, seed, dom):
    for i in range(5_000_000):
        if O.draw_pair(n, seed, i, dom) == (s, z):
            return i
    raise AssertionError("pair not found")


@pytest.mark.parametrize("opt", [0, 1, 2])
def test_wide_path_counts(M, opt):
    # sigma_sz = 16^16 = 2^64 does not fit 64 bits: the 128-bit re-run
    u, v, t, n, s, z = _layered(16, 16)
    g = M.Graph(u, v, t, n=n)
    o = O.Graph(u, v, t, n=n)
    i = _index_of_pair(n, s, z, 5, M.D_PAIR)
    got = g.sample_paths(opt, 5, i, 1, cap=n + 1)
    want = o.samples(opt, 5, i, 1, cap=n + 1)
    assert got == want and got[0][2] == 16 ** 16
    # a window of samples around it (mixed 64-bit and 128-bit samples)
    _cmp_samples(g.sample_paths(opt, 5, i - 40, 81, cap=n + 1), o.samples(opt, 5, i - 40, 81, cap=n + 1))


def test_path_count_beyond_128_bits(M):
    u, v, t, n, s, z = _layered(16, 32)       # 2^128
    g = M.Graph(u, v, t, n=n)
    i = _index_of_pair(n, s, z, 5, M.D_PAIR)
    with pytest.raises(M.MantraError) as ei:
        g.sample_paths(0, 5, i, 1)
    assert ei.value.code == 3
    o = O.Graph(u, v, t, n=n)
    with pytest.raises(O.OracleError):
        o.samples(0, 5, i, 1)


@pytest.mark.parametrize("case", [0, 1, 2, 4, 5])
@pytest.mark.parametrize("opt", [0, 1, 2])
def test_temporal_stats_bit_exact(M, case, opt):
    name, (u, v, t), n = _graphs()[case]
    g = M.Graph(u, v, t, n=n)
    o = O.Graph(u, v, t, n=n)
    st, reach = g.temporal_stats(opt, 0.05, 9, r_override=300, tau=0.9)
    oreach, odlb = o.stats_counts(opt, 9, 300)
    assert st["d_lb"] == odlb
    assert np.array_equal(reach, oreach)
    ref = O.stats_summary(oreach, odlb, g.n, 300, tau=0.9)
    for k in ("zeta", "psi", "rho"):
        assert st[k] == pytest.approx(ref[k], rel=XI_RTOL, abs=1e-300)
    assert st["d_tau"] == ref["d_tau"]


def test_temporal_stats_bursty_20k(M):
    u, v, t = synth.chung_lu_bursty()
    g = M.Graph(u, v, t)
    o = O.Graph(u, v, t)
    for opt in (0, 2):
        st, reach = g.temporal_stats(opt, 0.01, 3, r_override=6)
        oreach, odlb = o.stats_counts(opt, 3, 6)
        assert st["d_lb"] == odlb and np.array_equal(reach, oreach)
    # default r_s = ceil(ln n / eps^2) at eps = 0.1: 991 sources
    st, _ = g.temporal_stats(0, 0.1, 3)
    assert st["r"] == math.ceil(math.log(20000) / 0.01)


def test_invalid_arguments(M):
    u, v, t = synth.uniform_small(n=20, m=100, seed=2)
    g = M.Graph(u, v, t, n=20)
    for bad in (dict(eps=0.0), dict(eps=1.0), dict(delta=0.0), dict(delta=1.5)):
        kw = dict(eps=0.1, delta=0.1)
        kw.update(bad)
        with pytest.raises(M.MantraError) as ei:
            g.estimate(0, kw["eps"], kw["delta"], 1)
        assert ei.value.code == 1
    with pytest.raises(M.MantraError):
        g.estimate(0, 0.1, 0.1, 1, c=129)
    with pytest.raises(M.MantraError):
        M.Graph(np.array([0, 5]), np.array([1, 2]), np.array([1, 2]), n=4)      # id >= n
    with pytest.raises(M.MantraError):
        M.Graph(np.array([0]), np.array([0]), np.array([1]), n=1)              # n < 2
    with pytest.raises(M.MantraError):
        M.Graph(np.array([0]), np.array([1]), np.array([0xFFFFFFFE]), n=2)     # time too large


def test_degenerate_graphs(M):
    # no edges at all: every sample unreachable, estimates zero
    g = M.Graph(np.zeros(0, int), np.zeros(0, int), np.zeros(0, int), n=10)
    est, hits, info = g.estimate(0, 0.1, 0.1, 1)
    assert not hits.any() and not est.any() and info["sum_int_len"] == 0
    st, reach = g.temporal_stats(2, 0.1, 1, r_override=20)
    assert st["d_lb"] == 0 and st["zeta"] == 0.0
    # only self loops
    g = M.Graph(np.array([1, 2]), np.array([1, 2]), np.array([3, 4]), n=5)
    assert g.m == 0 and g.self_loops == 2
    # isolated nodes count in n(n-1)
    u, v, t = synth.uniform_small(n=30, m=300, seed=8)
    o = O.Graph(u, v, t, n=50)
    g = M.Graph(u, v, t, n=50)
    for opt in (0, 1, 2):
        _, hits, _ = g.estimate(opt, 0.1, 0.1, 2, fixed_r=500)
        _, ohits, _ = o.estimate(opt, 0.1, 0.1, 2, fixed_r=500)
        assert np.array_equal(hits, ohits)


def test_repeatable(M):
    u, v, t = synth.chung_lu_bursty(n=900, m=20000, seed=6)
    g = M.Graph(u, v, t)
    a = g.estimate(0, 0.05, 0.1, 11)
    b = g.estimate(0, 0.05, 0.1, 11)
    assert np.array_equal(a[1], b[1]) and a[2]["r"] == b[2]["r"]



def test_batch_equals_solo_and_oracle(M):
    """mantra_estimate_batch: uneven graphs, mixed optimalities and eps in one
    batch; every problem's result equals its solo mantra_estimate (bit for
    bit) and, for the small ones, the oracle."""
    specs = [(synth.chung_lu_bursty(n=600, m=9000, seed=41), 0, 0.08, 3),
             (synth.chung_lu_bursty(n=1500, m=30000, seed=42), 2, 0.05, 4),
             (synth.uniform_small(), 1, 0.06, 5),
             (synth.chung_lu_bursty(n=900, m=18000, seed=43), 2, 0.1, 6),
             (synth.chung_lu_bursty(n=3000, m=60000, seed=44), 1, 0.05, 7),
             (synth.uniform_small(n=50, m=600, seed=9), 0, 0.1, 8)]
    graphs = [M.Graph(*uvt) for uvt, _, _, _ in specs]
    probs = [dict(graph=g, opt=o, eps=e, delta=0.1, seed=sd) for g, (_, o, e, sd) in zip(graphs, specs)]
    probs.append(dict(graph=graphs[0], opt=2, eps=0.1, delta=0.1, seed=1, fixed_r=700))
    res = M.estimate_batch(probs)
    for p, (est, hits, info, st) in zip(probs, res):
        assert st == 0
        e2, h2, i2 = p["graph"].estimate(p["opt"], p["eps"], p["delta"], p["seed"], fixed_r=p.get("fixed_r", 0))
        assert np.array_equal(hits, h2) and np.array_equal(est.view(np.uint64), e2.view(np.uint64))
        for k in ("r", "rounds", "omega", "s1", "rade_num", "max_hits", "sum_int_len"):
            assert info[k] == i2[k], k
    for x in (0, 2, 5, 6):
        (u, v, t) = specs[min(x, 5)][0] if x < 6 else specs[0][0]
        p = probs[x]
        o = O.Graph(u, v, t, n=p["graph"].n)
        _, oh, oi = o.estimate(p["opt"], p["eps"], p["delta"], p["seed"], fixed_r=p.get("fixed_r", 0))
        assert np.array_equal(res[x][1], oh) and res[x][2]["r"] == oi["r"]


def test_pfm_list_overflow_fallback_bit_exact():
    """pfm samples whose contribution list would overflow are re-run by the
    in-order kernel; a child process with a tiny list capacity must give the
    oracle's per-sample results, estimates and Algorithm 2 counts."""
    import json
    import os
    import subprocess
    import sys
    code = r'''
import json, sys
sys.path.insert(0, ".")
import numpy as np
from paper_2304_08356_gb300 import build as B, synth
B.build()
from paper_2304_08356_gb300 import mantra as M
from oracle import oracle as O
u, v, t = synth.chung_lu_bursty(n=900, m=20000, seed=33)
g = M.Graph(u, v, t); o = O.Graph(u, v, t)
ok = g.sample_paths(2, 4, 0, 300, cap=g.n + 1) == o.samples(2, 4, 0, 300, cap=o.n + 1)
_, h, info = g.estimate(2, 0.1, 0.1, 4, fixed_r=400)
_, oh, _ = o.estimate(2, 0.1, 0.1, 4, fixed_r=400)
st, reach = g.temporal_stats(2, 0.1, 5, r_override=100)
oreach, _ = o.stats_counts(2, 5, 100)
print(json.dumps({"ok": bool(ok and np.array_equal(h, oh) and np.array_equal(reach, oreach)),
                  "wide": info["wide_samples"]}))
'''
    env = dict(os.environ, MANTRA_PFM_LIST_CAP="40", MANTRA_PFM_KERNEL="lane")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", code], cwd=root, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    res = json.loads(r.stdout.strip().splitlines()[-1])
    assert res["ok"] and res["wide"] > 0


@pytest.mark.parametrize("opt", [0, 2])
def test_vhat_mode_bit_exact(M, opt):
    """vhat_mode 1 (variance term of xi from the appendix's bound on W, the
    round's delta split evenly): same stopping round, hits and estimates as
    the oracle; xi and the variance term within 1e-12."""
    u, v, t = synth.chung_lu_bursty(n=1500, m=30000, seed=21)
    g = M.Graph(u, v, t)
    o = O.Graph(u, v, t)
    est, hits, info = g.estimate(opt, 0.05, 0.1, 7, vhat_mode=1)
    oest, ohits, oinfo = o.estimate(opt, 0.05, 0.1, 7, vhat_mode=1)
    for k in ("r", "rounds", "omega", "s1", "sum_int_len", "max_hits", "rade_num"):
        assert info[k] == oinfo[k], k
    assert np.array_equal(hits, ohits)
    for k in ("xi", "vhat"):
        assert info[k] == pytest.approx(oinfo[k], rel=XI_RTOL), k
    # the bound is never below W, so the run is at least as long as with vhat = W
    _, _, i0 = g.estimate(opt, 0.05, 0.1, 7)
    assert info["vhat"] >= info["max_hits"] / info["r"] and info["r"] >= i0["r"]
