"""Foremost-first shortest-foremost (fsfm: the earliest arrival at z, then
the fewest hops -- Buss et al.'s reading of Def. 1(2)) and temporal
closeness from Algorithm 2's searches, on the GPU against the oracle, bit for
bit: per-sample paths and counts (the 128-bit re-run included), the trk, ob
and RTB estimates and the edge families under fsfm, Algorithm 2's reach
counts, and the closeness sums of every optimality."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2304_08356_gb300 import synth
from test_gpu_parity import _graphs, _layered, _index_of_pair, _cmp_samples

pytestmark = pytest.mark.gpu
FSFM = 3
KEYS = ("r", "rounds", "omega", "s1", "bootstrap", "sum_int_len", "max_hits", "rade_num")


@pytest.fixture(scope="module")
def M():
    from paper_2304_08356_gb300 import build as B
    B.build()
    from paper_2304_08356_gb300 import mantra
    return mantra


@pytest.mark.parametrize("case", range(7))
def test_fsfm_sample_paths(M, case):
    _, (u, v, t), n = _graphs()[case]
    g = M.Graph(u, v, t, n=n)
    o = O.Graph(u, v, t, n=n)
    for dp, dq, i0, count in ((M.D_PAIR, M.D_PATH, 0, 500), (M.D_BOOT_PAIR, M.D_BOOT_PATH, 31, 60)):
        _cmp_samples(g.sample_paths(FSFM, 13, i0, count, dp, dq, cap=g.n + 1, edges=True),
                     o.samples(FSFM, 13, i0, count, dp, dq, cap=o.n + 1, edges=True))


def test_fsfm_wide_counts(M):
    u, v, t, n, s, z = _layered(16, 16)
    g = M.Graph(u, v, t, n=n)
    o = O.Graph(u, v, t, n=n)
    i = _index_of_pair(n, s, z, 5, M.D_PAIR)
    got = g.sample_paths(FSFM, 5, i, 1, cap=n + 1)
    assert got == o.samples(FSFM, 5, i, 1, cap=n + 1) and got[0][2] == 16 ** 16
    _cmp_samples(g.sample_paths(FSFM, 5, i - 30, 61, cap=n + 1), o.samples(FSFM, 5, i - 30, 61, cap=n + 1))


@pytest.mark.parametrize("case", [0, 2, 3, 4, 5, 6])
@pytest.mark.parametrize("kw", [dict(), dict(estimator=1), dict(estimator=2), dict(target=1), dict(target=2)])
def test_fsfm_estimates(M, case, kw):
    _, (u, v, t), n = _graphs()[case]
    g = M.Graph(u, v, t, n=n)
    o = O.Graph(u, v, t, n=n)
    r = 200 if kw.get("estimator") == 2 else 600
    est, hits, info = g.estimate(FSFM, 0.05, 0.1, 7, fixed_r=r, c=9, **kw)
    oest, ohits, oinfo = o.estimate(FSFM, 0.05, 0.1, 7, fixed_r=r, c=9, **kw)
    for k in KEYS:
        assert info[k] == oinfo[k], k
    assert np.array_equal(hits, ohits)
    assert np.array_equal(est.view(np.uint64), oest.view(np.uint64))


def test_fsfm_progressive_and_bench_graph(M):
    u, v, t = synth.chung_lu_bursty(n=1500, m=30000, seed=21)
    g = M.Graph(u, v, t)
    o = O.Graph(u, v, t)
    est, hits, info = g.estimate(FSFM, 0.04, 0.1, 5)
    oest, ohits, oinfo = o.estimate(FSFM, 0.04, 0.1, 5)
    assert np.array_equal(hits, ohits) and info["r"] == oinfo["r"] and info["rounds"] == oinfo["rounds"]
    u, v, t = synth.chung_lu_bursty(n=20000, m=500000, seed=1)
    g = M.Graph(u, v, t)
    o = O.Graph(u, v, t)
    _cmp_samples(g.sample_paths(FSFM, 3, 100, 24, cap=g.n + 1), o.samples(FSFM, 3, 100, 24, cap=o.n + 1))


@pytest.mark.parametrize("case", [0, 1, 2, 4, 5])
def test_fsfm_temporal_stats(M, case):
    _, (u, v, t), n = _graphs()[case]
    g = M.Graph(u, v, t, n=n)
    o = O.Graph(u, v, t, n=n)
    st, reach = g.temporal_stats(FSFM, 0.05, 9, r_override=300, tau=0.9)
    oreach, odlb = o.stats_counts(FSFM, 9, 300)
    assert st["d_lb"] == odlb
    assert np.array_equal(reach, oreach)


@pytest.mark.parametrize("case", [0, 2, 4, 5])
@pytest.mark.parametrize("opt", [0, 1, 2, 3])
def test_closeness(M, case, opt):
    _, (u, v, t), n = _graphs()[case]
    g = M.Graph(u, v, t, n=n)
    o = O.Graph(u, v, t, n=n)
    sm, cl, rs = g.temporal_closeness(opt, 0.05, 11, r_override=400)
    osm, ocl = o.closeness(opt, 11, 400)
    assert rs == 400
    assert np.array_equal(sm, osm)
    assert np.array_equal(cl.view(np.uint64), ocl.view(np.uint64))


def test_fsfm_batch_mixed(M):
    inst = [synth.chung_lu_bursty(n=300 + 150 * k, m=5000 + 2000 * k, seed=90 + k) for k in range(4)]
    graphs = [M.Graph(*x) for x in inst]
    probs = [dict(graph=gr, opt=(3, 0, 3, 2)[k], eps=0.05, delta=0.1, seed=40 + k, estimator=(0, 0, 1, 2)[k])
             for k, gr in enumerate(graphs)]
    res = M.estimate_batch(probs)
    for k, p in enumerate(probs):
        e, h, i = p["graph"].estimate(p["opt"], p["eps"], p["delta"], p["seed"], estimator=p["estimator"])
        assert res[k][3] == 0 and np.array_equal(res[k][1], h) and res[k][2]["r"] == i["r"], k
    o = O.Graph(*inst[0])
    _, oh, _ = o.estimate(3, 0.05, 0.1, 40)
    assert np.array_equal(res[0][1], oh)
