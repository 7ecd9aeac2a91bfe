"""The large and the many-graph workloads on the GPU.

* Chung-Lu n = 1,000,000, gamma 2.1, 20,000,000 temporal edges with t uniform
  in [0, 2^24): sampled samples of every optimality against the oracle one by
  one, Algorithm 2 reach counts against the oracle on a few sources, and the
  r_s = 256 stats run's invariants.
* Uneven bursty Chung-Lu graphs (n log-uniform in [500, 50,000], m = 20 n,
  optimality g mod 3, eps = 0.02) in one mantra_estimate_batch: every problem
  equals its solo mantra_estimate bit for bit, and the smallest ones equal the
  oracle."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2304_08356_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    from paper_2304_08356_gb300 import build as B
    B.build()
    from paper_2304_08356_gb300 import mantra
    return mantra


@pytest.fixture(scope="module")
def large():
    return synth.chung_lu_uniform_t(n=1_000_000, m=20_000_000, gamma=2.1, seed=1)


def test_large_graph_sampled_parity(M, large):
    u, v, t = large
    g = M.Graph(u, v, t, n=1_000_000)
    o = O.Graph(u, v, t, n=1_000_000)
    assert (g.n, g.m, g.slots) == (o.n, o.m, o.slots)
    for opt, i0, count in ((2, 11, 24), (0, 3, 1), (1, 7, 1)):
        got = g.sample_paths(opt, 5, i0, count, cap=1024)
        want = o.samples(opt, 5, i0, count, cap=1024)
        assert got == want, opt
    # Algorithm 2: pfm against the oracle on a few sources (an untruncated sh/sfm
    # oracle search at this size takes minutes), then the paper's r_s = 256 runs
    st, reach = g.temporal_stats(2, 0.01, 2, r_override=3)
    oreach, odlb = o.stats_counts(2, 2, 3)
    assert st["d_lb"] == odlb and np.array_equal(reach, oreach)
    for opt in (2, 1):
        st, reach = g.temporal_stats(opt, 0.01, 4, r_override=256)
        assert st["r"] == 256 and st["d_lb"] >= 1
        assert 0.0 < st["zeta"] <= 1.0 and st["psi"] >= 1.0
        assert int(reach[st["d_lb"]]) == int(reach.max())


def test_large_graph_fixed_r_estimate(M, large):
    """A fixed-r pfm estimate at full size: hits re-derived from the per-sample
    paths the same kernels return."""
    u, v, t = large
    g = M.Graph(u, v, t, n=1_000_000)
    r = 3000
    est, hits, info = g.estimate(2, 0.01, 0.1, 9, fixed_r=r)
    rows = g.sample_paths(2, 9, 0, r, cap=256)
    want = np.zeros(g.n, np.uint64)
    for (_, _, _, nodes) in rows:
        for x in nodes[1:-1]:
            want[x] += 1
    assert np.array_equal(hits, want)
    assert info["r"] == r and hits.sum() == info["sum_int_len"]


def test_uneven_batch(M):
    inst = synth.batch_instances(count=256)
    pick = list(range(0, 256, 4))                       # 64 of the 256 instances
    graphs = [M.Graph(*inst[x]) for x in pick]
    probs = [dict(graph=gr, opt=x % 3, eps=0.02, delta=0.1, seed=1000 + x) for gr, x in zip(graphs, pick)]
    res = M.estimate_batch(probs)
    assert all(st == 0 for (_, _, _, st) in res)
    assert all(info["bootstrap"] == 116 for (_, _, info, _) in res)
    # solo runs of a spread of problems, including the largest
    order = sorted(range(len(pick)), key=lambda y: graphs[y].n)
    for y in order[:3] + order[len(order) // 2: len(order) // 2 + 2] + order[-2:]:
        p = probs[y]
        e2, h2, i2 = p["graph"].estimate(p["opt"], p["eps"], p["delta"], p["seed"])
        est, hits, info, _ = res[y]
        assert np.array_equal(hits, h2) and np.array_equal(est.view(np.uint64), e2.view(np.uint64)), y
        for k in ("r", "rounds", "omega", "s1", "rade_num", "max_hits", "sum_int_len"):
            assert info[k] == i2[k], (y, k)
    # the oracle on the two smallest instances
    for y in order[:2]:
        p = probs[y]
        x = pick[y]
        o = O.Graph(*inst[x])
        _, oh, oi = o.estimate(p["opt"], p["eps"], p["delta"], p["seed"])
        assert np.array_equal(res[y][1], oh) and res[y][2]["r"] == oi["r"]
