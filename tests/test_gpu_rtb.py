"""The RTB estimator (paper App. C) on the GPU against the oracle, bit for
bit: every sample is a source s, and every vertex v gets f_v(s) = 1/(n-1)
sum_z sigma_sz(v) / sigma_sz from an untruncated search and a backward
dependency accumulation, every term rounded to 2^-32 units on both sides.
Covered: every optimality on the parity graphs, both pfm kernels, the
128-bit re-run, the progressive run, the bench-size graph, batches and the
server mixing RTB with the other estimators."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2304_08356_gb300 import synth
from test_gpu_parity import _graphs, _layered

pytestmark = pytest.mark.gpu
XI_RTOL = 1e-12
KEYS = ("r", "rounds", "omega", "s1", "bootstrap", "sum_int_len", "max_hits", "rade_num")


@pytest.fixture(scope="module")
def M():
    from paper_2304_08356_gb300 import build as B
    B.build()
    from paper_2304_08356_gb300 import mantra
    return mantra


@pytest.fixture(params=["lane", "cta"])
def pfm_kernel(request, monkeypatch):
    monkeypatch.setenv("MANTRA_PFM_KERNEL", request.param)
    return request.param


def _same(g, o, opt, eps=0.05, delta=0.1, seed=7, **kw):
    est, hits, info = g.estimate(opt, eps, delta, seed, estimator=2, **kw)
    oest, ohits, oinfo = o.estimate(opt, eps, delta, seed, estimator=2, **kw)
    for k in KEYS:
        assert info[k] == oinfo[k], k
    assert np.array_equal(hits, ohits)
    assert np.array_equal(est.view(np.uint64), oest.view(np.uint64))
    assert abs(info["xi"] - oinfo["xi"]) <= XI_RTOL * abs(oinfo["xi"])
    assert int(hits.sum()) == info["sum_int_len"]
    return est, hits, info


@pytest.mark.parametrize("case", range(7))
@pytest.mark.parametrize("opt", [0, 1, 2])
def test_rtb_fixed_r(M, pfm_kernel, case, opt):
    if opt != 2 and pfm_kernel == "cta":
        pytest.skip("the pfm kernel choice only affects pfm")
    _, (u, v, t), n = _graphs()[case]
    g = M.Graph(u, v, t, n=n)
    o = O.Graph(u, v, t, n=n)
    _same(g, o, opt, fixed_r=300, c=9)


@pytest.mark.parametrize("opt", [0, 1, 2])
def test_rtb_progressive(M, opt):
    u, v, t = synth.chung_lu_bursty(n=600, m=9000, seed=23)
    g = M.Graph(u, v, t)
    o = O.Graph(u, v, t)
    est, hits, info = _same(g, o, opt, eps=0.04)
    assert info["rounds"] >= 1 and (info["xi"] <= 0.04 or info["r"] >= info["omega"])


@pytest.mark.parametrize("opt", [0, 1, 2])
def test_rtb_wide_counts(M, opt):
    """The 16 x 16 layered graph: a full search from its source counts 2^64
    paths to the sink, so those samples run on the 128-bit kernels."""
    u, v, t, n, s, z = _layered(16, 16)
    g = M.Graph(u, v, t, n=n)
    o = O.Graph(u, v, t, n=n)
    hits_src = [i for i in range(400) if O.uniform64(n, 16, i, 0) == s]
    assert hits_src, "no sample from the source"
    _same(g, o, opt, seed=16, fixed_r=hits_src[0] + 1)


@pytest.mark.parametrize("opt", [0, 1, 2])
def test_rtb_bench_graph(M, opt):
    """The bench workload's graph (bursty Chung-Lu, n = 20,000, m = 500,000):
    a fixed-r RTB run of 6 full searches against the oracle."""
    u, v, t = synth.chung_lu_bursty(n=20000, m=500000, seed=1)
    g = M.Graph(u, v, t)
    o = O.Graph(u, v, t)
    _same(g, o, opt, seed=3, fixed_r=6)


def test_rtb_batch_and_server(M):
    inst = [synth.chung_lu_bursty(n=300 + 200 * k, m=5000 + 2000 * k, seed=80 + k) for k in range(6)]
    graphs = [M.Graph(*x) for x in inst]
    probs = [dict(graph=gr, opt=k % 3, eps=0.05, delta=0.1, seed=900 + k, estimator=(2, 0, 1)[k // 2 % 3])
             for k, gr in enumerate(graphs)]
    res = M.estimate_batch(probs)
    srv = M.Server()
    rids = [srv.submit(p["graph"], p["opt"], p["eps"], p["delta"], p["seed"], estimator=p["estimator"])
            for p in probs]
    served = [srv.wait(x, 300.0) for x in rids]
    srv.close()
    for k, p in enumerate(probs):
        e, h, i = p["graph"].estimate(p["opt"], p["eps"], p["delta"], p["seed"], estimator=p["estimator"])
        assert res[k][3] == 0
        for (e2, h2, i2) in ((res[k][0], res[k][1], res[k][2]), served[k]):
            assert np.array_equal(h2, h) and np.array_equal(e2.view(np.uint64), e.view(np.uint64)), k
            assert i2["r"] == i["r"] and i2["rade_num"] == i["rade_num"] and i2["max_hits"] == i["max_hits"], k
    o = O.Graph(*inst[1])
    _, oh, _ = o.estimate(1, 0.05, 0.1, 901, estimator=2)
    assert np.array_equal(res[1][1], oh)


def test_rtb_invalid(M):
    _, (u, v, t), n = _graphs()[0]
    g = M.Graph(u, v, t, n=n)
    for kw in (dict(target=1), dict(target=2), dict(estimator=3), dict(fixed_r=1 << 30, c=2)):
        kw.setdefault("estimator", 2)
        with pytest.raises(M.MantraError) as ei:
            g.estimate(0, 0.1, 0.1, 1, **kw)
        assert ei.value.code == 1
