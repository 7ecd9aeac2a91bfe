"""Temporal edge betweenness (paper App. A) on the GPU against the oracle, bit
for bit: edge ids, the temporal edges of every drawn path (every search
kernel, the 128-bit re-run included), hit counts and estimates over the
underlying and the temporal edges (solo, batched and served), and the
invariants that tie the three families to one another."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2304_08356_gb300 import synth
from test_gpu_parity import _graphs, _layered, _index_of_pair, _cmp_samples

pytestmark = pytest.mark.gpu


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


@pytest.mark.parametrize("case", range(7))
def test_edge_ids(M, case):
    _, (u, v, t), n = _graphs()[case]
    g = M.Graph(u, v, t, n=n)
    o = O.Graph(u, v, t, n=n)
    gu, gv, gt, gue, gnu = g.edge_ids()
    ou, ov, ot, oue, onu = o.edge_ids()
    assert gnu == onu
    for a, b in ((gu, ou), (gv, ov), (gt, ot), (gue, oue)):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("case", range(7))
@pytest.mark.parametrize("opt", [0, 1, 2])
def test_path_edges(M, pfm_kernel, case, opt):
    if opt != 2 and pfm_kernel == "cta":
        pytest.skip("the pfm kernel choice only affects pfm")
    _, (u, v, t), n = _graphs()[case]
    g = M.Graph(u, v, t, n=n)
    o = O.Graph(u, v, t, n=n)
    _cmp_samples(g.sample_paths(opt, 17, 0, 400, cap=g.n + 1, edges=True),
                 o.samples(opt, 17, 0, 400, cap=o.n + 1, edges=True))
    # every recorded edge joins consecutive path vertices, at strictly
    # increasing times (the paper's temporal paths are strict)
    eu, ev, et, _, _ = g.edge_ids()
    for (s, z, sig, path, pe) in g.sample_paths(opt, 17, 400, 100, cap=g.n + 1, edges=True):
        assert len(pe) == max(len(path) - 1, 0)
        for k, e in enumerate(pe):
            assert (eu[e], ev[e]) == (path[k], path[k + 1])
            if k:
                assert et[pe[k - 1]] < et[e]


@pytest.mark.parametrize("opt", [0, 1, 2])
def test_path_edges_wide(M, opt):
    u, v, t, n, s, z = _layered(16, 16)            # sigma_sz = 2^64: 128-bit re-run
    g = M.Graph(u, v, t, n=n)
    o = O.Graph(u, v, t, n=n)
    i = _index_of_pair(n, s, z, 5, M.D_PAIR)
    _cmp_samples(g.sample_paths(opt, 5, i - 20, 41, cap=n + 1, edges=True),
                 o.samples(opt, 5, i - 20, 41, cap=o.n + 1, edges=True))


def _check_estimate(g, o, opt, target, eps=0.05, seed=7, **kw):
    est, hits, info = g.estimate(opt, eps, 0.1, seed, target=target, **kw)
    oest, ohits, oinfo = o.estimate(opt, eps, 0.1, seed, target=target, **kw)
    for k in ("r", "rounds", "omega", "s1", "bootstrap", "sum_int_len", "max_hits", "rade_num"):
        assert info[k] == oinfo[k], k
    assert np.array_equal(hits, ohits)
    assert np.array_equal(est.view(np.uint64), oest.view(np.uint64))
    assert abs(info["xi"] - oinfo["xi"]) <= 1e-12 * abs(oinfo["xi"])
    return est, hits, info


@pytest.mark.parametrize("case", [0, 2, 3, 4, 5, 6])
@pytest.mark.parametrize("target", [1, 2])
@pytest.mark.parametrize("opt", [0, 1, 2])
def test_edge_estimate_bit_exact(M, case, target, opt):
    _, (u, v, t), n = _graphs()[case]
    g = M.Graph(u, v, t, n=n)
    o = O.Graph(u, v, t, n=n)
    est, hits, info = _check_estimate(g, o, opt, target)
    assert len(est) == g.family_size(target)


@pytest.mark.parametrize("target", [1, 2])
def test_edge_estimate_pfm_kernels(M, pfm_kernel, target):
    u, v, t = synth.chung_lu_bursty(n=1500, m=30000, seed=21)
    g = M.Graph(u, v, t)
    o = O.Graph(u, v, t)
    _check_estimate(g, o, 2, target, vhat_mode=1)


@pytest.mark.parametrize("opt", [0, 1, 2])
def test_family_invariants(M, opt):
    """One fixed-r run per family on the same samples: temporal-edge hits
    summed by underlying id give the underlying-edge hits; every path of l
    vertices adds l-1 edge hits and l-2 node hits (Sec. 3, App. A)."""
    u, v, t = synth.chung_lu_bursty(n=900, m=16000, seed=5)
    g = M.Graph(u, v, t)
    r = 5000
    _, hn, i0 = g.estimate(opt, 0.05, 0.1, 3, fixed_r=r, target=0)
    _, hu, i1 = g.estimate(opt, 0.05, 0.1, 3, fixed_r=r, target=1)
    _, ht, i2 = g.estimate(opt, 0.05, 0.1, 3, fixed_r=r, target=2)
    _, _, _, ue, nu = g.edge_ids()
    agg = np.zeros(nu, np.uint64)
    np.add.at(agg, ue, ht)
    assert np.array_equal(agg, hu)
    rows = g.sample_paths(opt, 3, 0, r, cap=g.n + 1, edges=True)
    reached = sum(1 for row in rows if len(row[3]) >= 2)
    assert i2["sum_int_len"] == int(ht.sum()) == i1["sum_int_len"]
    assert i2["sum_int_len"] == i0["sum_int_len"] + reached
    want = np.zeros(g.m, np.uint64)
    for row in rows:
        for e in row[4]:
            want[e] += 1
    assert np.array_equal(want, ht)


def test_mixed_targets_batch_and_server(M):
    inst = [synth.chung_lu_bursty(n=300 + 200 * k, m=6000 + 2000 * k, seed=40 + k) for k in range(6)]
    graphs = [M.Graph(*x) for x in inst]
    probs = [dict(graph=gr, opt=k % 3, eps=0.04, delta=0.1, seed=500 + k, target=(k // 2) % 3)
             for k, gr in enumerate(graphs)]
    res = M.estimate_batch(probs)
    srv = M.Server()
    rids = [srv.submit(p["graph"], p["opt"], p["eps"], p["delta"], p["seed"], target=p["target"]) for p in probs]
    served = [srv.wait(x, 120.0) for x in rids]
    srv.close()
    for k, p in enumerate(probs):
        e, h, i = p["graph"].estimate(p["opt"], p["eps"], p["delta"], p["seed"], target=p["target"])
        assert res[k][3] == 0
        for (e2, h2, i2) in ((res[k][0], res[k][1], res[k][2]), served[k]):
            assert np.array_equal(h2, h) and np.array_equal(e2.view(np.uint64), e.view(np.uint64)), k
            assert i2["r"] == i["r"] and i2["rade_num"] == i["rade_num"], k
    x = 4                                           # target 2, sfm
    o = O.Graph(*inst[x])
    _, oh, _ = o.estimate(probs[x]["opt"], 0.04, 0.1, probs[x]["seed"], target=probs[x]["target"])
    assert np.array_equal(res[x][1], oh)


def test_edgeless_family(M):
    """A graph whose only edges are self loops: no temporal edge survives, every
    sample is unreachable and the edge families are empty."""
    u, v, t = np.array([0, 1, 2]), np.array([0, 1, 2]), np.array([1, 2, 3])
    g = M.Graph(u, v, t, n=3)
    o = O.Graph(u, v, t, n=3)
    assert g.m == 0 and g.family_size(1) == 0 and g.family_size(2) == 0
    for target in (1, 2):
        est, hits, info = g.estimate(0, 0.1, 0.1, 1, target=target)
        oest, ohits, oinfo = o.estimate(0, 0.1, 0.1, 1, target=target)
        assert est.size == 0 and hits.size == 0 and oest.size == 0
        assert info["r"] == oinfo["r"] and info["sum_int_len"] == 0


def test_target_out_of_range(M):
    _, (u, v, t), n = _graphs()[0]
    g = M.Graph(u, v, t, n=n)
    with pytest.raises(M.MantraError) as ei:
        g.estimate(0, 0.1, 0.1, 1, target=3)
    assert ei.value.code == 1
