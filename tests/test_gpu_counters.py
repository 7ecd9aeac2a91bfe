"""The library's work counters (mantra_info: edges_scanned, sigma_adds,
states_new, frontier_vertices) against the oracle's, counted from the same
samples by their definitions, and the algorithmic bytes recomputed from them
with the byte model stated in include/mantra.h.  These counters are the
numerator of the reported roofline."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2304_08356_gb300 import synth
from test_gpu_parity import _graphs

pytestmark = pytest.mark.gpu
KEYS = ("edges_scanned", "sigma_adds", "states_new", "frontier_vertices")


@pytest.fixture(scope="module")
def M():
    from paper_2304_08356_gb300 import build as B
    B.build()
    from paper_2304_08356_gb300 import mantra
    return mantra


def alg_bytes(opt, info):
    """The byte model of include/mantra.h (64-bit path counts)."""
    e, u, s, f = (int(info[k]) for k in KEYS)
    if opt == 2:
        return 4 * e + (12 * e) // 32 + 24 * u
    return 24 * e + 8 * f + 12 * s


def _check(info, oinfo, opt):
    for k in KEYS:
        assert info[k] == oinfo[k], (k, info[k], oinfo[k])
    assert info["alg_bytes"] == alg_bytes(opt, oinfo)


@pytest.mark.parametrize("case", range(7))
@pytest.mark.parametrize("opt", [0, 1, 2, 3])
def test_fixed_r_counters_equal_oracle(M, case, opt):
    _, (u, v, t), n = _graphs()[case]
    g = M.Graph(u, v, t, n=n)
    o = O.Graph(u, v, t, n=n)
    _, hits, info = g.estimate(opt, 0.05, 0.1, 19, fixed_r=500)
    _, ohits, oinfo = o.estimate(opt, 0.05, 0.1, 19, fixed_r=500)
    assert np.array_equal(hits, ohits)
    _check(info, oinfo, opt)


@pytest.mark.parametrize("kernel", ["lane", "cta"])
def test_pfm_kernels_counters_equal_oracle(M, kernel, monkeypatch):
    monkeypatch.setenv("MANTRA_PFM_KERNEL", kernel)
    u, v, t = synth.chung_lu_bursty(n=1500, m=30000, seed=21)
    g = M.Graph(u, v, t)
    o = O.Graph(u, v, t)
    _, _, info = g.estimate(2, 0.05, 0.1, 7, fixed_r=700)
    _, _, oinfo = o.estimate(2, 0.05, 0.1, 7, fixed_r=700)
    _check(info, oinfo, 2)
    # the CTA kernel's walked edges include every DAG edge it counts paths over
    if kernel == "cta":
        assert info["edges_expanded"] >= info["sigma_adds"] > 0
    else:
        assert info["edges_expanded"] == 0


@pytest.mark.parametrize("opt", [0, 1, 2, 3])
def test_progressive_counters_include_the_bootstrap(M, opt):
    u, v, t = synth.chung_lu_bursty(n=1500, m=30000, seed=21)
    g = M.Graph(u, v, t)
    o = O.Graph(u, v, t)
    _, _, info = g.estimate(opt, 0.1, 0.1, 7)
    _, _, oinfo = o.estimate(opt, 0.1, 0.1, 7)
    assert (info["r"], info["bootstrap"]) == (oinfo["r"], oinfo["bootstrap"])
    _check(info, oinfo, opt)


@pytest.mark.parametrize("opt", [0, 1, 2])
def test_ob_counters_equal_oracle(M, opt):
    u, v, t = synth.uniform_small(n=60, m=900, t_lo=1, t_hi=8, seed=4)
    g = M.Graph(u, v, t, n=60)
    o = O.Graph(u, v, t, n=60)
    _, _, info = g.estimate(opt, 0.05, 0.1, 3, fixed_r=400, estimator=1)
    _, _, oinfo = o.estimate(opt, 0.05, 0.1, 3, fixed_r=400, estimator=1)
    _check(info, oinfo, opt)


@pytest.mark.parametrize("opt", [0, 1, 2])
def test_bench_graph_counters_equal_oracle(M, opt):
    """The bench workload's graph (bursty Chung-Lu n = 20,000, m = 500,000):
    a few hundred samples, counted on both sides."""
    u, v, t = synth.chung_lu_bursty()
    g = M.Graph(u, v, t)
    o = O.Graph(u, v, t)
    r = 30 if opt != 2 else 600
    _, _, info = g.estimate(opt, 0.01, 0.1, 5, fixed_r=r)
    _, _, oinfo = o.estimate(opt, 0.01, 0.1, 5, fixed_r=r)
    _check(info, oinfo, opt)
