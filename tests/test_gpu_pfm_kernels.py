"""Both prefix-foremost kernels (one lane per sample walking the time-sorted
stream; one CTA per sample with label-correcting arrivals and a Kahn pass
over the prefix-foremost DAG) against the oracle, bit for bit: per-sample
paths and path counts, hit counts and estimates, Algorithm 2 reach counts,
the 128-bit re-run of overflowed samples.  MANTRA_PFM_KERNEL selects the
kernel of every tick."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2304_08356_gb300 import synth
from test_gpu_parity import _graphs, _layered, _index_of_pair, _cmp_samples

pytestmark = pytest.mark.gpu

KERNELS = ["lane", "cta"]


@pytest.fixture(scope="module")
def M():
    from paper_2304_08356_gb300 import build as B
    B.build()
    from paper_2304_08356_gb300 import mantra
    return mantra


@pytest.fixture(params=KERNELS)
def kernel(request, monkeypatch):
    monkeypatch.setenv("MANTRA_PFM_KERNEL", request.param)
    return request.param


@pytest.mark.parametrize("case", range(7))
def test_pfm_sample_paths(M, kernel, case):
    _, (u, v, t), n = _graphs()[case]
    g = M.Graph(u, v, t, n=n)
    o = O.Graph(u, v, t, n=n)
    for dp, dq, i0, count in ((M.D_PAIR, M.D_PATH, 0, 700), (M.D_BOOT_PAIR, M.D_BOOT_PATH, 77, 33)):
        _cmp_samples(g.sample_paths(2, 13, i0, count, dp, dq, cap=g.n + 1),
                     o.samples(2, 13, i0, count, dp, dq, cap=o.n + 1))


def test_pfm_bursty_medium(M, kernel):
    u, v, t = synth.chung_lu_bursty(n=4000, m=90000, seed=17)
    g = M.Graph(u, v, t)
    o = O.Graph(u, v, t)
    _cmp_samples(g.sample_paths(2, 3, 1000, 150, cap=g.n + 1), o.samples(2, 3, 1000, 150, cap=o.n + 1))


def test_pfm_estimate(M, kernel):
    u, v, t = synth.chung_lu_bursty(n=1500, m=30000, seed=21)
    g = M.Graph(u, v, t)
    o = O.Graph(u, v, t)
    est, hits, info = g.estimate(2, 0.05, 0.1, 7)
    oest, ohits, oinfo = o.estimate(2, 0.05, 0.1, 7)
    for k in ("r", "rounds", "omega", "s1", "sum_int_len", "max_hits", "rade_num"):
        assert info[k] == oinfo[k], k
    assert np.array_equal(hits, ohits)
    assert np.array_equal(est.view(np.uint64), oest.view(np.uint64))


def test_pfm_wide_counts(M, kernel):
    # sigma_sz = 2^64: 64-bit overflow, re-run with 128-bit counts
    u, v, t, n, s, z = _layered(16, 16)
    g = M.Graph(u, v, t, n=n)
    o = O.Graph(u, v, t, n=n)
    i = _index_of_pair(n, s, z, 5, M.D_PAIR)
    got = g.sample_paths(2, 5, i, 1, cap=n + 1)
    assert got == o.samples(2, 5, i, 1, cap=n + 1) and got[0][2] == 16 ** 16
    _cmp_samples(g.sample_paths(2, 5, i - 40, 81, cap=n + 1), o.samples(2, 5, i - 40, 81, cap=o.n + 1))
    _, h, info = g.estimate(2, 0.1, 0.1, 5, fixed_r=300)
    _, oh, _ = o.estimate(2, 0.1, 0.1, 5, fixed_r=300)
    assert np.array_equal(h, oh)


@pytest.mark.parametrize("case", [0, 2, 4, 5])
def test_pfm_temporal_stats(M, kernel, case):
    _, (u, v, t), n = _graphs()[case]
    g = M.Graph(u, v, t, n=n)
    o = O.Graph(u, v, t, n=n)
    st, reach = g.temporal_stats(2, 0.05, 9, r_override=300, tau=0.9)
    oreach, odlb = o.stats_counts(2, 9, 300)
    assert st["d_lb"] == odlb
    assert np.array_equal(reach, oreach)


def test_pfm_bursty_20k_samples(M, kernel):
    """Full-size graph (n = 20,000, 500,000 contacts): sampled samples against
    the oracle one by one, and the counters both kernels report alike."""
    u, v, t = synth.chung_lu_bursty()
    g = M.Graph(u, v, t)
    o = O.Graph(u, v, t)
    _cmp_samples(g.sample_paths(2, 1, 5000, 12, cap=g.n + 1), o.samples(2, 1, 5000, 12, cap=o.n + 1))
    st, reach = g.temporal_stats(2, 0.01, 3, r_override=4)
    oreach, odlb = o.stats_counts(2, 3, 4)
    assert st["d_lb"] == odlb and np.array_equal(reach, oreach)


def test_pfm_kernels_agree_on_counters(M, monkeypatch):
    """edges_scanned (stream edges of each sample's scan window) and
    sigma_adds (prefix-foremost DAG edges) are properties of the samples,
    not of the kernel."""
    u, v, t = synth.chung_lu_bursty(n=3000, m=60000, seed=8)
    g = M.Graph(u, v, t)
    infos = {}
    for k in KERNELS:
        monkeypatch.setenv("MANTRA_PFM_KERNEL", k)
        _, h, info = g.estimate(2, 0.1, 0.1, 9, fixed_r=2000)
        infos[k] = (h, info)
    (h0, i0), (h1, i1) = infos["lane"], infos["cta"]
    assert np.array_equal(h0, h1)
    for key in ("edges_scanned", "sigma_adds", "sum_int_len", "rade_num"):
        assert i0[key] == i1[key], key


def test_pfm_cta_global_state_variant():
    """The CTA kernel with its arrival state in global memory (the variant
    graphs too large for shared memory take), forced in a child process."""
    import json
    import os
    import subprocess
    import sys
    code = r'''
import json, sys
sys.path.insert(0, ".")
sys.path.insert(0, "tests")
import numpy as np
from paper_2304_08356_gb300 import build as B, synth
B.build()
from paper_2304_08356_gb300 import mantra as M
from oracle import oracle as O
from test_gpu_parity import _graphs
ok = True
for case in (0, 2, 4, 5):
    _, (u, v, t), n = _graphs()[case]
    g = M.Graph(u, v, t, n=n); o = O.Graph(u, v, t, n=n)
    ok &= g.sample_paths(2, 6, 0, 400, cap=g.n + 1) == o.samples(2, 6, 0, 400, cap=o.n + 1)
    st, reach = g.temporal_stats(2, 0.1, 5, r_override=80)
    oreach, _ = o.stats_counts(2, 5, 80)
    ok &= bool(np.array_equal(reach, oreach))
u, v, t = synth.chung_lu_bursty(n=1500, m=30000, seed=21)
g = M.Graph(u, v, t); o = O.Graph(u, v, t)
_, h, _ = g.estimate(2, 0.1, 0.1, 4, fixed_r=600)
_, oh, _ = o.estimate(2, 0.1, 0.1, 4, fixed_r=600)
ok &= bool(np.array_equal(h, oh))
print(json.dumps({"ok": bool(ok)}))
'''
    env = dict(os.environ, MANTRA_PFM_KERNEL="cta", MANTRA_PFM_CTA_SMEM="0")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", code], cwd=root, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    assert json.loads(r.stdout.strip().splitlines()[-1])["ok"]
