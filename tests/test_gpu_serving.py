"""Serving loop (continuous batching): requests arriving while others run
give exactly the results of mantra_estimate alone; admission respects the
device-memory budget."""
import time

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
def graphs(M):
    specs = [synth.chung_lu_bursty(n=500, m=8000, seed=51), synth.chung_lu_bursty(n=2000, m=40000, seed=52),
             synth.uniform_small(), synth.chung_lu_bursty(n=1200, m=25000, seed=53)]
    return specs, [M.Graph(*s) for s in specs]


def _requests():
    rng = np.random.default_rng(3)
    out = []
    for k in range(14):
        out.append(dict(gi=int(rng.integers(0, 4)), opt=int(rng.integers(0, 3)),
                        eps=float(rng.choice([0.1, 0.07, 0.05])), seed=100 + k))
    return out


def test_served_equals_solo(M, graphs):
    specs, gs = graphs
    srv = M.Server()
    reqs = _requests()
    ids = []
    for k, r in enumerate(reqs):
        ids.append(srv.submit(gs[r["gi"]], r["opt"], r["eps"], 0.1, r["seed"]))
        if k % 4 == 3:
            time.sleep(0.02)             # later requests arrive while earlier ones run
    results = [srv.wait(i, timeout=300) for i in ids]
    st = srv.stats()
    srv.close()
    assert st["finished"] == len(reqs) and st["ticks"] > 0
    for r, (est, hits, info) in zip(reqs, results):
        e2, h2, i2 = gs[r["gi"]].estimate(r["opt"], r["eps"], 0.1, r["seed"])
        assert np.array_equal(hits, h2) and np.array_equal(est.view(np.uint64), e2.view(np.uint64))
        for k in ("r", "rounds", "omega", "s1", "rade_num"):
            assert info[k] == i2[k]
    # two requests also against the oracle
    for r, (est, hits, info) in list(zip(reqs, results))[:2]:
        u, v, t = specs[r["gi"]]
        o = O.Graph(u, v, t, n=gs[r["gi"]].n)
        _, oh, oi = o.estimate(r["opt"], r["eps"], 0.1, r["seed"])
        assert np.array_equal(hits, oh) and info["r"] == oi["r"]


def test_admission_budget_and_poll(M, graphs):
    specs, gs = graphs
    srv = M.Server(hbm_budget=1, max_active=0)     # budget below any request: one at a time
    ids = [srv.submit(gs[1], 2, 0.07, 0.1, 7 + k) for k in range(4)]
    seen_active = 0
    done = {}
    t0 = time.time()
    while len(done) < len(ids) and time.time() - t0 < 300:
        seen_active = max(seen_active, srv.stats()["active"])
        for i in ids:
            if i not in done:
                r = srv.poll(i)
                if r is not None:
                    done[i] = r
        time.sleep(0.002)
    srv.close()
    assert len(done) == len(ids) and seen_active <= 1
    for k, i in enumerate(ids):
        _, h2, _ = gs[1].estimate(2, 0.07, 0.1, 7 + k)
        assert np.array_equal(done[i][1], h2)


def test_admission_counts_the_search_workspace(M, graphs):
    """The shared search workspace counts against the budget: it is at least
    four CTAs per SM (>= 100 SMs) x 24 bytes per arrival slot, so a budget of
    that size admits one sh request at a time although the requests' own
    buffers are far smaller; the reported device state includes it."""
    _, gs = graphs
    g = gs[1]
    lower = 400 * 24 * g.slots
    srv = M.Server(hbm_budget=lower, max_active=0)
    ids = [srv.submit(g, 0, 0.07, 0.1, 21 + k) for k in range(3)]
    seen_active, seen_bytes, done = 0, 0, {}
    t0 = time.time()
    while len(done) < len(ids) and time.time() - t0 < 300:
        st = srv.stats()
        seen_active = max(seen_active, st["active"])
        if st["active"]:
            seen_bytes = max(seen_bytes, st["bytes_in_use"])
        for i in ids:
            if i not in done:
                r = srv.poll(i)
                if r is not None:
                    done[i] = r
        time.sleep(0.001)
    srv.close()
    assert len(done) == len(ids) and seen_active <= 1
    assert seen_bytes == 0 or seen_bytes >= lower
    for k, i in enumerate(ids):
        _, h2, _ = g.estimate(0, 0.07, 0.1, 21 + k)
        assert np.array_equal(done[i][1], h2)


def test_invalid_request_rejected(M, graphs):
    _, gs = graphs
    srv = M.Server()
    with pytest.raises(M.MantraError):
        srv.submit(gs[0], 0, 1.5, 0.1, 1)
    srv.close()
