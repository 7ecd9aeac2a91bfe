"""The autotuner (mantra_tune) and the launch choices it picks from: every
CTA shape and state placement of both search kernels gives the oracle's
results bit for bit, and a tuned graph's estimates equal the untuned ones."""
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
def bursty():
    return synth.chung_lu_bursty(n=4000, m=90000, seed=17)


@pytest.mark.parametrize("nt", ["256", "512", "1024"])
@pytest.mark.parametrize("smem", ["0", "1"])
def test_bfs_shapes_and_placements_equal_oracle(M, bursty, monkeypatch, nt, smem):
    monkeypatch.setenv("MANTRA_BFS_NT", nt)
    monkeypatch.setenv("MANTRA_BFS_SMEM", smem)
    g = M.Graph(*bursty)
    o = O.Graph(*bursty)
    for opt in (0, 1, 3):
        _, hits, info = g.estimate(opt, 0.05, 0.1, 3, fixed_r=1500)
        _, ohits, oinfo = o.estimate(opt, 0.05, 0.1, 3, fixed_r=1500)
        assert np.array_equal(hits, ohits), opt
        assert info["rade_num"] == oinfo["rade_num"] and info["edges_scanned"] == oinfo["edges_scanned"]
    g.free()


@pytest.mark.parametrize("nt", ["256", "512"])
@pytest.mark.parametrize("smem", ["0", "1", "16", "staged"])
def test_pfm_cta_shapes_and_placements_equal_oracle(M, bursty, monkeypatch, nt, smem):
    """Arrival state in shared memory (32-bit slots, or 16-bit offsets within
    each vertex's slots), in global memory, and in global memory with each
    chunk's out-edge tiles copied into shared memory by bulk copies (chunks
    whose tiles exceed the staging capacity walk global memory)."""
    monkeypatch.setenv("MANTRA_PFM_CTA_NT", nt)
    monkeypatch.setenv("MANTRA_PFM_CTA_SMEM", "0" if smem == "staged" else smem)
    monkeypatch.setenv("MANTRA_PFM_STAGE", "1" if smem == "staged" else "0")
    g = M.Graph(*bursty)
    o = O.Graph(*bursty)
    _, hits, info = g.estimate(2, 0.05, 0.1, 3, fixed_r=2000)
    _, ohits, oinfo = o.estimate(2, 0.05, 0.1, 3, fixed_r=2000)
    assert np.array_equal(hits, ohits)
    assert info["rade_num"] == oinfo["rade_num"] and info["sigma_adds"] == oinfo["sigma_adds"]
    g.free()


@pytest.mark.parametrize("k", [65534, 70001])
@pytest.mark.parametrize("nt", ["256", "512"])
def test_pfm_16bit_state_at_the_slot_limit(M, monkeypatch, k, nt):
    """A hub with k arrival slots: at 65,534 (the largest count the 16-bit
    state holds, offsets up to 65,533) the 16-bit mode runs; above it the
    launch falls back to 32-bit slots.  Both equal the oracle."""
    monkeypatch.setenv("MANTRA_PFM_CTA_SMEM", "16")
    monkeypatch.setenv("MANTRA_PFM_CTA_NT", nt)
    rng = np.random.default_rng(k)
    n = 300
    hub_t = rng.permutation(np.arange(1, k + 1))                     # k distinct times into vertex 1
    u = [rng.integers(2, n, k), rng.integers(0, n, 20000), np.ones(4000, np.int64)]
    v = [np.ones(k, np.int64), rng.integers(0, n, 20000), rng.integers(2, n, 4000)]
    t = [hub_t, rng.integers(1, k + 1, 20000), rng.integers(1, k + 1, 4000)]
    u, v, t = (np.concatenate(a).astype(np.uint32) for a in (u, v, t))
    g = M.Graph(u, v, t, n=n)
    o = O.Graph(u, v, t, n=n)
    into1 = v == 1
    assert len(np.unique(t[into1])) == k                              # the hub's slot count
    _, hits, info = g.estimate(2, 0.05, 0.1, 5, fixed_r=1500)
    _, ohits, oinfo = o.estimate(2, 0.05, 0.1, 5, fixed_r=1500)
    assert np.array_equal(hits, ohits)
    assert info["rade_num"] == oinfo["rade_num"] and info["sigma_adds"] == oinfo["sigma_adds"]
    g.free()


def test_tuned_estimates_equal_untuned(M, bursty):
    g = M.Graph(*bursty)
    before = {opt: g.estimate(opt, 0.05, 0.1, 11)[1:] for opt in (0, 1, 2, 3)}
    res = g.tune()
    assert res["bfs_threads"] in (256, 512, 1024) and res["pfm_threads"] in (256, 512)
    assert res["bfs_bitmap_shared"] in (0, 1) and res["pfm_state_shared"] in (0, 1) and res["pfm_staged"] in (0, 1)
    assert res["pfm_state16"] in (0, 1) and (not res["pfm_state16"] or res["pfm_state_shared"])
    assert res["bfs_resident_ctas"] > 0 and res["pfm_resident_ctas"] > 0 and res["probe_samples"] >= 1024
    for k in ("bfs_ms", "bfs_default_ms", "pfm_ms", "pfm_default_ms"):
        assert 0.0 < res[k] < 1e6, k
    for opt in (0, 1, 2, 3):
        hits, info = g.estimate(opt, 0.05, 0.1, 11)[1:]
        assert np.array_equal(hits, before[opt][0]), opt
        for k in ("r", "rounds", "omega", "s1", "rade_num", "max_hits", "sum_int_len", "edges_scanned"):
            assert info[k] == before[opt][1][k], (opt, k)
    # a batch mixing the tuned graph with an untuned one equals the solo runs
    h = M.Graph(*synth.chung_lu_bursty(n=1500, m=30000, seed=21))
    probs = [dict(graph=g, opt=o_, eps=0.05, delta=0.1, seed=11) for o_ in (0, 2)] + \
            [dict(graph=h, opt=o_, eps=0.05, delta=0.1, seed=5) for o_ in (1, 2)]
    res = M.estimate_batch(probs)
    for p, r in zip(probs, res):
        assert r[3] == 0
        assert np.array_equal(r[1], p["graph"].estimate(p["opt"], 0.05, 0.1, p["seed"])[1])
    g.free()
    h.free()
