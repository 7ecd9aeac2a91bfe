"""Complete hit vectors at the bench workload's full size (bursty Chung-Lu
n = 20,000, m = 500,000, the launch configuration the benchmark times)
against the oracle: every sample of the run is recomputed by the oracle, on
all host threads over disjoint sample ranges (the oracle's per-sample call
is unchanged; Philox indexing makes the ranges independent), and the hits,
the c-MCERA numerator and the wimpy maximum are recounted from its paths."""
import os
import threading

import numpy as np
import pytest

from oracle import oracle as O
from paper_2304_08356_gb300 import synth

pytestmark = pytest.mark.gpu
C_TRIALS = 25


@pytest.fixture(scope="module")
def M():
    from paper_2304_08356_gb300 import build as B
    B.build()
    from paper_2304_08356_gb300 import mantra
    return mantra


@pytest.fixture(scope="module")
def bench_graph():
    u, v, t = synth.chung_lu_bursty()
    return (u, v, t), O.Graph(u, v, t)


def oracle_recount(o, opt, seed, count, c=C_TRIALS, chunk=128):
    """(hits, S) over estimation samples 0..count-1: oracle paths on all host
    threads, each sample's internal vertices adding 1 to hits and its
    Rademacher signs to S."""
    n = o.n
    starts = list(range(0, count, chunk))
    lock = threading.Lock()
    pos = [0]
    parts = []

    def worker():
        while True:
            with lock:
                if pos[0] >= len(starts):
                    return
                i0 = starts[pos[0]]
                pos[0] += 1
            k = min(chunk, count - i0)
            smp = o.samples(opt, seed, i0, k, cap=256)
            rows, cols = [], []
            for q, (_, _, _, p) in enumerate(smp):
                for x in p[1:-1]:
                    rows.append(i0 + q)
                    cols.append(x)
            with lock:
                parts.append((rows, cols))

    ths = [threading.Thread(target=worker) for _ in range(max(1, os.cpu_count() or 1))]
    for th in ths:
        th.start()
    for th in ths:
        th.join()
    rows = np.array([r for p in parts for r in p[0]], np.int64)
    cols = np.array([x for p in parts for x in p[1]], np.int64)
    hits = np.bincount(cols, minlength=n).astype(np.uint64)
    # lambda_{j,i} = +1 when bit j of sample i's RADE block is set, else -1
    lam = np.zeros((count, c), np.int64)
    for i in np.unique(rows):
        w = O.philox([int(i) & 0xFFFFFFFF, int(i) >> 32, O.D_RADE, 0], [seed & 0xFFFFFFFF, seed >> 32])
        lam[i] = [1 if (w[j >> 5] >> (j & 31)) & 1 else -1 for j in range(c)]
    S = np.zeros((c, n), np.int64)
    for j in range(c):
        np.add.at(S[j], cols, lam[rows, j])
    return hits, S


def test_pfm_progressive_complete_hit_vector(M, bench_graph):
    """One progressive pfm run at eps = 0.01 (about 50,000 samples): every
    sample's path, hence the whole hit vector, N_R, H and sum |Int|, equals
    the oracle's."""
    (u, v, t), o = bench_graph
    g = M.Graph(u, v, t)
    est, hits, info = g.estimate(2, 0.01, 0.1, 1)
    r = info["r"]
    assert r > 20000
    H, S = oracle_recount(o, 2, 1, r)
    assert np.array_equal(hits, H)
    assert info["rade_num"] == int(S.max(axis=1).sum())
    assert info["max_hits"] == int(H.max()) and info["sum_int_len"] == int(H.sum())
    assert np.array_equal(est.view(np.uint64), (H.astype(np.float64) / r).view(np.uint64))
    g.free()


@pytest.mark.parametrize("opt", [0, 1])
def test_sh_sfm_fixed_r_complete_hit_vector(M, bench_graph, opt):
    """A fixed-r run of 640 sh / sfm samples at the bench size (an oracle sh
    search there takes about a second): the whole hit vector and N_R against
    the oracle's recount."""
    (u, v, t), o = bench_graph
    g = M.Graph(u, v, t)
    r = 640
    _, hits, info = g.estimate(opt, 0.01, 0.1, 3, fixed_r=r)
    H, S = oracle_recount(o, opt, 3, r)
    assert np.array_equal(hits, H)
    assert info["rade_num"] == int(S.max(axis=1).sum())
    g.free()
