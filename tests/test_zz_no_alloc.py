"""mantra_sample_paths_noalloc: the allocation-free entry point for callers
that cannot call cudaMalloc once running (device memory fixed after start-up,
or no allocator latency allowed between requests).  It must give exactly the
per-sample results of mantra_sample_paths, on consecutive calls that reuse its
fixed device scratch.  Collected last on purpose."""
import numpy as np
import pytest

from paper_2304_08356_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    from paper_2304_08356_gb300 import build as B
    B.build()
    from paper_2304_08356_gb300 import mantra
    return mantra


def _noalloc(M, g, opt, seed, i0, count, cap):
    import torch
    s = torch.zeros(count, dtype=torch.int32, device="cuda")
    z = torch.zeros(count, dtype=torch.int32, device="cuda")
    sig = torch.zeros(2 * count, dtype=torch.int64, device="cuda")
    ln = torch.zeros(count, dtype=torch.int32, device="cuda")
    nodes = torch.zeros(max(count * cap, 1), dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    rc = M.lib().mantra_sample_paths_noalloc(g.h, opt, seed, M.D_PAIR, M.D_PATH, i0, count, s.data_ptr(),
                                             z.data_ptr(), sig.data_ptr(), ln.data_ptr(), nodes.data_ptr(), cap,
                                             None)
    torch.cuda.synchronize()
    if rc != 0:
        return rc, None
    s, z, sig, ln, nodes = (x.cpu().numpy().view(np.uint32 if x.dtype == torch.int32 else np.uint64)
                            for x in (s, z, sig, ln, nodes))
    out = []
    for q in range(count):
        L = int(ln[q])
        out.append((int(s[q]), int(z[q]), (int(sig[2 * q + 1]) << 64) | int(sig[2 * q]),
                    [int(x) for x in nodes[q * cap:q * cap + min(L, cap)]]))
    return 0, out


@pytest.mark.parametrize("opt", [0, 1])
def test_noalloc_matches_sample_paths_two_calls(M, opt):
    u, v, t = synth.chung_lu_bursty(n=3000, m=60000, seed=12)
    g = M.Graph(u, v, t)
    cap = 64
    for i0, count in ((0, 700), (350, 900)):        # two calls in a row, overlapping ranges
        rc, got = _noalloc(M, g, opt, 5, i0, count, cap)
        assert rc == 0
        assert got == g.sample_paths(opt, 5, i0, count, cap=cap)


def test_noalloc_bench_size_graph(M):
    u, v, t = synth.chung_lu_bursty()                 # n = 20,000, 500,000 contacts
    g = M.Graph(u, v, t)
    for rep in range(2):
        rc, got = _noalloc(M, g, 0, 1, 100 * rep, 96, 32)
        assert rc == 0
        assert got == g.sample_paths(0, 1, 100 * rep, 96, cap=32)


def test_noalloc_rejects_oversized_and_pfm(M):
    u, v, t = synth.chung_lu_uniform_t(n=400_000, m=2_500_000, seed=3)   # ~2.5M slots: beyond 64 MiB
    g = M.Graph(u, v, t)
    rc, _ = _noalloc(M, g, 0, 1, 0, 8, 8)
    assert rc == 1
    u, v, t = synth.uniform_small()
    g = M.Graph(u, v, t, n=100)
    rc, _ = _noalloc(M, g, 2, 1, 0, 8, 8)
    assert rc == 1
