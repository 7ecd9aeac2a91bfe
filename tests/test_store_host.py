"""The host store builder (csrc/store.cu) against the store's definition (paper
Sec. 3: the temporal graph as a set of triples (u, v, t); the arrival slots and
the three orders are the layout of the library), run without a GPU through a
small driver.  Every array is rebuilt here from its definition with numpy
(lexicographic sorts, unique, searchsorted) and compared entry by entry, on
graphs that exercise one- and two-digit radix passes, the single-thread and
the threaded paths, duplicates, self loops, isolated vertices and invalid
input."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_2304_08356_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2304_08356_gb300", "csrc")
NAMES = ["out_ptr", "out_v", "out_t", "out_slot", "slot_ptr", "slot_t", "slot_v", "slot_in", "in_u", "in_slot",
         "st_u", "st_v", "st_t", "tmax_in", "tmin_out", "in_uedge", "slot_nout", "out_loff"]


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path_factory.mktemp("store") / "store_driver")
    cmd = [nvcc, "-O2", "-std=c++17", "-I", os.path.join(ROOT, "include"), "-I", CSRC,
           os.path.join(ROOT, "tests", "store_driver.cu"), os.path.join(CSRC, "store.cu"), "-lcudart", "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return exe


def run_builder(driver, tmp_path, u, v, t, n, threads=None):
    src, dst = str(tmp_path / "in.bin"), str(tmp_path / "out.bin")
    with open(src, "wb") as f:
        f.write(np.uint64(len(u)).tobytes() + np.uint32(n).tobytes())
        for a in (u, v, t):
            f.write(np.ascontiguousarray(a, dtype=np.uint32).tobytes())
    env = dict(os.environ)
    env.pop("MANTRA_STORE_THREADS", None)
    if threads is not None:
        env["MANTRA_STORE_THREADS"] = str(threads)
    subprocess.run([driver, src, dst], check=True, env=env)
    raw = open(dst, "rb").read()
    rc = int(np.frombuffer(raw, np.int32, 1, 0)[0])
    sc = np.frombuffer(raw, np.uint32, 8, 4)
    cn = np.frombuffer(raw, np.uint64, 2, 36)
    out = dict(rc=rc, n=int(sc[0]), m=int(sc[1]), A=int(sc[2]), n_uedge=int(sc[3]), cbound=int(sc[4]),
               max_slot_in=int(sc[5]), max_vslots=int(sc[6]), self_loops=int(cn[0]), duplicates=int(cn[1]))
    off = 52
    for name in NAMES:
        ln = int(np.frombuffer(raw, np.uint64, 1, off)[0])
        off += 8
        out[name] = np.frombuffer(raw, np.uint32, ln, off).copy()
        off += 4 * ln
    return out


def definition(u, v, t, n):
    """The store of the triples, from its definition."""
    u, v, t = (np.asarray(a, np.int64) for a in (u, v, t))
    n = n or int(max(u.max(initial=0), v.max(initial=0))) + 1
    keep = u != v
    tri = np.unique(np.stack([t[keep], u[keep], v[keep]], 1).reshape(-1, 3), axis=0)   # (t, u, v) order
    st_t, st_u, st_v = tri[:, 0], tri[:, 1], tri[:, 2]
    M = len(tri)
    d = dict(n=n, m=M, self_loops=int((~keep).sum()), duplicates=int(keep.sum()) - M,
             st_u=st_u, st_v=st_v, st_t=st_t)
    ino = np.lexsort((st_u, st_t, st_v))                   # in-CSR: (v, t, u)
    in_u, in_v, in_t = st_u[ino], st_v[ino], st_t[ino]
    new = np.ones(M, bool)
    new[1:] = (in_v[1:] != in_v[:-1]) | (in_t[1:] != in_t[:-1])
    first = np.flatnonzero(new)
    slot_t, slot_v = in_t[first], in_v[first]
    in_slot = np.cumsum(new) - 1
    inpos = np.empty(M, np.int64)
    inpos[ino] = np.arange(M)
    d.update(A=len(first), in_u=in_u, in_slot=in_slot, slot_t=slot_t, slot_v=slot_v,
             slot_in=np.append(first, M), slot_ptr=np.searchsorted(slot_v, np.arange(n + 1)))
    outo = np.lexsort((st_v, st_t, st_u))                  # out-CSR: (u, t, v)
    out_u, out_t = st_u[outo], st_t[outo]
    out_ptr = np.searchsorted(out_u, np.arange(n + 1))
    d.update(out_ptr=out_ptr, out_v=st_v[outo], out_t=out_t, out_slot=in_slot[inpos[outo]])
    # underlying edges: distinct (v, u) ranked in (v, u) order, per in-CSR position
    pairs, inv = np.unique(np.stack([in_v, in_u], 1).reshape(-1, 2), axis=0, return_inverse=True)
    d.update(in_uedge=inv.reshape(-1), n_uedge=len(pairs))
    cnt_s = np.diff(slot_ptr := d["slot_ptr"])
    d["tmax_in"] = np.where(cnt_s > 0, slot_t[np.maximum(slot_ptr[1:] - 1, 0)] if len(slot_t) else 0, 0)
    cnt_o = np.diff(out_ptr)
    d["tmin_out"] = np.where(cnt_o > 0, out_t[np.minimum(out_ptr[:-1], max(M - 1, 0))] if M else 0, 0)
    # first out-edge of v later than each slot (v, t): rows are in time order
    d["slot_nout"] = np.searchsorted((out_u << 32) | out_t, (slot_v << 32) | slot_t, side="right")
    # per out-edge, the head's slot offset within the head's slots (16-bit,
    # clamped to 0xFFFF), two entries per uint32 word, a trailing half 0
    loff = np.zeros(2 * ((M + 1) // 2), np.uint16)
    loff[:M] = np.minimum(d["out_slot"] - slot_ptr[d["out_v"]], 0xFFFF)
    d["out_loff"] = loff.view(np.uint32)
    per_slot = np.diff(d["slot_in"])
    vmax = np.zeros(n, np.int64)
    np.maximum.at(vmax, slot_v, per_slot)
    d.update(cbound=int(vmax.sum()), max_slot_in=int(vmax.max(initial=0)), max_vslots=int(cnt_s.max(initial=0)))
    return d


def check(driver, tmp_path, u, v, t, n=0, threads=None):
    got = run_builder(driver, tmp_path, u, v, t, n, threads)
    assert got["rc"] == 0
    ref = definition(u, v, t, n)
    for k in ("n", "m", "A", "n_uedge", "cbound", "max_slot_in", "max_vslots", "self_loops", "duplicates"):
        assert got[k] == ref[k], k
    for name in NAMES:
        assert np.array_equal(got[name].astype(np.int64), np.asarray(ref[name], np.int64)), name
    return got


def _random(seed, m, n, t_hi, loops=0.0, dup=0.0):
    rng = np.random.default_rng(seed)
    u = rng.integers(0, n, m, dtype=np.int64)
    v = rng.integers(0, n, m, dtype=np.int64)
    t = rng.integers(0, t_hi, m, dtype=np.int64)
    sel = rng.random(m) < loops
    v[sel] = u[sel]
    d = np.flatnonzero(rng.random(m) < dup)
    d = d[d > 0]
    u[d], v[d], t[d] = u[d - 1], v[d - 1], t[d - 1]
    return u, v, t


@pytest.mark.parametrize("case", [
    ("tiny", dict(seed=1, m=300, n=12, t_hi=5, loops=0.1, dup=0.2)),          # one thread
    ("dense_dups", dict(seed=2, m=200_000, n=500, t_hi=50, loops=0.02)),      # threaded, one digit
    ("wide_ids_times", dict(seed=3, m=150_000, n=300_000, t_hi=0xFFFFFFFE, loops=0.01, dup=0.05)),
    ("times_17_bits", dict(seed=4, m=90_000, n=70_000, t_hi=1 << 17)),
])
def test_store_matches_definition(driver, tmp_path, case):
    u, v, t = _random(**case[1])
    check(driver, tmp_path, u, v, t)


def test_store_bursty_bench_graph(driver, tmp_path):
    """The bench workload's graph (bursty Chung-Lu, n = 20,000, m = 500,000)."""
    u, v, t = synth.chung_lu_bursty(n=20000, m=500000, seed=1)
    got = check(driver, tmp_path, u, v, t)
    assert (got["n"], got["m"], got["A"]) == (20000, 499106, 498887)


def test_store_given_n_and_degenerate(driver, tmp_path):
    u, v, t = _random(5, 80_000, 900, 1000, loops=0.05)
    check(driver, tmp_path, u, v, t, n=1000)                 # isolated vertices at the end
    u = np.arange(70_000) % 50
    got = check(driver, tmp_path, u, u, u, n=50)             # only self loops: empty store
    assert got["m"] == 0 and got["self_loops"] == 70_000 and got["n_uedge"] == 0
    check(driver, tmp_path, np.array([0]), np.array([1]), np.array([0xFFFFFFFD]))


@pytest.mark.parametrize("bad", ["id_ge_n", "time", "n_one", "empty"])
def test_store_invalid(driver, tmp_path, bad):
    u, v, t = _random(6, 70_000, 100, 100)
    n = 100
    if bad == "id_ge_n":
        u[35_000] = 100
    elif bad == "time":
        t[1234] = 0xFFFFFFFE
    elif bad == "n_one":
        n = 1
    else:
        u = v = t = np.zeros(0, np.int64)
        n = 0
    assert run_builder(driver, tmp_path, u, v, t, n)["rc"] == 1


@pytest.mark.parametrize("threads", [1, 2, 3, 16])
def test_store_thread_counts(driver, tmp_path, threads):
    """Any team size gives the same store, including teams with more threads
    than records (empty chunks) and more threads than host cores."""
    for seed, m, n, t_hi in ((7, 5, 4, 3), (8, 40, 30, 6), (9, 3000, 700, 1 << 18), (10, 70_000, 90_000, 1000)):
        u, v, t = _random(seed, m, n, t_hi, loops=0.05, dup=0.1)
        check(driver, tmp_path, u, v, t, threads=threads)
    u, v, t = _random(11, 50, 20, 10)
    u[7] = 20
    assert run_builder(driver, tmp_path, u, v, t, 20, threads)["rc"] == 1


def test_store_head_offsets_clamp(driver, tmp_path):
    """A vertex with more than 65,535 arrival slots: its heads' offsets above
    0xFFFF are clamped (the 16-bit search state is then not used), the others
    are exact; an odd edge count leaves the trailing half word 0."""
    k = 70001
    u = np.concatenate([np.zeros(k, np.int64), [1, 1, 2, 3]])
    v = np.concatenate([np.ones(k, np.int64), [2, 3, 3, 2]])
    t = np.concatenate([np.arange(1, k + 1), [5, 70000, 9, 11]])
    got = check(driver, tmp_path, u, v, t)
    m = got["m"]
    assert got["max_vslots"] == k and m == k + 4 and m % 2 == 1
    lo = got["out_loff"].view(np.uint16)
    assert len(lo) == m + 1 and lo[m] == 0
    assert (lo[:m] == 0xFFFF).sum() == k - 0xFFFF

