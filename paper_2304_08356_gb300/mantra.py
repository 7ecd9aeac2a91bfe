"""Thin ctypes binding of libmantra.so (include/mantra.h).

Argument marshalling only: every step of the sampler runs in the library's
CUDA kernels.  Loading fails loudly when the library is missing; there is no
CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmantra.so")

SH, SFM, PFM, FSFM = 0, 1, 2, 3
OPT_NAMES = {"sh": SH, "sfm": SFM, "pfm": PFM, "fsfm": FSFM}
D_PAIR, D_PATH, D_RADE, D_BOOT_PAIR, D_BOOT_PATH, D_STATS = range(6)

ERRORS = {0: "MANTRA_OK", 1: "MANTRA_E_INVAL", 2: "MANTRA_E_NOMEM", 3: "MANTRA_E_OVERFLOW", 4: "MANTRA_E_CUDA",
          5: "MANTRA_E_TIMEOUT", 6: "MANTRA_E_CHECK", 7: "MANTRA_E_RNG", 8: "MANTRA_PENDING"}


class MantraError(RuntimeError):
    def __init__(self, code, where):
        super().__init__("%s: %s (%d)" % (where, ERRORS.get(code, "?"), code))
        self.code = code


class Opts(C.Structure):
    _fields_ = [("c", C.c_uint32), ("growth", C.c_double), ("fixed_r", C.c_uint64), ("bootstrap", C.c_uint64),
                ("delta_sched", C.c_int), ("out_device", C.c_int), ("stream", C.c_void_p), ("vhat_mode", C.c_int),
                ("target", C.c_int), ("estimator", C.c_int)]


class Info(C.Structure):
    _fields_ = [("r", C.c_uint64), ("rounds", C.c_uint64), ("omega", C.c_uint64), ("s1", C.c_uint64),
                ("bootstrap", C.c_uint64), ("sum_int_len", C.c_uint64), ("max_hits", C.c_uint64),
                ("rade_num", C.c_int64), ("xi", C.c_double), ("vhat", C.c_double), ("rho_hat", C.c_double),
                ("edges_scanned", C.c_uint64), ("sigma_adds", C.c_uint64), ("states_new", C.c_uint64),
                ("wide_samples", C.c_uint64), ("seconds", C.c_double), ("kernel_ms", C.c_double),
                ("search_launches", C.c_uint64), ("kernel_launches", C.c_uint64), ("alg_bytes", C.c_uint64),
                ("frontier_vertices", C.c_uint64), ("edges_expanded", C.c_uint64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class TuneResult(C.Structure):
    _fields_ = [("bfs_threads", C.c_uint32), ("bfs_bitmap_shared", C.c_uint32), ("pfm_threads", C.c_uint32),
                ("pfm_state_shared", C.c_uint32), ("bfs_resident_ctas", C.c_uint32), ("pfm_resident_ctas", C.c_uint32),
                ("bfs_ms", C.c_double), ("bfs_default_ms", C.c_double), ("pfm_ms", C.c_double),
                ("pfm_default_ms", C.c_double), ("probe_samples", C.c_uint64), ("pfm_probe_samples", C.c_uint64),
                ("pfm_staged", C.c_uint32), ("pfm_state16", C.c_uint32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Problem(C.Structure):
    _fields_ = [("graph", C.c_void_p), ("opt", C.c_int), ("eps", C.c_double), ("delta", C.c_double),
                ("seed", C.c_uint64), ("opts", C.POINTER(Opts)), ("est_out", C.c_void_p), ("hits_out", C.c_void_p),
                ("info", C.POINTER(Info)), ("status", C.c_int)]


class TStats(C.Structure):
    _fields_ = [("d_lb", C.c_uint32), ("d_tau", C.c_uint32), ("zeta", C.c_double), ("psi", C.c_double),
                ("rho", C.c_double), ("r", C.c_uint64), ("seconds", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


EXPORTS = ["mantra_graph_load", "mantra_graph_info", "mantra_graph_edges", "mantra_graph_free", "mantra_estimate",
           "mantra_estimate_batch", "mantra_tune",
           "mantra_temporal_stats", "mantra_temporal_closeness", "mantra_sample_paths", "mantra_sample_paths_noalloc", "mantra_strerror",
           "mantra_server_create", "mantra_server_submit", "mantra_server_poll", "mantra_server_wait",
           "mantra_server_stats", "mantra_server_destroy"]

_lib = None


def lib():
    """Load libmantra.so (built by paper_2304_08356_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libmantra.so is not built (%s); run paper_2304_08356_gb300.build.build()" % LIB_PATH)
    L = C.CDLL(LIB_PATH)
    u32p, u64p, dp = C.POINTER(C.c_uint32), C.POINTER(C.c_uint64), C.POINTER(C.c_double)
    L.mantra_graph_load.argtypes = [u32p, u32p, u32p, C.c_uint64, C.c_uint32, C.POINTER(C.c_void_p)]
    L.mantra_graph_info.argtypes = [C.c_void_p, u32p, u64p, u64p, u64p, u64p]
    L.mantra_graph_edges.argtypes = [C.c_void_p, u32p, u32p, u32p, u32p, u32p]
    L.mantra_graph_free.argtypes = [C.c_void_p]
    L.mantra_graph_free.restype = None
    L.mantra_estimate.argtypes = [C.c_void_p, C.c_int, C.c_double, C.c_double, C.c_uint64, C.POINTER(Opts),
                                  C.c_void_p, C.c_void_p, C.POINTER(Info)]
    L.mantra_estimate_batch.argtypes = [C.POINTER(Problem), C.c_uint32]
    L.mantra_tune.argtypes = [C.c_void_p, C.POINTER(TuneResult)]
    L.mantra_temporal_stats.argtypes = [C.c_void_p, C.c_int, C.c_double, C.c_uint64, C.c_uint64, C.c_double,
                                        C.POINTER(TStats), u64p, C.c_uint32]
    L.mantra_temporal_closeness.argtypes = [C.c_void_p, C.c_int, C.c_double, C.c_uint64, C.c_uint64, u64p, dp,
                                            u64p]
    L.mantra_sample_paths.argtypes = [C.c_void_p, C.c_int, C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint64,
                                      C.c_uint64, u32p, u32p, u64p, u32p, u32p, C.c_uint32, u32p]
    L.mantra_sample_paths_noalloc.argtypes = [C.c_void_p, C.c_int, C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint64,
                                              C.c_uint64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                              C.c_void_p, C.c_uint32, C.c_void_p]
    L.mantra_server_create.argtypes = [C.c_size_t, C.c_uint32, C.POINTER(C.c_void_p)]
    L.mantra_server_submit.argtypes = [C.c_void_p, C.c_void_p, C.c_int, C.c_double, C.c_double, C.c_uint64,
                                       C.POINTER(Opts), C.POINTER(C.c_uint64)]
    L.mantra_server_poll.argtypes = [C.c_void_p, C.c_uint64, C.c_void_p, C.c_void_p, C.POINTER(Info)]
    L.mantra_server_wait.argtypes = [C.c_void_p, C.c_uint64, C.c_double, C.c_void_p, C.c_void_p, C.POINTER(Info)]
    L.mantra_server_stats.argtypes = [C.c_void_p] + [C.POINTER(C.c_uint64)] * 5
    L.mantra_server_destroy.argtypes = [C.c_void_p]
    L.mantra_server_destroy.restype = None
    L.mantra_strerror.restype = C.c_char_p
    L.mantra_strerror.argtypes = [C.c_int]
    _lib = L
    return L


def _p(a, ct):
    return a.ctypes.data_as(C.POINTER(ct))


def _chk(code, where):
    if code != 0:
        raise MantraError(code, where)


def _opt(opt):
    return OPT_NAMES[opt] if isinstance(opt, str) else int(opt)


def strerror(code: int) -> str:
    return lib().mantra_strerror(code).decode()


class Graph:
    """A device-resident temporal graph (mantra_graph_load)."""

    def __init__(self, u, v, t, n: int = 0):
        u = np.ascontiguousarray(u, dtype=np.uint32)
        v = np.ascontiguousarray(v, dtype=np.uint32)
        t = np.ascontiguousarray(t, dtype=np.uint32)
        h = C.c_void_p()
        _chk(lib().mantra_graph_load(_p(u, C.c_uint32), _p(v, C.c_uint32), _p(t, C.c_uint32), u.size, n,
                                     C.byref(h)), "mantra_graph_load")
        self.h = h
        nn, m, sl, lp, dp_ = C.c_uint32(), C.c_uint64(), C.c_uint64(), C.c_uint64(), C.c_uint64()
        _chk(lib().mantra_graph_info(self.h, C.byref(nn), C.byref(m), C.byref(sl), C.byref(lp), C.byref(dp_)),
             "mantra_graph_info")
        self.n, self.m, self.slots, self.self_loops, self.duplicates = nn.value, m.value, sl.value, lp.value, dp_.value
        self._edges = None

    def edge_ids(self):
        """mantra_graph_edges -> (u, v, t, underlying id) per temporal edge id,
        and the number of underlying edges."""
        if self._edges is None:
            u = np.zeros(max(self.m, 1), np.uint32); v = np.zeros_like(u); t = np.zeros_like(u)
            ue = np.zeros_like(u); nu = C.c_uint32()
            _chk(lib().mantra_graph_edges(self.h, _p(u, C.c_uint32), _p(v, C.c_uint32), _p(t, C.c_uint32),
                                          _p(ue, C.c_uint32), C.byref(nu)), "mantra_graph_edges")
            self._edges = (u[:self.m], v[:self.m], t[:self.m], ue[:self.m], nu.value)
        return self._edges

    def family_size(self, target=0):
        """Entries of an estimate: nodes (0), underlying edges (1) or temporal edges (2)."""
        return self.n if target == 0 else (self.edge_ids()[4] if target == 1 else self.m)

    def free(self):
        if getattr(self, "h", None):
            lib().mantra_graph_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def estimate(self, opt, eps, delta, seed, c=0, growth=0.0, fixed_r=0, bootstrap=0, delta_sched=0,
                 est_out=None, hits_out=None, stream=None, vhat_mode=0, target=0, estimator=0):
        """mantra_estimate.  With est_out / hits_out given as integers they are
        device pointers (out_device = 1); otherwise host numpy arrays are
        returned.  target: 0 nodes, 1 underlying edges, 2 temporal edges;
        estimator: 0 trk, 1 ob, 2 RTB (ob and RTB hits in 2^-32 units).  Returns (est, hits, info dict)."""
        o = Opts(c, growth, fixed_r, bootstrap, delta_sched, 0, stream, vhat_mode, target, estimator)
        info = Info()
        if isinstance(est_out, int):
            o.out_device = 1
            _chk(lib().mantra_estimate(self.h, _opt(opt), eps, delta, seed, C.byref(o), C.c_void_p(est_out),
                                       C.c_void_p(hits_out) if hits_out else None, C.byref(info)),
                 "mantra_estimate")
            return None, None, info.as_dict()
        F = self.family_size(target) if target in (0, 1, 2) else self.n
        est = np.zeros(max(F, 1), np.float64)
        hits = np.zeros(max(F, 1), np.uint64)
        _chk(lib().mantra_estimate(self.h, _opt(opt), eps, delta, seed, C.byref(o), est.ctypes.data,
                                   hits.ctypes.data, C.byref(info)), "mantra_estimate")
        return est[:F], hits[:F], info.as_dict()

    def temporal_stats(self, opt, eps, seed, r_override=0, tau=0.9, reach_cap=None):
        """mantra_temporal_stats -> (stats dict, reach array)."""
        cap = reach_cap if reach_cap is not None else self.n
        reach = np.zeros(max(cap, 1), np.uint64)
        st = TStats()
        _chk(lib().mantra_temporal_stats(self.h, _opt(opt), eps, seed, r_override, tau, C.byref(st),
                                         _p(reach, C.c_uint64), cap), "mantra_temporal_stats")
        d = st.as_dict()
        return d, reach[:min(cap, d["d_lb"] + 1)].copy()

    def temporal_closeness(self, opt, eps, seed, r_override=0):
        """mantra_temporal_closeness -> (sums in 2^-32 units, closeness, r_s)."""
        sm = np.zeros(max(self.n, 1), np.uint64); cl = np.zeros(max(self.n, 1), np.float64)
        rs = C.c_uint64()
        _chk(lib().mantra_temporal_closeness(self.h, _opt(opt), eps, seed, r_override, _p(sm, C.c_uint64),
                                             _p(cl, C.c_double), C.byref(rs)), "mantra_temporal_closeness")
        return sm[:self.n], cl[:self.n], rs.value

    def tune(self):
        """mantra_tune: time the search kernels' launch choices on this graph
        and keep the fastest; returns the choice and the probe times."""
        out = TuneResult()
        _chk(lib().mantra_tune(self.h, C.byref(out)), "mantra_tune")
        return out.as_dict()

    def sample_paths(self, opt, seed, i0, count, dom_pair=D_PAIR, dom_path=D_PATH, cap=None, edges=False):
        """mantra_sample_paths -> list of (s, z, sigma, path) per sample; with
        edges=True a fifth entry, the path's temporal edge ids."""
        cap = cap if cap is not None else min(self.n + 1, 4096)
        s = np.zeros(count, np.uint32); z = np.zeros(count, np.uint32)
        sig = np.zeros(2 * count, np.uint64); ln = np.zeros(count, np.uint32)
        nodes = np.zeros(max(count * cap, 1), np.uint32)
        pe = np.zeros(max(count * cap, 1), np.uint32) if edges else None
        _chk(lib().mantra_sample_paths(self.h, _opt(opt), seed, dom_pair, dom_path, i0, count,
                                       _p(s, C.c_uint32), _p(z, C.c_uint32), _p(sig, C.c_uint64),
                                       _p(ln, C.c_uint32), _p(nodes, C.c_uint32), cap,
                                       _p(pe, C.c_uint32) if edges else None), "mantra_sample_paths")
        out = []
        for q in range(count):
            L = int(ln[q])
            row = (int(s[q]), int(z[q]), (int(sig[2 * q + 1]) << 64) | int(sig[2 * q]),
                   [int(x) for x in nodes[q * cap:q * cap + min(L, cap)]])
            if edges:
                row = row + ([int(x) for x in pe[q * cap:q * cap + min(max(L - 1, 0), cap)]],)
            out.append(row)
        return out


def estimate_batch(problems):
    """mantra_estimate_batch over a list of dicts with keys graph (Graph), opt,
    eps, delta, seed and optional c, growth, fixed_r, bootstrap, delta_sched,
    vhat_mode, target, estimator.  Returns a list of (est, hits, info dict, status)."""
    k = len(problems)
    arr = (Problem * k)()
    keep = []
    outs = []
    for x, p in enumerate(problems):
        g = p["graph"]
        o = Opts(p.get("c", 0), p.get("growth", 0.0), p.get("fixed_r", 0), p.get("bootstrap", 0),
                 p.get("delta_sched", 0), 0, None, p.get("vhat_mode", 0), p.get("target", 0), p.get("estimator", 0))
        F = g.family_size(p.get("target", 0))
        est = np.zeros(max(F, 1), np.float64)
        hits = np.zeros(max(F, 1), np.uint64)
        info = Info()
        keep += [o, est, hits, info]
        arr[x].graph = g.h.value if isinstance(g.h, C.c_void_p) else g.h
        arr[x].opt = _opt(p["opt"])
        arr[x].eps = p["eps"]
        arr[x].delta = p["delta"]
        arr[x].seed = p["seed"]
        arr[x].opts = C.pointer(o)
        arr[x].est_out = est.ctypes.data
        arr[x].hits_out = hits.ctypes.data
        arr[x].info = C.pointer(info)
        outs.append((est[:F], hits[:F], info))
    lib().mantra_estimate_batch(arr, k)
    return [(e, h, i.as_dict(), arr[x].status) for x, (e, h, i) in enumerate(outs)]


PENDING = 8


class Server:
    """Continuous-batching request server (mantra_server_*)."""

    def __init__(self, hbm_budget: int = 0, max_active: int = 0):
        h = C.c_void_p()
        _chk(lib().mantra_server_create(hbm_budget, max_active, C.byref(h)), "mantra_server_create")
        self.h = h
        self._n = {}

    def submit(self, graph, opt, eps, delta, seed, c=0, growth=0.0, fixed_r=0, bootstrap=0, delta_sched=0,
               vhat_mode=0, target=0, estimator=0):
        o = Opts(c, growth, fixed_r, bootstrap, delta_sched, 0, None, vhat_mode, target, estimator)
        rid = C.c_uint64()
        _chk(lib().mantra_server_submit(self.h, graph.h, _opt(opt), eps, delta, seed, C.byref(o), C.byref(rid)),
             "mantra_server_submit")
        self._n[rid.value] = graph.family_size(target)
        return rid.value

    def _result(self, rc, rid, est, hits, info):
        if rc == PENDING:
            return None
        self._n.pop(rid, None)
        _chk(rc, "mantra_server result")
        return est, hits, info.as_dict()

    def poll(self, rid):
        n = self._n[rid]
        est = np.zeros(max(n, 1), np.float64); hits = np.zeros(max(n, 1), np.uint64); info = Info()
        rc = lib().mantra_server_poll(self.h, rid, est.ctypes.data, hits.ctypes.data, C.byref(info))
        return self._result(rc, rid, est[:n], hits[:n], info)

    def wait(self, rid, timeout=0.0):
        n = self._n[rid]
        est = np.zeros(max(n, 1), np.float64); hits = np.zeros(max(n, 1), np.uint64); info = Info()
        rc = lib().mantra_server_wait(self.h, rid, timeout, est.ctypes.data, hits.ctypes.data, C.byref(info))
        return self._result(rc, rid, est[:n], hits[:n], info)

    def stats(self):
        v = [C.c_uint64() for _ in range(5)]
        _chk(lib().mantra_server_stats(self.h, *[C.byref(x) for x in v]), "mantra_server_stats")
        return dict(zip(("queued", "active", "finished", "ticks", "bytes_in_use"), [x.value for x in v]))

    def close(self):
        if getattr(self, "h", None):
            lib().mantra_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
