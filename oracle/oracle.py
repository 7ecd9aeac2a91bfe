"""ctypes wrapper of the MANTRA CPU oracle (mantra_oracle.cpp).

TEST INFRASTRUCTURE ONLY: the tests, the package smoke check and the
benchmark's CPU-baseline leg load this; the product path never does.

Optimality codes: 0 = sh (shortest), 1 = sfm (shortest-foremost),
2 = pfm (prefix-foremost), Def. 1 of the paper.
Random-stream domains: 0 PAIR, 1 PATH, 2 RADE, 3 BOOT_PAIR, 4 BOOT_PATH,
5 STATS.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mantra_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")

SH, SFM, PFM = 0, 1, 2
D_PAIR, D_PATH, D_RADE, D_BOOT_PAIR, D_BOOT_PATH, D_STATS = range(6)


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (plain -O2, no target-specific flags)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


class Info(C.Structure):
    _fields_ = [("r", C.c_uint64), ("rounds", C.c_uint64), ("omega", C.c_uint64), ("s1", C.c_uint64),
                ("bootstrap", C.c_uint64), ("sum_int_len", C.c_uint64), ("max_hits", C.c_uint64),
                ("rade_num", C.c_int64), ("xi", C.c_double), ("vhat", C.c_double), ("rho_hat", C.c_double),
                ("edges_scanned", C.c_uint64), ("sigma_adds", C.c_uint64), ("states_new", C.c_uint64),
                ("frontier_vertices", C.c_uint64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        u32p, u64p, dp = C.POINTER(C.c_uint32), C.POINTER(C.c_uint64), C.POINTER(C.c_double)
        L.orc_philox.argtypes = [u32p, u32p, u32p]
        L.orc_uniform64.argtypes = [C.c_uint64, C.c_uint64, C.c_uint64, C.c_uint32, u64p]
        L.orc_draw_pair.argtypes = [C.c_uint32, C.c_uint64, C.c_uint64, C.c_uint32, u32p, u32p]
        L.orc_rademacher.argtypes = [C.c_uint64, C.c_uint64, C.c_uint32]
        L.orc_graph_new.restype = C.c_void_p
        L.orc_graph_new.argtypes = [u32p, u32p, u32p, C.c_uint64, C.c_uint32]
        L.orc_graph_free.argtypes = [C.c_void_p]
        L.orc_graph_info.argtypes = [C.c_void_p, u32p, u64p, u64p, u64p, u64p]
        L.orc_graph_edges.argtypes = [C.c_void_p, u32p, u32p, u32p]
        L.orc_sigma.argtypes = [C.c_void_p, C.c_int, C.c_uint32, C.c_uint32, u64p, u64p, C.POINTER(C.c_int64)]
        L.orc_unrank.argtypes = [C.c_void_p, C.c_int, C.c_uint32, C.c_uint32, C.c_uint64, C.c_uint64,
                                 u32p, C.POINTER(C.c_int64), C.c_uint32, u32p]
        L.orc_samples.argtypes = [C.c_void_p, C.c_int, C.c_uint64, C.c_uint64, C.c_uint64, C.c_uint32,
                                  C.c_uint32, u32p, u32p, u64p, u64p, u32p, u32p, C.c_uint32, u32p]
        L.orc_edge_ids.argtypes = [C.c_void_p, u32p, u32p, u32p, u32p, u32p]
        L.orc_work.argtypes = [C.c_void_p, C.c_int, C.c_uint64, C.c_uint64, C.c_uint64, C.c_uint32, C.c_uint32,
                               u64p]
        L.orc_sd_bound.restype = C.c_double
        L.orc_sd_bound.argtypes = [C.c_double] * 6
        L.orc_xi_from_R.restype = C.c_double
        L.orc_xi_from_R.argtypes = [C.c_double] * 4
        L.orc_omega_bound.restype = C.c_double
        L.orc_omega_bound.argtypes = [C.c_double] * 4
        L.orc_estimate.argtypes = [C.c_void_p, C.c_int, C.c_double, C.c_double, C.c_uint64, C.c_uint32,
                                   C.c_double, C.c_uint64, C.c_uint64, C.c_int, C.c_int, C.c_int, C.c_int, dp,
                                   u64p, C.POINTER(Info)]
        L.orc_through.argtypes = [C.c_void_p, C.c_int, C.c_uint32, C.c_uint32, u64p, u64p, u64p, u64p]
        L.orc_fixed32.argtypes = [C.c_uint64] * 4
        L.orc_fixed32.restype = C.c_uint64
        L.orc_rtb_values.argtypes = [C.c_void_p, C.c_int, C.c_uint64, C.c_uint64, C.c_uint32, u64p]
        L.orc_muldiv_round.argtypes = [C.c_uint64] * 5
        L.orc_muldiv_round.restype = C.c_uint64
        L.orc_wimpy_variance_bound.argtypes = [C.c_double, C.c_double, C.c_double]
        L.orc_wimpy_variance_bound.restype = C.c_double
        L.orc_stats.argtypes = [C.c_void_p, C.c_int, C.c_uint64, C.c_uint64, C.c_int, u64p, u32p]
        L.orc_exact_bc.argtypes = [C.c_void_p, C.c_int, dp]
        L.orc_closeness.argtypes = [C.c_void_p, C.c_int, C.c_uint64, C.c_uint64, u64p, dp]
        _lib = L
    return _lib


def _p(a, ct):
    return a.ctypes.data_as(C.POINTER(ct))


class OracleError(RuntimeError):
    pass


def _chk(st):
    if st != 0:
        raise OracleError("oracle status %d" % st)


def philox(ctr, key):
    c = np.asarray(ctr, dtype=np.uint32)
    k = np.asarray(key, dtype=np.uint32)
    o = np.zeros(4, dtype=np.uint32)
    lib().orc_philox(_p(c, C.c_uint32), _p(k, C.c_uint32), _p(o, C.c_uint32))
    return [int(x) for x in o]


def uniform64(N, seed, i, domain):
    x = C.c_uint64()
    _chk(lib().orc_uniform64(N, seed, i, domain, C.byref(x)))
    return x.value


def draw_pair(n, seed, i, domain=D_PAIR):
    s, z = C.c_uint32(), C.c_uint32()
    _chk(lib().orc_draw_pair(n, seed, i, domain, C.byref(s), C.byref(z)))
    return s.value, z.value


def rademacher(seed, i, j):
    return lib().orc_rademacher(seed, i, j)


def sd_bound(Rc, W, vhat, delta, r, c):
    return lib().orc_sd_bound(Rc, W, vhat, delta, r, c)


def xi_from_R(R, vhat, delta, r):
    return lib().orc_xi_from_R(R, vhat, delta, r)


def omega_bound(vhat, rho, eps, delta):
    return lib().orc_omega_bound(vhat, rho, eps, delta)


def wimpy_variance_bound(W, delta, r):
    return lib().orc_wimpy_variance_bound(W, delta, r)


class Graph:
    """A deduplicated temporal graph held by the oracle."""

    def __init__(self, u, v, t, n: int = 0):
        u = np.ascontiguousarray(u, dtype=np.uint32)
        v = np.ascontiguousarray(v, dtype=np.uint32)
        t = np.ascontiguousarray(t, dtype=np.uint32)
        self._keep = (u, v, t)
        self.h = lib().orc_graph_new(_p(u, C.c_uint32), _p(v, C.c_uint32), _p(t, C.c_uint32), u.size, n)
        nn, m, sl, slf, dup = C.c_uint32(), C.c_uint64(), C.c_uint64(), C.c_uint64(), C.c_uint64()
        lib().orc_graph_info(self.h, C.byref(nn), C.byref(m), C.byref(sl), C.byref(slf), C.byref(dup))
        self.n, self.m, self.slots = nn.value, m.value, sl.value
        self.self_loops, self.duplicates = slf.value, dup.value

    def __del__(self):
        if getattr(self, "h", None):
            lib().orc_graph_free(self.h)
            self.h = None

    def edges(self):
        u = np.zeros(self.m, np.uint32); v = np.zeros(self.m, np.uint32); t = np.zeros(self.m, np.uint32)
        lib().orc_graph_edges(self.h, _p(u, C.c_uint32), _p(v, C.c_uint32), _p(t, C.c_uint32))
        return u, v, t

    def sigma(self, opt, s, z):
        """(sigma_sz as int, d): d = hop length (sh/sfm, 0 if unreachable) or
        fa(z) (pfm, -1 if unreachable)."""
        lo, hi, d = C.c_uint64(), C.c_uint64(), C.c_int64()
        _chk(lib().orc_sigma(self.h, opt, s, z, C.byref(lo), C.byref(hi), C.byref(d)))
        return (hi.value << 64) | lo.value, d.value

    def unrank(self, opt, s, z, x, cap=None, with_times=False):
        """Path named by x in [0, sigma_sz): vertices s..z (and, with
        with_times, the arrival time at each vertex, -1 for the source)."""
        cap = cap or (self.n + 1)
        buf = np.zeros(cap, np.uint32)
        tim = np.zeros(cap, np.int64)
        ln = C.c_uint32()
        _chk(lib().orc_unrank(self.h, opt, s, z, x & ((1 << 64) - 1), x >> 64, _p(buf, C.c_uint32),
                              _p(tim, C.c_int64), cap, C.byref(ln)))
        path = [int(q) for q in buf[:ln.value]]
        if with_times:
            return path, [int(q) for q in tim[:ln.value]]
        return path

    def samples(self, opt, seed, i0, count, dom_pair=D_PAIR, dom_path=D_PATH, cap=None, edges=False):
        """Per-sample (s, z, sigma, path) for sample indices i0..i0+count-1;
        with edges=True a fifth entry, the path's temporal edge ids."""
        cap = cap or min(self.n + 1, 4096)
        s = np.zeros(count, np.uint32); z = np.zeros(count, np.uint32)
        lo = np.zeros(count, np.uint64); hi = np.zeros(count, np.uint64)
        ln = np.zeros(count, np.uint32); paths = np.zeros(count * cap, np.uint32)
        pe = np.zeros(count * cap, np.uint32) if edges else None
        _chk(lib().orc_samples(self.h, opt, seed, i0, count, dom_pair, dom_path, _p(s, C.c_uint32),
                               _p(z, C.c_uint32), _p(lo, C.c_uint64), _p(hi, C.c_uint64), _p(ln, C.c_uint32),
                               _p(paths, C.c_uint32), cap, _p(pe, C.c_uint32) if edges else None))
        out = []
        for q in range(count):
            row = (int(s[q]), int(z[q]), (int(hi[q]) << 64) | int(lo[q]),
                   [int(x) for x in paths[q * cap:q * cap + ln[q]]])
            if edges:
                row = row + ([int(x) for x in pe[q * cap:q * cap + max(int(ln[q]) - 1, 0)]],)
            out.append(row)
        return out

    def work(self, opt, seed, i0, count, dom_pair=D_PAIR, dom_path=D_PATH):
        """Per-sample work counters of the searches (escan, eadd, snew, fseg),
        an array of shape (count, 4); definitions in mantra_oracle.cpp
        (search_work)."""
        out = np.zeros(4 * count, np.uint64)
        _chk(lib().orc_work(self.h, opt, seed, i0, count, dom_pair, dom_path, _p(out, C.c_uint64)))
        return out.reshape(count, 4)

    def edge_ids(self):
        """(u, v, t, underlying id) per temporal edge id, and the number of
        underlying edges."""
        u = np.zeros(self.m, np.uint32); v = np.zeros(self.m, np.uint32); t = np.zeros(self.m, np.uint32)
        ue = np.zeros(self.m, np.uint32); nu = C.c_uint32()
        lib().orc_edge_ids(self.h, _p(u, C.c_uint32), _p(v, C.c_uint32), _p(t, C.c_uint32), _p(ue, C.c_uint32),
                           C.byref(nu))
        return u, v, t, ue, nu.value

    def estimate(self, opt, eps, delta, seed, c=25, growth=1.2, fixed_r=0, bootstrap=0, delta_sched=0, vhat_mode=0,
                 target=0, estimator=0):
        """Algorithm 1; target 0 nodes, 1 underlying edges, 2 temporal edges;
        estimator 0 trk (App. C), 1 ob (Sec. 4.1), 2 RTB (App. C); ob and RTB
        hits are in 2^-32 units."""
        F = self.n if target == 0 else (self.edge_ids()[4] if target == 1 else self.m)
        est = np.zeros(max(F, 1), np.float64)
        hits = np.zeros(max(F, 1), np.uint64)
        info = Info()
        _chk(lib().orc_estimate(self.h, opt, eps, delta, seed, c, growth, fixed_r, bootstrap, delta_sched, vhat_mode,
                                target, estimator, _p(est, C.c_double), _p(hits, C.c_uint64), C.byref(info)))
        est, hits = est[:F], hits[:F]
        return est, hits, info.as_dict()

    def through(self, opt, s, z):
        """(sigma_sz, [sigma_sz(v) for v in range(n)]): optimal paths through v."""
        lo = np.zeros(self.n, np.uint64); hi = np.zeros(self.n, np.uint64)
        slo = C.c_uint64(); shi = C.c_uint64()
        _chk(lib().orc_through(self.h, opt, s, z, _p(lo, C.c_uint64), _p(hi, C.c_uint64), C.byref(slo),
                               C.byref(shi)))
        return (shi.value << 64) | slo.value, [(int(b) << 64) | int(a) for a, b in zip(lo, hi)]

    def rtb_values(self, opt, seed, i, dom=D_PAIR):
        """RTB values f_v(s) of sample i in 2^-32 units (n entries)."""
        q = np.zeros(self.n, np.uint64)
        _chk(lib().orc_rtb_values(self.h, opt, seed, i, dom, _p(q, C.c_uint64)))
        return q

    def closeness(self, opt, seed, r_s):
        """(per-vertex sums of round(2^32 / d), closeness estimates) over
        Algorithm 2's r_s sources."""
        sm = np.zeros(self.n, np.uint64); cl = np.zeros(self.n, np.float64)
        _chk(lib().orc_closeness(self.h, opt, seed, r_s, _p(sm, C.c_uint64), _p(cl, C.c_double)))
        return sm, cl

    def stats_counts(self, opt, seed, r_s, all_sources=False):
        """(reach[0..D_LB], D_LB): cumulative reach counts per hop (Algorithm 2)."""
        reach = np.zeros(max(self.n, 1), np.uint64)
        d = C.c_uint32()
        _chk(lib().orc_stats(self.h, opt, seed, r_s, 1 if all_sources else 0, _p(reach, C.c_uint64),
                             C.byref(d)))
        return reach[:d.value + 1].copy(), d.value

    def exact_bc(self, opt):
        bc = np.zeros(self.n, np.float64)
        _chk(lib().orc_exact_bc(self.h, opt, _p(bc, C.c_double)))
        return bc


def stats_summary(reach, d_lb, n, r_s, tau=0.9):
    """Host formulas of Algorithm 2 from integer reach counts:
    Rhat[h] = (n / r_s) R[h]; Psi = sum_{h=1}^{D_LB} (Rhat[h]-Rhat[h-1]) h / Rhat[D_LB];
    D_tau = min{h : Rhat[h]/Rhat[D_LB] >= tau}; zeta = Rhat[D_LB] / (n(n-1));
    rho = zeta * (Psi - 1) (mean internal-node count over all ordered pairs)."""
    Rh = [(n / r_s) * float(x) for x in reach]
    top = Rh[d_lb]
    if top == 0.0:
        return {"d_lb": d_lb, "d_tau": 0, "zeta": 0.0, "psi": 0.0, "rho": 0.0}
    psi = 0.0
    for h in range(1, d_lb + 1):
        psi += (Rh[h] - Rh[h - 1]) * h
    psi /= top
    d_tau = next(h for h in range(d_lb + 1) if Rh[h] / top >= tau)
    zeta = top / (n * (n - 1))
    return {"d_lb": d_lb, "d_tau": d_tau, "zeta": zeta, "psi": psi, "rho": zeta * (psi - 1.0)}


def sample_size_bootstrap(eps, delta):
    """s' = ceil(ln(1/delta) / eps) (footnote of Sec. 4.4)."""
    return int(math.ceil(math.log(1.0 / delta) / eps))


def fixed32(a: int, b: int) -> int:
    """The oracle's ob rounding: the integer nearest 2^32 a / b (ties up), 0 <= a <= b < 2^128."""
    M = (1 << 64) - 1
    return lib().orc_fixed32(a & M, a >> 64, b & M, b >> 64)


def muldiv_round(a: int, x: int, d: int) -> int:
    """The oracle's RTB rounding: floor(a x / d + 1/2), a <= d < 2^128, x < 2^64."""
    M = (1 << 64) - 1
    return lib().orc_muldiv_round(a & M, a >> 64, x, d & M, d >> 64)
