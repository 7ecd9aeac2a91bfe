"""Pins of the oracle's progressive-sampling control (paper Sec. 4.4,
Algorithm 1; Theorem 1; the closed form of omega at the end of the proof of
Theorem 3), each recomputed here from the per-sample paths with Python's own
arithmetic, and each chosen so that the plausible slip named in its docstring
changes the compared value.  No GPU."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2304_08356_gb300 import synth

C_TRIALS = 25


def _graph():
    u, v, t = synth.chung_lu_bursty(n=400, m=6000, seed=3)
    return O.Graph(u, v, t)


def _recount(g, opt, seed, count, dom_pair, dom_path, c=C_TRIALS):
    """(hits, S, sum of internal lengths) over samples 0..count-1, from the
    oracle's per-sample paths and the Rademacher bits of each sample's block."""
    n = g.n
    H = np.zeros(n, np.int64)
    S = np.zeros((c, n), np.int64)
    tot = 0
    for i, (_, _, _, p) in enumerate(g.samples(opt, seed, 0, count, dom_pair=dom_pair, dom_path=dom_path)):
        inner = p[1:-1]
        if not inner:
            continue
        w = O.philox([i & 0xFFFFFFFF, i >> 32, O.D_RADE, 0], [seed & 0xFFFFFFFF, seed >> 32])
        lam = np.array([1 if (w[j >> 5] >> (j & 31)) & 1 else -1 for j in range(c)], np.int64)
        for x in inner:
            H[x] += 1
            S[:, x] += lam
        tot += len(inner)
    return H, S, tot


def _xi(NR, H, r, c, delta_i):
    """Theorem 1: xi from the c-MCERA numerator N_R, the largest hit count H
    (wimpy variance W = H / r, vhat = W) and the round's confidence delta_i."""
    L = math.log(4.0 / delta_i)
    Rc = NR / (c * r)
    W = H / r
    Rt = Rc + math.sqrt(4.0 * W * L / (c * r))
    R = Rt + L / r + math.sqrt((L / r) ** 2 + 2.0 * L * Rt / r)
    return 2.0 * R + math.sqrt(2.0 * L * (W + 4.0 * R) / r) + L / (3.0 * r)


def _xi_r0(v0, delta_1, s):
    """Theorem 1's xi with the Rademacher bound set to 0 (the bootstrap's
    schedule test of Sec. 4.4)."""
    L = math.log(4.0 / delta_1)
    return 2.0 * 0.0 + math.sqrt(2.0 * L * (v0 + 4.0 * 0.0) / s) + L / (3.0 * s)


def _bootstrap(g, opt, seed, eps, delta):
    sb = int(math.ceil(math.log(1.0 / delta) / eps))
    H, _, tot = _recount(g, opt, seed, sb, O.D_BOOT_PAIR, O.D_BOOT_PATH)
    v0 = int(H.max()) / sb
    rho = tot / sb
    return sb, v0, rho


def _omega(v0, rho, eps, delta_omega):
    return math.ceil(((2.0 * v0 + 2.0 * eps / 3.0) / eps ** 2) * (math.log(2.0 * rho / v0) + math.log(1.0 / delta_omega)))


@pytest.mark.parametrize("opt,eps,seed", [(0, 0.05, 5), (1, 0.04, 2), (2, 0.03, 7)])
def test_omega_uses_half_delta_and_the_bootstrap(opt, eps, seed):
    """omega = ceil(((2 v0 + 2 eps/3) / eps^2)(ln(2 rho / v0) + ln(2/delta)))
    with v0 = max bootstrap hits / s' and rho = mean internal length of the s'
    bootstrap paths (Algorithm 1 calls the sample-size bound with delta/2).
    Slips caught: delta instead of delta/2; v0 or rho from the wrong samples."""
    g = _graph()
    delta = 0.1
    _, _, info = g.estimate(opt, eps, delta, seed)
    sb, v0, rho = _bootstrap(g, opt, seed, eps, delta)
    assert info["bootstrap"] == sb
    assert info["rho_hat"] == pytest.approx(rho, rel=1e-12)
    want = _omega(v0, rho, eps, delta / 2.0)
    assert info["omega"] == want
    assert _omega(v0, rho, eps, delta) != want          # the case separates delta from delta/2


@pytest.mark.parametrize("sched", [0, 1])
@pytest.mark.parametrize("opt,eps,seed", [(0, 0.05, 5), (1, 0.04, 2), (2, 0.03, 7), (0, 0.02, 11)])
def test_s1_is_the_least_size_meeting_eps_with_r_zero(opt, eps, seed, sched):
    """s_1 = the least s in [s', omega] with xi(R = 0; v0, delta_1, s) <= eps,
    found here by a linear scan (the oracle bisects); omega when none; delta_1
    = delta/4 (delta/2^(i+1), i = 1), or delta/2 with the printed schedule.
    Slips caught: an off-by-one bisection, delta_1 = delta/2^i in the default
    schedule, v0 taken after the degenerate-case adjustment wrongly."""
    g = _graph()
    delta = 0.1
    _, _, info = g.estimate(opt, eps, delta, seed, delta_sched=sched)
    sb, v0, rho = _bootstrap(g, opt, seed, eps, delta)
    omega = info["omega"]
    d1 = delta / 4.0 if sched == 0 else delta / 2.0
    s1 = next((s for s in range(sb, omega + 1) if _xi_r0(v0, d1, s) <= eps), omega)
    if sb >= omega:
        s1 = omega
    assert info["s1"] == s1
    assert sb < s1 < omega                               # the scan ends strictly inside the range
    other = delta / 2.0 if sched == 0 else delta / 4.0
    s1_other = next((s for s in range(sb, omega + 1) if _xi_r0(v0, other, s) <= eps), omega)
    assert s1_other != s1                                # the case separates the two schedules
    # the boundary is not a near-tie in double precision
    assert abs(_xi_r0(v0, d1, s1) - eps) > 1e-9 * eps


@pytest.mark.parametrize("sched", [0, 1])
@pytest.mark.parametrize("opt,eps,seed", [(0, 0.05, 5), (1, 0.04, 2), (0, 0.04, 7)])
def test_round_i_reports_theorem1_at_delta_over_2_pow_i_plus_1(opt, eps, seed, sched):
    """After the last round i the reported xi is Theorem 1 at delta_i =
    delta/2^(i+1) (delta/2^i with the printed schedule), with N_R and H
    recounted from the r estimation paths; the round count follows the
    schedule s_i = min(omega, ceil(1.2 s_(i-1))) from s_1.  Slips caught:
    delta/2^i in the default schedule (or the reverse), a round index off by
    one, N_R or H taken over the wrong samples."""
    g = _graph()
    delta = 0.1
    _, hits, info = g.estimate(opt, eps, delta, seed, delta_sched=sched)
    r, rounds = info["r"], info["rounds"]
    assert rounds >= 2
    H, S, tot = _recount(g, opt, seed, r, O.D_PAIR, O.D_PATH)
    assert np.array_equal(hits.astype(np.int64), H)
    NR = int(S.max(axis=1).sum())
    assert info["rade_num"] == NR and info["max_hits"] == int(H.max()) and info["sum_int_len"] == tot
    di = delta / 2.0 ** (rounds + 1) if sched == 0 else delta / 2.0 ** rounds
    want = _xi(NR, int(H.max()), r, C_TRIALS, di)
    assert info["xi"] == pytest.approx(want, rel=1e-12)
    off = _xi(NR, int(H.max()), r, C_TRIALS, di * 2.0)   # the index one round off
    assert abs(off - want) > 1e-6 * want
    s = info["s1"]
    for _ in range(rounds - 1):
        s = min(info["omega"], math.ceil(1.2 * s))
    assert s == r
    # stopping rule: every earlier round had r < omega and xi > eps (checked
    # on the round before the last, recounted the same way)
    prev = info["s1"]
    for _ in range(rounds - 2):
        prev = min(info["omega"], math.ceil(1.2 * prev))
    Hp, Sp, _ = _recount(g, opt, seed, prev, O.D_PAIR, O.D_PATH)
    dp = delta / 2.0 ** rounds if sched == 0 else delta / 2.0 ** (rounds - 1)
    assert prev < info["omega"]
    assert _xi(int(Sp.max(axis=1).sum()), int(Hp.max()), prev, C_TRIALS, dp) > eps
