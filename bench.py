"""Benchmark of the MANTRA hot path on one GB300 (or N, one process each).

Workload (default): Chung-Lu temporal graph, n = 20,000, degree exponent 2.3,
500,000 bursty contacts (K ~ Geometric(0.3) per static edge, Exp(mean 1000)
gaps, t in [0, 1e6]); progressive MCERA sampling at eps = 0.01, delta = 0.1,
c = 25.  One step = one complete Algorithm 1 run (bootstrap, schedule, rounds
until the stopping rule) for each of sh, sfm and pfm with a fresh seed per
step, run as one mantra_estimate_batch (default) or as three mantra_estimate
calls (--mode sequential; also timed after the main region on the same seeds).
Metric: sampled (s,z) pairs per second, bootstrap and estimation samples of the
three optimalities together.  Inputs are synthetic (the
paper's data sets are not available).  After the timed region, one batched
step each of temporal edge betweenness (App. A), of the ob estimator
(Sec. 4.1) and of the RTB estimator (App. C; its samples are sources, so
its rate counts sources) on the same workload is reported under
secondary.next_rows (--no-next skips them).

Other workloads, after the headline, on one GPU (each leg has a flag that
skips it):
* secondary.large_graph: Chung-Lu n = 10^6, gamma 2.1, 2*10^7 edges with t
  uniform in [0, 2^24) -- one Algorithm 1 run each of sfm and pfm at
  eps = 0.005, Algorithm 2 at r_s = 256, per-kernel rooflines, the oracle on
  the host cores for pfm (--no-large);
* secondary.batch_256: 256 uneven bursty graphs in one mantra_estimate_batch
  against 256 sequential calls (--no-batch256);
* serving: 64 resident graphs (n log-spaced in [1000, 200000], m = 25 n),
  2,000 Poisson requests at 200/s, served (continuous batching) against one
  request at a time (--serve-graphs 0 skips it).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun each rank runs its own steps on its own GPU (different seeds,
no collective on the data path); value = all ranks' samples / max-rank time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

EPS, DELTA, C_TRIALS = 0.01, 0.1, 25
OPTS = ("sh", "sfm", "pfm")
OPTS_ALL = ("sh", "sfm", "pfm")
METRIC = "sampled pairs/sec at eps=0.01 (sh+sfm+pfm)"
WORKLOAD = "chung_lu_bursty n=20000 gamma=2.3 m=500000 eps=0.01 delta=0.1 c=25"
PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
TRAFFIC = os.path.join(ROOT, "profiles", "traffic.txt")


def bench_config(world: int) -> dict:
    """The config object of the bench line, the same for both arms."""
    return {"workload": WORKLOAD, "parallelism": "replicas" if world > 1 else "single",
            "l2": "GPU arm: flushed between steps (256 MiB write), per-step CUDA events; reference arm: host cores"}


def workload():
    from paper_2304_08356_gb300 import synth
    return synth.chung_lu_bursty(n=20000, m=500000, gamma=2.3, seed=1)


def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("LOCAL_RANK", "0"))


def max_over_ranks(x: float, world: int) -> float:
    """Max of a float over ranks (identity for one rank)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1])); mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


KSRC = {"k_bfs": "k_bfs.cu", "k_pfm_cta": "k_pfm_cta.cu", "k_pfm": "k_pfm.cu"}


def kernel_source_digest(kernel: str):
    """Digest of one kernel's source and the shared device header."""
    h = hashlib.sha256()
    for f in (KSRC[kernel], "mantra_dev.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2304_08356_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel: str, alg_bytes_per_launch: float):
    """DRAM bytes per launch for this kernel source, or None.

    profiles/traffic.txt holds, per kernel and source digest, the ratio of
    ncu's dram__bytes_read.sum + dram__bytes_write.sum to the library's
    algorithmic bytes over the same launches; a launch's traffic is that
    ratio times its algorithmic bytes."""
    if not os.path.exists(TRAFFIC):
        return None
    dig = kernel_source_digest(kernel.split("@")[0])
    for line in open(TRAFFIC):
        f = line.split()
        if len(f) >= 3 and not line.startswith("#") and f[0] == kernel and f[1] == dig:
            return float(f[2]) * alg_bytes_per_launch
    return None


def serving_workload(num_graphs, n_lo, n_hi, edges_per_node, num_requests, rate, seed=7):
    """Resident bursty Chung-Lu graphs (n log-spaced, m = edges_per_node * n) and
    Poisson-arriving requests: (arrival time, graph, optimality, eps, seed)."""
    from paper_2304_08356_gb300 import synth
    ns = np.unique(np.round(np.exp(np.linspace(np.log(n_lo), np.log(n_hi), num_graphs))).astype(int))
    graphs = [synth.chung_lu_bursty(n=int(n), m=edges_per_node * int(n), gamma=2.3, seed=500 + k)
              for k, n in enumerate(ns)]
    rng = np.random.default_rng(seed)
    arrivals = np.cumsum(rng.exponential(1.0 / rate, size=num_requests))
    reqs = [(float(arrivals[k]), int(rng.integers(0, len(graphs))), OPTS_ALL[int(rng.integers(0, 3))],
             float(rng.choice([0.05, 0.02, 0.01])), 10_000 + k) for k in range(num_requests)]
    return graphs, reqs


def run_serving(M, graphs_uvt, reqs):
    """p50/p99 latency and throughput of the served (continuous batching) and
    the plain one-request-at-a-time GPU paths on the same request trace."""
    import threading as th
    gs = [M.Graph(*uvt) for uvt in graphs_uvt]
    # warm both paths (workspaces, captured tick)
    for g in gs[:2]:
        g.estimate("pfm", 0.05, DELTA, 1, c=C_TRIALS)
        g.estimate("sh", 0.05, DELTA, 1, c=C_TRIALS)

    def summarize(lat, t_first, t_last, samples):
        lat = np.sort(np.array(lat))
        return {"p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
                "mean_s": float(lat.mean()), "requests_per_s": len(lat) / (t_last - t_first),
                "pairs_per_s": samples / (t_last - t_first)}

    # plain: requests in arrival order, one mantra_estimate at a time
    t0 = time.perf_counter()
    lat, samples, t_end = [], 0, t0
    for (arr, gi, opt, eps, sd) in reqs:
        now = time.perf_counter() - t0
        if now < arr:
            time.sleep(arr - now)
        _, _, info = gs[gi].estimate(opt, eps, DELTA, sd, c=C_TRIALS)
        t_end = time.perf_counter()
        lat.append(t_end - t0 - arr)
        samples += info["r"] + info["bootstrap"]
    plain = summarize(lat, t0 + reqs[0][0], t_end, samples)

    # served: submissions at arrival times, completions collected by a waiter
    srv = M.Server()
    ids = [None] * len(reqs)
    done_t = [None] * len(reqs)
    infos = [None] * len(reqs)
    t0 = time.perf_counter()

    def client():
        for k, (arr, gi, opt, eps, sd) in enumerate(reqs):
            now = time.perf_counter() - t0
            if now < arr:
                time.sleep(arr - now)
            ids[k] = srv.submit(gs[gi], opt, eps, DELTA, sd, c=C_TRIALS)

    ct = th.Thread(target=client)
    ct.start()
    pending = set(range(len(reqs)))
    while pending:
        for k in list(pending):
            if ids[k] is None:
                continue
            r = srv.poll(ids[k])
            if r is not None:
                done_t[k] = time.perf_counter()
                infos[k] = r[2]
                pending.discard(k)
        time.sleep(0.0005)
    ct.join()
    st = srv.stats()
    srv.close()
    lat = [done_t[k] - t0 - reqs[k][0] for k in range(len(reqs))]
    samples = sum(i["r"] + i["bootstrap"] for i in infos)
    served = summarize(lat, t0 + reqs[0][0], max(done_t), samples)
    served["ticks"] = st["ticks"]
    for g in gs:
        g.free()
    return plain, served


LARGE = ("chung_lu_uniform_t n=1000000 gamma=2.1 m=20000000 t<2^24; Algorithm 1 sfm and pfm at eps=0.005 "
         "delta=0.1 c=25; Algorithm 2 pfm and sfm at eps=0.01 r_s=256")
BATCH = "256 bursty Chung-Lu graphs, n log-uniform in [500, 50000], m = 20 n, optimality g mod 3, eps=0.02 delta=0.1 c=25"


def kernel_rooflines(info, opt, peak, ms=None):
    """Achieved GB/s of the search kernels of one Algorithm 1 run, from the
    library's counters (byte models of include/mantra.h) and kernel time."""
    ms = info["kernel_ms"] if ms is None else ms
    out = {}
    if opt == "pfm":
        own = 12 * info["edges_expanded"] + 24 * info["sigma_adds"]
        out["k_pfm_cta"] = {"achieved": info["alg_bytes"] / (ms / 1e3) / 1e9,
                            "achieved_own_model": own / (ms / 1e3) / 1e9,
                            "alg_bytes": info["alg_bytes"], "own_model_bytes": own, "ms": ms,
                            "launches": info["search_launches"]}
        out["k_pfm_cta"]["frac"] = out["k_pfm_cta"]["achieved"] / peak
        out["k_pfm_cta"]["frac_own_model"] = out["k_pfm_cta"]["achieved_own_model"] / peak
    else:
        out["k_bfs"] = {"achieved": info["alg_bytes"] / (ms / 1e3) / 1e9, "alg_bytes": info["alg_bytes"], "ms": ms,
                        "launches": info["search_launches"]}
        out["k_bfs"]["frac"] = out["k_bfs"]["achieved"] / peak
    for k in out:
        tr = recorded_traffic(k + "@large", out[k]["alg_bytes"] / max(1, out[k]["launches"]))
        out[k]["traffic_per_launch"] = tr
        out[k]["unit"] = "GB/s"
    return out


def run_large(M, torch, peak, cpu=True):
    """Config 3 (the HBM-bound case): one Algorithm 1 run each of sfm and pfm
    at eps = 0.005 after a warm-up, device outputs, L2 flushed before each,
    CUDA events on the library's stream; then Algorithm 2 with r_s = 256."""
    from paper_2304_08356_gb300 import synth
    u, v, t = synth.chung_lu_uniform_t(n=1_000_000, m=20_000_000, gamma=2.1, seed=1)
    g = M.Graph(u, v, t, n=1_000_000)
    tuned = g.tune()
    st = torch.cuda.Stream()
    est = torch.empty(g.n, dtype=torch.float64, device="cuda")
    hits = torch.empty(g.n, dtype=torch.int64, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    for opt in ("sfm", "pfm"):
        g.estimate(opt, 0.05, DELTA, 7, c=C_TRIALS, fixed_r=600, est_out=est.data_ptr(), hits_out=hits.data_ptr(),
                   stream=st.cuda_stream)
    torch.cuda.synchronize()
    infos, ms = {}, {}
    for opt in ("sfm", "pfm"):
        flush.zero_()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st)
        _, _, infos[opt] = g.estimate(opt, 0.005, DELTA, 2024, c=C_TRIALS, est_out=est.data_ptr(),
                                      hits_out=hits.data_ptr(), stream=st.cuda_stream)
        e1.record(st)
        e1.synchronize()
        ms[opt] = e0.elapsed_time(e1)
    stats = {}
    for opt in ("pfm", "sfm"):
        s_, _ = g.temporal_stats(opt, 0.01, 4, r_override=256)
        stats[opt] = {k: s_[k] for k in ("d_lb", "d_tau", "zeta", "psi", "r", "seconds")}
    n_s = {o: infos[o]["r"] + infos[o]["bootstrap"] for o in infos}
    roof = {}
    for o in ("sfm", "pfm"):
        roof.update(kernel_rooflines(infos[o], o, peak))
    out = {"workload": LARGE, "pairs_per_s": sum(n_s.values()) / (sum(ms.values()) / 1e3),
           "per_opt": {o: {"pairs_per_s": n_s[o] / (ms[o] / 1e3), "ms": ms[o], "r": infos[o]["r"],
                           "omega": infos[o]["omega"], "rounds": infos[o]["rounds"],
                           "temporal_edge_GBps": infos[o]["alg_bytes"] / (ms[o] / 1e3) / 1e9,
                           "edges_per_s": infos[o]["edges_scanned"] / (ms[o] / 1e3)} for o in infos},
           "algorithm2_r_s_256": stats, "roofline": roof, "autotune": tuned,
           "l2": "flushed before each run (256 MiB write); CUDA events around each Algorithm 1 run"}
    if cpu:
        # the oracle on the host cores over the first pfm estimation samples of the
        # same run (an sfm oracle search at this size takes minutes per sample)
        from oracle import oracle as O
        og = O.Graph(u, v, t, n=1_000_000)
        cores = host_cores()
        rates, counts = cpu_oracle_rates(u, v, t, 2024, budget_s=20.0, threads=cores, graph=og, opts=("pfm",))
        out["cpu_baseline"] = {"value": rates["pfm"], "unit": "pairs/s", "cores": cores, "kind": "oracle",
                               "sample": "first %d pfm estimation samples of the same seed on %d host threads, "
                                         "20 s of wall time; sfm not timed (minutes per oracle sample)"
                                         % (counts["pfm"], cores),
                               "gpu_pfm_pairs_per_s": n_s["pfm"] / (ms["pfm"] / 1e3)}
    g.free()
    del flush, est, hits
    torch.cuda.empty_cache()
    return out


def run_batch256(M, torch):
    """Config 4: 256 uneven graphs, every problem's Algorithm 1 in one
    mantra_estimate_batch (one persistent launch per kernel family and tick)
    against 256 sequential mantra_estimate calls on the same arguments."""
    from paper_2304_08356_gb300 import synth
    inst = synth.batch_instances()
    gs = [M.Graph(*uvt) for uvt in inst]
    names = ("sh", "sfm", "pfm")
    probs = [dict(graph=gs[k], opt=names[k % 3], eps=0.02, delta=DELTA, seed=77 + k, c=C_TRIALS)
             for k in range(len(gs))]
    M.estimate_batch([dict(p, seed=1) for p in probs[:8]])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    res = M.estimate_batch(probs)
    t_batch = time.perf_counter() - t0
    for r in res:
        if r[3] != 0:
            raise M.MantraError(r[3], "mantra_estimate_batch (256 graphs)")
    n_b = sum(r[2]["r"] + r[2]["bootstrap"] for r in res)
    t0 = time.perf_counter()
    n_q, same = 0, True
    for p, r in zip(probs, res):
        _, h, info = p["graph"].estimate(p["opt"], p["eps"], p["delta"], p["seed"], c=C_TRIALS)
        n_q += info["r"] + info["bootstrap"]
        same = same and bool(np.array_equal(h, r[1]))
    t_seq = time.perf_counter() - t0
    for g in gs:
        g.free()
    return {"workload": BATCH, "batched": {"pairs_per_s": n_b / t_batch, "s": t_batch},
            "sequential": {"pairs_per_s": n_q / t_seq, "s": t_seq}, "samples": n_b,
            "batched_equals_sequential": same, "timing": "host wall clock around each whole call sequence"}


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_oracle_rates(u, v, t, seed, budget_s=6.0, threads=1, graph=None, opts=None):
    """Oracle pairs/s per optimality on a bounded prefix of the estimation
    samples.  With threads > 1 the oracle's per-sample call runs on that many
    host threads over disjoint sample indices (the call releases the GIL; the
    oracle itself is unchanged), and the rate is samples / wall time."""
    from oracle import oracle as O
    g = graph if graph is not None else O.Graph(u, v, t)
    rates, counts = {}, {}
    for name in (opts or OPTS):
        opt = {"sh": 0, "sfm": 1, "pfm": 2}[name]
        k = 1 if opt != 2 else 64
        lock = threading.Lock()
        nxt = [0]
        t0 = time.perf_counter()
        deadline = t0 + budget_s

        def worker():
            done = 0
            while time.perf_counter() < deadline:
                with lock:
                    i0 = nxt[0]
                    nxt[0] += k
                g.samples(opt, seed, i0, k, cap=64)
                done += k
            return done

        if threads <= 1:
            done = worker()
        else:
            ths, res = [], [0] * threads
            for x in range(threads):
                th = threading.Thread(target=lambda x=x: res.__setitem__(x, worker()))
                th.start()
                ths.append(th)
            for th in ths:
                th.join()
            done = sum(res)
        dt = time.perf_counter() - t0
        rates[name] = done / dt
        counts[name] = done
    return rates, counts


def run_reference(args):
    """The reference arm: the CPU oracle as it stands, on the host cores."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    from oracle import oracle as O
    u, v, t = workload()
    g = O.Graph(u, v, t)
    cores = host_cores()
    per_step_budget = max(1.0, 20.0 / max(1, args.steps + args.warmup))
    for _ in range(args.warmup):
        cpu_oracle_rates(u, v, t, 1, budget_s=per_step_budget / 4, threads=cores, graph=g)
    # equal numbers of samples per optimality: time per sample triple = sum_o 1/rate_o
    tot_s, tot_n = 0.0, 0
    for k in range(args.steps):
        rates, counts = cpu_oracle_rates(u, v, t, 100 + k, budget_s=per_step_budget / 3, threads=cores, graph=g)
        tot_s += sum(1.0 / rates[o] for o in OPTS)
        tot_n += len(OPTS)
    value = tot_n / tot_s
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": 0,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * tot_s / max(1, args.steps),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic (seeded Chung-Lu bursty)", "config": bench_config(1),
            "cpu_baseline": {"value": value, "unit": "pairs/s", "cores": cores, "kind": "oracle",
                             "sample": "per step: the first estimation samples of sh, sfm and pfm on %d host "
                                       "threads, %.1f s of wall time each; equal sample counts per optimality "
                                       "(harmonic mean of the rates)" % (cores, per_step_budget / 3)},
            "e2e": {"value": value, "unit": "pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def run_probe(M, args):
    """Kernel time of fixed-r estimates (one warm run, best of 3), one JSON line."""
    from paper_2304_08356_gb300 import synth
    if args.probe_graph:
        n, m = (int(x) for x in args.probe_graph.split(","))
        u, v, t = synth.chung_lu_bursty(n=n, m=m, seed=77)
        wl = "bursty Chung-Lu n=%d, m=%d contacts, seed 77" % (n, m)
    else:
        u, v, t = workload()
        wl = WORKLOAD
    g = M.Graph(u, v, t)
    out = {}
    for name in OPTS:
        g.estimate(name, EPS, DELTA, 7, c=C_TRIALS, fixed_r=args.probe)
        best, info, hits = 1e300, None, None
        for _ in range(3):
            _, hits, info = g.estimate(name, EPS, DELTA, 7, c=C_TRIALS, fixed_r=args.probe)
            best = min(best, info["kernel_ms"])
        out[name] = {"kernel_ms": round(best, 3), "r": args.probe, "edges_expanded": info["edges_expanded"],
                     "alg_bytes": info["alg_bytes"], "hits_sha256_16": hashlib.sha256(hits.tobytes()).hexdigest()[:16]}
    print(json.dumps({"probe": out, "workload": wl,
                      "launch_env": {k: v_ for k, v_ in os.environ.items() if k.startswith("MANTRA_")}}))
    g.free()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-next", action="store_true", help="skip the edge-betweenness and ob legs")
    ap.add_argument("--opts", default="sh,sfm,pfm", help="optimalities per step (profiling subsets)")
    ap.add_argument("--serve-graphs", type=int, default=64, help="serving leg: resident graphs (0: skip)")
    ap.add_argument("--serve-requests", type=int, default=2000, help="serving leg: requests")
    ap.add_argument("--serve-nmax", type=int, default=200000, help="serving leg: largest graph's n")
    ap.add_argument("--no-large", action="store_true", help="skip the n = 10^6, m = 2*10^7 leg")
    ap.add_argument("--no-tune", action="store_true",
                    help="run the bench graph with the default launch choices (no mantra_tune probes)")
    ap.add_argument("--no-batch256", action="store_true", help="skip the 256-graph batching leg")
    ap.add_argument("--mode", default="batched", choices=["batched", "sequential"],
                    help="batched: one mantra_estimate_batch over the optimalities per step; "
                         "sequential: one mantra_estimate per optimality")
    ap.add_argument("--probe", type=int, default=0,
                    help="instead of the bench: time a fixed-r estimate of this many samples per optimality "
                         "(best kernel time of 3 after one warm run, default or MANTRA_* launch choices) and exit")
    ap.add_argument("--probe-graph", default="",
                    help="with --probe: N,M for a bursty Chung-Lu graph of N nodes and M contacts (seed 77) "
                         "instead of the bench graph")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    global OPTS
    OPTS = tuple(x for x in args.opts.split(",") if x)

    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    from paper_2304_08356_gb300 import build as B
    if rank == 0:
        B.build()
    barrier(world)
    import paper_2304_08356_gb300.mantra as M

    if args.probe:
        return run_probe(M, args)
    u, v, t = workload()
    g = M.Graph(u, v, t)
    tuned = None if args.no_tune else g.tune()   # the autotuner's launch choices (results do not depend on them)
    stream = torch.cuda.Stream()
    est_dev = torch.empty(g.n, dtype=torch.float64, device="cuda")
    hits_dev = torch.empty(g.n, dtype=torch.int64, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def step_sequential(seed):
        infos = {}
        for name in OPTS:
            _, _, info = g.estimate(name, EPS, DELTA, seed, c=C_TRIALS, est_out=est_dev.data_ptr(),
                                    hits_out=hits_dev.data_ptr(), stream=stream.cuda_stream)
            infos[name] = info
        return infos

    def step_batched(seed):
        res = M.estimate_batch([dict(graph=g, opt=name, eps=EPS, delta=DELTA, seed=seed, c=C_TRIALS)
                                for name in OPTS])
        for (_, _, _, st) in res:
            if st != 0:
                raise M.MantraError(st, "mantra_estimate_batch")
        return {name: r[2] for name, r in zip(OPTS, res)}

    step = step_batched if args.mode == "batched" else step_sequential

    seed0 = 1_000_003 * (rank + 1)
    for w in range(args.warmup):
        step(seed0 + w)
    torch.cuda.synchronize()

    # ---------------- device-resident timed region ----------------
    infos_all, ms_steps = [], []
    with ClockSampler(torch.cuda.current_device()) as clk:
        barrier(world)
        torch.cuda.synchronize()
        for k in range(args.steps):
            flush.zero_()                    # L2 flush between steps (256 MiB write), outside the events
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            infos_all.append(step(seed0 + 1000 + k))
            e1.record(stream)
            e1.synchronize()
            ms_steps.append(e0.elapsed_time(e1))
        torch.cuda.synchronize()
        barrier(world)
    total_ms = sum(ms_steps)
    samples = sum(i["r"] + i["bootstrap"] for st in infos_all for i in st.values())
    t_max = max_over_ranks(total_ms / 1000.0, world)
    samples_all = sum_over_ranks(float(samples), world)
    value = samples_all / t_max

    # sequential pass on the same seeds: one mantra_estimate per optimality, each
    # tick running a single kernel family -- its tick times give the per-kernel
    # durations of the roofline, and its rate is the plain (unbatched) figure
    seq_infos, seq_ms = [], []
    n_seq = min(args.steps, 2)
    for k in range(n_seq):
        flush.zero_()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        seq_infos.append(step_sequential(seed0 + 1000 + k))
        e1.record(stream)
        e1.synchronize()
        seq_ms.append(e0.elapsed_time(e1))
    seq_rate = sum(i["r"] + i["bootstrap"] for st in seq_infos for i in st.values()) / (sum(seq_ms) / 1000.0)

    # the same workload for the other estimators (edge betweenness over the
    # temporal edges, App. A; the ob estimator, Sec. 4.1; the RTB estimator,
    # App. C, whose samples are sources): one batched step each
    next_rows = {}
    for label, kw in (() if args.no_next else (("edge_betweenness_temporal", dict(target=2)),
                                               ("ob_estimator", dict(estimator=1)),
                                               ("rtb_estimator", dict(estimator=2)))):
        flush.zero_()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        res = M.estimate_batch([dict(graph=g, opt=name, eps=EPS, delta=DELTA, seed=seed0 + 1000, c=C_TRIALS, **kw)
                                for name in OPTS])
        e1.record(stream)
        e1.synchronize()
        for (_, _, _, st) in res:
            if st != 0:
                raise M.MantraError(st, "mantra_estimate_batch (%s)" % label)
        ms = e0.elapsed_time(e1)
        n_s = sum(r[2]["r"] + r[2]["bootstrap"] for r in res)
        next_rows[label] = {"pairs_per_s": n_s / (ms / 1000.0), "ms": ms,
                            "r": {o: r[2]["r"] for o, r in zip(OPTS, res)},
                            "kernel_ms": {o: r[2]["kernel_ms"] for o, r in zip(OPTS, res)}}

    # dominant kernel: search time per optimality family (sequential pass)
    pfm_kernel = "k_pfm" if os.environ.get("MANTRA_PFM_KERNEL") == "lane" else "k_pfm_cta"
    fam = {k: tuple(o for o in v_ if o in OPTS) for k, v_ in {"k_bfs": ("sh", "sfm"), pfm_kernel: ("pfm",)}.items()}
    fam = {k: v_ for k, v_ in fam.items() if v_}
    kms = {k: sum(st[o]["kernel_ms"] for st in seq_infos for o in os_) for k, os_ in fam.items()}
    kbytes = {k: sum(st[o]["alg_bytes"] for st in seq_infos for o in os_) for k, os_ in fam.items()}
    klaunch = {k: sum(st[o]["search_launches"] for st in seq_infos for o in os_) for k, os_ in fam.items()}
    dom = max(kms, key=kms.get)
    peaks = json.load(open(PEAKS)) if os.path.exists(PEAKS) else {}
    peak = peaks.get("hbm_gbs", 6800.0)
    achieved = (kbytes[dom] / klaunch[dom]) / (kms[dom] / klaunch[dom] / 1000.0) / 1e9
    traffic = recorded_traffic(dom, kbytes[dom] / klaunch[dom])
    alg_gbps = sum(st[o]["alg_bytes"] for st in infos_all for o in OPTS) / (total_ms / 1000.0) / 1e9
    edges = sum(st[o]["edges_scanned"] for st in infos_all for o in OPTS)
    launches = sum(st[o]["kernel_launches"] for st in infos_all for o in OPTS)

    # ---------------- end to end through the C ABI with host buffers ----------------
    pin_u = torch.from_numpy(u).pin_memory().numpy()
    pin_v = torch.from_numpy(v).pin_memory().numpy()
    pin_t = torch.from_numpy(t).pin_memory().numpy()
    e2e_s, e2e_n = 0.0, 0
    barrier(world)
    for k in range(0 if args.no_e2e else max(1, min(args.steps, 2))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g2 = M.Graph(pin_u, pin_v, pin_t)
        if args.mode == "batched":
            res = M.estimate_batch([dict(graph=g2, opt=name, eps=EPS, delta=DELTA, seed=seed0 + 5000 + k,
                                         c=C_TRIALS) for name in OPTS])
            e2e_n += sum(r[2]["r"] + r[2]["bootstrap"] for r in res)
        else:
            for name in OPTS:
                est, hits, info = g2.estimate(name, EPS, DELTA, seed0 + 5000 + k, c=C_TRIALS)
                e2e_n += info["r"] + info["bootstrap"]
        g2.free()
        e2e_s += time.perf_counter() - t0
    e2e_val = sum_over_ranks(float(e2e_n), world) / max(max_over_ranks(e2e_s, world), 1e-9)
    # the store's 17 uint32 arrays (9 of m entries, 4 of A, 4 of n, 3 extra
    # row ends) go up; each problem's est (f64) and hits (u64) come back
    h2d = 4 * (9 * g.m + 4 * g.slots + 4 * g.n + 3)
    d2h = len(OPTS) * 16 * g.n

    serving = None
    if args.serve_graphs > 0 and rank == 0:
        sg, sr = serving_workload(args.serve_graphs, 1000, args.serve_nmax, 25, args.serve_requests, 200.0)
        plain, served = run_serving(M, sg, sr)
        serving = {"workload": "%d resident bursty Chung-Lu graphs, n log-spaced in [1000, %d], m = 25 n; "
                               "%d Poisson requests at 200/s, optimality uniform, eps uniform in "
                               "{0.05, 0.02, 0.01}, delta 0.1" % (len(sg), args.serve_nmax, len(sr)),
                   "served": served, "plain": plain}

    large = batch256 = None
    if rank == 0 and world == 1:
        if not args.no_large:
            large = run_large(M, torch, peak, cpu=not args.no_cpu_baseline)
        if not args.no_batch256:
            batch256 = run_batch256(M, torch)

    line = None
    if rank == 0:
        cpu = None
        if not args.no_cpu_baseline and world == 1:
            from oracle import oracle as O
            og = O.Graph(u, v, t)
            cores = host_cores()
            per_opt = {o: sum(st[o]["r"] + st[o]["bootstrap"] for st in infos_all) for o in OPTS}
            rates1, counts1 = cpu_oracle_rates(u, v, t, 1, budget_s=3.0, graph=og)
            rates, counts = cpu_oracle_rates(u, v, t, 1, budget_s=3.0, threads=cores, graph=og)
            t_cpu = sum(per_opt[o] / rates[o] for o in OPTS)
            t_cpu1 = sum(per_opt[o] / rates1[o] for o in OPTS)
            cpu = {"value": sum(per_opt.values()) / t_cpu, "unit": "pairs/s", "cores": cores, "kind": "oracle",
                   "sample": "first %d/%d/%d estimation samples (sh/sfm/pfm) on %d host threads, 3 s of wall time "
                             "each, weighted by the GPU run's per-optimality sample counts"
                             % (counts["sh"], counts["sfm"], counts["pfm"], cores),
                   "per_opt_pairs_per_s": {o: round(rates[o], 2) for o in OPTS},
                   "single_thread": {"value": sum(per_opt.values()) / t_cpu1, "cores": 1,
                                     "sample": "first %d/%d/%d samples, 3 s each"
                                               % (counts1["sh"], counts1["sfm"], counts1["pfm"])}}
        line = {"metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": t_max * 1000.0 / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic (seeded Chung-Lu bursty)",
                "config": bench_config(world),
                "secondary": {"samples_per_step": samples / args.steps,
                              "per_opt_r": {o: [st[o]["r"] for st in infos_all] for o in OPTS},
                              "temporal_edge_GBps": alg_gbps, "edges_per_s": edges / (total_ms / 1000.0),
                              "sequential_pairs_per_s": seq_rate, "sequential_kernel_ms": kms,
                              "mode": args.mode, "next_rows": next_rows, "autotune": tuned,
                              "large_graph": large, "batch_256": batch256},
                "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                             "frac": achieved / peak, "traffic": traffic, "timing": "sequential pass, tick events",
                             "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)" if peaks else "fallback"},
                "cpu_baseline": cpu,
                "e2e": {"value": e2e_val, "unit": "pairs/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
                "gpu_launches": launches,
                "serving": serving,
                "clocks": clk.summary()}
        print(json.dumps(line))
    g.free()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
