/*
 * mantra.h -- C ABI of the GB300 MANTRA library (libmantra.so).
 *
 * MANTRA (arXiv 2304.08356) estimates the temporal betweenness of every node
 * of a directed temporal graph by sampling node pairs, drawing one optimal
 * temporal path per pair and counting how often each node is an internal
 * node of the drawn paths; progressive sampling stops when a bound built on
 * Monte Carlo Empirical Rademacher Averages (c-MCERA) reaches the target
 * accuracy.  All per-sample work runs in CUDA kernels for sm_103a.
 *
 * Conventions (every call):
 *   - returns a status code (MANTRA_OK = 0); nothing is thrown across the ABI;
 *   - output buffers are caller-allocated HOST memory unless stated otherwise;
 *   - a graph handle is owned by the library until mantra_graph_free; calls
 *     on one graph are serialised by the library (a graph may be shared
 *     between threads);
 *   - sample i of a run uses Philox4x32-10 blocks with key = seed and counter
 *     (i_lo, i_hi, domain, attempt), so a result depends only on
 *     (graph, optimality, eps, delta, seed, options), never on launch shape.
 *
 * Optimalities (paper Sec. 3, Def. 1): MANTRA_SH shortest; MANTRA_SFM
 * shortest-foremost (minimum hops, then earliest arrival at z -- the reading
 * fixed by the worked example in the paper's App. A figure); MANTRA_PFM
 * prefix-foremost; MANTRA_FSFM the other reading of Def. 1(2), Buss et al.'s
 * order: the earliest arrival at z first, then the fewest hops among those
 * paths (Algorithm 2 distance: the hops of v's earliest appearance).  A
 * temporal path uses strictly increasing times and starts
 * at (s, -inf); identical (u,v,t) triples are one edge; self loops are
 * dropped.
 */
#ifndef MANTRA_H
#define MANTRA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mantra_graph mantra_graph; /* opaque, device resident */

typedef enum { MANTRA_SH = 0, MANTRA_SFM = 1, MANTRA_PFM = 2, MANTRA_FSFM = 3 } mantra_opt;

enum {
    MANTRA_OK = 0,
    MANTRA_E_INVAL = 1,    /* bad argument (NULL pointer, eps/delta outside (0,1), n < 2, id >= n, c outside [1,128], time > 2^32-3) */
    MANTRA_E_NOMEM = 2,    /* device or host allocation failed */
    MANTRA_E_OVERFLOW = 3, /* a path count sigma_sz exceeded 2^128 - 1 */
    MANTRA_E_CUDA = 4,     /* a CUDA runtime call failed */
    MANTRA_E_TIMEOUT = 5,  /* a bounded wait gave up: the staged pfm variant's wait for its bulk copies,
                              or mantra_server_wait */
    MANTRA_E_CHECK = 6,    /* an internal consistency check failed on the device */
    MANTRA_E_RNG = 7,      /* 65536 consecutive rejections in a uniform draw */
    MANTRA_PENDING = 8     /* serving: the request has not finished yet (not an error) */
};

/* Options of mantra_estimate (paper Algorithm 1).  Zero-initialise and set
 * fields, or pass NULL for the defaults. */
typedef struct {
    uint32_t c;          /* Monte Carlo trials of the c-MCERA; 0 = 25 (paper Sec. 5) */
    double growth;       /* geometric schedule factor s_i = growth * s_{i-1}; 0 = 1.2 */
    uint64_t fixed_r;    /* > 0: no bootstrap and no stopping test, exactly fixed_r samples */
    uint64_t bootstrap;  /* bootstrap sample count s'; 0 = ceil(ln(1/delta)/eps) */
    int delta_sched;     /* 0: round i uses delta/2^(i+1) (union bound totals delta); 1: delta/2^i as printed */
    int out_device;      /* 1: est_out / hits_out are DEVICE pointers (no device-to-host copy) */
    void* stream;        /* cudaStream_t to run on; NULL = the graph's own stream */
    int vhat_mode;       /* 0: the variance term of xi is the empirical wimpy variance W (as Algorithm 1
                            passes it); 1: the appendix's variance bound from W,
                            W + L/r + sqrt((L/r)^2 + 2 W L / r) with L = ln(2/delta_i), the round's
                            delta_i split evenly between it and xi */
    int target;          /* what is estimated (paper App. A): 0 = temporal betweenness of the n
                            nodes (Sec. 3); 1 = of the underlying edges (u,v), one entry per
                            distinct ordered pair with a temporal edge, id = rank in (v,u) order;
                            2 = of the m temporal edges, id = rank in (v,t,u) order.  An edge
                            counts once for every sampled path that traverses it, first and last
                            edge included.  Ids: mantra_graph_edges. */
    int estimator;       /* 0 = trk (App. C): hits of one drawn optimal path per sample; 1 = ob
                            (Sec. 4.1, target 0 only): every vertex v gets f_v = sigma_sz(v) /
                            sigma_sz, the share of the optimal s-z paths with v internal, carried
                            as the nearest multiple of 2^-32 (ties up) so that all sums are exact
                            integers.  With ob, hits_out, info->max_hits (largest sum of the
                            rounded f_v^2), info->rade_num and info->sum_int_len are in units of
                            2^-32, est = hits / (r 2^32), and c * r must stay below 2^31
                            (MANTRA_E_INVAL for fixed_r, or when omega exceeds it).  2 = RTB
                            (App. C, target 0 only): a sample is a source s drawn uniformly
                            from the n vertices and every v != s gets f_v(s) = 1/(n-1) sum_z
                            sigma_sz(v) / sigma_sz, from one untruncated search and a backward
                            dependency accumulation in which every term is rounded to 2^-32;
                            units and limits as for ob. */
} mantra_opts;

/* Diagnostics of one mantra_estimate call. */
typedef struct {
    uint64_t r;              /* samples in the estimate (|S_i| at the stop) */
    uint64_t rounds;         /* progressive-sampling rounds */
    uint64_t omega;          /* sample-size cap omega (0 with fixed_r) */
    uint64_t s1;             /* first schedule size s_1 */
    uint64_t bootstrap;      /* bootstrap samples s' */
    uint64_t sum_int_len;    /* sum over samples of |Int(tp_i)| (= sum_v hits_v) */
    uint64_t max_hits;       /* H = max_v hits_v */
    int64_t rade_num;        /* N_R = sum_j max_v S[j][v] */
    double xi;               /* final supremum-deviation bound (Theorem 1) */
    double vhat;             /* final variance term of xi: W = H / r, or its bound (vhat_mode 1) */
    double rho_hat;          /* bootstrap estimate of the mean internal length */
    /* Work counters, summed over every sample of the call (bootstrap included).
     * Per sh / sfm sample (levels F_k = the states (v,t) at hop level k with t <
     * tz = z's latest in-edge time, F_0 = {(s,-inf)}; the search stops on the
     * level that reaches z, or when F_k is empty):
     *   edges_scanned = per level k that is searched: z's in-edges (the pull
     *                   test), plus, when level k is pushed, every out-edge
     *                   (u,v,t) of each vertex u of F_k with t' < t < tz for
     *                   u's earliest t' in F_k (all out-edges of s at k = 0);
     *   sigma_adds    = those pushed edges whose head (v,t) is new on level k+1;
     *   states_new    = |F_1| + ... + |F_K| over the pushed levels' successors;
     *   frontier_vertices = distinct vertices of every searched level (1 for F_0).
     * fsfm has no pull test and pushes out-edges with t <= tz.  Per pfm sample
     * (fa = earliest arrival, te = fa(z), or tz when z is unreachable):
     *   edges_scanned = time-sorted edges (u,v,t) with v != s and
     *                   tmin_out(s) <= t <= te (the paper's scan window);
     *   sigma_adds    = prefix-foremost DAG edges (w,v,fa(v)), v != s,
     *                   fa(w) < fa(v) <= te;  states_new = frontier_vertices = 0.
     * Samples with no out-edge at s or no in-edge at z count nothing. */
    uint64_t edges_scanned;  /* E_scan (above) */
    uint64_t sigma_adds;     /* U (above) */
    uint64_t states_new;     /* S_new (above) */
    uint64_t wide_samples;   /* samples re-run with 128-bit path counts */
    double seconds;          /* wall time of the call */
    double kernel_ms;        /* device time of the search kernels (CUDA events) */
    uint64_t search_launches;/* search-kernel launches */
    uint64_t kernel_launches;/* all kernel launches of the call (search, reduction, normalisation) */
    uint64_t alg_bytes;      /* algorithmic bytes of the search kernels (64-bit path counts):
                                sh / sfm: 24 * edges_scanned (12 B edge record, 4 B level test, 8 B
                                path-count update) + 8 * frontier_vertices (row bounds) + 12 *
                                states_new (state set-up and frontier entry);
                                pfm: 4 * edges_scanned (fa(u) per sample and edge) + 12 *
                                edges_scanned / 32 (the edge record, shared by 32 samples) + 24 *
                                sigma_adds (sigma(u) read, sigma(v) read-modify-write) */
    uint64_t frontier_vertices; /* F (above) */
    uint64_t edges_expanded; /* pfm, one CTA per sample (the default pfm kernel): out-edges walked by
                                the earliest-arrival rounds plus prefix-foremost DAG edges walked by the
                                path-count pass; that kernel's own algorithmic bytes are 12 per walked
                                edge (8 B record, 4 B arrival test or count read) + 24 * sigma_adds.
                                0 for sh / sfm and for the stream-scan kernel */
} mantra_info;

/* Output of mantra_temporal_stats (paper App. D, Algorithm 2). */
typedef struct {
    uint32_t d_lb;   /* largest hop distance seen (diameter lower bound D_LB) */
    uint32_t d_tau;  /* effective diameter: least h with Rhat[h]/Rhat[D_LB] >= tau */
    double zeta;     /* temporal connectivity rate Rhat[D_LB] / (n(n-1)) */
    double psi;      /* average temporal distance over connected pairs */
    double rho;      /* zeta * (psi - 1): mean internal-node count over all ordered pairs */
    uint64_t r;      /* number of sampled sources r_s */
    double seconds;
} mantra_tstats;

/* Build the device-resident temporal-edge store from m host triples.
 * u, v, t: host arrays of m entries (copied; the caller keeps ownership).
 * n: number of nodes; 0 = max id + 1.  Ids must be < n, times <= 2^32-3,
 * fewer than 2^32-16 triples without self loops (else MANTRA_E_INVAL).
 * Duplicate triples are kept once, self loops dropped (counts reported by
 * mantra_graph_info).  The store is built on up to 16 host threads into
 * host buffers that the device's engine keeps for later loads (page-locked
 * while at most 256 MB, then uploaded by DMA).  Paper Sec. 3 (temporal
 * graph). */
int mantra_graph_load(const uint32_t* u, const uint32_t* v, const uint32_t* t, uint64_t m, uint32_t n,
                      mantra_graph** out);

/* Sizes: n, deduplicated edges, arrival slots (distinct (v,t) with an in-edge),
 * dropped self loops, dropped duplicates.  Any output pointer may be NULL. */
int mantra_graph_info(const mantra_graph* g, uint32_t* n, uint64_t* m_dedup, uint64_t* slots,
                      uint64_t* self_loops_dropped, uint64_t* duplicates_dropped);

/* The edge ids of mantra_opts.target 1 and 2 (paper App. A).  Temporal edge
 * e (0 <= e < m_dedup) is (u_out[e], v_out[e], t_out[e]); the m_dedup triples
 * come in (v, t, u) order, so e is the triple's rank in that order.
 * uedge_out[e] is the id of its underlying edge (u,v): the rank of (v,u) among
 * the distinct ordered pairs, sorted by v then u; *n_underlying receives their
 * number.  u_out, v_out, t_out, uedge_out: host arrays of m_dedup entries
 * (may be NULL only when m_dedup = 0). */
int mantra_graph_edges(const mantra_graph* g, uint32_t* u_out, uint32_t* v_out, uint32_t* t_out,
                       uint32_t* uedge_out, uint32_t* n_underlying);

void mantra_graph_free(mantra_graph* g);

/* Algorithm 1 (MANTRA): progressive sampling of (s,z) pairs with the
 * temporal Riondato-Kornaropoulos estimator (App. C), c-MCERA stopping rule
 * (Theorem 1) and sample cap omega (Theorem 3's closed form).
 * est_out: F doubles, est_x = hits_x / r (IEEE division), where F is the size
 * of the estimated family (opts->target: n nodes, the underlying edges, or
 * m_dedup temporal edges); nothing is written when F = 0.  hits_out: F
 * uint64 or NULL.  info: or NULL.  With opts->out_device = 1 both outputs are
 * device pointers.  Returns MANTRA_E_INVAL for eps/delta outside (0,1),
 * c outside [1,128], r >= 2^31. */
int mantra_estimate(const mantra_graph* g, mantra_opt opt, double eps, double delta, uint64_t seed,
                    const mantra_opts* opts, double* est_out, uint64_t* hits_out, mantra_info* info);

/* One problem of mantra_estimate_batch: the arguments of mantra_estimate,
 * plus the per-problem status written by the call. */
typedef struct {
    const mantra_graph* graph;
    mantra_opt opt;
    double eps, delta;
    uint64_t seed;
    const mantra_opts* opts;   /* NULL = defaults; stream is ignored */
    double* est_out;           /* F entries (see mantra_estimate; host, or device with opts->out_device) */
    uint64_t* hits_out;        /* F entries or NULL */
    mantra_info* info;         /* or NULL */
    int status;                /* out: this problem's status code */
} mantra_problem;

/* Algorithm 1 for `count` problems at once (batched, on one device).  Every
 * launch carries the pending samples of all unfinished problems: one
 * persistent launch per search kernel over a device task table (graph,
 * sample range), one reduction for all problems' rounds, one readback; each
 * problem follows its own bootstrap, schedule and stopping rule, so each
 * result is identical to mantra_estimate on the same arguments.  Returns the
 * first failing problem's status (each problem's own status is in .status). */
int mantra_estimate_batch(mantra_problem* probs, uint32_t count);

/* Autotuner (no counterpart in the paper; it sets how the library runs, not
 * what it computes).  For one graph it times the launch choices of the two
 * search kernels on probes -- fixed-r estimates of the graph itself, one per
 * candidate and the same seed for all, each timed by the library's CUDA events
 * -- and keeps the fastest for that graph:
 *   sh / sfm (k_bfs): CTA size 256, 512 or 1024 threads (how many samples run
 *     at once per SM, and the frontier tile a CTA scans per pass) x the
 *     visited bitmap in shared or in global memory (shared only where it fits);
 *   pfm (CTA kernel): CTA size 256 or 512 x the arrival state in shared
 *     memory (as 32-bit arrival slots, or as 16-bit offsets within each
 *     vertex's slots when no vertex has more than 65,534 slots), in global
 *     memory, or in global memory with each chunk's out-edge tiles copied
 *     into shared memory by bulk (TMA) copies.
 * A probe is sized like one of Algorithm 1's large rounds: about 100 ms of
 * kernel time by a calibration run of the defaults, between 8 and 64 samples
 * per SM.  Every candidate runs within the same workspace, whose size is bounded by
 * the engine's share of free device memory.  Later calls whose largest graph
 * of that kernel family is g use g's choice (ticks of small bootstraps keep
 * their 1024-thread shape).  Results never depend on the choice: sample i
 * draws from Philox counters fixed by (seed, i).  Call it before sharing g
 * between threads; a tuned graph can be tuned again. */
typedef struct {
    uint32_t bfs_threads;        /* chosen sh/sfm CTA size */
    uint32_t bfs_bitmap_shared;  /* 1: the visited bitmap in shared memory */
    uint32_t pfm_threads;        /* chosen pfm CTA size */
    uint32_t pfm_state_shared;   /* 1: the arrival state in shared memory */
    uint32_t bfs_resident_ctas;  /* samples in flight of the choice (resident CTAs) */
    uint32_t pfm_resident_ctas;
    double bfs_ms, bfs_default_ms;   /* sh probe kernel time: the choice, the defaults */
    double pfm_ms, pfm_default_ms;   /* pfm probe kernel time: the choice, the defaults */
    uint64_t probe_samples;      /* samples per sh probe run */
    uint64_t pfm_probe_samples;  /* samples per pfm probe run */
    uint32_t pfm_staged;         /* 1: global state with the edge tiles staged by bulk copies */
    uint32_t pfm_state16;        /* 1: the shared arrival state as 16-bit slot offsets */
} mantra_tune_result;

int mantra_tune(mantra_graph* g, mantra_tune_result* out);

/* Algorithm 2: r_s = r_override (or ceil(ln n / eps^2) when 0) full searches
 * from sources drawn uniformly from [0,n) (Philox domain 5).  reach_out (or
 * NULL): reach_cap entries, reach_out[h] = number of (source, v != source)
 * pairs at distance <= h (cumulative, unscaled), for h <= min(D_LB, cap-1).
 * Distances: sh / sfm -- hop level of v's first appearance; pfm -- minimum
 * hops among prefix-foremost paths. */
int mantra_temporal_stats(const mantra_graph* g, mantra_opt opt, double eps, uint64_t seed, uint64_t r_override,
                          double tau, mantra_tstats* out, uint64_t* reach_out, uint32_t reach_cap);

/* Temporal closeness from Algorithm 2's searches (the paper's App. D remarks
 * that they approximate closeness; the harmonic form is the reading used
 * here): the same r_s sources as mantra_temporal_stats (r_override, or
 * ceil(ln n / eps^2)), each a full search.  sum_out[v] (or NULL): the sum
 * over the sources u_k != v that reach v of round(2^32 / d(u_k, v)), ties up
 * (the distance of mantra_temporal_stats); closeness_out[v] = sum[v] n /
 * (2^32 r_s (n-1)) estimates 1/(n-1) sum_{u != v} 1/d(u, v).  *r_out (or
 * NULL) receives r_s.  Host arrays of n entries. */
int mantra_temporal_closeness(const mantra_graph* g, mantra_opt opt, double eps, uint64_t seed, uint64_t r_override,
                              uint64_t* sum_out, double* closeness_out, uint64_t* r_out);

/* Diagnostic: run the per-sample path computation of Algorithm 1's Update
 * step for sample indices i0 .. i0+count-1 of the given Philox domains
 * (0/1: estimation pair/path, 3/4: bootstrap pair/path) without
 * accumulating, and return per sample: s, z, sigma_sz (two uint64 words per
 * sample: low, high), the number of vertices of the drawn path (0 when z is
 * unreachable) and the path's vertices s .. z (cap per sample; longer paths
 * are truncated in nodes but len is exact).  edges_out (or NULL): cap per
 * sample, the temporal-edge ids (mantra_graph_edges) of the path's len-1
 * edges in order from s, truncated at cap.  All outputs host arrays. */
int mantra_sample_paths(const mantra_graph* g, mantra_opt opt, uint64_t seed, uint32_t dom_pair, uint32_t dom_path,
                        uint64_t i0, uint64_t count, uint32_t* s_out, uint32_t* z_out, uint64_t* sigma_out,
                        uint32_t* len_out, uint32_t* nodes_out, uint32_t cap, uint32_t* edges_out);

/* Allocation-free variant of mantra_sample_paths for MANTRA_SH and
 * MANTRA_SFM.  The paper has no counterpart.  It is for callers that cannot
 * call cudaMalloc once they are running: a process whose device memory is
 * fixed after start-up, or code that must not pay an allocator's latency or
 * risk its failure between requests.  The call allocates nothing: the search
 * scratch and launch counters live in one fixed 64 MiB __device__ array that
 * every GPU loading the library holds until exit.
 *   g: a graph loaded earlier with mantra_graph_load, on the device that is
 *   current for this call (MANTRA_E_INVAL otherwise); s_dev, z_dev, len_dev:
 *   count uint32 DEVICE buffers; sigma_dev: 2*count uint64 (low, high words);
 *   nodes_dev: count*cap uint32 (may be NULL when cap = 0); stream: a
 *   cudaStream_t of that same device, or NULL (legacy default stream).  Outputs are those of
 *   mantra_sample_paths, indexed by (sample index - i0).
 * The first call made on a device looks up the array's device address
 * (cudaGetSymbolAddress); make that first call before any stream capture.
 * Every call uses the same array and leaves its contents behind; each call
 * clears what must start at zero.  Calls that overlap on the GPU (two streams,
 * two threads, two graphs) race on the array: serialise them.
 * Returns MANTRA_E_INVAL for pfm, for a graph whose search scratch does not
 * fit the fixed array (roughly 44 bytes per arrival slot plus 52 per node,
 * plus 16 per arrival slot of the vertex with the most slots, for one CTA,
 * plus 8 bytes per requested sample), and MANTRA_E_OVERFLOW
 * when a path count exceeds 64 bits (this variant has no 128-bit re-run). */
int mantra_sample_paths_noalloc(const mantra_graph* g, mantra_opt opt, uint64_t seed, uint32_t dom_pair,
                                uint32_t dom_path, uint64_t i0, uint64_t count, uint32_t* s_dev, uint32_t* z_dev,
                                uint64_t* sigma_dev, uint32_t* len_dev, uint32_t* nodes_dev, uint32_t cap,
                                void* stream);

/* ---- Serving (continuous batching over resident graphs) ----
 * A server owns a host thread that runs Algorithm 1 for many requests at
 * once.  Requests queue in arrival order and are admitted while the device
 * state of the running requests and the candidate fits `hbm_budget` bytes
 * (0 = half of free device memory): each request's own buffers (hits,
 * Rademacher sums, estimates: about 16 + 4c bytes per entry of the estimated
 * family) plus the search workspaces shared by all, sized for the largest
 * graph of each search family (sh/sfm; pfm) among them, counted for four
 * (sh/sfm) or six (pfm) CTAs per SM (per CTA about 28 bytes per arrival
 * slot and 28 per node for sh/sfm, 44 and 52 with the ob / RTB scratch; 56
 * per node plus 4 per unit of the graph's path-count bound for pfm), and
 * fewer than
 * `max_active` (0 = 256) run; a request is always admitted when none is
 * running.  Each tick launches the pending samples of every running request
 * together; finished requests leave between ticks and queued ones join at the
 * next tick.  A request's result equals mantra_estimate on the same
 * arguments.  Graphs must stay loaded while their requests are pending. */
typedef struct mantra_server mantra_server;

int mantra_server_create(size_t hbm_budget, uint32_t max_active, mantra_server** out);

/* Queues a request (opts: as mantra_estimate; out_device must be 0; stream is
 * ignored).  req_id receives its id. */
int mantra_server_submit(mantra_server* srv, const mantra_graph* g, mantra_opt opt, double eps, double delta,
                         uint64_t seed, const mantra_opts* opts, uint64_t* req_id);

/* MANTRA_PENDING while the request runs or waits; otherwise the request's
 * status, with est_out (F doubles, F as in mantra_estimate), hits_out (F, or
 * NULL) and info (or NULL)
 * filled when it is MANTRA_OK.  A finished request is retired by this call. */
int mantra_server_poll(mantra_server* srv, uint64_t req_id, double* est_out, uint64_t* hits_out, mantra_info* info);

/* As poll, blocking up to timeout_s seconds (<= 0: no limit). */
int mantra_server_wait(mantra_server* srv, uint64_t req_id, double timeout_s, double* est_out, uint64_t* hits_out,
                       mantra_info* info);

/* Queue length, running requests, finished requests, ticks run, and the
 * running requests' admitted device state (their buffers plus the shared
 * search workspaces as counted for admission; 0 when none runs). */
int mantra_server_stats(mantra_server* srv, uint64_t* queued, uint64_t* active, uint64_t* finished,
                        uint64_t* ticks, uint64_t* bytes_in_use);

/* Drops queued requests, lets running ones finish, stops the thread. */
void mantra_server_destroy(mantra_server* srv);

const char* mantra_strerror(int code);

#ifdef __cplusplus
}
#endif

#endif /* MANTRA_H */
