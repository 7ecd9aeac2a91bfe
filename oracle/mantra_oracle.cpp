// MANTRA CPU oracle -- TEST INFRASTRUCTURE ONLY.
//
// A plain, slow, obviously-correct restatement of the per-sample temporal
// path computation of MANTRA (Cruciani, "MANTRA: Temporal Betweenness
// Centrality Approximation through Sampling", arXiv 2304.08356) and of the
// host-side bounds around it.  Only the test-suite, the package's smoke check
// and the benchmark's CPU-baseline leg may load this library; the product
// path never calls it.  It shares no code, header or table with the CUDA
// library.
//
// Sections followed (paper numbering):
//   Sec. 3 "Preliminaries"  -- temporal graph, temporal path, Def. 1
//                              (sh / sfm / pfm), D, rho, Lemma 1, SD, c-MCERA,
//                              wimpy variance, Theorem 1 (the SD bound xi).
//   Sec. 4.2 / App. B       -- the MCERA sample bound omega (closed form at the
//                              end of the proof of Theorem 3).
//   Sec. 4.4, Algorithm 1   -- the progressive sampler.
//   App. C, "temporal Riondato-Kornaropoulos" estimator and Theorem on the
//                              path sampler -- backward path draw with
//                              probability 1/sigma_sz.
//   Sec. 4.1, the ob estimator -- f_v(s,z) = sigma_sz(v) / sigma_sz, carried
//                              as fixed point with 32 fraction bits.
//   App. C, the RTB estimator  -- f_v(s) = 1/(n-1) sum_z sigma_sz(v) / sigma_sz
//                              from one full search and a backward dependency
//                              accumulation, each term in 2^-32 units.
//   App. D, Algorithm 2     -- reach counts per hop, D_LB, D_tau, zeta, Psi.
//
// Readings where the paper is silent or garbled (same list in the design
// notes): source appearance (s,-inf); strict time increase; duplicate
// (u,v,t) triples deduplicated, self loops dropped; sfm = minimum hops first,
// then earliest arrival at z (Figure "example_tp" caption); canonical
// predecessor order for the path draw (in-edges by ascending w, then the
// predecessor's appearances by ascending time); delta_i = delta/2^(i+1);
// vhat = W, or (vhat_mode 1) the appendix's variance bound with its garbled
// square-root term read as 2 W ln(1/delta)/r; natural logarithms; pfm
// distance = minimum hops among pfm paths; ob values rounded to the nearest
// multiple of 2^-32 (ties up), their squares for the wimpy variance rounded
// the same way from the rounded value.
//
// Parity unpinned (no value printed in the paper; pinned only by special
// cases, monotonicity, Theorem 1's guarantee and a coverage simulation): the
// floating-point bounds xi, omega, the s_1 search and the variance bound.
//
// Integers: path counts are exact unsigned 128-bit; a count that would exceed
// 2^128-1 is reported as an overflow error.

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <mutex>
#include <set>
#include <tuple>
#include <utility>
#include <vector>

typedef unsigned __int128 u128;

namespace {

// ---------------------------------------------------------------------------
// Philox4x32-10 counter-based generator, written from its published
// definition (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
// as 1, 2, 3", SC'11): 10 rounds of two 32x32->64 multiplies with the round
// function (c0,c1,c2,c3) -> (hi(M1*c2)^c1^k0, lo(M1*c2), hi(M0*c0)^c3^k1,
// lo(M0*c0)), the key bumped by the Weyl constants between rounds.
// ---------------------------------------------------------------------------
const uint32_t PHILOX_M0 = 0xD2511F53u;
const uint32_t PHILOX_M1 = 0xCD9E8D57u;
const uint32_t PHILOX_W0 = 0x9E3779B9u;
const uint32_t PHILOX_W1 = 0xBB67AE85u;

void philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
    uint32_t c[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { k0 += PHILOX_W0; k1 += PHILOX_W1; }
        uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)c[0];
        uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)c[2];
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c[1] ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c[3] ^ k1;
        uint32_t n3 = lo0;
        c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
    }
    out[0] = c[0]; out[1] = c[1]; out[2] = c[2]; out[3] = c[3];
}

// Random-stream domains (counter word 2).
enum { D_PAIR = 0, D_PATH = 1, D_RADE = 2, D_BOOT_PAIR = 3, D_BOOT_PATH = 4, D_STATS = 5 };
const uint32_t MAX_ATTEMPTS = 1u << 16;

// One Philox block for (seed, sample index i, domain, attempt).
void block_for(uint64_t seed, uint64_t i, uint32_t domain, uint32_t attempt, uint32_t out[4]) {
    uint32_t ctr[4] = {(uint32_t)i, (uint32_t)(i >> 32), domain, attempt};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    philox4x32_10(ctr, key, out);
}

// Uniform integer in [0, N), N >= 1, by masking the low 64 bits of a block
// to the smallest 2^k - 1 >= N - 1 and rejecting values >= N (a rejected
// value moves to the next attempt counter).  Returns false after
// MAX_ATTEMPTS rejections.
bool uniform_below64(uint64_t N, uint64_t seed, uint64_t i, uint32_t domain, uint64_t* x) {
    uint64_t mask = 0;
    while (mask < N - 1) mask = (mask << 1) | 1u;
    for (uint32_t a = 0; a < MAX_ATTEMPTS; ++a) {
        uint32_t w[4];
        block_for(seed, i, domain, a, w);
        uint64_t val = ((uint64_t)w[1] << 32) | w[0];
        val &= mask;
        if (val < N) { *x = val; return true; }
    }
    return false;
}

// Same with all 128 bits of the block (for path counts).
bool uniform_below128(u128 N, uint64_t seed, uint64_t i, uint32_t domain, u128* x) {
    u128 mask = 0;
    while (mask < N - 1) mask = (mask << 1) | 1u;
    for (uint32_t a = 0; a < MAX_ATTEMPTS; ++a) {
        uint32_t w[4];
        block_for(seed, i, domain, a, w);
        u128 val = ((u128)w[3] << 96) | ((u128)w[2] << 64) | ((u128)w[1] << 32) | (u128)w[0];
        val &= mask;
        if (val < N) { *x = val; return true; }
    }
    return false;
}

// Sample space of the ob / trk estimators (Sec. 4.1): ordered pairs (s,z),
// s != z, uniform.  x in [0, n(n-1)) ; s = x / (n-1) ; z' = x mod (n-1) ;
// z = z' + [z' >= s].
bool draw_pair(uint32_t n, uint64_t seed, uint64_t i, uint32_t domain, uint32_t* s, uint32_t* z) {
    uint64_t N = (uint64_t)n * (uint64_t)(n - 1);
    uint64_t x;
    if (!uniform_below64(N, seed, i, domain, &x)) return false;
    uint64_t ss = x / (uint64_t)(n - 1);
    uint64_t zz = x % (uint64_t)(n - 1);
    if (zz >= ss) zz += 1;
    *s = (uint32_t)ss; *z = (uint32_t)zz;
    return true;
}

// Rademacher sign lambda_{j,i} (Sec. 3, c-MCERA): bit j of the 128-bit block
// for (seed, i, RADE, 0); bit 1 -> +1, bit 0 -> -1.
int rademacher(uint64_t seed, uint64_t i, uint32_t j) {
    uint32_t w[4];
    block_for(seed, i, D_RADE, 0, w);
    return ((w[j >> 5] >> (j & 31)) & 1u) ? 1 : -1;
}

// ---------------------------------------------------------------------------
// Temporal graph (Sec. 3): a set of temporal edges (u,v,t).  Identical triples
// name the same vertex appearances, so they are kept once; self loops are
// dropped (the path sampler's theorem assumes none).
// ---------------------------------------------------------------------------
struct Graph {
    uint32_t n = 0;
    std::vector<std::tuple<uint32_t, uint32_t, uint32_t>> edges;   // (u,v,t), sorted by (t,u,v)
    std::vector<std::vector<std::pair<uint32_t, uint32_t>>> out;  // out[u] = (v,t), ascending t
    std::vector<std::vector<std::pair<uint32_t, uint32_t>>> in;   // in[v]  = (w,t)
    uint64_t self_loops = 0;
    uint64_t duplicates = 0;
    // Edge betweenness (App. A): temporal edge (u,v,t) -> id = its rank in
    // (v,t,u) order; underlying edge (u,v) -> id = its rank in (v,u) order.
    // Built on first use (edge_ids), once, by whichever thread needs them.
    mutable std::once_flag ids_once;
    mutable std::map<std::tuple<uint32_t, uint32_t, uint32_t>, uint32_t> tid;   // key (v,t,u)
    mutable std::map<std::pair<uint32_t, uint32_t>, uint32_t> uid;              // key (v,u)
    mutable std::vector<uint32_t> t2u;                                          // temporal id -> underlying id
};

// The edge ids of the Graph (ranks of the deduplicated triples in (v,t,u)
// order, of the distinct pairs in (v,u) order).
const Graph& edge_ids(const Graph& G) {
    std::call_once(G.ids_once, [&G]() {
        for (const auto& e : G.edges) {                                  // (u,v,t)
            G.tid[std::make_tuple(std::get<1>(e), std::get<2>(e), std::get<0>(e))] = 0;
            G.uid[std::make_pair(std::get<1>(e), std::get<0>(e))] = 0;
        }
        uint32_t r = 0;
        for (auto& kv : G.tid) kv.second = r++;
        r = 0;
        for (auto& kv : G.uid) kv.second = r++;
        G.t2u.assign(G.tid.size(), 0);
        for (const auto& kv : G.tid)
            G.t2u[kv.second] = G.uid.at(std::make_pair(std::get<0>(kv.first), std::get<2>(kv.first)));
    });
    return G;
}

const int64_t NEG_INF = -1;                 // the source appearance (s, -inf)
const int64_t POS_INF = INT64_MAX;

// A vertex appearance (v, t): v reached at time t.
typedef std::pair<uint32_t, int64_t> App;
struct State { uint32_t level; u128 sigma; };

bool add_checked(u128 a, u128 b, u128* r) {
    u128 s = a + b;
    if (s < a) return false;
    *r = s;
    return true;
}

// OPT_FSFM: foremost-first shortest-foremost (Buss et al.'s order, the other
// reading of Def. 1(2)): the earliest arrival at z first, then the fewest hops.
enum { OPT_SH = 0, OPT_SFM = 1, OPT_PFM = 2, OPT_FSFM = 3 };
enum { OK = 0, E_INVAL = 1, E_OVERFLOW = 3, E_RNG = 7 };

// Result of a forward search from s (truncated at z when z is given).
struct Search {
    // sh / sfm: appearance states with (level, sigma)
    std::map<App, State> st;
    uint32_t d = 0;              // level of z's first appearance (0 = not reached)
    // pfm: earliest arrival, path counts, minimum hops per vertex
    std::vector<int64_t> fa;
    std::vector<u128> sig;
    std::vector<uint32_t> hop;
    int status = OK;
};

// (*)-temporal BFS for sh and sfm over vertex appearances.  Level 0 is
// (s,-inf).  From every appearance (u,t') on level k, each out-edge (u,v,t)
// with t > t' reaches (v,t); if (v,t) has no level yet it gets level k+1, and
// every such (appearance, edge) pair adds sigma(u,t') to sigma(v,t).  The
// additions are grouped by u: an out-edge (u,v,t) adds the total sigma of u's
// level-k appearances earlier than t (same sum, taken per edge).  With a
// target z the search stops after the first level that holds an appearance
// of z; with no target (z = n) it runs until the frontier is empty.
Search tbfs_levels(const Graph& G, uint32_t s, uint32_t z, int64_t tmax = POS_INF) {
    Search R;
    App src(s, NEG_INF);
    R.st[src] = State{0, 1};
    std::vector<App> frontier(1, src);
    uint32_t k = 0;
    while (!frontier.empty()) {
        std::sort(frontier.begin(), frontier.end());
        std::vector<App> next;
        size_t g0 = 0;
        while (g0 < frontier.size()) {
            const uint32_t u = frontier[g0].first;
            size_t g1 = g0;
            while (g1 < frontier.size() && frontier[g1].first == u) ++g1;
            // running totals of sigma over u's level-k appearances, ascending in time
            std::vector<int64_t> times;
            std::vector<u128> prefix;
            u128 run = 0;
            for (size_t q = g0; q < g1; ++q) {
                if (!add_checked(run, R.st[frontier[q]].sigma, &run)) { R.status = E_OVERFLOW; return R; }
                times.push_back(frontier[q].second);
                prefix.push_back(run);
            }
            for (const auto& e : G.out[u]) {                      // out[u] is sorted by time
                int64_t t = e.second;
                if (t > tmax) break;                              // beyond the time bound
                size_t cnt = std::lower_bound(times.begin(), times.end(), t) - times.begin();
                if (cnt == 0) continue;                           // no appearance of u before t
                const u128 add = prefix[cnt - 1];
                App b(e.first, t);
                auto it = R.st.find(b);
                if (it == R.st.end()) {
                    R.st[b] = State{k + 1, add};
                    next.push_back(b);
                } else if (it->second.level == k + 1) {
                    if (!add_checked(it->second.sigma, add, &it->second.sigma)) {
                        R.status = E_OVERFLOW;
                        return R;
                    }
                }
            }
            g0 = g1;
        }
        k += 1;
        bool hit_z = false;
        for (const App& b : next) if (b.first == z) hit_z = true;
        if (hit_z) { R.d = k; return R; }
        frontier.swap(next);
    }
    return R;
}

// Prefix-foremost search (Def. 1(3)): scan all temporal edges in time order.
// fa[s] = -inf; an edge (u,v,t) with v != s, fa[u] < t and fa[v] in {inf, t}
// sets fa[v] = t, adds sigma[u] to sigma[v] and lowers hop[v] to hop[u]+1.
// Within one timestamp the test fa[u] < t ignores values set at that
// timestamp, so the order of equal-time edges does not matter.
Search pfm_scan(const Graph& G, uint32_t s) {
    Search R;
    R.fa.assign(G.n, POS_INF);
    R.sig.assign(G.n, 0);
    R.hop.assign(G.n, UINT32_MAX);
    R.fa[s] = NEG_INF;
    R.sig[s] = 1;
    R.hop[s] = 0;
    for (const auto& e : G.edges) {
        uint32_t u = std::get<0>(e), v = std::get<1>(e);
        int64_t t = std::get<2>(e);
        if (v == s) continue;
        if (!(R.fa[u] < t)) continue;
        if (R.fa[v] != POS_INF && R.fa[v] != t) continue;
        R.fa[v] = t;
        if (!add_checked(R.sig[v], R.sig[u], &R.sig[v])) { R.status = E_OVERFLOW; return R; }
        R.hop[v] = std::min(R.hop[v], R.hop[u] + 1);
    }
    return R;
}

// Endpoint appearances of z in the sh / sfm search, ascending in time.
// sh keeps every appearance of z on level d; sfm only the earliest one;
// fsfm the earliest appearance of z at any level (its level is R.d).
std::vector<App> endpoints(const Search& R, uint32_t z, int opt) {
    std::vector<App> ends;
    if (R.d == 0) return ends;
    if (opt == OPT_FSFM) {
        auto it = R.st.lower_bound(App(z, NEG_INF));
        if (it != R.st.end() && it->first.first == z) ends.push_back(it->first);
        return ends;
    }
    for (auto it = R.st.lower_bound(App(z, NEG_INF)); it != R.st.end() && it->first.first == z; ++it)
        if (it->second.level == R.d) ends.push_back(it->first);
    if (opt == OPT_SFM && !ends.empty()) ends.resize(1);
    return ends;
}

// sigma_sz: the number of (*)-optimal temporal paths from s to z.
int count_paths(const Graph& G, int opt, uint32_t s, uint32_t z, Search* out, u128* sigma) {
    if (opt == OPT_PFM) {
        *out = pfm_scan(G, s);
        if (out->status != OK) return out->status;
        *sigma = (out->fa[z] == POS_INF) ? 0 : out->sig[z];
        return OK;
    }
    if (opt == OPT_FSFM) {
        // every appearance of z that some path reaches: search without the
        // first-level stop, up to z's latest in-edge time; the earliest one
        // is the endpoint, with the fewest hops (its level)
        int64_t tz = -1;
        for (const auto& e : G.in[z]) tz = std::max<int64_t>(tz, e.second);
        *out = tbfs_levels(G, s, G.n, tz);
        if (out->status != OK) return out->status;
        out->d = 0;
        auto it = out->st.lower_bound(App(z, NEG_INF));
        if (z != s && it != out->st.end() && it->first.first == z) out->d = it->second.level;
    } else {
        *out = tbfs_levels(G, s, z);
    }
    if (out->status != OK) return out->status;
    u128 tot = 0;
    for (const App& a : endpoints(*out, z, opt))
        if (!add_checked(tot, out->st.at(a).sigma, &tot)) return E_OVERFLOW;
    *sigma = tot;
    return OK;
}

// Backward draw of one optimal path (App. C, temporal Riondato-Kornaropoulos
// estimator): x in [0, sigma_sz) names one path.  At each step the candidates
// are taken in a fixed order, each weighted by its path count, and the first
// whose running weight exceeds x is chosen (x drops by the weight before it).
//   sh / sfm end : appearances of z on level d by ascending time.
//   sh / sfm step: from (v,t_v) on level k, in-edges (w,v,t_v) by ascending w,
//                  then appearances (w,t_w) on level k-1 with t_w < t_v by
//                  ascending t_w; on level 0 only (s,-inf), weight 1.
//   pfm step     : from v (reached at fa[v]), in-edges (w,v,fa[v]) by
//                  ascending w with fa[w] < fa[v], weight sigma[w].
// The vertices are returned from s to z.
int unrank_path(const Graph& G, int opt, uint32_t s, uint32_t z, const Search& R, u128 x,
                std::vector<uint32_t>* path, std::vector<int64_t>* times = nullptr) {
    std::vector<uint32_t> rev;
    std::vector<int64_t> rev_t;
    if (opt == OPT_PFM) {
        uint32_t v = z;
        rev.push_back(z);
        rev_t.push_back(R.fa[z]);
        while (v != s) {
            std::vector<uint32_t> cands;
            for (const auto& e : G.in[v])
                if ((int64_t)e.second == R.fa[v] && R.fa[e.first] < R.fa[v]) cands.push_back(e.first);
            std::sort(cands.begin(), cands.end());
            u128 cum = 0;
            bool picked = false;
            for (uint32_t w : cands) {
                u128 wt = R.sig[w];
                if (x < cum + wt) { x -= cum; v = w; picked = true; break; }
                cum += wt;
            }
            if (!picked) return E_INVAL;
            rev.push_back(v);
            rev_t.push_back(R.fa[v]);
        }
    } else {
        std::vector<App> ends = endpoints(R, z, opt);
        App cur;
        bool picked = false;
        u128 cum = 0;
        for (const App& a : ends) {
            u128 wt = R.st.at(a).sigma;
            if (x < cum + wt) { x -= cum; cur = a; picked = true; break; }
            cum += wt;
        }
        if (!picked) return E_INVAL;
        rev.push_back(z);
        rev_t.push_back(cur.second);
        uint32_t k = R.d;
        while (k > 0) {
            // candidates for (cur.first, cur.second) on level k
            std::vector<uint32_t> ws;
            for (const auto& e : G.in[cur.first])
                if ((int64_t)e.second == cur.second) ws.push_back(e.first);
            std::sort(ws.begin(), ws.end());
            cum = 0;
            picked = false;
            App nxt;
            for (uint32_t w : ws) {
                std::vector<App> apps;
                if (k - 1 == 0) {
                    if (w == s) apps.push_back(App(s, NEG_INF));
                } else {
                    for (auto it = R.st.lower_bound(App(w, NEG_INF)); it != R.st.end() && it->first.first == w; ++it)
                        if (it->second.level == k - 1 && it->first.second < cur.second) apps.push_back(it->first);
                }
                for (const App& a : apps) {          // map order = ascending time
                    u128 wt = R.st.at(a).sigma;
                    if (x < cum + wt) { x -= cum; nxt = a; picked = true; break; }
                    cum += wt;
                }
                if (picked) break;
            }
            if (!picked) return E_INVAL;
            cur = nxt;
            rev.push_back(cur.first);
            rev_t.push_back(cur.second);
            k -= 1;
        }
    }
    path->assign(rev.rbegin(), rev.rend());
    if (times) times->assign(rev_t.rbegin(), rev_t.rend());
    return OK;
}

// ---------------------------------------------------------------------------
// Work of one sample's search (the exact counters behind the algorithmic-byte
// model of the measurement; no paper passage defines them, they restate what
// the search of Sec. 3 / Def. 1 must touch).  tz = z's latest in-edge time.
// sh / sfm / fsfm: F_k = the appearances (v,t) on hop level k with t < tz
// (fsfm: t <= tz), F_0 = {(s,-inf)}.  sh / sfm search levels 0 .. d-1 when z
// is reached on level d (levels 0 .. d-2 are expanded), or every non-empty
// level when z is unreachable (all expanded); fsfm searches and expands every
// non-empty level.
//   escan  per searched level: |in(z)| (sh / sfm test whether the level
//          reaches z); per expanded level: for each vertex u of F_k, the
//          out-edges (u,v,t) with t > u's earliest time in F_k and t < tz
//          (fsfm: t <= tz); every out-edge of s on level 0;
//   eadd   those expanded edges whose head (v,t) is on level k+1;
//   snew   the sizes of the levels that follow the expanded ones;
//   fseg   the distinct vertices of every searched level (1 on level 0).
// pfm: te = fa(z), or tz when z is unreachable;
//   escan  edges (u,v,t) with v != s and (earliest out-edge time of s) <= t <= te;
//   eadd   edges (w,v,t) with v != s, t = fa(v) <= te and fa(w) < fa(v)
//          (the prefix-foremost DAG);  snew = fseg = 0.
// A sample whose s has no out-edge, or whose z has no in-edge, counts nothing.
// ---------------------------------------------------------------------------
struct Work { uint64_t escan = 0, eadd = 0, snew = 0, fseg = 0; };

void search_work(const Graph& G, int opt, uint32_t s, uint32_t z, const Search& R, Work* w) {
    *w = Work();
    if (G.out[s].empty() || G.in[z].empty()) return;
    int64_t tz = -1;
    for (const auto& e : G.in[z]) tz = std::max<int64_t>(tz, e.second);
    if (opt == OPT_PFM) {
        int64_t ts = POS_INF;
        for (const auto& e : G.out[s]) ts = std::min<int64_t>(ts, e.second);
        const int64_t te = (R.fa[z] == POS_INF) ? tz : R.fa[z];
        for (const auto& e : G.edges) {
            const uint32_t u = std::get<0>(e), v = std::get<1>(e);
            const int64_t t = std::get<2>(e);
            if (v == s) continue;
            if (ts <= t && t <= te) w->escan += 1;
            if (t == R.fa[v] && t <= te && R.fa[u] < R.fa[v]) w->eadd += 1;
        }
        return;
    }
    const bool fsfm = opt == OPT_FSFM;
    auto keep = [&](int64_t t) { return fsfm ? t <= tz : t < tz; };
    // the kept appearances by level
    std::vector<std::vector<App>> lev(1, std::vector<App>(1, App(s, NEG_INF)));
    for (const auto& kv : R.st) {
        const uint32_t k = kv.second.level;
        if (k == 0 || !keep(kv.first.second)) continue;
        if (lev.size() <= k) lev.resize(k + 1);
        lev[k].push_back(kv.first);
    }
    // searched levels 0 .. last_searched, expanded levels 0 .. last_expanded
    int64_t last_searched, last_expanded;
    const bool reached = !fsfm && R.d > 0;
    if (reached) {
        last_searched = (int64_t)R.d - 1;
        last_expanded = (int64_t)R.d - 2;
    } else {
        int64_t K = 0;
        for (size_t k = 0; k < lev.size(); ++k) if (!lev[k].empty()) K = (int64_t)k;
        last_searched = last_expanded = K;
    }
    for (int64_t k = 0; k <= last_searched; ++k) {
        // lev[k] is in map order: grouped by vertex, ascending in time
        std::map<uint32_t, int64_t> first_time;
        for (const App& a : lev[k]) if (!first_time.count(a.first)) first_time[a.first] = a.second;
        w->fseg += first_time.size();
        if (!fsfm) w->escan += G.in[z].size();
        if (k > last_expanded) continue;
        for (const auto& ut : first_time) {
            for (const auto& e : G.out[ut.first]) {
                const int64_t t = e.second;
                if (!(t > ut.second) || !keep(t)) continue;
                w->escan += 1;
                auto it = R.st.find(App(e.first, t));
                if (it != R.st.end() && it->second.level == (uint32_t)k + 1) w->eadd += 1;
            }
        }
        if ((size_t)k + 1 < lev.size()) w->snew += lev[k + 1].size();
    }
}

struct Sample {
    uint32_t s = 0, z = 0;
    u128 sigma = 0;
    std::vector<uint32_t> path;   // s .. z, empty when z is unreachable
    std::vector<uint32_t> edges;  // temporal edge ids of the path, s to z
    Work work;                    // the search's work counters
};

// One sample of Algorithm 1's Update step: draw (s,z), count optimal paths,
// draw x uniform in [0, sigma_sz), unrank the path (and, with want_edges, list
// the temporal edge ids of its edges).
int one_sample(const Graph& G, int opt, uint64_t seed, uint64_t i, uint32_t dom_pair, uint32_t dom_path,
               Sample* out, bool want_edges = false) {
    if (!draw_pair(G.n, seed, i, dom_pair, &out->s, &out->z)) return E_RNG;
    Search R;
    int st = count_paths(G, opt, out->s, out->z, &R, &out->sigma);
    if (st != OK) return st;
    search_work(G, opt, out->s, out->z, R, &out->work);
    out->path.clear();
    if (out->sigma == 0) return OK;                       // unreachable: empty path
    u128 x;
    if (!uniform_below128(out->sigma, seed, i, dom_path, &x)) return E_RNG;
    std::vector<int64_t> times;
    int st2 = unrank_path(G, opt, out->s, out->z, R, x, &out->path, &times);
    if (st2 != OK) return st2;
    out->edges.clear();
    if (want_edges)
        for (size_t k = 0; k + 1 < out->path.size(); ++k)      // edge (path[k], path[k+1], times[k+1])
            out->edges.push_back(edge_ids(G).tid.at(std::make_tuple(out->path[k + 1], (uint32_t)times[k + 1], out->path[k])));
    return OK;
}

// sigma_sz(v) for every v (Sec. 3): the number of (*)-optimal paths from s to
// z with v as an internal node.  A path through an appearance a of v splits
// into an optimal path s -> a (counted by the forward search) and an optimal
// continuation a -> z; the continuations beta are counted backward from z's
// endpoint appearances over the optimal-path DAG (Brandes-style).  A path
// visits v at most once, so the products over v's appearances add up.
// `through` gets n entries (0 for s, z and vertices on no optimal path).
void through_counts(const Graph& G, int opt, uint32_t s, uint32_t z, const Search& R, std::vector<u128>* through) {
    const uint32_t n = G.n;
    through->assign(n, 0);
    if (opt == OPT_PFM) {
        // beta[v] = number of pfm continuations from v to z, over the DAG of
        // edges (w,v,fa[v]) with fa[w] < fa[v], in decreasing fa.
        if (R.fa[z] == POS_INF) return;
        std::vector<u128> beta(n, 0);
        beta[z] = 1;
        std::vector<uint32_t> order;
        for (uint32_t v = 0; v < n; ++v) if (R.fa[v] != POS_INF) order.push_back(v);
        std::sort(order.begin(), order.end(), [&](uint32_t a, uint32_t b) { return R.fa[a] > R.fa[b]; });
        for (uint32_t v : order) {
            if (beta[v] == 0 || v == s) continue;
            for (const auto& e : G.in[v])
                if ((int64_t)e.second == R.fa[v] && R.fa[e.first] < R.fa[v]) beta[e.first] += beta[v];
        }
        for (uint32_t v = 0; v < n; ++v) if (v != s && v != z) (*through)[v] = R.sig[v] * beta[v];
        return;
    }
    std::map<App, u128> beta;
    for (const App& a : endpoints(R, z, opt)) beta[a] = 1;
    for (uint32_t k = R.d; k >= 1; --k) {
        for (auto& kv : R.st) {
            if (kv.second.level != k) continue;
            auto bi = beta.find(kv.first);
            if (bi == beta.end() || bi->second == 0) continue;
            for (const auto& e : G.in[kv.first.first]) {
                if ((int64_t)e.second != kv.first.second) continue;
                uint32_t w = e.first;
                if (k - 1 == 0) {
                    if (w == s) beta[App(s, NEG_INF)] += bi->second;
                    continue;
                }
                for (auto it = R.st.lower_bound(App(w, NEG_INF)); it != R.st.end() && it->first.first == w; ++it)
                    if (it->second.level == k - 1 && it->first.second < kv.first.second) beta[it->first] += bi->second;
            }
        }
    }
    for (auto& kv : beta) {
        uint32_t v = kv.first.first;
        if (v == s || v == z) continue;
        (*through)[v] += R.st.at(kv.first).sigma * kv.second;
    }
}

// a / b (0 <= a <= b, b >= 1) as a multiple of 2^-32, rounded to nearest with
// ties up: the integer nearest to 2^32 a / b.  Binary long division of a * 2^32
// by b, one quotient bit per step, then one more step decides the rounding;
// the remainder is kept below b, so 2 * remainder fits in 129 bits (the
// carry out of bit 127 is tracked).
uint64_t fixed32(u128 a, u128 b) {
    if (a >= b) return (uint64_t)1 << 32;
    u128 rem = a;               // invariant: rem < b
    uint64_t q = 0;
    for (int bit = 0; bit < 33; ++bit) {
        const bool carry = (rem >> 127) != 0;
        rem <<= 1;              // true value: rem + carry * 2^128
        const bool ge = carry || rem >= b;
        if (ge) rem -= b;       // wraps back below b when carry is set
        if (bit < 32) q = (q << 1) | (ge ? 1u : 0u);
        else if (ge) q += 1;    // the 33rd bit: 2 * remainder >= b rounds up
    }
    return q;
}

// floor(a * x / d + 1/2) for a <= d (d >= 1), x < 2^64: the quotient is at
// most x + 1.  The product is formed exactly (192 bits as hi:lo) and divided
// by schoolbook binary long division when it does not fit 128 bits.
uint64_t muldiv_round(u128 a, uint64_t x, u128 d) {
    const u128 M64 = ~(u128)0 >> 64;
    if ((a >> 64) == 0) {                       // a * x < 2^128
        const u128 nprod = a * (u128)x;
        const u128 q0 = nprod / d, r0 = nprod % d;
        return (uint64_t)q0 + ((r0 >= d - r0) ? 1u : 0u);   // 2 r0 >= d, without overflow
    }
    // 192-bit product: a = ah 2^64 + al, a x = ah x 2^64 + al x
    const u128 al = a & M64, ah = a >> 64;
    const u128 p0 = al * (u128)x, p1 = ah * (u128)x;
    u128 lo = p0 + (p1 << 64);
    u128 hi = (p1 >> 64) + ((lo < p0) ? 1 : 0);   // carry out of the low 128 bits
    // long division of (hi:lo) by d, bit by bit from the top (hi < 2^64)
    u128 rem = 0;
    uint64_t q = 0;
    for (int bit = 191; bit >= 0; --bit) {
        const bool top = (rem >> 127) != 0;
        const unsigned b = bit >= 128 ? (unsigned)((hi >> (bit - 128)) & 1) : (unsigned)((lo >> bit) & 1);
        rem = (rem << 1) | b;
        const bool ge = top || rem >= d;
        if (ge) rem -= d;
        if (bit < 64) q = (q << 1) | (ge ? 1u : 0u);
        else if (ge) return ~(uint64_t)0;       // quotient >= 2^64: impossible for a <= d
    }
    const bool top = (rem >> 127) != 0;
    return q + ((top || (rem << 1) >= d) ? 1u : 0u);
}

// One RTB sample (App. C): q[v] = f_v(s) in 2^-32 units for every v != s.
// Full search from s.  sh / sfm: the endpoint states of a vertex v are its
// states on its first level d_v (sfm: only the earliest of them), and
// eps(b) = sigma(b) / sigma_{s,v_b} for an endpoint b, else 0.  pfm: every
// reached vertex is its own endpoint (eps = 1).  Levels (or decreasing fa)
// from the last down: for every optimal-DAG edge a -> b,
//   delta(a) += round(sigma(a) * (eps(b) + delta(b)) / sigma(b)),
// then f_v = round(sum of delta over v's states / (n-1)).
int rtb_values(const Graph& G, int opt, uint64_t seed, uint64_t i, uint32_t dom, std::vector<uint64_t>* q) {
    const uint32_t n = G.n;
    q->assign(n, 0);
    uint64_t s64;
    if (!uniform_below64(n, seed, i, dom, &s64)) return E_RNG;
    const uint32_t s = (uint32_t)s64;
    const uint64_t ONE = (uint64_t)1 << 32;
    std::vector<uint64_t> sum(n, 0);
    if (opt == OPT_PFM) {
        Search R = pfm_scan(G, s);
        if (R.status != OK) return R.status;
        std::vector<uint64_t> delta(n, 0);
        std::vector<uint32_t> order;
        for (uint32_t v = 0; v < n; ++v) if (v != s && R.fa[v] != POS_INF) order.push_back(v);
        std::sort(order.begin(), order.end(), [&](uint32_t a, uint32_t b) { return R.fa[a] > R.fa[b]; });
        for (uint32_t x : order) {
            const uint64_t X = ONE + delta[x];
            for (const auto& e : G.in[x]) {
                const uint32_t w = e.first;
                if ((int64_t)e.second != R.fa[x] || !(R.fa[w] < R.fa[x]) || w == s) continue;
                delta[w] += muldiv_round(R.sig[w], X, R.sig[x]);
            }
        }
        for (uint32_t v = 0; v < n; ++v) sum[v] = delta[v];
    } else {
        Search R = tbfs_levels(G, s, n);
        if (R.status != OK) return R.status;
        // first level and endpoint states per vertex
        std::vector<uint32_t> dv(n, UINT32_MAX);
        for (const auto& kv : R.st)
            if (kv.first.first != s) dv[kv.first.first] = std::min(dv[kv.first.first], kv.second.level);
        std::map<App, bool> is_end;
        std::vector<u128> sv(n, 0);             // sigma_{s,v}
        std::vector<bool> taken(n, false);
        for (const auto& kv : R.st) {           // map order: by vertex, then ascending time
            const uint32_t v = kv.first.first;
            if (v == s) continue;
            if (opt == OPT_FSFM) {                // the earliest state of v, at any level
                if (taken[v]) continue;
            } else {
                if (kv.second.level != dv[v]) continue;
                if (opt == OPT_SFM && taken[v]) continue;
            }
            taken[v] = true;
            is_end[kv.first] = true;
            if (!add_checked(sv[v], kv.second.sigma, &sv[v])) return E_OVERFLOW;
        }
        uint32_t D = 0;
        for (const auto& kv : R.st) D = std::max(D, kv.second.level);
        std::map<App, uint64_t> delta;
        for (uint32_t k = D; k >= 2; --k) {
            for (const auto& kv : R.st) {
                if (kv.second.level != k) continue;
                const App b = kv.first;
                uint64_t X = delta.count(b) ? delta[b] : 0;
                if (is_end.count(b)) X += (uint64_t)fixed32(kv.second.sigma, sv[b.first]);
                if (X == 0) continue;
                for (const auto& e : G.in[b.first]) {
                    if ((int64_t)e.second != b.second) continue;
                    const uint32_t w = e.first;
                    for (auto it = R.st.lower_bound(App(w, NEG_INF)); it != R.st.end() && it->first.first == w; ++it)
                        if (it->second.level == k - 1 && it->first.second < b.second)
                            delta[it->first] += muldiv_round(it->second.sigma, X, kv.second.sigma);
                }
            }
        }
        for (const auto& kv : delta) sum[kv.first.first] += kv.second;
    }
    for (uint32_t v = 0; v < n; ++v)
        if (v != s && sum[v]) (*q)[v] = muldiv_round(1, sum[v], n - 1);
    return OK;
}

// The ob functions of one sample (Sec. 4.1): q[v] = fixed32(sigma_sz(v), sigma_sz)
// for the internal vertices v on some optimal path (all 0 when z is
// unreachable).
int ob_values(const Graph& G, int opt, uint64_t seed, uint64_t i, uint32_t dom_pair,
              std::vector<std::pair<uint32_t, uint64_t>>* vals, Work* work = nullptr) {
    vals->clear();
    uint32_t s, z;
    if (!draw_pair(G.n, seed, i, dom_pair, &s, &z)) return E_RNG;
    Search R;
    u128 sg;
    int st = count_paths(G, opt, s, z, &R, &sg);
    if (st != OK) return st;
    if (work) search_work(G, opt, s, z, R, work);
    if (sg == 0) return OK;
    std::vector<u128> th;
    through_counts(G, opt, s, z, R, &th);
    for (uint32_t v = 0; v < G.n; ++v)
        if (th[v] != 0) vals->push_back(std::make_pair(v, fixed32(th[v], sg)));
    return OK;
}

// ---------------------------------------------------------------------------
// Bounds (Sec. 3 Theorem 1; proof of Theorem 3).
// ---------------------------------------------------------------------------
// xi of Theorem 1 for c-MCERA value Rc, wimpy variance W, variance bound vhat,
// confidence delta and r samples.
// Last line of Theorem 1: xi from the Rademacher bound R.
double xi_from_R(double Rb, double vhat, double delta, double r) {
    double L = std::log(4.0 / delta);
    return 2.0 * Rb + std::sqrt(2.0 * L * (vhat + 4.0 * Rb) / r) + L / (3.0 * r);
}

double sd_bound(double Rc, double W, double vhat, double delta, double r, double c) {
    double L = std::log(4.0 / delta);
    double Rt = Rc + std::sqrt(4.0 * W * L / (c * r));
    double Rb = Rt + L / r + std::sqrt((L / r) * (L / r) + 2.0 * L * Rt / r);
    return xi_from_R(Rb, vhat, delta, r);
}

// omega: the closed-form sample bound at the end of the proof of Theorem 3,
// ((2 vhat + 2 eps / 3) / eps^2) (ln(2 rho / vhat) + ln(1/delta)).
double omega_bound(double vhat, double rho, double eps, double delta) {
    return ((2.0 * vhat + 2.0 * eps / 3.0) / (eps * eps)) * (std::log(2.0 * rho / vhat) + std::log(1.0 / delta));
}

// Variance bound from the empirical wimpy variance (the self-bounding
// proposition of the appendix, adapted from Pellegrina & Vandin): with
// probability >= 1 - delta, sup_f Var(f) <= W + L/r + sqrt((L/r)^2 + 2 W L / r),
// L = ln(1/delta).  The printed square-root term is garbled; it is read as the
// same self-bounding form as the R bound of Theorem 1 (2 L x / r).
double wimpy_variance_bound(double W, double delta, double r) {
    const double L = std::log(1.0 / delta);
    return W + L / r + std::sqrt((L / r) * (L / r) + 2.0 * W * L / r);
}

double delta_round(double delta, uint64_t i, int sched) {
    return sched == 1 ? delta / std::ldexp(1.0, (int)i) : delta / std::ldexp(1.0, (int)(i + 1));
}

}  // namespace

// ===========================================================================
// C API for the tests (ctypes)
// ===========================================================================
extern "C" {

struct orc_info {
    uint64_t r, rounds, omega, s1, bootstrap, sum_int_len, max_hits;
    int64_t rade_num;
    double xi, vhat, rho_hat;
    // work counters of the trk and ob searches (search_work), bootstrap
    // included; 0 for RTB
    uint64_t edges_scanned, sigma_adds, states_new, frontier_vertices;
};

void orc_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) { philox4x32_10(ctr, key, out); }

int orc_uniform64(uint64_t N, uint64_t seed, uint64_t i, uint32_t domain, uint64_t* x) {
    return uniform_below64(N, seed, i, domain, x) ? OK : E_RNG;
}

int orc_draw_pair(uint32_t n, uint64_t seed, uint64_t i, uint32_t domain, uint32_t* s, uint32_t* z) {
    return draw_pair(n, seed, i, domain, s, z) ? OK : E_RNG;
}

int orc_rademacher(uint64_t seed, uint64_t i, uint32_t j) { return rademacher(seed, i, j); }

void* orc_graph_new(const uint32_t* u, const uint32_t* v, const uint32_t* t, uint64_t m, uint32_t n) {
    Graph* G = new Graph();
    uint32_t nn = n;
    if (nn == 0) for (uint64_t e = 0; e < m; ++e) nn = std::max(nn, std::max(u[e], v[e]) + 1);
    G->n = nn;
    // the distinct (t,u,v) triples without self loops, ascending
    std::vector<std::tuple<uint32_t, uint32_t, uint32_t>> seen;
    seen.reserve(m);
    for (uint64_t e = 0; e < m; ++e) {
        if (u[e] == v[e]) { G->self_loops++; continue; }
        seen.push_back(std::make_tuple(t[e], u[e], v[e]));
    }
    std::sort(seen.begin(), seen.end());
    const size_t all = seen.size();
    seen.erase(std::unique(seen.begin(), seen.end()), seen.end());
    G->duplicates = all - seen.size();
    G->out.assign(nn, {});
    G->in.assign(nn, {});
    for (const auto& k : seen) {                                  // ascending (t,u,v)
        uint32_t tt = std::get<0>(k), uu = std::get<1>(k), vv = std::get<2>(k);
        G->edges.push_back(std::make_tuple(uu, vv, tt));
        G->out[uu].push_back(std::make_pair(vv, tt));             // so out[u] ascends in t
        G->in[vv].push_back(std::make_pair(uu, tt));
    }
    return G;
}

void orc_graph_free(void* g) { delete (Graph*)g; }

void orc_graph_info(const void* g, uint32_t* n, uint64_t* m, uint64_t* slots, uint64_t* self_loops,
                    uint64_t* duplicates) {
    const Graph* G = (const Graph*)g;
    std::vector<std::pair<uint32_t, uint32_t>> apps;             // arrival appearances (v,t)
    apps.reserve(G->edges.size());
    for (const auto& e : G->edges) apps.push_back(std::make_pair(std::get<1>(e), std::get<2>(e)));
    std::sort(apps.begin(), apps.end());
    *n = G->n; *m = G->edges.size();
    *slots = std::unique(apps.begin(), apps.end()) - apps.begin();
    *self_loops = G->self_loops; *duplicates = G->duplicates;
}

// Deduplicated edges, sorted by (t,u,v).
void orc_graph_edges(const void* g, uint32_t* u, uint32_t* v, uint32_t* t) {
    const Graph* G = (const Graph*)g;
    for (size_t e = 0; e < G->edges.size(); ++e) {
        u[e] = std::get<0>(G->edges[e]); v[e] = std::get<1>(G->edges[e]); t[e] = std::get<2>(G->edges[e]);
    }
}

// sigma_sz for a given pair and optimality; d = hop length of the optimal
// paths for sh/sfm (0 when unreachable), fa(z) for pfm (-1 when unreachable).
int orc_sigma(const void* g, int opt, uint32_t s, uint32_t z, uint64_t* lo, uint64_t* hi, int64_t* d) {
    const Graph* G = (const Graph*)g;
    Search R;
    u128 sg;
    int st = count_paths(*G, opt, s, z, &R, &sg);
    if (st != OK) return st;
    *lo = (uint64_t)sg; *hi = (uint64_t)(sg >> 64);
    if (opt == OPT_PFM) *d = (R.fa[z] == POS_INF) ? -1 : R.fa[z];
    else *d = R.d;
    return OK;
}

// The path named by integer x (0 <= x < sigma_sz); vertices s..z.
// times[q] = arrival time at path[q] (-1 for the source appearance).
int orc_unrank(const void* g, int opt, uint32_t s, uint32_t z, uint64_t x_lo, uint64_t x_hi,
               uint32_t* path, int64_t* times, uint32_t cap, uint32_t* len) {
    const Graph* G = (const Graph*)g;
    Search R;
    u128 sg;
    int st = count_paths(*G, opt, s, z, &R, &sg);
    if (st != OK) return st;
    u128 x = ((u128)x_hi << 64) | x_lo;
    if (x >= sg) return E_INVAL;
    std::vector<uint32_t> p;
    std::vector<int64_t> tt;
    st = unrank_path(*G, opt, s, z, R, x, &p, &tt);
    if (st != OK) return st;
    if (p.size() > cap) return E_INVAL;
    for (size_t q = 0; q < p.size(); ++q) { path[q] = p[q]; times[q] = tt[q]; }
    *len = (uint32_t)p.size();
    return OK;
}

// Samples i0 .. i0+count-1 of the given domains: pair, sigma and the drawn
// path (full vertex list s..z; len 0 when unreachable).
// Per-sample results; path_edges (optional) receives the temporal edge ids of
// each path (len - 1 of them) at the same offsets as paths.
int orc_samples(const void* g, int opt, uint64_t seed, uint64_t i0, uint64_t count, uint32_t dom_pair,
                uint32_t dom_path, uint32_t* s, uint32_t* z, uint64_t* sig_lo, uint64_t* sig_hi, uint32_t* len,
                uint32_t* paths, uint32_t cap, uint32_t* path_edges) {
    const Graph* G = (const Graph*)g;
    for (uint64_t q = 0; q < count; ++q) {
        Sample S;
        int st = one_sample(*G, opt, seed, i0 + q, dom_pair, dom_path, &S, path_edges != nullptr);
        if (st != OK) return st;
        s[q] = S.s; z[q] = S.z;
        sig_lo[q] = (uint64_t)S.sigma; sig_hi[q] = (uint64_t)(S.sigma >> 64);
        len[q] = (uint32_t)S.path.size();
        if (S.path.size() > cap) return E_INVAL;
        for (size_t p = 0; p < S.path.size(); ++p) paths[q * cap + p] = S.path[p];
        if (path_edges)
            for (size_t p = 0; p < S.edges.size(); ++p) path_edges[q * cap + p] = S.edges[p];
    }
    return OK;
}

// Work counters (search_work) of samples i0 .. i0+count-1 of the given
// domains: out[4q .. 4q+3] = escan, eadd, snew, fseg of sample i0+q.
int orc_work(const void* g, int opt, uint64_t seed, uint64_t i0, uint64_t count, uint32_t dom_pair,
             uint32_t dom_path, uint64_t* out) {
    const Graph* G = (const Graph*)g;
    for (uint64_t q = 0; q < count; ++q) {
        Sample S;
        int st = one_sample(*G, opt, seed, i0 + q, dom_pair, dom_path, &S);
        if (st != OK) return st;
        out[4 * q] = S.work.escan; out[4 * q + 1] = S.work.eadd;
        out[4 * q + 2] = S.work.snew; out[4 * q + 3] = S.work.fseg;
    }
    return OK;
}

// Edge ids: for temporal edge id e, its (u, v, t) and its underlying edge id;
// *n_underlying = the number of underlying edges.
void orc_edge_ids(const void* g, uint32_t* u, uint32_t* v, uint32_t* t, uint32_t* uedge, uint32_t* n_underlying) {
    const Graph* G = &edge_ids(*(const Graph*)g);
    for (const auto& kv : G->tid) {
        const uint32_t e = kv.second;
        v[e] = std::get<0>(kv.first); t[e] = std::get<1>(kv.first); u[e] = std::get<2>(kv.first);
        uedge[e] = G->t2u[e];
    }
    *n_underlying = (uint32_t)G->uid.size();
}

// sigma_sz(v) for all v (lo/hi 64-bit halves, n entries each); returns the
// status, sigma_sz in *sig_lo / *sig_hi.
// RTB values of sample i (n entries, 2^-32 units).
int orc_rtb_values(const void* g, int opt, uint64_t seed, uint64_t i, uint32_t dom, uint64_t* q) {
    std::vector<uint64_t> v;
    int st = rtb_values(*(const Graph*)g, opt, seed, i, dom, &v);
    if (st != OK) return st;
    for (size_t k = 0; k < v.size(); ++k) q[k] = v[k];
    return OK;
}

uint64_t orc_muldiv_round(uint64_t a_lo, uint64_t a_hi, uint64_t x, uint64_t d_lo, uint64_t d_hi) {
    return muldiv_round(((u128)a_hi << 64) | a_lo, x, ((u128)d_hi << 64) | d_lo);
}

int orc_through(const void* g, int opt, uint32_t s, uint32_t z, uint64_t* lo, uint64_t* hi, uint64_t* sig_lo,
                uint64_t* sig_hi) {
    const Graph* G = (const Graph*)g;
    Search R;
    u128 sg;
    int st = count_paths(*G, opt, s, z, &R, &sg);
    if (st != OK) return st;
    *sig_lo = (uint64_t)sg; *sig_hi = (uint64_t)(sg >> 64);
    std::vector<u128> th(G->n, 0);
    if (sg != 0) through_counts(*G, opt, s, z, R, &th);
    for (uint32_t v = 0; v < G->n; ++v) { lo[v] = (uint64_t)th[v]; hi[v] = (uint64_t)(th[v] >> 64); }
    return OK;
}

uint64_t orc_fixed32(uint64_t a_lo, uint64_t a_hi, uint64_t b_lo, uint64_t b_hi) {
    return fixed32(((u128)a_hi << 64) | a_lo, ((u128)b_hi << 64) | b_lo);
}

double orc_sd_bound(double Rc, double W, double vhat, double delta, double r, double c) {
    return sd_bound(Rc, W, vhat, delta, r, c);
}

double orc_xi_from_R(double Rb, double vhat, double delta, double r) { return xi_from_R(Rb, vhat, delta, r); }

double orc_wimpy_variance_bound(double W, double delta, double r) { return wimpy_variance_bound(W, delta, r); }

double orc_omega_bound(double vhat, double rho, double eps, double delta) {
    return omega_bound(vhat, rho, eps, delta);
}

// Algorithm 1 (MANTRA).  fixed_r > 0 runs exactly fixed_r samples with no
// bootstrap and no stopping test.  Outputs est[x] = hits[x] / r.
// vhat_mode 0: vhat = W in xi (as Algorithm 1 passes it); 1: vhat = the
// variance bound above, delta_i split evenly between it and xi.
// target 0: the functions are the nodes (f_v = 1 when v is an internal node
// of the drawn path); 1: the underlying edges, 2: the temporal edges (App. A;
// f_e = 1 when the drawn path uses e, first and last edge included), indexed
// by the ids of the Graph.
// estimator 0: trk (App. C, the drawn path's hits); 1: ob (Sec. 4.1, nodes
// only): f_v = sigma_sz(v) / sigma_sz as q = fixed32(.) in 2^-32 units, so
// hits, S, N_R, the wimpy sums (of square32(q)) and sum_int_len are all in
// 2^-32 units and est = hits / (r 2^32); no path is drawn.  ob needs c r < 2^31
// (fixed_r, and omega) so that |N_R| fits int64; max_hits then reports the
// largest wimpy sum.  2: RTB (App. C, nodes only): sample i is a source s
// drawn uniformly from the pair stream's domain, f_v(s) from rtb_values, with
// the same units and limits as ob.
int orc_estimate(const void* g, int opt, double eps, double delta, uint64_t seed, uint32_t c, double growth,
                 uint64_t fixed_r, uint64_t bootstrap, int delta_sched, int vhat_mode, int target, int estimator,
                 double* est, uint64_t* hits_out, orc_info* info) {
    const Graph* G = (const Graph*)g;
    const uint32_t n = G->n;
    if (n < 2 || !(eps > 0 && eps < 1) || !(delta > 0 && delta < 1) || c < 1 || c > 128) return E_INVAL;
    if (target < 0 || target > 2) return E_INVAL;
    if (estimator < 0 || estimator > 2 || (estimator != 0 && target != 0)) return E_INVAL;
    const bool ob = estimator != 0;             // ob and RTB: fractional values in 2^-32 units
    // ob sums are in units of 2^-32; |N_R| <= c r 2^32 must fit int64
    const double scale = ob ? 4294967296.0 : 1.0;
    if (ob && (double)fixed_r * (double)c >= 2147483648.0) return E_INVAL;
    if (target != 0) edge_ids(*G);
    const uint32_t F = target == 0 ? n : (uint32_t)(target == 1 ? G->uid.size() : G->tid.size());
    std::vector<uint64_t> hits(F, 0);
    std::vector<uint64_t> wsq(F, 0);                                        // ob: sum_i f_x(s_i)^2 (2^-32 units)
    std::vector<std::vector<int64_t>> S(c, std::vector<int64_t>(F, 0));     // S[j][x] = sum_i lambda_{j,i} f_x(s_i)
    uint64_t sum_int = 0;
    orc_info I;
    std::memset(&I, 0, sizeof(I));

    // The functions of the family that are 1 on a sample.
    auto items_of = [&](const Sample& sm, std::vector<uint32_t>* it) {
        it->clear();
        if (target == 0) {
            for (size_t p = 1; p + 1 < sm.path.size(); ++p) it->push_back(sm.path[p]);
        } else {
            for (uint32_t e : sm.edges) it->push_back(target == 1 ? G->t2u[e] : e);
        }
    };
    // f^2 of an ob value q = 2^32 f, rounded back to 2^-32 units (ties up).
    auto square32 = [](uint64_t q) { return (uint64_t)(((u128)q * q + ((u128)1 << 31)) >> 32); };
    // Update step for samples [a, b): hits and Rademacher sums (Algorithm 1).
    // the fractional functions of sample i (ob: pair (s,z); RTB: source s)
    auto count_work = [&](const Work& w) {
        I.edges_scanned += w.escan; I.sigma_adds += w.eadd; I.states_new += w.snew; I.frontier_vertices += w.fseg;
    };
    auto frac_values = [&](uint64_t i, uint32_t dom, std::vector<std::pair<uint32_t, uint64_t>>* vals) -> int {
        if (estimator == 1) {
            Work w;
            const int st = ob_values(*G, opt, seed, i, dom, vals, &w);
            count_work(w);
            return st;
        }
        std::vector<uint64_t> q;
        int st = rtb_values(*G, opt, seed, i, dom, &q);
        vals->clear();
        for (uint32_t v = 0; v < n; ++v) if (q[v]) vals->push_back(std::make_pair(v, q[v]));
        return st;
    };
    auto run = [&](uint64_t a, uint64_t b) -> int {
        std::vector<uint32_t> it;
        std::vector<std::pair<uint32_t, uint64_t>> vals;
        for (uint64_t i = a; i < b; ++i) {
            if (ob) {
                int st = frac_values(i, D_PAIR, &vals);
                if (st != OK) return st;
                for (const auto& vq : vals) {
                    hits[vq.first] += vq.second;
                    wsq[vq.first] += square32(vq.second);
                    sum_int += vq.second;
                    for (uint32_t j = 0; j < c; ++j) S[j][vq.first] += rademacher(seed, i, j) * (int64_t)vq.second;
                }
                continue;
            }
            Sample sm;
            int st = one_sample(*G, opt, seed, i, D_PAIR, D_PATH, &sm, target != 0);
            if (st != OK) return st;
            count_work(sm.work);
            items_of(sm, &it);
            for (uint32_t x : it) {
                hits[x] += 1;
                sum_int += 1;
                for (uint32_t j = 0; j < c; ++j) S[j][x] += rademacher(seed, i, j);
            }
        }
        return OK;
    };
    // N_R = sum_j max_x S[j][x] (sup over the whole family, no absolute value),
    // H = max_x hits[x]; both 0 for an empty family.
    auto reduce = [&](int64_t* NR, uint64_t* H) {
        int64_t tot = 0;
        for (uint32_t j = 0; j < c && F > 0; ++j) {
            int64_t mx = S[j][0];
            for (uint32_t x = 1; x < F; ++x) mx = std::max(mx, S[j][x]);
            tot += mx;
        }
        uint64_t h = 0;
        for (uint32_t x = 0; x < F; ++x) h = std::max(h, ob ? wsq[x] : hits[x]);   // trk: f^2 = f
        *NR = tot; *H = h;
    };
    auto vhat_of = [&](uint64_t H, uint64_t r, uint64_t round) {
        double W = (double)H / ((double)r * scale);
        if (vhat_mode != 1) return W;
        return wimpy_variance_bound(W, delta_round(delta, round, delta_sched) / 2.0, (double)r);
    };
    auto xi_of = [&](int64_t NR, uint64_t H, uint64_t r, uint64_t round) {
        double Rc = (double)NR / ((double)c * (double)r * scale);
        double W = (double)H / ((double)r * scale);
        double di = delta_round(delta, round, delta_sched);
        if (vhat_mode == 1) di /= 2.0;
        return sd_bound(Rc, W, vhat_of(H, r, round), di, (double)r, (double)c);
    };

    uint64_t r = 0;
    if (fixed_r > 0) {
        int st = run(0, fixed_r);
        if (st != OK) return st;
        r = fixed_r;
        int64_t NR; uint64_t H;
        reduce(&NR, &H);
        I.rounds = 1; I.rade_num = NR; I.max_hits = H;
        I.xi = xi_of(NR, H, r, 1);
        I.vhat = vhat_of(H, r, 1);
    } else {
        // Bootstrap (DrawSufficientSampleSize with delta/2): s' samples from
        // their own streams, not part of S.
        uint64_t sb = bootstrap ? bootstrap : (uint64_t)std::ceil(std::log(1.0 / delta) / eps);
        std::vector<uint64_t> hb(F, 0);
        uint64_t sum_b = 0;
        std::vector<uint32_t> it;
        std::vector<std::pair<uint32_t, uint64_t>> vals;
        for (uint64_t i = 0; i < sb; ++i) {
            if (ob) {                       // hb: sum of f^2 (the wimpy numerator), sum_b: sum of f
                int st = frac_values(i, D_BOOT_PAIR, &vals);
                if (st != OK) return st;
                for (const auto& vq : vals) { hb[vq.first] += square32(vq.second); sum_b += vq.second; }
                continue;
            }
            Sample sm;
            int st = one_sample(*G, opt, seed, i, D_BOOT_PAIR, D_BOOT_PATH, &sm, target != 0);
            if (st != OK) return st;
            count_work(sm.work);
            items_of(sm, &it);
            for (uint32_t x : it) { hb[x] += 1; sum_b += 1; }
        }
        uint64_t Hb = 0;
        for (uint32_t x = 0; x < F; ++x) Hb = std::max(Hb, hb[x]);
        double v0 = (double)Hb / ((double)sb * scale);
        double rho = (double)sum_b / ((double)sb * scale);
        if (v0 == 0.0 || rho == 0.0) { v0 = 1.0 / (double)sb; rho = std::max(rho, v0); }
        uint64_t omega = (uint64_t)std::ceil(omega_bound(v0, rho, eps, delta / 2.0));
        if (omega < 1) omega = 1;
        if (ob && (double)omega * (double)c >= 2147483648.0) return E_INVAL;
        // SamplingSchedule: least s in [s', omega] with xi(R = 0) <= eps.
        uint64_t s1;
        double d1 = delta_round(delta, 1, delta_sched);
        // Theorem 1's xi with R set to 0 (Sec. 4.4, bootstrap phase).
        auto xi0 = [&](uint64_t s) { return xi_from_R(0.0, v0, d1, (double)s); };
        if (sb >= omega) s1 = omega;
        else if (xi0(omega) > eps) s1 = omega;
        else {
            uint64_t lo = sb, hi = omega;              // xi0(hi) <= eps
            while (lo < hi) {
                uint64_t mid = lo + (hi - lo) / 2;
                if (xi0(mid) <= eps) hi = mid; else lo = mid + 1;
            }
            s1 = lo;
        }
        I.bootstrap = sb; I.omega = omega; I.s1 = s1; I.rho_hat = rho;
        uint64_t target = s1, round = 0;
        while (true) {
            round += 1;
            int st = run(r, target);
            if (st != OK) return st;
            r = target;
            int64_t NR; uint64_t H;
            reduce(&NR, &H);
            double xi = xi_of(NR, H, r, round);
            I.rounds = round; I.rade_num = NR; I.max_hits = H; I.xi = xi; I.vhat = vhat_of(H, r, round);
            if (r >= omega || xi <= eps) break;
            uint64_t nt = (uint64_t)std::ceil(growth * (double)target);
            if (nt <= target) nt = target + 1;
            target = std::min(omega, nt);
        }
    }
    I.r = r;
    I.sum_int_len = sum_int;
    for (uint32_t x = 0; x < F; ++x) {
        est[x] = (double)hits[x] / ((double)r * scale);
        if (hits_out) hits_out[x] = hits[x];
    }
    if (info) *info = I;
    return OK;
}

// Hop distances from u (UINT32_MAX: unreached; u itself excluded).
// sh / sfm: level of v's first appearance; fsfm: level of v's earliest
// appearance; pfm: minimum hops among prefix-foremost paths.
int distances_from(const Graph& G, int opt, uint32_t u, std::vector<uint32_t>* dist) {
    const uint32_t n = G.n;
    dist->assign(n, UINT32_MAX);
    if (opt == OPT_PFM) {
        Search R = pfm_scan(G, u);
        if (R.status != OK) return R.status;
        for (uint32_t v = 0; v < n; ++v) if (v != u && R.fa[v] != POS_INF) (*dist)[v] = R.hop[v];
        return OK;
    }
    Search R = tbfs_levels(G, u, n);
    if (R.status != OK) return R.status;
    std::vector<bool> seen(n, false);
    for (const auto& kv : R.st) {             // map order: by vertex, then ascending time
        const uint32_t x = kv.first.first;
        if (x == u) continue;
        if (opt == OPT_FSFM) {                // hops of the earliest appearance
            if (!seen[x]) (*dist)[x] = kv.second.level;
            seen[x] = true;
        } else {
            (*dist)[x] = std::min((*dist)[x], kv.second.level);
        }
    }
    return OK;
}

// Algorithm 2: r_s full searches from sources u_k (uniform in [0,n) from the
// STATS stream, or every node once when all_sources != 0).  cnt[h] counts
// reached nodes v != u at distance h (distances_from); reach[h] = sum_{h' <= h}
// cnt[h'].  reach must hold n entries; returns D_LB.
int orc_stats(const void* g, int opt, uint64_t seed, uint64_t r_s, int all_sources, uint64_t* reach,
              uint32_t* d_lb) {
    const Graph* G = (const Graph*)g;
    const uint32_t n = G->n;
    std::vector<uint64_t> cnt(n + 1, 0);
    uint32_t D = 0;
    uint64_t count = all_sources ? n : r_s;
    std::vector<uint32_t> dist;
    for (uint64_t k = 0; k < count; ++k) {
        uint64_t u64;
        if (all_sources) u64 = k;
        else if (!uniform_below64(n, seed, k, D_STATS, &u64)) return E_RNG;
        int st = distances_from(*G, opt, (uint32_t)u64, &dist);
        if (st != OK) return st;
        for (uint32_t v = 0; v < n; ++v)
            if (dist[v] != UINT32_MAX) { cnt[dist[v]] += 1; D = std::max(D, dist[v]); }
    }
    uint64_t acc = 0;
    for (uint32_t h = 0; h < n; ++h) { acc += cnt[h]; reach[h] = acc; }
    *d_lb = D;
    return OK;
}

// Temporal closeness from Algorithm 2's searches (the appendix remarks that
// they give a fast closeness approximation; the harmonic form is the reading
// used here): over the same r_s sources, sum[v] = sum_k round(2^32 / d(u_k, v))
// (ties up; 0 when unreached or u_k = v), and
//   closeness[v] = sum[v] n / (2^32 r_s (n-1)),
// an unbiased estimate of 1/(n-1) sum_{u != v} 1/d(u,v) up to the rounding.
int orc_closeness(const void* g, int opt, uint64_t seed, uint64_t r_s, uint64_t* sum, double* closeness) {
    const Graph* G = (const Graph*)g;
    const uint32_t n = G->n;
    std::vector<uint32_t> dist;
    for (uint32_t v = 0; v < n; ++v) sum[v] = 0;
    for (uint64_t k = 0; k < r_s; ++k) {
        uint64_t u64;
        if (!uniform_below64(n, seed, k, D_STATS, &u64)) return E_RNG;
        int st = distances_from(*G, opt, (uint32_t)u64, &dist);
        if (st != OK) return st;
        for (uint32_t v = 0; v < n; ++v)
            if (dist[v] != UINT32_MAX) sum[v] += (((uint64_t)1 << 33) + dist[v]) / (2 * (uint64_t)dist[v]);
    }
    for (uint32_t v = 0; v < n; ++v)
        closeness[v] = ((double)sum[v] * (double)n) / (4294967296.0 * (double)r_s * (double)(n - 1));
    return OK;
}

// Exact (*)-temporal betweenness (Sec. 3): b_v = 1/(n(n-1)) sum_{s != v != z}
// sigma_sz(v) / sigma_sz, with sigma_sz(v) from through_counts.  Long double
// accumulation.  Small graphs only.
int orc_exact_bc(const void* g, int opt, double* bc) {
    const Graph* G = (const Graph*)g;
    const uint32_t n = G->n;
    std::vector<long double> acc(n, 0.0L);
    for (uint32_t s = 0; s < n; ++s) {
        for (uint32_t z = 0; z < n; ++z) {
            if (s == z) continue;
            Search R;
            u128 sg;
            int st = count_paths(*G, opt, s, z, &R, &sg);
            if (st != OK) return st;
            if (sg == 0) continue;
            std::vector<u128> through;
            through_counts(*G, opt, s, z, R, &through);
            for (uint32_t v = 0; v < n; ++v)
                if (through[v]) acc[v] += (long double)through[v] / (long double)sg;
        }
    }
    long double norm = (long double)n * (long double)(n - 1);
    for (uint32_t v = 0; v < n; ++v) bc[v] = (double)(acc[v] / norm);
    return OK;
}

}  // extern "C"
