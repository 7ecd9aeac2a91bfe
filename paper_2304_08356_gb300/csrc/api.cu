// Host side of libmantra.so: the temporal-edge store, the Algorithm 1 driver
// (bootstrap, sampling schedule, rounds, stopping test), Algorithm 2's host
// formulas and the C ABI declared in include/mantra.h.
#include "mantra.h"
#include "mantra_dev.cuh"

#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

using namespace mantra;

struct mantra_graph {
    uint32_t n = 0, A = 0, m = 0;
    uint64_t self_loops = 0, duplicates = 0;
    DevGraph dg{};
    void* dmem = nullptr;
    cudaStream_t stream = nullptr;
    int device = 0, num_sms = 0;
    size_t smem_optin = 0;
    std::mutex mu;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    // search workspaces (allocated on first use, kept with the graph)
    char* bfs_mem = nullptr; BfsWs bws{}; int bfs_grid = 0; size_t bfs_smem = 0;
    char* pfm_mem = nullptr; PfmWs pws{}; int pfm_grid = 0; size_t pfm_bytes = 0;
    // run buffers
    char* run_mem = nullptr; size_t run_bytes = 0; uint32_t run_c = 0; uint64_t run_cap = 0;
    u64* hits = nullptr; int* S = nullptr; u64* ctr = nullptr; int* status = nullptr;
    long long* rowmax = nullptr; u64* hmax = nullptr; uint64_t* ovf = nullptr; uint64_t* ovf2 = nullptr;
    u64* cnt = nullptr; u64* dmax = nullptr; double* est = nullptr;
    u64* host_ctr = nullptr;   // pinned mirror: counters, status, rowmax, hmax
};

namespace {

#define CU(x) do { cudaError_t e_ = (x); if (e_ != cudaSuccess) return MANTRA_E_CUDA; } while (0)

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

struct HostEdge { uint32_t t, u, v; };

// ---------------------------------------------------------------------------
// Temporal-edge store (paper Sec. 3: the temporal graph; the paper's own code
// keeps a sparse n x |T| table, here every arrival appearance (v,t) gets a
// dense slot id).
// ---------------------------------------------------------------------------
int build_store(const uint32_t* u, const uint32_t* v, const uint32_t* t, uint64_t m, uint32_t n, mantra_graph* G) {
    if (n == 0) {
        for (uint64_t e = 0; e < m; ++e) n = std::max(n, std::max(u[e], v[e]) + 1);
    }
    if (n < 2) return MANTRA_E_INVAL;
    std::vector<HostEdge> es;
    try { es.reserve(m); } catch (...) { return MANTRA_E_NOMEM; }
    uint64_t loops = 0;
    for (uint64_t e = 0; e < m; ++e) {
        if (u[e] >= n || v[e] >= n || t[e] > 0xFFFFFFFDu) return MANTRA_E_INVAL;
        if (u[e] == v[e]) { ++loops; continue; }
        es.push_back(HostEdge{t[e], u[e], v[e]});
    }
    auto by_tuv = [](const HostEdge& a, const HostEdge& b) {
        if (a.t != b.t) return a.t < b.t;
        if (a.u != b.u) return a.u < b.u;
        return a.v < b.v;
    };
    std::sort(es.begin(), es.end(), by_tuv);
    auto same = [](const HostEdge& a, const HostEdge& b) { return a.t == b.t && a.u == b.u && a.v == b.v; };
    const size_t before = es.size();
    es.erase(std::unique(es.begin(), es.end(), same), es.end());
    if (es.size() >= 0xFFFFFFF0ull) return MANTRA_E_INVAL;
    const uint32_t M = (uint32_t)es.size();
    G->n = n; G->m = M; G->self_loops = loops; G->duplicates = before - es.size();

    std::vector<uint32_t> st_u(M), st_v(M), st_t(M);
    for (uint32_t e = 0; e < M; ++e) { st_u[e] = es[e].u; st_v[e] = es[e].v; st_t[e] = es[e].t; }

    // in-CSR by (v, t, u) and slots
    std::vector<HostEdge> ein(es);
    std::sort(ein.begin(), ein.end(), [](const HostEdge& a, const HostEdge& b) {
        if (a.v != b.v) return a.v < b.v;
        if (a.t != b.t) return a.t < b.t;
        return a.u < b.u;
    });
    std::vector<uint32_t> in_u(M), in_slot(M), slot_t, slot_v, slot_in, slot_ptr(n + 1, 0);
    slot_t.reserve(M); slot_v.reserve(M); slot_in.reserve(M + 1);
    for (uint32_t e = 0; e < M; ++e) {
        if (e == 0 || ein[e].v != ein[e - 1].v || ein[e].t != ein[e - 1].t) {
            slot_t.push_back(ein[e].t); slot_v.push_back(ein[e].v); slot_in.push_back(e);
            slot_ptr[ein[e].v + 1] += 1;
        }
        in_u[e] = ein[e].u;
        in_slot[e] = (uint32_t)slot_t.size() - 1;
    }
    const uint32_t A = (uint32_t)slot_t.size();
    slot_in.push_back(M);
    for (uint32_t x = 0; x < n; ++x) slot_ptr[x + 1] += slot_ptr[x];
    G->A = A;

    // out-CSR by (u, t, v)
    std::vector<HostEdge> eo(std::move(ein));
    std::sort(eo.begin(), eo.end(), [](const HostEdge& a, const HostEdge& b) {
        if (a.u != b.u) return a.u < b.u;
        if (a.t != b.t) return a.t < b.t;
        return a.v < b.v;
    });
    std::vector<uint32_t> out_ptr(n + 1, 0), out_v(M), out_t(M), out_slot(M);
    for (uint32_t e = 0; e < M; ++e) {
        out_ptr[eo[e].u + 1] += 1;
        out_v[e] = eo[e].v; out_t[e] = eo[e].t;
        const uint32_t* b = slot_t.data() + slot_ptr[eo[e].v];
        const uint32_t* f = slot_t.data() + slot_ptr[eo[e].v + 1];
        out_slot[e] = (uint32_t)(std::lower_bound(b, f, eo[e].t) - slot_t.data());
    }
    for (uint32_t x = 0; x < n; ++x) out_ptr[x + 1] += out_ptr[x];
    std::vector<uint32_t> tmax_in(n, 0), tmin_out(n, 0);
    for (uint32_t x = 0; x < n; ++x) {
        if (slot_ptr[x + 1] > slot_ptr[x]) tmax_in[x] = slot_t[slot_ptr[x + 1] - 1];
        if (out_ptr[x + 1] > out_ptr[x]) tmin_out[x] = out_t[out_ptr[x]];
    }

    // one device allocation for the whole store
    struct Arr { const std::vector<uint32_t>* h; const uint32_t** d; };
    Arr arrs[] = {{&out_ptr, &G->dg.out_ptr}, {&out_v, &G->dg.out_v}, {&out_t, &G->dg.out_t},
                  {&out_slot, &G->dg.out_slot}, {&slot_ptr, &G->dg.slot_ptr}, {&slot_t, &G->dg.slot_t},
                  {&slot_v, &G->dg.slot_v}, {&slot_in, &G->dg.slot_in}, {&in_u, &G->dg.in_u},
                  {&in_slot, &G->dg.in_slot}, {&st_u, &G->dg.st_u}, {&st_v, &G->dg.st_v},
                  {&st_t, &G->dg.st_t}, {&tmax_in, &G->dg.tmax_in}, {&tmin_out, &G->dg.tmin_out}};
    size_t total = 0;
    for (auto& a : arrs) total += al256((a.h->size() + 1) * 4);
    if (cudaMalloc(&G->dmem, total) != cudaSuccess) return MANTRA_E_NOMEM;
    size_t off = 0;
    for (auto& a : arrs) {
        char* p = (char*)G->dmem + off;
        if (!a.h->empty()) CU(cudaMemcpyAsync(p, a.h->data(), a.h->size() * 4, cudaMemcpyHostToDevice, G->stream));
        *a.d = (const uint32_t*)p;
        off += al256((a.h->size() + 1) * 4);
    }
    CU(cudaStreamSynchronize(G->stream));
    G->dg.n = n; G->dg.A = A; G->dg.m = M;
    return MANTRA_OK;
}

size_t free_device_bytes() {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) return 0;
    return fr;
}

// Search workspaces: one region per CTA (sh/sfm) or per warp (pfm), sized to
// at most `budget` bytes.  The sigma arrays and global bitmaps start zeroed;
// every sample leaves them zeroed.
int ensure_bfs_ws(mantra_graph* G, cudaStream_t st) {
    if (G->bfs_mem) return MANTRA_OK;
    const size_t smem = bfs_smem_bytes(G->A);
    const bool in_smem = smem + 1024 <= G->smem_optin;
    const size_t region = bfs_region_bytes(G->n, G->A, in_smem, &G->bws);
    const size_t budget = free_device_bytes() / 3;
    int grid = G->num_sms;
    if ((size_t)grid * region > budget) grid = (int)std::max<size_t>(1, budget / region);
    if (cudaMalloc(&G->bfs_mem, (size_t)grid * region) != cudaSuccess) { G->bfs_mem = nullptr; return MANTRA_E_NOMEM; }
    CU(cudaMemsetAsync(G->bfs_mem, 0, (size_t)grid * region, st));
    G->bws.base = G->bfs_mem;
    G->bws.stride = region;
    G->bfs_grid = grid;
    G->bfs_smem = in_smem ? smem : 0;
    CU(bfs_configure(G->bfs_smem));
    return MANTRA_OK;
}

// pfm: one region per warp (32 samples), grown to the largest launch seen, at
// most one warp slot per 32 resident threads and at most a third of free memory.
int ensure_pfm_ws(mantra_graph* G, uint64_t count) {
    const int wpb = pfm_threads() / 32;
    const uint64_t max_warps = (uint64_t)G->num_sms * 32;
    const uint64_t want = std::min<uint64_t>(std::max<uint64_t>((count + 31) / 32, 1), max_warps);
    const uint64_t have = (uint64_t)G->pfm_grid * wpb;
    if (G->pfm_mem && have >= want) return MANTRA_OK;
    const size_t region = pfm_region_bytes(G->n, &G->pws);
    if (G->pfm_mem) { cudaFree(G->pfm_mem); G->pfm_mem = nullptr; }
    const size_t budget = free_device_bytes() / 3;
    uint64_t warps = std::min<uint64_t>(want, std::max<size_t>(budget / region, (size_t)wpb));
    const int blocks = (int)((warps + wpb - 1) / wpb);
    if (cudaMalloc(&G->pfm_mem, (size_t)blocks * wpb * region) != cudaSuccess) {
        G->pfm_mem = nullptr; G->pfm_grid = 0; return MANTRA_E_NOMEM;
    }
    G->pws.base = G->pfm_mem;
    G->pws.stride = region;
    G->pfm_grid = blocks;
    G->pfm_bytes = (size_t)blocks * wpb * region;
    return MANTRA_OK;
}

// Run buffers for n nodes, c trials and up to `cap` samples per launch.
int ensure_run(mantra_graph* G, uint32_t c, uint64_t cap) {
    if (G->run_mem && G->run_c >= c && G->run_cap >= cap) return MANTRA_OK;
    if (G->run_mem) { cudaFree(G->run_mem); G->run_mem = nullptr; }
    if (!G->host_ctr) {
        if (cudaMallocHost(&G->host_ctr, 4096) != cudaSuccess) { G->host_ctr = nullptr; return MANTRA_E_NOMEM; }
    }
    const uint32_t n = G->n;
    c = std::max(c, 25u);
    cap = std::max<uint64_t>(cap, 1024);
    size_t o = 0;
    const size_t o_hits = o; o = al256(o + (size_t)n * 8);
    const size_t o_S = o;    o = al256(o + (size_t)c * n * 4);
    const size_t o_ctr = o;  o = al256(o + 4096);   // counters + status + rowmax + hmax + dmax (mirrors host_ctr)
    const size_t o_ovf = o;  o = al256(o + cap * 8);
    const size_t o_ovf2 = o; o = al256(o + cap * 8);
    const size_t o_cnt = o;  o = al256(o + ((size_t)n + 2) * 8);
    const size_t o_est = o;  o = al256(o + (size_t)n * 8);
    if (cudaMalloc(&G->run_mem, o) != cudaSuccess) { G->run_mem = nullptr; return MANTRA_E_NOMEM; }
    char* b = G->run_mem;
    G->hits = (u64*)(b + o_hits);
    G->S = (int*)(b + o_S);
    G->ctr = (u64*)(b + o_ctr);                     // [0, 8): counters
    G->status = (int*)(b + o_ctr + 64);             // one int
    G->hmax = (u64*)(b + o_ctr + 128);
    G->dmax = (u64*)(b + o_ctr + 136);
    G->rowmax = (long long*)(b + o_ctr + 256);      // up to 128 rows
    G->ovf = (uint64_t*)(b + o_ovf);
    G->ovf2 = (uint64_t*)(b + o_ovf2);
    G->cnt = (u64*)(b + o_cnt);
    G->est = (double*)(b + o_est);
    G->run_bytes = o; G->run_c = c; G->run_cap = cap;
    return MANTRA_OK;
}

struct LaunchTotals {
    uint64_t sum_int = 0, escan = 0, eadd = 0, snew = 0, fseg = 0, wide = 0, launches = 0;
    double kernel_ms = 0;
};

// Algorithmic bytes of search work (64-bit path counts):
//   pfm    4 B fa(u) per (sample, edge) + the 12 B edge shared by the 32 samples of a
//          warp + 24 B per path-count update (sigma(u) read, sigma(v) read-modify-write)
//   sh/sfm 12 B edge record + 12 B level test and path-count update per examined edge,
//          8 B row bounds per frontier vertex, 12 B per discovered state
uint64_t alg_bytes_of(bool pfm, uint64_t escan, uint64_t eadd, uint64_t snew, uint64_t fseg) {
    if (pfm) return 4ull * escan + (12ull * escan) / 32 + 24ull * eadd;
    return 24ull * escan + 8ull * fseg + 12ull * snew;
}

void log_launch(bool pfm, bool wide, const Job& j, const u64* h, float ms) {
    static const bool on = std::getenv("MANTRA_LOG_LAUNCHES") != nullptr;
    if (!on) return;
    std::fprintf(stderr, "mantra-launch kernel=%s%s samples=%llu escan=%llu eadd=%llu snew=%llu fseg=%llu "
                 "alg_bytes=%llu ms=%.4f\n", pfm ? "k_pfm" : "k_bfs", wide ? "<wide>" : "",
                 (unsigned long long)j.count, (unsigned long long)h[C_ESCAN], (unsigned long long)h[C_EADD],
                 (unsigned long long)h[C_SNEW], (unsigned long long)h[C_FSEG],
                 (unsigned long long)alg_bytes_of(pfm, h[C_ESCAN], h[C_EADD], h[C_SNEW], h[C_FSEG]), ms);
}

// One search launch over sample indices [i0, i0+count) (Algorithm 1's
// Update step, or Algorithm 2's searches when job.stats), followed by a
// 128-bit re-run of the samples whose 64-bit path counts overflowed.
int run_samples(mantra_graph* G, Job job, cudaStream_t st, LaunchTotals* tot) {
    if (job.count == 0) return MANTRA_OK;
    const bool pfm = job.opt == MANTRA_PFM;
    int rc = pfm ? ensure_pfm_ws(G, job.count) : ensure_bfs_ws(G, st);
    if (rc != MANTRA_OK) return rc;
    if (job.count > G->run_cap) return MANTRA_E_INVAL;
    job.ctr = G->ctr; job.status = G->status; job.ovf_list = G->ovf;
    CU(cudaMemsetAsync(G->ctr, 0, 64 + 4, st));
    CU(cudaEventRecord(G->ev0, st));
    if (pfm) CU(launch_pfm(G->dg, job, G->pws, G->pfm_grid, false, st));
    else CU(launch_bfs(G->dg, job, G->bws, G->bfs_grid, G->bfs_smem, false, st));
    CU(cudaEventRecord(G->ev1, st));
    CU(cudaMemcpyAsync(G->host_ctr, G->ctr, 72, cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    float ms = 0;
    CU(cudaEventElapsedTime(&ms, G->ev0, G->ev1));
    tot->kernel_ms += ms;
    tot->launches += 1;
    u64 h[9];
    std::memcpy(h, G->host_ctr, 72);
    log_launch(pfm, false, job, h, ms);
    int status = (int)(h[8] & 0xFFFFFFFFu);
    if (status != 0) return status;
    tot->sum_int += h[C_SUMINT]; tot->escan += h[C_ESCAN]; tot->eadd += h[C_EADD]; tot->snew += h[C_SNEW];
    tot->fseg += h[C_FSEG];
    const uint64_t novf = h[C_NOVF];
    if (novf) {
        Job w = job;
        w.idx_list = G->ovf;
        w.count = novf;
        w.ovf_list = G->ovf2;
        CU(cudaMemsetAsync(G->ctr, 0, 64 + 4, st));
        CU(cudaEventRecord(G->ev0, st));
        if (pfm) CU(launch_pfm(G->dg, w, G->pws, G->pfm_grid, true, st));
        else CU(launch_bfs(G->dg, w, G->bws, G->bfs_grid, G->bfs_smem, true, st));
        CU(cudaEventRecord(G->ev1, st));
        CU(cudaMemcpyAsync(G->host_ctr, G->ctr, 72, cudaMemcpyDeviceToHost, st));
        CU(cudaStreamSynchronize(st));
        CU(cudaEventElapsedTime(&ms, G->ev0, G->ev1));
        tot->kernel_ms += ms;
        tot->launches += 1;
        std::memcpy(h, G->host_ctr, 72);
        log_launch(pfm, true, w, h, ms);
        status = (int)(h[8] & 0xFFFFFFFFu);
        if (status != 0) return status;
        tot->sum_int += h[C_SUMINT]; tot->escan += h[C_ESCAN]; tot->eadd += h[C_EADD]; tot->snew += h[C_SNEW];
        tot->fseg += h[C_FSEG];
        tot->wide += novf;
    }
    return MANTRA_OK;
}

// Reduction after a round: N_R = sum_j max_v S[j][v] and H = max_v hits[v].
int round_reduce(mantra_graph* G, uint32_t c, bool with_S, cudaStream_t st, int64_t* NR, uint64_t* H) {
    CU(launch_round_reduce(with_S ? G->S : nullptr, G->hits, G->n, with_S ? c : 0, G->rowmax, G->hmax, st));
    CU(cudaMemcpyAsync((char*)G->host_ctr + 128, G->hmax, 8, cudaMemcpyDeviceToHost, st));
    if (with_S) CU(cudaMemcpyAsync((char*)G->host_ctr + 256, G->rowmax, (size_t)c * 8, cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    std::memcpy(H, (char*)G->host_ctr + 128, 8);
    int64_t s = 0;
    if (with_S) {
        for (uint32_t j = 0; j < c; ++j) {
            long long x;
            std::memcpy(&x, (char*)G->host_ctr + 256 + 8 * j, 8);
            s += x;
        }
    }
    *NR = s;
    return MANTRA_OK;
}

// Theorem 1 (supremum-deviation bound) pieces, natural logarithms.
double xi_given_R(double R, double vhat, double delta_i, double r) {
    const double L = std::log(4.0 / delta_i);
    return 2.0 * R + std::sqrt(2.0 * L * (vhat + 4.0 * R) / r) + L / (3.0 * r);
}

double xi_from_mcera(double Rc, double W, double vhat, double delta_i, double r, double c) {
    const double L = std::log(4.0 / delta_i);
    const double Rt = Rc + std::sqrt(4.0 * W * L / (c * r));
    const double R = Rt + L / r + std::sqrt((L / r) * (L / r) + 2.0 * L * Rt / r);
    return xi_given_R(R, vhat, delta_i, r);
}

// Closed form of the MCERA sample bound (end of the proof of Theorem 3).
double omega_closed_form(double vhat, double rho, double eps, double delta) {
    return ((2.0 * vhat + 2.0 * eps / 3.0) / (eps * eps)) * (std::log(2.0 * rho / vhat) + std::log(1.0 / delta));
}

double delta_of_round(double delta, uint64_t i, int sched) {
    return sched == 1 ? delta / std::ldexp(1.0, (int)i) : delta / std::ldexp(1.0, (int)(i + 1));
}

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

int init_graph_device(mantra_graph* G) {
    CU(cudaGetDevice(&G->device));
    CU(cudaDeviceGetAttribute(&G->num_sms, cudaDevAttrMultiProcessorCount, G->device));
    int optin = 0;
    CU(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, G->device));
    G->smem_optin = (size_t)optin;
    CU(cudaStreamCreateWithFlags(&G->stream, cudaStreamNonBlocking));
    CU(cudaEventCreate(&G->ev0));
    CU(cudaEventCreate(&G->ev1));
    return MANTRA_OK;
}

}  // namespace

namespace mantra {

// Read-only view of a loaded graph for the library's other translation units.
const DevGraph* graph_view(const mantra_graph* g, uint32_t* n, uint32_t* A, int* num_sms, size_t* smem_optin,
                           std::mutex** mu) {
    mantra_graph* G = const_cast<mantra_graph*>(g);
    *n = G->n; *A = G->A; *num_sms = G->num_sms; *smem_optin = G->smem_optin; *mu = &G->mu;
    return &G->dg;
}

}  // namespace mantra

extern "C" {

const char* mantra_strerror(int code) {
    switch (code) {
        case MANTRA_OK: return "ok";
        case MANTRA_E_INVAL: return "invalid argument";
        case MANTRA_E_NOMEM: return "out of memory";
        case MANTRA_E_OVERFLOW: return "path count exceeds 128 bits";
        case MANTRA_E_CUDA: return "CUDA runtime error";
        case MANTRA_E_TIMEOUT: return "device wait timed out";
        case MANTRA_E_CHECK: return "device consistency check failed";
        case MANTRA_E_RNG: return "random draw rejected too often";
        default: return "unknown error";
    }
}

int mantra_graph_load(const uint32_t* u, const uint32_t* v, const uint32_t* t, uint64_t m, uint32_t n,
                      mantra_graph** out) {
    if (!out || (m > 0 && (!u || !v || !t))) return MANTRA_E_INVAL;
    *out = nullptr;
    mantra_graph* G = new (std::nothrow) mantra_graph();
    if (!G) return MANTRA_E_NOMEM;
    int rc = init_graph_device(G);
    if (rc == MANTRA_OK) rc = build_store(u, v, t, m, n, G);
    if (rc != MANTRA_OK) { mantra_graph_free(G); return rc; }
    *out = G;
    return MANTRA_OK;
}

int mantra_graph_info(const mantra_graph* g, uint32_t* n, uint64_t* m_dedup, uint64_t* slots,
                      uint64_t* self_loops_dropped, uint64_t* duplicates_dropped) {
    if (!g) return MANTRA_E_INVAL;
    if (n) *n = g->n;
    if (m_dedup) *m_dedup = g->m;
    if (slots) *slots = g->A;
    if (self_loops_dropped) *self_loops_dropped = g->self_loops;
    if (duplicates_dropped) *duplicates_dropped = g->duplicates;
    return MANTRA_OK;
}

void mantra_graph_free(mantra_graph* g) {
    if (!g) return;
    if (g->stream) cudaStreamSynchronize(g->stream);
    if (g->dmem) cudaFree(g->dmem);
    if (g->bfs_mem) cudaFree(g->bfs_mem);
    if (g->pfm_mem) cudaFree(g->pfm_mem);
    if (g->run_mem) cudaFree(g->run_mem);
    if (g->host_ctr) cudaFreeHost(g->host_ctr);
    if (g->ev0) cudaEventDestroy(g->ev0);
    if (g->ev1) cudaEventDestroy(g->ev1);
    if (g->stream) cudaStreamDestroy(g->stream);
    delete g;
}

int mantra_estimate(const mantra_graph* gc, mantra_opt opt, double eps, double delta, uint64_t seed,
                    const mantra_opts* opts, double* est_out, uint64_t* hits_out, mantra_info* info) {
    if (!gc || !est_out) return MANTRA_E_INVAL;
    if (!(eps > 0.0 && eps < 1.0) || !(delta > 0.0 && delta < 1.0)) return MANTRA_E_INVAL;
    if (opt != MANTRA_SH && opt != MANTRA_SFM && opt != MANTRA_PFM) return MANTRA_E_INVAL;
    mantra_opts o{};
    if (opts) o = *opts;
    const uint32_t c = o.c ? o.c : 25;
    const double growth = o.growth > 0 ? o.growth : 1.2;
    if (c < 1 || c > 128 || growth <= 1.0) return MANTRA_E_INVAL;
    mantra_graph* G = const_cast<mantra_graph*>(gc);
    std::lock_guard<std::mutex> lock(G->mu);
    const double t0 = now_s();
    cudaStream_t st = o.stream ? (cudaStream_t)o.stream : G->stream;
    const uint32_t n = G->n;
    const uint64_t RMAX = 0x7FFFFFFFull;

    mantra_info I;
    std::memset(&I, 0, sizeof(I));
    LaunchTotals T;

    Job base{};
    base.seed = seed; base.opt = (int)opt; base.c = c;

    uint64_t r = 0, reduces = 0;
    int rc;
    if (o.fixed_r > 0) {
        if (o.fixed_r > RMAX) return MANTRA_E_INVAL;
        if ((rc = ensure_run(G, c, o.fixed_r)) != MANTRA_OK) return rc;
        CU(cudaMemsetAsync(G->hits, 0, (size_t)n * 8, st));
        CU(cudaMemsetAsync(G->S, 0, (size_t)c * n * 4, st));
        Job j = base;
        j.i0 = 0; j.count = o.fixed_r; j.dom_pair = DOM_PAIR; j.dom_path = DOM_PATH;
        j.hits = G->hits; j.S = G->S;
        if ((rc = run_samples(G, j, st, &T)) != MANTRA_OK) return rc;
        r = o.fixed_r;
        int64_t NR; uint64_t H;
        if ((rc = round_reduce(G, c, true, st, &NR, &H)) != MANTRA_OK) return rc;
        reduces += 1;
        I.rounds = 1; I.rade_num = NR; I.max_hits = H;
        const double W = (double)H / (double)r;
        I.vhat = W;
        I.xi = xi_from_mcera((double)NR / ((double)c * (double)r), W, W, delta_of_round(delta, 1, o.delta_sched),
                             (double)r, (double)c);
    } else {
        // bootstrap: DrawSufficientSampleSize(G, s', delta/2)
        const uint64_t sb = o.bootstrap ? o.bootstrap : (uint64_t)std::ceil(std::log(1.0 / delta) / eps);
        if (sb > RMAX) return MANTRA_E_INVAL;
        if ((rc = ensure_run(G, c, std::max<uint64_t>(sb, 4096))) != MANTRA_OK) return rc;
        CU(cudaMemsetAsync(G->hits, 0, (size_t)n * 8, st));
        Job jb = base;
        jb.i0 = 0; jb.count = sb; jb.dom_pair = DOM_BOOT_PAIR; jb.dom_path = DOM_BOOT_PATH;
        jb.hits = G->hits; jb.S = nullptr;
        LaunchTotals TB;
        if ((rc = run_samples(G, jb, st, &TB)) != MANTRA_OK) return rc;
        int64_t NRb; uint64_t Hb;
        if ((rc = round_reduce(G, c, false, st, &NRb, &Hb)) != MANTRA_OK) return rc;
        reduces += 1;
        double v0 = (double)Hb / (double)sb;
        double rho = (double)TB.sum_int / (double)sb;
        if (v0 == 0.0 || rho == 0.0) { v0 = 1.0 / (double)sb; rho = std::max(rho, v0); }
        const double om = std::ceil(omega_closed_form(v0, rho, eps, delta / 2.0));
        if (!(om <= (double)RMAX)) return MANTRA_E_INVAL;
        const uint64_t omega = std::max<uint64_t>(1, (uint64_t)om);
        // SamplingSchedule: least s in [s', omega] with xi(R = 0) <= eps
        const double d1 = delta_of_round(delta, 1, o.delta_sched);
        uint64_t s1;
        if (sb >= omega || xi_given_R(0.0, v0, d1, (double)omega) > eps) s1 = omega;
        else {
            uint64_t lo = sb, hi = omega;
            while (lo < hi) {
                const uint64_t mid = lo + (hi - lo) / 2;
                if (xi_given_R(0.0, v0, d1, (double)mid) <= eps) hi = mid; else lo = mid + 1;
            }
            s1 = lo;
        }
        I.bootstrap = sb; I.omega = omega; I.s1 = s1; I.rho_hat = rho;
        T.kernel_ms += TB.kernel_ms; T.launches += TB.launches; T.escan += TB.escan; T.eadd += TB.eadd;
        T.snew += TB.snew; T.fseg += TB.fseg; T.wide += TB.wide;
        if ((rc = ensure_run(G, c, omega)) != MANTRA_OK) return rc;
        CU(cudaMemsetAsync(G->hits, 0, (size_t)n * 8, st));
        CU(cudaMemsetAsync(G->S, 0, (size_t)c * n * 4, st));
        uint64_t target = s1, round = 0;
        while (true) {
            round += 1;
            Job j = base;
            j.i0 = r; j.count = target - r; j.dom_pair = DOM_PAIR; j.dom_path = DOM_PATH;
            j.hits = G->hits; j.S = G->S;
            if ((rc = run_samples(G, j, st, &T)) != MANTRA_OK) return rc;
            r = target;
            int64_t NR; uint64_t H;
            if ((rc = round_reduce(G, c, true, st, &NR, &H)) != MANTRA_OK) return rc;
            reduces += 1;
            const double W = (double)H / (double)r;
            const double xi = xi_from_mcera((double)NR / ((double)c * (double)r), W, W,
                                            delta_of_round(delta, round, o.delta_sched), (double)r, (double)c);
            I.rounds = round; I.rade_num = NR; I.max_hits = H; I.xi = xi; I.vhat = W;
            if (r >= omega || xi <= eps) break;
            uint64_t nt = (uint64_t)std::ceil(growth * (double)target);
            if (nt <= target) nt = target + 1;
            target = std::min(omega, nt);
        }
    }
    I.r = r;
    I.sum_int_len = T.sum_int;
    // est_v = hits_v / r
    double* est_dev = o.out_device ? est_out : G->est;
    CU(launch_normalise(G->hits, n, r, est_dev, st));
    if (!o.out_device) CU(cudaMemcpyAsync(est_out, G->est, (size_t)n * 8, cudaMemcpyDeviceToHost, st));
    if (hits_out)
        CU(cudaMemcpyAsync(hits_out, G->hits, (size_t)n * 8,
                           o.out_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    if (info) {
        I.edges_scanned = T.escan; I.sigma_adds = T.eadd; I.states_new = T.snew; I.wide_samples = T.wide;
        I.kernel_ms = T.kernel_ms; I.search_launches = T.launches;
        I.kernel_launches = T.launches + reduces + 1;
        I.alg_bytes = alg_bytes_of(opt == MANTRA_PFM, T.escan, T.eadd, T.snew, T.fseg);
        I.seconds = now_s() - t0;
        *info = I;
    }
    return MANTRA_OK;
}

int mantra_temporal_stats(const mantra_graph* gc, mantra_opt opt, double eps, uint64_t seed, uint64_t r_override,
                          double tau, mantra_tstats* out, uint64_t* reach_out, uint32_t reach_cap) {
    if (!gc || !out) return MANTRA_E_INVAL;
    if (!(eps > 0.0 && eps < 1.0) || !(tau >= 0.0 && tau <= 1.0)) return MANTRA_E_INVAL;
    if (opt != MANTRA_SH && opt != MANTRA_SFM && opt != MANTRA_PFM) return MANTRA_E_INVAL;
    mantra_graph* G = const_cast<mantra_graph*>(gc);
    std::lock_guard<std::mutex> lock(G->mu);
    const double t0 = now_s();
    const uint32_t n = G->n;
    const uint64_t rs = r_override ? r_override : (uint64_t)std::ceil(std::log((double)n) / (eps * eps));
    int rc;
    if ((rc = ensure_run(G, 25, rs)) != MANTRA_OK) return rc;
    cudaStream_t st = G->stream;
    CU(cudaMemsetAsync(G->cnt, 0, ((size_t)n + 2) * 8, st));
    CU(cudaMemsetAsync(G->dmax, 0, 8, st));
    Job j{};
    j.seed = seed; j.i0 = 0; j.count = rs; j.opt = (opt == MANTRA_PFM) ? MANTRA_PFM : MANTRA_SH;
    j.stats = 1; j.cnt = G->cnt; j.dmax = G->dmax;
    LaunchTotals T;
    if ((rc = run_samples(G, j, st, &T)) != MANTRA_OK) return rc;
    std::vector<u64> cnt((size_t)n + 1);
    u64 dmax = 0;
    CU(cudaMemcpyAsync(cnt.data(), G->cnt, ((size_t)n + 1) * 8, cudaMemcpyDeviceToHost, st));
    CU(cudaMemcpyAsync(&dmax, G->dmax, 8, cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    const uint32_t D = (uint32_t)dmax;
    std::vector<u64> R((size_t)D + 1);
    u64 acc = 0;
    for (uint32_t h = 0; h <= D; ++h) { acc += cnt[h]; R[h] = acc; }
    if (reach_out)
        for (uint32_t h = 0; h < reach_cap; ++h) reach_out[h] = (h <= D) ? R[h] : acc;
    // Algorithm 2's host formulas: Rhat[h] = (n/r) R[h]
    std::vector<double> Rh((size_t)D + 1);
    for (uint32_t h = 0; h <= D; ++h) Rh[h] = ((double)n / (double)rs) * (double)R[h];
    mantra_tstats S{};
    S.d_lb = D; S.r = rs;
    const double top = Rh[D];
    if (top > 0.0) {
        double psi = 0.0;
        for (uint32_t h = 1; h <= D; ++h) psi += (Rh[h] - Rh[h - 1]) * (double)h;
        psi /= top;
        uint32_t dt = 0;
        while (dt < D && !(Rh[dt] / top >= tau)) ++dt;
        S.psi = psi; S.d_tau = dt;
        S.zeta = top / ((double)n * (double)(n - 1));
        S.rho = S.zeta * (psi - 1.0);
    }
    S.seconds = now_s() - t0;
    *out = S;
    return MANTRA_OK;
}

int mantra_sample_paths(const mantra_graph* gc, mantra_opt opt, uint64_t seed, uint32_t dom_pair, uint32_t dom_path,
                        uint64_t i0, uint64_t count, uint32_t* s_out, uint32_t* z_out, uint64_t* sigma_out,
                        uint32_t* len_out, uint32_t* nodes_out, uint32_t cap) {
    if (!gc || !s_out || !z_out || !sigma_out || !len_out || (cap > 0 && !nodes_out)) return MANTRA_E_INVAL;
    if (opt != MANTRA_SH && opt != MANTRA_SFM && opt != MANTRA_PFM) return MANTRA_E_INVAL;
    if (dom_pair > 5 || dom_path > 5) return MANTRA_E_INVAL;
    if (count == 0) return MANTRA_OK;
    mantra_graph* G = const_cast<mantra_graph*>(gc);
    std::lock_guard<std::mutex> lock(G->mu);
    int rc;
    if ((rc = ensure_run(G, 25, count)) != MANTRA_OK) return rc;
    cudaStream_t st = G->stream;
    const size_t capn = std::max<uint32_t>(cap, 1);
    const size_t bytes = al256(count * 4) * 3 + al256(count * 16) + al256(count * capn * 4);
    char* d = nullptr;
    if (cudaMalloc(&d, bytes) != cudaSuccess) return MANTRA_E_NOMEM;
    Job j{};
    j.seed = seed; j.i0 = i0; j.count = count; j.dom_pair = dom_pair; j.dom_path = dom_path; j.opt = (int)opt;
    size_t o = 0;
    j.rec_s = (uint32_t*)(d + o); o += al256(count * 4);
    j.rec_z = (uint32_t*)(d + o); o += al256(count * 4);
    j.rec_len = (uint32_t*)(d + o); o += al256(count * 4);
    j.rec_sig = (u64*)(d + o); o += al256(count * 16);
    j.rec_nodes = (uint32_t*)(d + o);
    j.rec_cap = (uint32_t)capn;
    LaunchTotals T;
    rc = run_samples(G, j, st, &T);
    if (rc == MANTRA_OK) {
        cudaError_t e = cudaSuccess;
        if (e == cudaSuccess) e = cudaMemcpyAsync(s_out, j.rec_s, count * 4, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(z_out, j.rec_z, count * 4, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(len_out, j.rec_len, count * 4, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(sigma_out, j.rec_sig, count * 16, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess && cap > 0)
            e = cudaMemcpyAsync(nodes_out, j.rec_nodes, count * (size_t)cap * 4, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) rc = MANTRA_E_CUDA;
    }
    cudaFree(d);
    return rc;
}

}  // extern "C"
