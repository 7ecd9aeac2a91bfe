// Host side of libmantra.so: the temporal-edge store, the per-device engine
// that runs every search as a tick over a task table (one persistent launch
// per kernel family, a multi-problem round reduction and one readback,
// captured once as a CUDA graph and replayed), the Algorithm 1 state machine
// (bootstrap, sampling schedule, rounds, stopping test) for one or many
// problems at once, Algorithm 2's host formulas and the C ABI declared in
// include/mantra.h.
#include "mantra.h"
#include "mantra_dev.cuh"
#include "store.h"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <deque>
#include <thread>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <vector>

using namespace mantra;

// Launch choices of the search kernels for one graph (mantra_tune); 0 / -1
// leave the engine's defaults.
struct Knobs {
    int bfs_nt = 0;      // sh/sfm CTA size: 256, 512 or 1024
    int bfs_smem = -1;   // visited bitmap: 1 shared memory, 0 global
    int pfm_nt = 0;      // pfm CTA size: 256 or 512
    int pfm_mode = -1;   // pfm arrival state: 1 shared memory, 0 global, 2 global with the out-edge tiles
                         // staged in shared memory by bulk copies
};

// Out-edges per chunk the staged pfm variant copies into shared memory (the
// out_v and out_slot tiles, 32 KB each; a chunk with more edges is walked from
// global memory).
constexpr uint32_t PFM_STAGE_CAP = 8192;

struct mantra_graph {
    uint32_t n = 0, A = 0, m = 0, n_uedge = 0;
    uint64_t self_loops = 0, duplicates = 0;
    DevGraph dg{};
    void* dmem = nullptr;
    int device = 0;
    Knobs knobs;         // set by mantra_tune
};

namespace {

// Failing CUDA runtime calls become MANTRA_E_CUDA; with MANTRA_DEBUG set the
// call and the runtime's message go to stderr.
int cuda_fail(cudaError_t e, const char* what, int line) {
    static const bool dbg = std::getenv("MANTRA_DEBUG") != nullptr;
    if (dbg) std::fprintf(stderr, "mantra: %s failed at api.cu:%d: %s\n", what, line, cudaGetErrorString(e));
    return MANTRA_E_CUDA;
}
#define CU(x) do { cudaError_t e_ = (x); if (e_ != cudaSuccess) return cuda_fail(e_, #x, __LINE__); } while (0)

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

// ---------------------------------------------------------------------------
// Temporal-edge store (paper Sec. 3: the temporal graph; the paper's own code
// keeps a sparse n x |T| table, here every arrival appearance (v,t) gets a
// dense slot id).  The host team of store.cu builds the arrays; this uploads
// them into one device allocation, each array from its page-locked buffer.
// ---------------------------------------------------------------------------
int upload_store(const StoreHost& H, mantra_graph* G, cudaStream_t st) {
    const uint32_t** dst[SA_COUNT] = {};
    dst[SA_OUT_PTR] = &G->dg.out_ptr;   dst[SA_OUT_V] = &G->dg.out_v;       dst[SA_OUT_T] = &G->dg.out_t;
    dst[SA_OUT_SLOT] = &G->dg.out_slot; dst[SA_SLOT_PTR] = &G->dg.slot_ptr; dst[SA_SLOT_T] = &G->dg.slot_t;
    dst[SA_SLOT_V] = &G->dg.slot_v;     dst[SA_SLOT_IN] = &G->dg.slot_in;   dst[SA_IN_U] = &G->dg.in_u;
    dst[SA_IN_SLOT] = &G->dg.in_slot;   dst[SA_ST_U] = &G->dg.st_u;         dst[SA_ST_V] = &G->dg.st_v;
    dst[SA_ST_T] = &G->dg.st_t;         dst[SA_TMAX_IN] = &G->dg.tmax_in;   dst[SA_TMIN_OUT] = &G->dg.tmin_out;
    dst[SA_IN_UEDGE] = &G->dg.in_uedge; dst[SA_SLOT_NOUT] = &G->dg.slot_nout;
    const uint32_t* loff_words = nullptr;   // 16-bit entries, two per word
    dst[SA_OUT_LOFF] = &loff_words;
    size_t total = 0;
    for (int k = 0; k < SA_COUNT; ++k) total += al256((H.len[k] + 1) * 4);
    if (cudaMalloc(&G->dmem, total) != cudaSuccess) return MANTRA_E_NOMEM;
    size_t off = 0;
    for (int k = 0; k < SA_COUNT; ++k) {
        char* p = (char*)G->dmem + off;
        if (H.len[k]) CU(cudaMemcpyAsync(p, H.arr[k], H.len[k] * 4, cudaMemcpyHostToDevice, st));
        *dst[k] = (const uint32_t*)p;
        off += al256((H.len[k] + 1) * 4);
    }
    CU(cudaStreamSynchronize(st));
    G->dg.out_loff = reinterpret_cast<const unsigned short*>(loff_words);
    G->n = H.n; G->m = H.m; G->A = H.A; G->n_uedge = H.n_uedge;
    G->self_loops = H.self_loops; G->duplicates = H.duplicates;
    G->dg.n = H.n; G->dg.A = H.A; G->dg.m = H.m; G->dg.n_uedge = H.n_uedge;
    G->dg.cbound = H.cbound; G->dg.max_slot_in = H.max_slot_in; G->dg.max_vslots = H.max_vslots;
    return MANTRA_OK;
}


size_t free_device_bytes() {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) return 0;
    return fr;
}

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// ---------------------------------------------------------------------------
// Device memory pool: blocks kept by exact (256-rounded) size and reused by
// later problems; at most kPoolCacheBytes stay cached.
// ---------------------------------------------------------------------------
constexpr size_t kPoolCacheBytes = (size_t)8 << 30;

struct DevPool {
    std::multimap<size_t, void*> free_blocks;
    size_t cached = 0;
    void* get(size_t bytes) {
        bytes = al256(std::max<size_t>(bytes, 256));
        auto it = free_blocks.find(bytes);
        if (it != free_blocks.end()) {
            void* p = it->second;
            free_blocks.erase(it);
            cached -= bytes;
            return p;
        }
        void* p = nullptr;
        if (cudaMalloc(&p, bytes) != cudaSuccess) {
            release_all();
            if (cudaMalloc(&p, bytes) != cudaSuccess) return nullptr;
        }
        return p;
    }
    void put(void* p, size_t bytes) {
        if (!p) return;
        bytes = al256(std::max<size_t>(bytes, 256));
        if (cached + bytes > kPoolCacheBytes) { cudaFree(p); return; }
        free_blocks.emplace(bytes, p);
        cached += bytes;
    }
    void release_all() {
        for (auto& kv : free_blocks) cudaFree(kv.second);
        free_blocks.clear();
        cached = 0;
    }
};

// Per-problem result slot of a tick: search counters, device status word,
// and the round reduction's outputs.
constexpr size_t SLOT_BYTES = 1152;
constexpr size_t SLOT_STATUS = 64, SLOT_HMAX = 72, SLOT_ROWMAX = 80;

struct LaunchTotals {
    uint64_t sum_int = 0, escan = 0, eadd = 0, snew = 0, fseg = 0, xedge = 0, wide = 0, launches = 0;
    double kernel_ms = 0;
    void add_counters(const u64* c) {
        sum_int += c[C_SUMINT]; escan += c[C_ESCAN]; eadd += c[C_EADD]; snew += c[C_SNEW]; fseg += c[C_FSEG];
        xedge += c[C_XEDGE];
    }
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

// One entry of a tick: a graph and a sample range, plus an optional round
// reduction over its hits (and red_c rows of S).
struct TickItem {
    const mantra_graph* G = nullptr;
    Job job{};
    bool reduce = false;
    uint32_t red_c = 0;
};

struct TickOut {
    std::vector<const char*> slot;   // host copy of each item's result slot
    double bfs_ms = 0, pfm_ms = 0;
    bool had_bfs = false, had_pfm = false;
};

// ---------------------------------------------------------------------------
// Engine: one per device.  Owns the search workspaces (sized for the largest
// graph seen), the task tables of a tick (pinned host copy + device copy) and
// the captured tick graph.  Every public call locks `mu` for its duration.
// ---------------------------------------------------------------------------
struct Engine {
    std::mutex mu;
    StoreBuilder store;        // host buffers of graph loads (mantra_graph_load)
    int device = -1, num_sms = 0;
    size_t smem_optin = 0;
    cudaStream_t sa = nullptr, sb = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr, e_b0 = nullptr, e_b1 = nullptr, e_p0 = nullptr, e_p1 = nullptr;
    cudaEvent_t e_t0 = nullptr, e_t1 = nullptr;   // around a graph launch (events inside graphs cannot be timed)
    bool last_tick_graph = false;
    // search workspaces
    // sh/sfm: regions for the largest resident grid of any CTA shape (s: 0 =
    // 256, 1 = 512, 2 = 1024 threads) and visited-bitmap placement (p: 0 =
    // global, 1 = shared memory); bfs_grids[s][p] = resident CTAs (0: the
    // placement does not fit)
    char* bfs_mem = nullptr; BfsWs bws{}; size_t bfs_smem = 0; uint32_t bfs_n = 0, bfs_A = 0, bfs_z = 0;
    int bfs_grids[3][2] = {};
    int bfs_rule_smem = 0;     // default placement: shared only while it keeps the 512-thread residency
    int bfs_grid = 0;          // resident CTAs of the default (512 threads, default placement)
    bool bfs_dl = false;       // the regions carry the ob / RTB scratch
    int tick_bfs_nt = 512;     // sh/sfm CTA size of the current tick
    int tick_bfs_sm = 0;       // its bitmap placement
    bool tick_frac = false;    // the tick has an ob or RTB problem on the sh/sfm kernel
    char* pfm_mem = nullptr; PfmWs pws{}; int pfm_grid = 0; uint32_t pfm_n = 0, pfm_lcap = 0; uint64_t pfm_warps = 0;
    // pfm, one CTA per sample: shapes 0 = 256, 1 = 512 threads; modes 0 = state
    // in global memory, 1 = in shared memory, 2 = global with staged edge tiles,
    // 3 = in shared memory as 16-bit slot offsets
    char* pc_mem = nullptr; PfmCtaWs pcws{}; int pc_grid = 0; uint32_t pc_n = 0, pc_cb = 0;
    int pc_grids[2][4] = {};
    size_t pc_smem = 0;
    int tick_pc_nt = 512, tick_pc_sm = 0;
    bool tick_cta = false;   // pfm samples of the current tick run one per CTA
    // tick tables
    uint32_t cap = 0;
    char* tab_h = nullptr; char* tab_d = nullptr; size_t tab_bytes = 0;
    char* slot_h = nullptr; char* slot_d = nullptr;
    size_t o_hdr = 0, o_work = 0, o_ub = 0, o_up = 0, o_tb = 0, o_tp = 0, o_ri = 0, o_rs = 0;
    int red_grid = 0;
    // captured ticks, by launch configuration (tick_key)
    std::map<int, cudaGraphExec_t> gexec;
    bool use_graph = true;
    DevPool pool;

    int init(int dev) {
        device = dev;
        CU(cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev));
        int optin = 0;
        CU(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
        smem_optin = (size_t)optin;
        // the pfm stream gets the higher priority: its small latency-bound blocks are
        // placed first and the persistent sh/sfm CTAs take the remaining SMs
        int lo_pri = 0, hi_pri = 0;
        CU(cudaDeviceGetStreamPriorityRange(&lo_pri, &hi_pri));
        CU(cudaStreamCreateWithPriority(&sa, cudaStreamNonBlocking, lo_pri));
        CU(cudaStreamCreateWithPriority(&sb, cudaStreamNonBlocking, hi_pri));
        CU(cudaEventCreateWithFlags(&ev_fork, cudaEventDisableTiming));
        CU(cudaEventCreateWithFlags(&ev_join, cudaEventDisableTiming));
        CU(cudaEventCreate(&e_b0)); CU(cudaEventCreate(&e_b1));
        CU(cudaEventCreate(&e_p0)); CU(cudaEventCreate(&e_p1));
        CU(cudaEventCreate(&e_t0)); CU(cudaEventCreate(&e_t1));
        red_grid = num_sms * 4;
        if (const char* env = std::getenv("MANTRA_NO_GRAPH")) use_graph = env[0] == '0';
        return MANTRA_OK;
    }

    void invalidate_graph() {
        for (auto& kv : gexec)
            if (kv.second) cudaGraphExecDestroy(kv.second);
        gexec.clear();
    }

    static int shape_of(int nt) { return nt == 256 ? 0 : (nt == 1024 ? 2 : 1); }

    int tick_key() const {
        return (tick_cta ? 1 : 0) | (shape_of(tick_bfs_nt) << 1) | (tick_bfs_sm << 3) | ((tick_frac ? 1 : 0) << 4) |
               ((tick_pc_nt == 256 ? 0 : 1) << 5) | (tick_pc_sm << 6);   // tick_pc_sm: the pfm mode (2 bits)
    }

    // Table block layout: header | 2 work counters | unit starts (bfs, pfm) |
    // tasks (bfs, pfm) | reduction items | reduction row starts.
    int ensure_tables(uint32_t need) {
        if (tab_h && need <= cap) return MANTRA_OK;
        uint32_t nc = std::max<uint32_t>(64, cap);
        while (nc < need) nc *= 2;
        if (tab_h) { cudaFreeHost(tab_h); tab_h = nullptr; }
        if (tab_d) { cudaFree(tab_d); tab_d = nullptr; }
        if (slot_h) { cudaFreeHost(slot_h); slot_h = nullptr; }
        if (slot_d) { cudaFree(slot_d); slot_d = nullptr; }
        size_t o = 0;
        o_hdr = o;  o = al256(o + 16);
        o_work = o; o = al256(o + 16);
        o_ub = o;   o = al256(o + (size_t)(nc + 1) * 8);
        o_up = o;   o = al256(o + (size_t)(nc + 1) * 8);
        o_tb = o;   o = al256(o + (size_t)nc * sizeof(Task));
        o_tp = o;   o = al256(o + (size_t)nc * sizeof(Task));
        o_ri = o;   o = al256(o + (size_t)nc * sizeof(ReduceItem));
        o_rs = o;   o = al256(o + (size_t)(nc + 1) * 4);
        tab_bytes = o;
        if (cudaMallocHost((void**)&tab_h, tab_bytes) != cudaSuccess) { tab_h = nullptr; return MANTRA_E_NOMEM; }
        if (cudaMalloc((void**)&tab_d, tab_bytes) != cudaSuccess) { tab_d = nullptr; return MANTRA_E_NOMEM; }
        if (cudaMallocHost((void**)&slot_h, (size_t)nc * SLOT_BYTES) != cudaSuccess) { slot_h = nullptr; return MANTRA_E_NOMEM; }
        if (cudaMalloc((void**)&slot_d, (size_t)nc * SLOT_BYTES) != cudaSuccess) { slot_d = nullptr; return MANTRA_E_NOMEM; }
        std::memset(tab_h, 0, tab_bytes);
        cap = nc;
        invalidate_graph();
        return MANTRA_OK;
    }

    // sh/sfm: one region per resident CTA of the largest grid over CTA shapes
    // and bitmap placements, at most 60 % of free memory.  Every region holds
    // a global visited bitmap as well, so the placement is chosen per launch.
    // Device bytes of the search workspaces for graphs with these maxima (sh/sfm:
    // n, A, slots per vertex, ob/RTB scratch; pfm: n, cbound), at the largest
    // grid of any CTA shape (256-thread CTAs: four per SM for k_bfs, six for
    // k_pfm_cta) and without the free-memory caps of ensure_bfs /
    // ensure_pfm_cta: an upper estimate of what those allocate.
    size_t ws_estimate(uint32_t n, uint32_t A, uint32_t zc, bool dl, uint32_t pn, uint32_t cb) const {
        size_t b = 0;
        const size_t sms = (size_t)std::max(num_sms, 1);
        if (n) { BfsWs w{}; b += 4 * sms * bfs_region_bytes(n, A, zc, false, dl, &w); }
        if (pn) { PfmCtaWs w{}; b += 6 * sms * pfm_cta_region_bytes(pn, cb, false, &w); }
        return b;
    }

    int ensure_bfs(uint32_t n, uint32_t A, uint32_t zc, bool dl) {
        if (bfs_mem && n <= bfs_n && A <= bfs_A && zc <= bfs_z && (!dl || bfs_dl)) return MANTRA_OK;
        n = std::max(n, bfs_n);
        A = std::max(A, bfs_A);
        zc = std::max(zc, bfs_z);
        dl = dl || bfs_dl;
        if (bfs_mem) { cudaStreamSynchronize(sa); cudaFree(bfs_mem); bfs_mem = nullptr; }
        const int nts[3] = {256, 512, 1024};
        const size_t smem = bfs_smem_bytes(A);
        size_t stat = 0;
        for (int nt : nts) stat = std::max(stat, bfs_static_smem(nt));
        const bool fit = smem + stat + 1024 <= smem_optin;
        if (fit) CU(bfs_configure(smem));
        int per[3][2] = {};
        for (int s = 0; s < 3; ++s) {
            CU(bfs_blocks_per_sm(nts[s], 0, &per[s][0]));
            if (fit) CU(bfs_blocks_per_sm(nts[s], smem, &per[s][1]));
        }
        // default placement: the bitmap goes to shared memory only while two
        // 512-thread CTAs per SM stay resident (on a 798k-slot graph one CTA per
        // SM with the bitmap took 64 ms where two without it took 49 ms);
        // MANTRA_BFS_SMEM=0 forces global memory, =1 shared whenever it fits
        bfs_rule_smem = (fit && per[1][1] >= per[1][0]) ? 1 : 0;
        if (const char* env = std::getenv("MANTRA_BFS_SMEM")) {
            if (env[0] == '0') bfs_rule_smem = 0;
            else if (env[0] == '1') bfs_rule_smem = fit ? 1 : 0;
        }
        const size_t region = bfs_region_bytes(n, A, zc, false, dl, &bws);
        // the search regions may take 60 % of free memory: on the n = 10^6,
        // m = 2*10^7 graph one region is about half a GB and every SM should
        // keep its resident CTAs
        const size_t budget = (size_t)((double)free_device_bytes() * 0.6);
        int grid = 0;
        for (int s = 0; s < 3; ++s)
            for (int p = 0; p < 2; ++p) grid = std::max(grid, num_sms * per[s][p]);
        grid = std::max(grid, 1);
        // MANTRA_BFS_GRID caps the resident CTAs
        if (const char* env = std::getenv("MANTRA_BFS_GRID")) grid = std::max(1, std::min(grid, std::atoi(env)));
        if ((size_t)grid * region > budget) grid = (int)std::max<size_t>(1, budget / region);
        if (cudaMalloc(&bfs_mem, (size_t)grid * region) != cudaSuccess) { bfs_mem = nullptr; return MANTRA_E_NOMEM; }
        CU(cudaMemsetAsync(bfs_mem, 0, (size_t)grid * region, sa));
        bws.base = bfs_mem;
        bws.stride = region;
        for (int s = 0; s < 3; ++s)
            for (int p = 0; p < 2; ++p) bfs_grids[s][p] = per[s][p] > 0 ? std::min(grid, num_sms * per[s][p]) : 0;
        bfs_grid = bfs_grids[1][bfs_rule_smem];
        bfs_smem = fit ? smem : 0;
        bfs_n = n; bfs_A = A; bfs_z = zc; bfs_dl = dl;
        invalidate_graph();
        return MANTRA_OK;
    }

    // pfm: one region per warp (32 samples), at most one warp per 32 resident
    // threads of the GPU and at most a third of free memory.
    int ensure_pfm(uint32_t n, uint32_t lcap, uint64_t warps) {
        const int wpb = pfm_threads() / 32;
        warps = std::min<uint64_t>(std::max<uint64_t>(warps, (uint64_t)wpb), (uint64_t)num_sms * 32);
        // MANTRA_PFM_LIST_CAP lowers the contribution-list capacity (tests of the
        // in-order fallback taken by samples whose list would overflow)
        if (const char* env = std::getenv("MANTRA_PFM_LIST_CAP")) {
            const long v = std::strtol(env, nullptr, 10);
            if (v > 0 && (uint64_t)v < lcap) lcap = (uint32_t)v;
        }
        lcap = std::max<uint32_t>(32, std::min<uint32_t>(lcap, 1u << 20));
        if (pfm_mem && n <= pfm_n && lcap <= pfm_lcap && warps <= pfm_warps) return MANTRA_OK;
        n = std::max(n, pfm_n);
        lcap = std::max(lcap, pfm_lcap);
        warps = std::max<uint64_t>(warps, pfm_warps);
        if (pfm_mem) { cudaStreamSynchronize(sb); cudaStreamSynchronize(sa); cudaFree(pfm_mem); pfm_mem = nullptr; }
        const size_t region = pfm_region_bytes(n, lcap, &pws);
        const size_t budget = free_device_bytes() / 3;
        uint64_t w = std::min<uint64_t>(warps, std::max<size_t>(budget / region, (size_t)wpb));
        const int blocks = (int)((w + wpb - 1) / wpb);
        if (cudaMalloc(&pfm_mem, (size_t)blocks * wpb * region) != cudaSuccess) { pfm_mem = nullptr; return MANTRA_E_NOMEM; }
        pws.base = pfm_mem;
        pws.stride = region;
        pfm_grid = blocks;
        pfm_n = n;
        pfm_lcap = lcap;
        pfm_warps = (uint64_t)blocks * wpb;
        invalidate_graph();
        return MANTRA_OK;
    }

    // pfm with one CTA per sample: one region per resident CTA of the largest
    // grid over CTA shapes and state placements, at most a third of free
    // memory.  Every region holds the arrival state in global memory as well,
    // so the placement (shared memory when it fits) is chosen per launch.
    int ensure_pfm_cta(uint32_t n, uint32_t cb) {
        if (pc_mem && n <= pc_n && cb <= pc_cb) return MANTRA_OK;
        n = std::max(n, pc_n);
        cb = std::max(cb, pc_cb);
        if (pc_mem) { cudaStreamSynchronize(sb); cudaStreamSynchronize(sa); cudaFree(pc_mem); pc_mem = nullptr; }
        const int nts[2] = {256, 512};
        const size_t smem = pfm_cta_smem_bytes(n, false), smem16 = pfm_cta_smem_bytes(n, true);
        const size_t stat = std::max(pfm_cta_static_smem(256), pfm_cta_static_smem(512)) + 1024;
        const bool fit = smem + stat <= smem_optin, fit16 = smem16 + stat <= smem_optin;
        const size_t stage = pfm_cta_stage_bytes(PFM_STAGE_CAP);
        CU(pfm_cta_configure(std::max({fit ? smem : 0, fit16 ? smem16 : 0, stage})));
        int per[2][4] = {};
        for (int s = 0; s < 2; ++s) {
            CU(pfm_cta_blocks_per_sm(nts[s], 0, 0, &per[s][0]));
            if (fit) CU(pfm_cta_blocks_per_sm(nts[s], 1, smem, &per[s][1]));
            CU(pfm_cta_blocks_per_sm(nts[s], 0, stage, &per[s][2]));
            if (fit16) CU(pfm_cta_blocks_per_sm(nts[s], 2, smem16, &per[s][3]));
        }
        const size_t region = pfm_cta_region_bytes(n, cb, false, &pcws);
        int grid = 0;
        for (int s = 0; s < 2; ++s)
            for (int p = 0; p < 4; ++p) grid = std::max(grid, num_sms * per[s][p]);
        grid = std::max(grid, 1);
        if (const char* env = std::getenv("MANTRA_PFM_GRID")) grid = std::max(1, std::min(grid, std::atoi(env)));
        const size_t budget = free_device_bytes() / 3;
        if ((size_t)grid * region > budget) grid = (int)std::max<size_t>(1, budget / region);
        if (cudaMalloc(&pc_mem, (size_t)grid * region) != cudaSuccess) { pc_mem = nullptr; return MANTRA_E_NOMEM; }
        pcws.base = pc_mem;
        pcws.stride = region;
        for (int s = 0; s < 2; ++s)
            for (int p = 0; p < 4; ++p) pc_grids[s][p] = per[s][p] > 0 ? std::min(grid, num_sms * per[s][p]) : 0;
        pc_grid = pc_grids[1][fit ? 1 : 0];
        pc_smem = fit ? smem : 0;
        pc_n = n;
        pc_cb = cb;
        invalidate_graph();
        return MANTRA_OK;
    }

    // The tick as stream work: tables up, slots cleared, both search
    // families on two streams, the round reduction, slots down.
    int enqueue(bool wide) {
        CU(cudaMemcpyAsync(tab_d, tab_h, tab_bytes, cudaMemcpyHostToDevice, sa));
        CU(cudaMemsetAsync(slot_d, 0, (size_t)cap * SLOT_BYTES, sa));
        CU(cudaEventRecord(ev_fork, sa));
        CU(cudaStreamWaitEvent(sb, ev_fork, 0));
        const uint32_t* hdr = (const uint32_t*)(tab_d + o_hdr);
        u64* work = (u64*)(tab_d + o_work);
        if (bfs_mem) {
            CU(cudaEventRecord(e_b0, sa));
            BfsWs w = bws;
            w.nt = tick_bfs_nt;
            w.bits_in_smem = tick_bfs_sm;
            CU(launch_bfs((const Task*)(tab_d + o_tb), (const uint64_t*)(tab_d + o_ub), hdr + 0, work + 0, w,
                          bfs_grids[shape_of(tick_bfs_nt)][tick_bfs_sm], tick_bfs_sm ? bfs_smem : 0, wide, tick_frac,
                          sa));
            CU(cudaEventRecord(e_b1, sa));
        }
        if (tick_cta && !wide && pc_mem) {
            CU(cudaEventRecord(e_p0, sb));
            PfmCtaWs w = pcws;
            w.nt = tick_pc_nt;
            w.fa_in_smem = tick_pc_sm == 1 ? 1 : (tick_pc_sm == 3 ? 2 : 0);
            w.stage_cap = tick_pc_sm == 2 ? PFM_STAGE_CAP : 0u;
            CU(launch_pfm_cta((const Task*)(tab_d + o_tp), (const uint64_t*)(tab_d + o_up), hdr + 1, work + 1, w,
                              pc_grids[tick_pc_nt == 256 ? 0 : 1][tick_pc_sm], sb));
            CU(cudaEventRecord(e_p1, sb));
        } else if (!tick_cta && pfm_mem) {
            CU(cudaEventRecord(e_p0, sb));
            CU(launch_pfm((const Task*)(tab_d + o_tp), (const uint64_t*)(tab_d + o_up), hdr + 1, work + 1, pws,
                          pfm_grid, wide, sb));
            CU(cudaEventRecord(e_p1, sb));
        }
        CU(cudaEventRecord(ev_join, sb));
        CU(cudaStreamWaitEvent(sa, ev_join, 0));
        CU(launch_round_reduce((const ReduceItem*)(tab_d + o_ri), (const uint32_t*)(tab_d + o_rs), hdr + 2, red_grid,
                               sa));
        CU(cudaMemcpyAsync(slot_h, slot_d, (size_t)cap * SLOT_BYTES, cudaMemcpyDeviceToHost, sa));
        return MANTRA_OK;
    }

    int launch_tick(bool wide) {
        last_tick_graph = false;
        if (wide || !use_graph) return enqueue(wide);
        const int gk = tick_key();
        if (!gexec.count(gk)) {
            cudaGraph_t graph = nullptr;
            CU(cudaStreamBeginCapture(sa, cudaStreamCaptureModeThreadLocal));
            const int rc = enqueue(false);
            const cudaError_t e = cudaStreamEndCapture(sa, &graph);
            if (rc != MANTRA_OK || e != cudaSuccess) {
                if (graph) cudaGraphDestroy(graph);
                use_graph = false;                    // capture unavailable: run the same work directly
                return enqueue(false);
            }
            cudaGraphExec_t ex = nullptr;
            const cudaError_t ei = cudaGraphInstantiate(&ex, graph, 0);
            cudaGraphDestroy(graph);
            if (ei != cudaSuccess) { use_graph = false; return enqueue(false); }
            gexec[gk] = ex;
        }
        CU(cudaEventRecord(e_t0, sa));
        CU(cudaGraphLaunch(gexec[gk], sa));
        CU(cudaEventRecord(e_t1, sa));
        last_tick_graph = true;
        return MANTRA_OK;
    }
};

std::mutex g_engines_mu;
Engine* g_engines[64];

int engine_for(int dev, Engine** out) {
    if (dev < 0 || dev >= 64) return MANTRA_E_CUDA;
    std::lock_guard<std::mutex> lock(g_engines_mu);
    if (!g_engines[dev]) {
        Engine* E = new (std::nothrow) Engine();
        if (!E) return MANTRA_E_NOMEM;
        int cur = 0;
        CU(cudaGetDevice(&cur));
        if (cur != dev) CU(cudaSetDevice(dev));
        const int rc = E->init(dev);
        if (cur != dev) cudaSetDevice(cur);
        if (rc != MANTRA_OK) { delete E; return rc; }
        g_engines[dev] = E;
    }
    *out = g_engines[dev];
    return MANTRA_OK;
}

// Milliseconds between two recorded events; 0 (and the runtime's error state
// cleared) when the pair cannot be timed.
double elapsed_ms(cudaEvent_t a, cudaEvent_t b) {
    float ms = 0;
    const cudaError_t e = cudaEventElapsedTime(&ms, a, b);
    if (e != cudaSuccess) {
        static const bool dbg = std::getenv("MANTRA_DEBUG") != nullptr;
        if (dbg) std::fprintf(stderr, "mantra: cudaEventElapsedTime: %s\n", cudaGetErrorString(e));
        (void)cudaGetLastError();
        return 0.0;
    }
    return ms;
}

// One line per tick item on stderr (MANTRA_LOG_LAUNCHES): kernel, launch
// shape (threads) and state mode (k_bfs: bitmap placement; k_pfm_cta: the
// engine's mode 0..3), the item's counters and algorithmic bytes, the
// kernel's event time.
void log_item(const TickItem& it, bool wide, bool cta, int nt, int mode, const u64* c, double ms) {
    static const bool on = std::getenv("MANTRA_LOG_LAUNCHES") != nullptr;
    if (!on) return;
    const bool pfm = it.job.opt == MANTRA_PFM;
    std::fprintf(stderr, "mantra-launch kernel=%s%s nt=%d mode=%d samples=%llu escan=%llu eadd=%llu snew=%llu "
                 "fseg=%llu xedge=%llu alg_bytes=%llu ms=%.4f\n", pfm ? (cta ? "k_pfm_cta" : "k_pfm") : "k_bfs",
                 wide ? "<wide>" : "", nt, mode, (unsigned long long)it.job.count, (unsigned long long)c[C_ESCAN],
                 (unsigned long long)c[C_EADD], (unsigned long long)c[C_SNEW], (unsigned long long)c[C_FSEG],
                 (unsigned long long)c[C_XEDGE],
                 (unsigned long long)alg_bytes_of(pfm, c[C_ESCAN], c[C_EADD], c[C_SNEW], c[C_FSEG]), ms);
}

// Which pfm kernel a narrow tick uses.  The lane kernel's launch costs at
// least one warp's serial walk over the stream and its per-warp state grows
// with 32 n; the CTA kernel measured faster at every launch size on the
// n = 20,000 bursty graph (1.8 vs 70 ms for 231 samples, 82 vs 126 ms for
// 42,521).  The lane kernel stays the 128-bit re-run.
// MANTRA_PFM_KERNEL=lane|cta forces one of them.
bool pfm_use_cta() {
    const char* env = std::getenv("MANTRA_PFM_KERNEL");
    return !(env && std::strcmp(env, "lane") == 0);
}

// One tick over `items` (narrow kernels, captured graph), or with `wide` the
// 128-bit kernels launched directly.  Fills each item's ctr/status pointers.
int run_tick(Engine& E, std::vector<TickItem>& items, bool wide, TickOut* out) {
    const uint32_t k = (uint32_t)items.size();
    int rc;
    if ((rc = E.ensure_tables(std::max<uint32_t>(k, 1))) != MANTRA_OK) return rc;
    uint32_t bn = 0, bA = 0, bz = 0, pn = 0, plc = 0, pz = 0;
    const mantra_graph* gb = nullptr;   // the tick's largest sh/sfm graph: its knobs apply
    const mantra_graph* gp = nullptr;   // the tick's largest pfm graph
    uint64_t pwarps = 0, bsamples = 0;
    bool any_b = false, any_p = false, frac = false, dl = false;
    for (const TickItem& it : items) {
        if (it.job.opt == MANTRA_PFM) {
            any_p = true; pn = std::max(pn, it.G->n); plc = std::max(plc, it.G->dg.cbound);
            pz = std::max(pz, it.G->dg.max_vslots);
            if (!gp || it.G->n > gp->n) gp = it.G;
            pwarps += (it.job.count + 31) / 32;
        } else {
            any_b = true; bn = std::max(bn, it.G->n); bA = std::max(bA, it.G->A);
            bz = std::max(bz, it.G->dg.max_vslots);
            if (!gb || it.G->A > gb->A) gb = it.G;
            bsamples += it.job.count;
            frac |= it.job.ob || it.job.rtb || it.job.opt == 3;
            dl |= it.job.ob || it.job.rtb;
        }
    }
    E.tick_frac = frac;
    const bool cta = any_p && !wide && pfm_use_cta();
    if (any_b && (rc = E.ensure_bfs(bn, bA, bz, dl)) != MANTRA_OK) return rc;
    if (any_p && cta && (rc = E.ensure_pfm_cta(pn, plc)) != MANTRA_OK) return rc;
    if (any_p && !cta && (rc = E.ensure_pfm(pn, plc, pwarps)) != MANTRA_OK) return rc;
    E.tick_cta = cta;
    // sh/sfm CTA shape: 1024 threads for ticks of at most two samples per resident
    // 1024-thread CTA (shorter per-sample latency), else two 512-thread CTAs per SM
    // (measured on the n = 20,000 bursty graph: 1.9 vs 2.7 ms for 231 samples,
    // 42.5 vs 40.4 ms for 26,702), or the shape and bitmap placement mantra_tune
    // chose for the graph; MANTRA_BFS_NT=256|512|1024 forces a shape
    if (any_b) {
        const bool small = bsamples <= 2ull * (uint64_t)E.bfs_grids[2][E.bfs_rule_smem];
        int nt = small ? 1024 : 512, sm = E.bfs_rule_smem;
        if (gb && !small && gb->knobs.bfs_nt) nt = gb->knobs.bfs_nt;
        if (gb && !small && gb->knobs.bfs_smem >= 0) sm = gb->knobs.bfs_smem;
        if (const char* env = std::getenv("MANTRA_BFS_NT")) {
            const int v = std::atoi(env);
            nt = v == 1024 ? 1024 : (v == 256 ? 256 : 512);
        }
        if (!E.bfs_grids[Engine::shape_of(nt)][sm]) sm = 0;   // the placement does not fit this shape
        E.tick_bfs_nt = nt;
        E.tick_bfs_sm = sm;
    }
    // pfm CTA shape and arrival-state mode: 512 threads with the state in shared
    // memory when it fits, or the graph's tuned choice; MANTRA_PFM_CTA_NT=256,
    // MANTRA_PFM_CTA_SMEM=0 (global state), =16 (shared, 16-bit offsets) and
    // MANTRA_PFM_STAGE=1 (global state, staged edge tiles) force the others.
    // The 16-bit state needs every pfm graph of the tick to have at most
    // 0xFFFE slots per vertex.
    if (any_p && cta) {
        int nt = 512, sm = E.pc_grids[1][1] || E.pc_grids[1][3] ? 1 : 0;
        if (gp && gp->knobs.pfm_nt) nt = gp->knobs.pfm_nt;
        if (gp && gp->knobs.pfm_mode >= 0) sm = gp->knobs.pfm_mode;
        if (const char* env = std::getenv("MANTRA_PFM_CTA_NT")) nt = std::atoi(env) == 256 ? 256 : 512;
        if (const char* env = std::getenv("MANTRA_PFM_CTA_SMEM"))
            sm = env[0] == '0' ? 0 : (std::atoi(env) == 16 ? 3 : (sm == 3 ? 1 : sm));
        if (const char* env = std::getenv("MANTRA_PFM_STAGE")) sm = env[0] == '1' ? 2 : (sm == 2 ? 0 : sm);
        const int sh = nt == 256 ? 0 : 1;
        if (sm == 3 && pz > PFM_W16_MAX_VSLOTS) sm = 1;
        // the untuned shared state: 16-bit offsets where they keep more CTAs resident
        if (sm == 1 && !(gp && gp->knobs.pfm_mode >= 0) && pz <= PFM_W16_MAX_VSLOTS &&
            E.pc_grids[sh][3] > E.pc_grids[sh][1])
            sm = 3;
        if (!E.pc_grids[sh][sm]) sm = 0;
        E.tick_pc_nt = nt;
        E.tick_pc_sm = sm;
    }
    // host tables
    uint32_t* hdr = (uint32_t*)(E.tab_h + E.o_hdr);
    u64* work = (u64*)(E.tab_h + E.o_work);
    uint64_t* ub = (uint64_t*)(E.tab_h + E.o_ub);
    uint64_t* up = (uint64_t*)(E.tab_h + E.o_up);
    Task* tb = (Task*)(E.tab_h + E.o_tb);
    Task* tp = (Task*)(E.tab_h + E.o_tp);
    ReduceItem* ri = (ReduceItem*)(E.tab_h + E.o_ri);
    uint32_t* rs = (uint32_t*)(E.tab_h + E.o_rs);
    uint32_t nb = 0, np = 0, nr = 0;
    ub[0] = 0; up[0] = 0; rs[0] = 0;
    for (uint32_t x = 0; x < k; ++x) {
        TickItem& it = items[x];
        char* slot = E.slot_d + (size_t)x * SLOT_BYTES;
        it.job.ctr = (u64*)slot;
        it.job.status = (int*)(slot + SLOT_STATUS);
        Task t{it.G->dg, it.job};
        if (it.job.opt == MANTRA_PFM) {
            tp[np] = t;
            up[np + 1] = up[np] + (cta ? it.job.count : (it.job.count + 31) / 32);
            ++np;
        }
        else { tb[nb] = t; ub[nb + 1] = ub[nb] + it.job.count; ++nb; }
        if (it.reduce) {
            ri[nr] = ReduceItem{it.job.S, it.job.S64, (it.job.ob || it.job.rtb) ? it.job.wsq : it.job.hits, it.job.fam,
                                it.red_c,
                                (long long*)(slot + SLOT_ROWMAX),
                                (u64*)(slot + SLOT_HMAX)};
            rs[nr + 1] = rs[nr] + it.red_c + 1;
            ++nr;
        }
    }
    hdr[0] = nb; hdr[1] = np; hdr[2] = nr;
    work[0] = 0; work[1] = 0;
    if ((rc = E.launch_tick(wide)) != MANTRA_OK) return rc;
    CU(cudaStreamSynchronize(E.sa));
    out->slot.resize(k);
    for (uint32_t x = 0; x < k; ++x) out->slot[x] = E.slot_h + (size_t)x * SLOT_BYTES;
    out->had_bfs = nb > 0 && E.bfs_mem;
    out->had_pfm = np > 0 && (cta ? E.pc_mem != nullptr : E.pfm_mem != nullptr);
    if (E.last_tick_graph) {
        // a graph tick is timed as a whole: table upload, searches, reduction, readback
        const double t = elapsed_ms(E.e_t0, E.e_t1);
        out->bfs_ms = out->had_bfs ? t : 0.0;
        out->pfm_ms = out->had_pfm ? t : 0.0;
    } else {
        out->bfs_ms = out->had_bfs ? elapsed_ms(E.e_b0, E.e_b1) : 0.0;
        out->pfm_ms = out->had_pfm ? elapsed_ms(E.e_p0, E.e_p1) : 0.0;
    }
    for (uint32_t x = 0; x < k; ++x)
        if (items[x].job.opt == MANTRA_PFM)
            log_item(items[x], wide, cta, cta ? E.tick_pc_nt : 32, cta ? E.tick_pc_sm : 0, (const u64*)out->slot[x],
                     out->pfm_ms);
        else
            log_item(items[x], wide, cta, E.tick_bfs_nt, E.tick_bfs_sm, (const u64*)out->slot[x], out->bfs_ms);
    return MANTRA_OK;
}

// A tick followed, for items whose 64-bit path counts overflowed, by a
// 128-bit re-run of those samples (and their reductions).  counters[x]
// receives both passes' counters; slot_out[x] the slot whose reduction
// outputs are current.
struct TickResult {
    std::vector<std::vector<char>> slot;   // current reduction outputs per item (copied)
    std::vector<LaunchTotals> tot;         // per item counters, kernel time and launches
    std::vector<int> status;
};

int run_tick_full(Engine& E, std::vector<TickItem>& items, uint64_t** ovf_lists, TickResult* R) {
    TickOut out;
    int rc = run_tick(E, items, false, &out);
    if (rc != MANTRA_OK) return rc;
    const uint32_t k = (uint32_t)items.size();
    R->slot.assign(k, std::vector<char>(SLOT_BYTES));
    R->tot.assign(k, LaunchTotals());
    R->status.assign(k, MANTRA_OK);
    std::vector<uint32_t> wide_ix;
    std::vector<TickItem> witems;
    for (uint32_t x = 0; x < k; ++x) {
        std::memcpy(R->slot[x].data(), out.slot[x], SLOT_BYTES);
        const u64* c = (const u64*)out.slot[x];
        int st;
        std::memcpy(&st, out.slot[x] + SLOT_STATUS, 4);
        R->status[x] = st;
        R->tot[x].add_counters(c);
        R->tot[x].launches += 1;
        R->tot[x].kernel_ms += items[x].job.opt == MANTRA_PFM ? out.pfm_ms : out.bfs_ms;
        if (st == MANTRA_OK && c[C_NOVF] > 0) {
            TickItem w = items[x];
            w.job.idx_list = ovf_lists[x];
            w.job.count = c[C_NOVF];
            wide_ix.push_back(x);
            witems.push_back(w);
        }
    }
    if (!witems.empty()) {
        TickOut wout;
        if ((rc = run_tick(E, witems, true, &wout)) != MANTRA_OK) return rc;
        for (size_t y = 0; y < witems.size(); ++y) {
            const uint32_t x = wide_ix[y];
            const u64* c = (const u64*)wout.slot[y];
            int st;
            std::memcpy(&st, wout.slot[y] + SLOT_STATUS, 4);
            if (st != MANTRA_OK) R->status[x] = st;
            R->tot[x].add_counters(c);
            R->tot[x].launches += 1;
            R->tot[x].wide += witems[y].job.count;
            R->tot[x].kernel_ms += witems[y].job.opt == MANTRA_PFM ? wout.pfm_ms : wout.bfs_ms;
            // reduction outputs of the wide tick include every sample of the round
            std::memcpy(R->slot[x].data() + SLOT_HMAX, wout.slot[y] + SLOT_HMAX, SLOT_BYTES - SLOT_HMAX);
        }
    }
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

// Appendix proposition (after Pellegrina & Vandin): with probability >= 1 - delta
// the largest estimator variance is at most W + L/r + sqrt((L/r)^2 + 2 W L / r),
// L = ln(1/delta); the printed square-root term is read in the self-bounding form
// of Theorem 1's R bound.
double wimpy_variance_bound(double W, double delta, double r) {
    const double L = std::log(1.0 / delta);
    return W + L / r + std::sqrt((L / r) * (L / r) + 2.0 * W * L / r);
}

double delta_of_round(double delta, uint64_t i, int sched) {
    return sched == 1 ? delta / std::ldexp(1.0, (int)i) : delta / std::ldexp(1.0, (int)(i + 1));
}

// ---------------------------------------------------------------------------
// Algorithm 1 for one problem, as a state machine advanced by ticks:
// BOOT (s' bootstrap samples) -> ROUND (schedule s_1, s_2, ...) -> DONE.
// ---------------------------------------------------------------------------
constexpr uint64_t RMAX = 0x7FFFFFFFull;

struct Problem {
    const mantra_graph* G = nullptr;
    int opt = 0;
    double eps = 0, delta = 0;
    uint64_t seed = 0;
    uint32_t c = 25;
    double growth = 1.2;
    uint64_t fixed_r = 0, boot = 0;
    int dsched = 0, vhat_mode = 0;
    int fam_target = 0;       // mantra_opts.target: 0 nodes, 1 underlying edges, 2 temporal edges
    int estimator = 0;        // mantra_opts.estimator: 0 trk (App. C), 1 ob (Sec. 4.1), 2 RTB (App. C)
    double* est_out = nullptr;
    uint64_t* hits_out = nullptr;
    bool out_device = false;
    mantra_info* info_out = nullptr;
    // device state
    u64* hits = nullptr; int* S = nullptr; double* est = nullptr; uint64_t* ovf = nullptr;
    u64* wsq = nullptr;       // ob: sums of f^2 (the wimpy variance's numerators)
    size_t b_hits = 0, b_S = 0, b_est = 0, b_ovf = 0, b_wsq = 0;
    uint64_t ovf_cap = 0;
    // progress: the current phase covers sample indices [phase_begin, phase_end);
    // pos = the next index to run (a phase may span several ticks)
    enum { BOOT, ROUND, DONE } phase = BOOT;
    uint64_t sb = 0, omega = 0, s1 = 0, r = 0, target = 0, round = 0, reduces = 0;
    uint64_t pos = 0, boot_sum_int = 0;
    LaunchTotals T;
    mantra_info I{};
    int status = MANTRA_OK;
    double t0 = 0;

    int validate() const {
        if (!G || (!est_out && !out_device)) return MANTRA_E_INVAL;
        if (!(eps > 0.0 && eps < 1.0) || !(delta > 0.0 && delta < 1.0)) return MANTRA_E_INVAL;
        if (opt != MANTRA_SH && opt != MANTRA_SFM && opt != MANTRA_PFM && opt != MANTRA_FSFM) return MANTRA_E_INVAL;
        if (c < 1 || c > 128 || !(growth > 1.0)) return MANTRA_E_INVAL;
        if (fixed_r > RMAX) return MANTRA_E_INVAL;
        if (out_device && !est_out) return MANTRA_E_INVAL;
        if (vhat_mode != 0 && vhat_mode != 1) return MANTRA_E_INVAL;
        if (fam_target < 0 || fam_target > 2) return MANTRA_E_INVAL;
        if (estimator < 0 || estimator > 2 || (estimator != 0 && fam_target != 0)) return MANTRA_E_INVAL;
        if (estimator != 0 && !ob_r_ok(fixed_r)) return MANTRA_E_INVAL;
        return MANTRA_OK;
    }

    // ob and RTB sums are in units of 2^-32 (f_v carried as the nearest
    // multiple): |N_R| <= c r 2^32 must fit int64, so c r < 2^31.
    double scale() const { return estimator != 0 ? 4294967296.0 : 1.0; }
    bool ob_r_ok(uint64_t rr) const { return (double)rr * (double)c < 2147483648.0; }

    // Size F of the estimated family (App. A for the edge families).
    uint32_t family() const { return fam_target == 0 ? G->n : (fam_target == 1 ? G->n_uedge : G->m); }

    // bytes of device state held while the problem runs (admission footprint)
    size_t footprint() const {
        const size_t f = std::max<uint32_t>(family(), 1);
        if (estimator != 0) return al256(f * 8) * 3 + al256((size_t)c * f * 8) + al256(8 * 4096);
        return al256(f * 8) * 2 + al256((size_t)c * f * 4) + al256(8 * 4096);
    }

    int grow_ovf(Engine& E, uint64_t need) {
        if (need <= ovf_cap) return MANTRA_OK;
        uint64_t nc = std::max<uint64_t>(4096, ovf_cap);
        while (nc < need) nc *= 2;
        if (ovf) E.pool.put(ovf, b_ovf);
        b_ovf = nc * 8;
        ovf = (uint64_t*)E.pool.get(b_ovf);
        if (!ovf) { ovf_cap = 0; return MANTRA_E_NOMEM; }
        ovf_cap = nc;
        return MANTRA_OK;
    }

    int start(Engine& E) {
        t0 = now_s();
        const size_t f = std::max<uint32_t>(family(), 1);
        b_hits = f * 8; b_S = (size_t)c * f * (estimator != 0 ? 8 : 4); b_est = f * 8;
        hits = (u64*)E.pool.get(b_hits);
        S = (int*)E.pool.get(b_S);
        est = out_device ? nullptr : (double*)E.pool.get(b_est);
        if (!hits || !S || (!out_device && !est)) return MANTRA_E_NOMEM;
        CU(cudaMemsetAsync(hits, 0, b_hits, E.sa));
        CU(cudaMemsetAsync(S, 0, b_S, E.sa));
        if (estimator != 0) {
            b_wsq = f * 8;
            wsq = (u64*)E.pool.get(b_wsq);
            if (!wsq) return MANTRA_E_NOMEM;
            CU(cudaMemsetAsync(wsq, 0, b_wsq, E.sa));
        }
        pos = 0; boot_sum_int = 0;
        if (fixed_r > 0) {
            phase = ROUND; target = fixed_r; r = 0;
        } else {
            sb = boot ? boot : (uint64_t)std::ceil(std::log(1.0 / delta) / eps);
            if (sb > RMAX) return MANTRA_E_INVAL;
            phase = BOOT;
        }
        return grow_ovf(E, phase == BOOT ? sb : target);
    }

    // Samples left in the current phase.
    uint64_t remaining() const { return phase == BOOT ? sb - pos : (phase == ROUND ? target - pos : 0); }

    // The next sample range, at most quota samples; the round reduction runs
    // on the tick that completes the phase.
    int item(Engine& E, TickItem* it, uint64_t quota = ~0ull) {
        it->G = G;
        Job& j = it->job;
        j = Job{};
        j.seed = seed; j.opt = opt; j.c = c; j.hits = hits;
        j.target = fam_target; j.fam = family();
        j.ob = estimator == 1; j.rtb = estimator == 2; j.wsq = wsq;
        const uint64_t left = remaining();
        j.i0 = pos; j.count = std::min(left, quota);
        if (phase == BOOT) {
            j.dom_pair = DOM_BOOT_PAIR; j.dom_path = DOM_BOOT_PATH; j.S = nullptr; j.S64 = nullptr;
            it->red_c = 0;
        } else {
            j.dom_pair = DOM_PAIR; j.dom_path = DOM_PATH;
            if (estimator != 0) { j.S = nullptr; j.S64 = (long long*)S; }
            else { j.S = S; j.S64 = nullptr; }
            it->red_c = c;
        }
        it->reduce = j.count == left;
        const int rc = grow_ovf(E, j.count);
        j.ovf_list = ovf;
        return rc;
    }

    // Advances the state after a tick of `count` samples (slot: counters, and
    // the reduction outputs when the tick completed the phase).
    int consume(Engine& E, const char* slot, const LaunchTotals& tt, uint64_t count) {
        T.kernel_ms += tt.kernel_ms; T.launches += tt.launches; T.escan += tt.escan; T.eadd += tt.eadd;
        T.snew += tt.snew; T.fseg += tt.fseg; T.xedge += tt.xedge; T.wide += tt.wide;
        if (phase == BOOT) boot_sum_int += tt.sum_int;
        else T.sum_int += tt.sum_int;
        pos += count;
        if (remaining() > 0) return MANTRA_OK;
        u64 H;
        std::memcpy(&H, slot + SLOT_HMAX, 8);
        reduces += 1;
        if (phase == BOOT) {
            // DrawSufficientSampleSize(G, s', delta/2) and SamplingSchedule
            double v0 = (double)H / ((double)sb * scale());
            double rho = (double)boot_sum_int / ((double)sb * scale());
            if (v0 == 0.0 || rho == 0.0) { v0 = 1.0 / (double)sb; rho = std::max(rho, v0); }
            const double om = std::ceil(omega_closed_form(v0, rho, eps, delta / 2.0));
            if (!(om <= (double)RMAX)) return MANTRA_E_INVAL;
            if (estimator != 0 && !ob_r_ok((uint64_t)std::max(om, 1.0))) return MANTRA_E_INVAL;
            omega = std::max<uint64_t>(1, (uint64_t)om);
            const double d1 = delta_of_round(delta, 1, dsched);
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
            CU(cudaMemsetAsync(hits, 0, b_hits, E.sa));
            if (wsq) CU(cudaMemsetAsync(wsq, 0, b_wsq, E.sa));
            phase = ROUND; r = 0; pos = 0; target = s1; round = 0;
            return MANTRA_OK;
        }
        r = target;
        round += 1;
        int64_t NR = 0;
        for (uint32_t jj = 0; jj < c; ++jj) {
            long long x;
            std::memcpy(&x, slot + SLOT_ROWMAX + 8 * jj, 8);
            NR += x;
        }
        const double W = (double)H / ((double)r * scale());
        double di = delta_of_round(delta, round, dsched), vh = W;
        if (vhat_mode == 1) {            // variance bound from W, delta_i split evenly
            di /= 2.0;
            vh = wimpy_variance_bound(W, di, (double)r);
        }
        const double xi = xi_from_mcera((double)NR / ((double)c * (double)r * scale()), W, vh, di, (double)r, (double)c);
        I.rounds = round; I.rade_num = NR; I.max_hits = H; I.xi = xi; I.vhat = vh;
        if (fixed_r > 0 || r >= omega || xi <= eps) { phase = DONE; return MANTRA_OK; }
        uint64_t nt = (uint64_t)std::ceil(growth * (double)target);
        if (nt <= target) nt = target + 1;
        target = std::min(omega, nt);
        return MANTRA_OK;
    }

    // est = hits / r, outputs copied (enqueued on E.sa; caller synchronises).
    int finish(Engine& E) {
        I.r = r;
        I.sum_int_len = T.sum_int;
        double* dst = out_device ? est_out : est;
        const uint32_t f = family();
        if (f > 0) {
            CU(launch_normalise(hits, f, (double)r * scale(), dst, E.sa));
            if (!out_device) CU(cudaMemcpyAsync(est_out, est, (size_t)f * 8, cudaMemcpyDeviceToHost, E.sa));
            if (hits_out)
                CU(cudaMemcpyAsync(hits_out, hits, (size_t)f * 8,
                                   out_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, E.sa));
        }
        I.edges_scanned = T.escan; I.sigma_adds = T.eadd; I.states_new = T.snew; I.wide_samples = T.wide;
        I.kernel_ms = T.kernel_ms; I.search_launches = T.launches;
        I.kernel_launches = T.launches + reduces + (f > 0 ? 1 : 0);
        I.alg_bytes = alg_bytes_of(opt == MANTRA_PFM, T.escan, T.eadd, T.snew, T.fseg);
        I.frontier_vertices = opt == MANTRA_PFM ? 0 : T.fseg;
        I.edges_expanded = opt == MANTRA_PFM ? T.xedge : 0;
        return MANTRA_OK;
    }

    void release(Engine& E) {
        E.pool.put(hits, b_hits); E.pool.put(S, b_S); E.pool.put(est, b_est); E.pool.put(ovf, b_ovf);
        E.pool.put(wsq, b_wsq);
        hits = nullptr; S = nullptr; est = nullptr; ovf = nullptr; ovf_cap = 0; wsq = nullptr;
    }
};

int problem_from(const mantra_graph* g, mantra_opt opt, double eps, double delta, uint64_t seed,
                 const mantra_opts* opts, double* est_out, uint64_t* hits_out, mantra_info* info, Problem* p) {
    mantra_opts o{};
    if (opts) o = *opts;
    p->G = g; p->opt = (int)opt; p->eps = eps; p->delta = delta; p->seed = seed;
    p->c = o.c ? o.c : 25;
    p->growth = o.growth > 0 ? o.growth : 1.2;
    p->fixed_r = o.fixed_r; p->boot = o.bootstrap; p->dsched = o.delta_sched;
    p->vhat_mode = o.vhat_mode;
    p->fam_target = o.target;
    p->estimator = o.estimator;
    p->est_out = est_out; p->hits_out = hits_out; p->out_device = o.out_device != 0; p->info_out = info;
    return p->validate();
}

// Runs Algorithm 1 for every problem together: each tick carries the next
// sample range of every unfinished problem.  Per-problem statuses are kept;
// the return value is the first failure, or MANTRA_OK.
// One tick for every running problem of `ps`: each contributes its next
// sample range; results advance each problem's state.  Returns false when no
// problem had work.
bool tick_problems(Engine& E, std::vector<Problem*>& ps, uint64_t budget_bfs = ~0ull, uint64_t budget_pfm = ~0ull) {
    std::vector<Problem*> act;
    std::vector<TickItem> items;
    std::vector<uint64_t*> ovfs;
    for (Problem* p : ps) {
        if (p->status != MANTRA_OK || p->phase == Problem::DONE) continue;
        uint64_t& left = p->opt == MANTRA_PFM ? budget_pfm : budget_bfs;
        if (left == 0) continue;                      // waits for a later tick
        TickItem it;
        const int rc = p->item(E, &it, left);
        if (rc != MANTRA_OK) { p->status = rc; continue; }
        left -= it.job.count;
        act.push_back(p); items.push_back(it); ovfs.push_back(p->ovf);
    }
    if (act.empty()) return false;
    TickResult R;
    const int rc = run_tick_full(E, items, ovfs.data(), &R);
    if (rc != MANTRA_OK) {
        for (Problem* p : act) p->status = rc;
        return true;
    }
    for (size_t x = 0; x < act.size(); ++x) {
        if (R.status[x] != MANTRA_OK) { act[x]->status = R.status[x]; continue; }
        const int st = act[x]->consume(E, R.slot[x].data(), R.tot[x], items[x].job.count);
        if (st != MANTRA_OK) act[x]->status = st;
    }
    return true;
}

// Outputs of finished (or failed) problems, buffers returned to the pool.
void finish_problems(Engine& E, std::vector<Problem*>& ps) {
    for (Problem* p : ps)
        if (p->status == MANTRA_OK) p->status = p->finish(E);
    const cudaError_t se = cudaStreamSynchronize(E.sa);
    for (Problem* p : ps) {
        if (se != cudaSuccess && p->status == MANTRA_OK) p->status = MANTRA_E_CUDA;
        p->I.seconds = now_s() - p->t0;
        if (p->info_out && p->status == MANTRA_OK) *p->info_out = p->I;
        p->release(E);
    }
}

// Runs Algorithm 1 for every problem together: each tick carries the next
// sample range of every unfinished problem.  Per-problem statuses are kept;
// the return value is the first failure, or MANTRA_OK.
int run_problems(Engine& E, std::vector<Problem*>& ps) {
    for (Problem* p : ps)
        if (p->status == MANTRA_OK) p->status = p->start(E);
    while (tick_problems(E, ps)) {
    }
    finish_problems(E, ps);
    for (Problem* p : ps)
        if (p->status != MANTRA_OK) return p->status;
    return MANTRA_OK;
}

// Orders the engine's streams after a caller stream, and the caller stream
// after the engine's work.
struct StreamJoin {
    Engine& E;
    cudaStream_t user;
    cudaEvent_t ev = nullptr;
    StreamJoin(Engine& e, void* s) : E(e), user((cudaStream_t)s) {
        if (user && cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) == cudaSuccess) {
            cudaEventRecord(ev, user);
            cudaStreamWaitEvent(E.sa, ev, 0);
        }
    }
    ~StreamJoin() {
        if (ev) {
            cudaEventRecord(ev, E.sa);
            cudaStreamWaitEvent(user, ev, 0);
            cudaEventDestroy(ev);
        }
    }
};

int current_engine(const mantra_graph* g, Engine** E) {
    int dev = g ? g->device : 0;
    if (!g) {
        if (cudaGetDevice(&dev) != cudaSuccess) return MANTRA_E_CUDA;
    }
    return engine_for(dev, E);
}

// ---------------------------------------------------------------------------
// Serving loop (continuous batching).  Requests wait in a FIFO queue and are
// admitted while the device state fits the budget: the running requests' own
// buffers plus the search workspaces sized for the largest running graph of
// each search family, the candidate included (one request is always admitted
// when none is running).  A tick carries a bounded number of
// samples per search family, about SERVER_TICK_PER_CTA per resident CTA,
// handed out in arrival order: the oldest running requests get their whole
// pending range first (a round may span ticks), so requests complete close
// to arrival order while every tick still fills the GPU.  Finished requests
// leave between ticks and queued ones join at the next tick.  Results wait
// on the host until polled.
// ---------------------------------------------------------------------------
constexpr uint64_t SERVER_TICK_PER_CTA = 32;

struct Request {
    uint64_t id = 0;
    Problem p;
    std::vector<double> est;
    std::vector<uint64_t> hits;
    mantra_info info{};
    int state = 0;            // 0 queued, 1 running, 2 finished
    bool started = false;
    size_t footprint = 0;
};

struct Server {
    Engine* E = nullptr;
    size_t budget = 0;
    uint32_t max_active = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request*> queue;
    std::vector<Request*> active;
    std::map<uint64_t, Request*> reqs;
    size_t used = 0;
    uint64_t next_id = 1, ticks = 0, finished = 0;
    bool stop = false;
    std::thread th;

    // Search workspace for the running requests and (if given) one more.
    size_t ws_for(const Request* extra) const {
        uint32_t n = 0, A = 0, z = 0, pn = 0, cb = 0;
        bool dl = false;
        auto add = [&](const Request* r) {
            const mantra_graph* G = r->p.G;
            if (!G) return;
            if (r->p.opt == MANTRA_PFM) {
                pn = std::max(pn, G->n); cb = std::max(cb, G->dg.cbound);
            } else {
                n = std::max(n, G->n); A = std::max(A, G->A); z = std::max(z, G->dg.max_vslots);
                dl = dl || r->p.estimator != 0;
            }
        };
        for (const Request* r : active) add(r);
        if (extra) add(extra);
        return E->ws_estimate(n, A, z, dl, pn, cb);
    }

    void loop() {
        std::unique_lock<std::mutex> lk(mu);
        while (true) {
            while (!queue.empty() && active.size() < max_active) {
                Request* r = queue.front();
                if (!active.empty() && used + r->footprint + ws_for(r) > budget) break;
                queue.pop_front();
                r->state = 1;
                used += r->footprint;
                active.push_back(r);
            }
            if (active.empty()) {
                if (stop) break;
                cv_work.wait(lk);
                continue;
            }
            std::vector<Request*> batch = active;
            lk.unlock();
            {
                std::lock_guard<std::mutex> elk(E->mu);
                std::vector<Problem*> ps;
                for (Request* r : batch) {
                    if (!r->started) {
                        r->started = true;
                        if (r->p.status == MANTRA_OK) r->p.status = r->p.start(*E);
                    }
                    ps.push_back(&r->p);
                }
                // per-family tick budgets (MANTRA_SERVER_TICK_SAMPLES overrides)
                uint64_t bb = SERVER_TICK_PER_CTA * (uint64_t)(E->bfs_grid ? E->bfs_grid : 2 * E->num_sms);
                uint64_t bp = SERVER_TICK_PER_CTA * (uint64_t)(E->pc_grid ? E->pc_grid : 2 * E->num_sms);
                if (const char* env = std::getenv("MANTRA_SERVER_TICK_SAMPLES")) {
                    const long long v = std::atoll(env);
                    if (v > 0) bb = bp = (uint64_t)v;
                }
                tick_problems(*E, ps, bb, bp);
                std::vector<Problem*> fin;
                for (Request* r : batch)
                    if (r->p.status != MANTRA_OK || r->p.phase == Problem::DONE) fin.push_back(&r->p);
                if (!fin.empty()) finish_problems(*E, fin);
            }
            lk.lock();
            ++ticks;
            for (auto it = active.begin(); it != active.end();) {
                Request* r = *it;
                if (r->p.status != MANTRA_OK || r->p.phase == Problem::DONE) {
                    r->state = 2;
                    used -= r->footprint;
                    ++finished;
                    it = active.erase(it);
                } else {
                    ++it;
                }
            }
            cv_done.notify_all();
        }
    }
};

// Copies a finished request's outputs and retires it (server lock held).
int take_result(Server* S, std::map<uint64_t, Request*>::iterator it, double* est_out, uint64_t* hits_out,
                mantra_info* info) {
    Request* r = it->second;
    const int st = r->p.status;
    if (st == MANTRA_OK) {
        const size_t f = r->p.family();
        if (est_out && f) std::memcpy(est_out, r->est.data(), f * 8);
        if (hits_out && f) std::memcpy(hits_out, r->hits.data(), f * 8);
        if (info) *info = r->info;
    }
    S->reqs.erase(it);
    delete r;
    return st;
}

}  // namespace

namespace mantra {

// Read-only view of a loaded graph for the library's other translation units.
int graph_view(const mantra_graph* g, const DevGraph** dg, int* device, uint32_t* n, uint32_t* A, int* num_sms,
               size_t* smem_optin, std::mutex** mu) {
    Engine* E = nullptr;
    const int rc = engine_for(g->device, &E);
    if (rc != MANTRA_OK) return rc;
    if (!E) return MANTRA_E_CUDA;
    *dg = &g->dg;
    *device = g->device;
    *n = g->n; *A = g->A;
    *num_sms = E->num_sms;
    *smem_optin = E->smem_optin;
    *mu = &E->mu;
    return MANTRA_OK;
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
        case MANTRA_PENDING: return "request still running";
        default: return "unknown error";
    }
}

int mantra_graph_load(const uint32_t* u, const uint32_t* v, const uint32_t* t, uint64_t m, uint32_t n,
                      mantra_graph** out) {
    if (!out || (m > 0 && (!u || !v || !t))) return MANTRA_E_INVAL;
    *out = nullptr;
    mantra_graph* G = new (std::nothrow) mantra_graph();
    if (!G) return MANTRA_E_NOMEM;
    Engine* E = nullptr;
    int rc = MANTRA_OK;
    if (cudaGetDevice(&G->device) != cudaSuccess) rc = MANTRA_E_CUDA;
    if (rc == MANTRA_OK) rc = engine_for(G->device, &E);
    if (rc == MANTRA_OK) {
        std::lock_guard<std::mutex> lock(E->mu);
        StoreHost H;
        rc = E->store.build(u, v, t, m, n, &H);
        if (rc == MANTRA_OK) rc = upload_store(H, G, E->sa);
        E->store.trim();
    }
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

int mantra_graph_edges(const mantra_graph* g, uint32_t* u_out, uint32_t* v_out, uint32_t* t_out,
                       uint32_t* uedge_out, uint32_t* n_underlying) {
    if (!g || !n_underlying) return MANTRA_E_INVAL;
    *n_underlying = g->n_uedge;
    const uint32_t M = g->m;
    if (M == 0) return MANTRA_OK;
    if (!u_out || !v_out || !t_out || !uedge_out) return MANTRA_E_INVAL;
    std::vector<uint32_t> slot_v, slot_t, in_slot;
    try { slot_v.resize(g->A); slot_t.resize(g->A); in_slot.resize(M); } catch (...) { return MANTRA_E_NOMEM; }
    if (cudaMemcpy(u_out, g->dg.in_u, (size_t)M * 4, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(uedge_out, g->dg.in_uedge, (size_t)M * 4, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(in_slot.data(), g->dg.in_slot, (size_t)M * 4, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(slot_v.data(), g->dg.slot_v, (size_t)g->A * 4, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(slot_t.data(), g->dg.slot_t, (size_t)g->A * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
        return MANTRA_E_CUDA;
    for (uint32_t e = 0; e < M; ++e) { v_out[e] = slot_v[in_slot[e]]; t_out[e] = slot_t[in_slot[e]]; }
    return MANTRA_OK;
}

void mantra_graph_free(mantra_graph* g) {
    if (!g) return;
    Engine* E = nullptr;
    if (g->dmem && engine_for(g->device, &E) == MANTRA_OK) {
        std::lock_guard<std::mutex> lock(E->mu);
        cudaStreamSynchronize(E->sa);
        cudaStreamSynchronize(E->sb);
        cudaFree(g->dmem);
    } else if (g->dmem) {
        cudaFree(g->dmem);
    }
    delete g;
}

int mantra_estimate(const mantra_graph* g, mantra_opt opt, double eps, double delta, uint64_t seed,
                    const mantra_opts* opts, double* est_out, uint64_t* hits_out, mantra_info* info) {
    if (!g || !est_out) return MANTRA_E_INVAL;
    Problem p;
    int rc = problem_from(g, opt, eps, delta, seed, opts, est_out, hits_out, info, &p);
    if (rc != MANTRA_OK) return rc;
    Engine* E = nullptr;
    if ((rc = current_engine(g, &E)) != MANTRA_OK) return rc;
    std::lock_guard<std::mutex> lock(E->mu);
    StreamJoin join(*E, opts ? opts->stream : nullptr);
    std::vector<Problem*> ps{&p};
    return run_problems(*E, ps);
}

int mantra_tune(mantra_graph* g, mantra_tune_result* out) {
    if (!g || !out) return MANTRA_E_INVAL;
    Engine* E = nullptr;
    int rc = current_engine(g, &E);
    if (rc != MANTRA_OK) return rc;
    // probes: fixed-r estimates with the same seed for every candidate; a
    // candidate's time is the smaller kernel time of two runs (the first run of
    // a configuration also allocates).  The knobs serve Algorithm 1's large
    // rounds, so a probe is sized like one: about 100 ms of kernel time by a
    // calibration run of the defaults, between 8 and 64 samples per SM.
    const uint64_t r_lo = 8ull * (uint64_t)E->num_sms, r_hi = 64ull * (uint64_t)E->num_sms;
    uint64_t r = r_lo;
    std::vector<double> est(std::max<uint32_t>(g->n, 1));
    auto probe = [&](mantra_opt opt, const Knobs& k, double* ms) -> int {
        g->knobs = k;
        mantra_opts o{};
        o.c = 25;
        o.fixed_r = r;
        *ms = 1e300;
        for (int rep = 0; rep < 2; ++rep) {
            mantra_info I{};
            const int st = mantra_estimate(g, opt, 0.05, 0.1, 0x7E57ull, &o, est.data(), nullptr, &I);
            if (st != MANTRA_OK) return st;
            *ms = std::min(*ms, I.kernel_ms);
        }
        return MANTRA_OK;
    };
    const Knobs none{};
    Knobs best{};
    auto size_probe = [&](mantra_opt opt) -> int {
        r = r_lo;
        double ms = 0;
        const int st = probe(opt, none, &ms);
        if (st != MANTRA_OK) return st;
        const double per = ms > 0 ? ms / (double)r_lo : 0.0;
        r = per > 0 ? (uint64_t)std::min<double>((double)r_hi, std::max<double>((double)r_lo, 100.0 / per)) : r_hi;
        return MANTRA_OK;
    };
    // sh/sfm: CTA shape x visited-bitmap placement (shared memory only where it fits)
    if ((rc = size_probe(MANTRA_SH)) != MANTRA_OK) { g->knobs = none; return rc; }
    out->probe_samples = r;
    if ((rc = probe(MANTRA_SH, none, &out->bfs_default_ms)) != MANTRA_OK) { g->knobs = none; return rc; }
    out->bfs_ms = 1e300;
    for (int nt : {256, 512, 1024})
        for (int sm = 0; sm < 2; ++sm) {
            if (!E->bfs_grids[Engine::shape_of(nt)][sm]) continue;
            Knobs k = none;
            k.bfs_nt = nt; k.bfs_smem = sm;
            double ms = 0;
            if ((rc = probe(MANTRA_SH, k, &ms)) != MANTRA_OK) { g->knobs = none; return rc; }
            if (ms < out->bfs_ms) { out->bfs_ms = ms; best.bfs_nt = nt; best.bfs_smem = sm; }
        }
    // pfm (one CTA per sample): CTA shape x arrival-state placement
    if ((rc = size_probe(MANTRA_PFM)) != MANTRA_OK) { g->knobs = none; return rc; }
    out->pfm_probe_samples = r;
    if ((rc = probe(MANTRA_PFM, none, &out->pfm_default_ms)) != MANTRA_OK) { g->knobs = none; return rc; }
    out->pfm_ms = 1e300;
    for (int nt : {256, 512})
        for (int sm = 0; sm < 4; ++sm) {
            if (!E->pc_grids[nt == 256 ? 0 : 1][sm]) continue;
            if (sm == 3 && g->dg.max_vslots > PFM_W16_MAX_VSLOTS) continue;
            Knobs k = none;
            k.pfm_nt = nt; k.pfm_mode = sm;
            double ms = 0;
            if ((rc = probe(MANTRA_PFM, k, &ms)) != MANTRA_OK) { g->knobs = none; return rc; }
            if (ms < out->pfm_ms) { out->pfm_ms = ms; best.pfm_nt = nt; best.pfm_mode = sm; }
        }
    g->knobs = best;
    out->bfs_threads = (uint32_t)best.bfs_nt;
    out->bfs_bitmap_shared = best.bfs_smem > 0 ? 1u : 0u;
    out->pfm_threads = (uint32_t)best.pfm_nt;               // 0: the stream-scan pfm kernel is forced
    out->pfm_state_shared = best.pfm_mode == 1 || best.pfm_mode == 3 ? 1u : 0u;
    out->pfm_staged = best.pfm_mode == 2 ? 1u : 0u;
    out->pfm_state16 = best.pfm_mode == 3 ? 1u : 0u;
    out->bfs_resident_ctas = best.bfs_nt ? (uint32_t)E->bfs_grids[Engine::shape_of(best.bfs_nt)][best.bfs_smem] : 0u;
    out->pfm_resident_ctas = best.pfm_nt ? (uint32_t)E->pc_grids[best.pfm_nt == 256 ? 0 : 1][best.pfm_mode] : 0u;
    if (!best.pfm_nt) out->pfm_ms = out->pfm_default_ms;
    return MANTRA_OK;
}

int mantra_estimate_batch(mantra_problem* probs, uint32_t count) {
    if (!probs && count) return MANTRA_E_INVAL;
    if (count == 0) return MANTRA_OK;
    std::vector<Problem> P(count);
    std::vector<Problem*> ptrs;
    Engine* E = nullptr;
    int first = MANTRA_OK;
    for (uint32_t x = 0; x < count; ++x) {
        mantra_problem& q = probs[x];
        q.status = problem_from(q.graph, q.opt, q.eps, q.delta, q.seed, q.opts, q.est_out, q.hits_out, q.info, &P[x]);
        if (q.status == MANTRA_OK && q.graph) {
            Engine* e = nullptr;
            q.status = current_engine(q.graph, &e);
            if (q.status == MANTRA_OK && E && e != E) q.status = MANTRA_E_INVAL;   // one device per batch
            if (q.status == MANTRA_OK) E = e;
        }
        if (q.status == MANTRA_OK) ptrs.push_back(&P[x]);
        else if (first == MANTRA_OK) first = q.status;
    }
    if (!E) return first == MANTRA_OK ? MANTRA_E_INVAL : first;
    {
        std::lock_guard<std::mutex> lock(E->mu);
        const int rc = run_problems(*E, ptrs);
        if (first == MANTRA_OK) first = rc;
    }
    for (uint32_t x = 0; x < count; ++x)
        if (probs[x].status == MANTRA_OK) probs[x].status = P[x].status;
    return first;
}

// Algorithm 2's searches: r_s full searches from sources drawn from the STATS
// stream; hc[h] = reached (source, v) pairs at distance h, *dm = the largest
// distance; with clos_out (n entries) also the per-vertex closeness sums.
int stats_run(const mantra_graph* g, mantra_opt opt, uint64_t rs, uint64_t seed, std::vector<u64>* hc, u64* dm,
              uint64_t* clos_out) {
    if (opt != MANTRA_SH && opt != MANTRA_SFM && opt != MANTRA_PFM && opt != MANTRA_FSFM) return MANTRA_E_INVAL;
    Engine* E = nullptr;
    int rc;
    if ((rc = current_engine(g, &E)) != MANTRA_OK) return rc;
    std::lock_guard<std::mutex> lock(E->mu);
    const uint32_t n = g->n;
    const size_t b_cnt = ((size_t)n + 2) * 8;
    const size_t b_clos = clos_out ? al256((size_t)n * 8) : 0;
    const size_t b_all = al256(b_cnt) + 256 + al256(rs * 8) + b_clos;
    char* blk = (char*)E->pool.get(b_all);
    if (!blk) return MANTRA_E_NOMEM;
    u64* cnt = (u64*)blk;
    u64* dmax = (u64*)(blk + al256(b_cnt));
    u64* clos = clos_out ? (u64*)(blk + al256(b_cnt) + 256 + al256(rs * 8)) : nullptr;
    CU(cudaMemsetAsync(blk, 0, al256(b_cnt) + 256, E->sa));
    if (clos) CU(cudaMemsetAsync(clos, 0, b_clos, E->sa));
    std::vector<TickItem> items(1);
    items[0].G = g;
    Job& j = items[0].job;
    // sh and sfm share their distances (first level); fsfm and pfm have their own
    j.seed = seed; j.i0 = 0; j.count = rs;
    j.opt = (opt == MANTRA_PFM || opt == MANTRA_FSFM) ? (int)opt : (int)MANTRA_SH;
    j.stats = 1; j.cnt = cnt; j.dmax = dmax; j.clos = clos;
    j.ovf_list = (uint64_t*)(blk + al256(b_cnt) + 256);       // pfm lists that overflowed: re-run in order
    TickResult TR;
    uint64_t* ovfs[1] = {j.ovf_list};
    rc = run_tick_full(*E, items, ovfs, &TR);
    hc->assign((size_t)n + 1, 0);
    *dm = 0;
    if (rc == MANTRA_OK && TR.status[0] != MANTRA_OK) rc = TR.status[0];
    if (rc == MANTRA_OK) {
        if (cudaMemcpyAsync(hc->data(), cnt, ((size_t)n + 1) * 8, cudaMemcpyDeviceToHost, E->sa) != cudaSuccess ||
            cudaMemcpyAsync(dm, dmax, 8, cudaMemcpyDeviceToHost, E->sa) != cudaSuccess ||
            (clos && cudaMemcpyAsync(clos_out, clos, (size_t)n * 8, cudaMemcpyDeviceToHost, E->sa) != cudaSuccess) ||
            cudaStreamSynchronize(E->sa) != cudaSuccess)
            rc = MANTRA_E_CUDA;
    }
    E->pool.put(blk, b_all);
    return rc;
}

int mantra_temporal_stats(const mantra_graph* g, mantra_opt opt, double eps, uint64_t seed, uint64_t r_override,
                          double tau, mantra_tstats* out, uint64_t* reach_out, uint32_t reach_cap) {
    if (!g || !out) return MANTRA_E_INVAL;
    if (!(eps > 0.0 && eps < 1.0) || !(tau >= 0.0 && tau <= 1.0)) return MANTRA_E_INVAL;
    const double t0 = now_s();
    const uint32_t n = g->n;
    const uint64_t rs = r_override ? r_override : (uint64_t)std::ceil(std::log((double)n) / (eps * eps));
    std::vector<u64> hc;
    u64 dm = 0;
    const int rc = stats_run(g, opt, rs, seed, &hc, &dm, nullptr);
    if (rc != MANTRA_OK) return rc;
    const uint32_t D = (uint32_t)dm;
    std::vector<u64> R((size_t)D + 1);
    u64 acc = 0;
    for (uint32_t h = 0; h <= D; ++h) { acc += hc[h]; R[h] = acc; }
    if (reach_out)
        for (uint32_t h = 0; h < reach_cap; ++h) reach_out[h] = (h <= D) ? R[h] : acc;
    // Algorithm 2's host formulas: Rhat[h] = (n / r) R[h]
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

int mantra_temporal_closeness(const mantra_graph* g, mantra_opt opt, double eps, uint64_t seed, uint64_t r_override,
                              uint64_t* sum_out, double* closeness_out, uint64_t* r_out) {
    if (!g || !closeness_out) return MANTRA_E_INVAL;
    if (!(eps > 0.0 && eps < 1.0)) return MANTRA_E_INVAL;
    const uint32_t n = g->n;
    const uint64_t rs = r_override ? r_override : (uint64_t)std::ceil(std::log((double)n) / (eps * eps));
    std::vector<u64> hc;
    std::vector<uint64_t> sum(n, 0);
    u64 dm = 0;
    const int rc = stats_run(g, opt, rs, seed, &hc, &dm, sum.data());
    if (rc != MANTRA_OK) return rc;
    for (uint32_t v = 0; v < n; ++v) {
        if (sum_out) sum_out[v] = sum[v];
        closeness_out[v] = ((double)sum[v] * (double)n) / (4294967296.0 * (double)rs * (double)(n - 1));
    }
    if (r_out) *r_out = rs;
    return MANTRA_OK;
}

int mantra_sample_paths(const mantra_graph* g, mantra_opt opt, uint64_t seed, uint32_t dom_pair, uint32_t dom_path,
                        uint64_t i0, uint64_t count, uint32_t* s_out, uint32_t* z_out, uint64_t* sigma_out,
                        uint32_t* len_out, uint32_t* nodes_out, uint32_t cap, uint32_t* edges_out) {
    if (!g || !s_out || !z_out || !sigma_out || !len_out || (cap > 0 && !nodes_out)) return MANTRA_E_INVAL;
    if (opt != MANTRA_SH && opt != MANTRA_SFM && opt != MANTRA_PFM && opt != MANTRA_FSFM) return MANTRA_E_INVAL;
    if (dom_pair > 5 || dom_path > 5) return MANTRA_E_INVAL;
    if (count == 0) return MANTRA_OK;
    Engine* E = nullptr;
    int rc;
    if ((rc = current_engine(g, &E)) != MANTRA_OK) return rc;
    std::lock_guard<std::mutex> lock(E->mu);
    const size_t capn = std::max<uint32_t>(cap, 1);
    const size_t bytes = al256(count * 4) * 3 + al256(count * 16) + al256(count * capn * 4) * 2 + al256(count * 8);
    char* d = (char*)E->pool.get(bytes);
    if (!d) return MANTRA_E_NOMEM;
    std::vector<TickItem> items(1);
    items[0].G = g;
    Job& j = items[0].job;
    j.seed = seed; j.i0 = i0; j.count = count; j.dom_pair = dom_pair; j.dom_path = dom_path; j.opt = (int)opt;
    size_t o = 0;
    j.rec_s = (uint32_t*)(d + o); o += al256(count * 4);
    j.rec_z = (uint32_t*)(d + o); o += al256(count * 4);
    j.rec_len = (uint32_t*)(d + o); o += al256(count * 4);
    j.rec_sig = (u64*)(d + o); o += al256(count * 16);
    j.rec_nodes = (uint32_t*)(d + o); o += al256(count * capn * 4);
    j.rec_edges = edges_out ? (uint32_t*)(d + o) : nullptr; o += al256(count * capn * 4);
    j.ovf_list = (uint64_t*)(d + o);
    j.rec_cap = (uint32_t)capn;
    TickResult R;
    uint64_t* ovfs[1] = {j.ovf_list};
    rc = run_tick_full(*E, items, ovfs, &R);
    if (rc == MANTRA_OK && R.status[0] != MANTRA_OK) rc = R.status[0];
    if (rc == MANTRA_OK) {
        cudaError_t e = cudaSuccess;
        if (e == cudaSuccess) e = cudaMemcpyAsync(s_out, j.rec_s, count * 4, cudaMemcpyDeviceToHost, E->sa);
        if (e == cudaSuccess) e = cudaMemcpyAsync(z_out, j.rec_z, count * 4, cudaMemcpyDeviceToHost, E->sa);
        if (e == cudaSuccess) e = cudaMemcpyAsync(len_out, j.rec_len, count * 4, cudaMemcpyDeviceToHost, E->sa);
        if (e == cudaSuccess) e = cudaMemcpyAsync(sigma_out, j.rec_sig, count * 16, cudaMemcpyDeviceToHost, E->sa);
        if (e == cudaSuccess && cap > 0)
            e = cudaMemcpyAsync(nodes_out, j.rec_nodes, count * (size_t)cap * 4, cudaMemcpyDeviceToHost, E->sa);
        if (e == cudaSuccess && cap > 0 && edges_out)
            e = cudaMemcpyAsync(edges_out, j.rec_edges, count * (size_t)cap * 4, cudaMemcpyDeviceToHost, E->sa);
        if (e == cudaSuccess) e = cudaStreamSynchronize(E->sa);
        if (e != cudaSuccess) rc = MANTRA_E_CUDA;
    }
    E->pool.put(d, bytes);
    return rc;
}

int mantra_server_create(size_t hbm_budget, uint32_t max_active, mantra_server** out) {
    if (!out) return MANTRA_E_INVAL;
    *out = nullptr;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return MANTRA_E_CUDA;
    Engine* E = nullptr;
    int rc = engine_for(dev, &E);
    if (rc != MANTRA_OK) return rc;
    Server* S = new (std::nothrow) Server();
    if (!S) return MANTRA_E_NOMEM;
    S->E = E;
    S->budget = hbm_budget ? hbm_budget : free_device_bytes() / 2;
    S->max_active = max_active ? max_active : 256;
    try {
        S->th = std::thread([S, dev]() {
            cudaSetDevice(dev);
            S->loop();
        });
    } catch (...) {
        delete S;
        return MANTRA_E_NOMEM;
    }
    *out = reinterpret_cast<mantra_server*>(S);
    return MANTRA_OK;
}

int mantra_server_submit(mantra_server* srv, const mantra_graph* g, mantra_opt opt, double eps, double delta,
                         uint64_t seed, const mantra_opts* opts, uint64_t* req_id) {
    Server* S = reinterpret_cast<Server*>(srv);
    if (!S || !g || !req_id) return MANTRA_E_INVAL;
    if (opts && opts->out_device) return MANTRA_E_INVAL;     // served results are host arrays
    Request* r = new (std::nothrow) Request();
    if (!r) return MANTRA_E_NOMEM;
    const int tgt = opts ? opts->target : 0;
    const uint32_t fam = tgt == 1 ? g->n_uedge : (tgt == 2 ? g->m : g->n);
    try {
        r->est.assign(std::max<uint32_t>(fam, 1), 0.0);
        r->hits.assign(std::max<uint32_t>(fam, 1), 0);
    } catch (...) {
        delete r;
        return MANTRA_E_NOMEM;
    }
    const int rc = problem_from(g, opt, eps, delta, seed, opts, r->est.data(), r->hits.data(), &r->info, &r->p);
    if (rc != MANTRA_OK) { delete r; return rc; }
    r->footprint = r->p.footprint();
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->stop) { delete r; return MANTRA_E_INVAL; }
    r->id = S->next_id++;
    S->reqs[r->id] = r;
    S->queue.push_back(r);
    *req_id = r->id;
    S->cv_work.notify_one();
    return MANTRA_OK;
}

int mantra_server_poll(mantra_server* srv, uint64_t req_id, double* est_out, uint64_t* hits_out, mantra_info* info) {
    Server* S = reinterpret_cast<Server*>(srv);
    if (!S) return MANTRA_E_INVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(req_id);
    if (it == S->reqs.end()) return MANTRA_E_INVAL;
    if (it->second->state != 2) return MANTRA_PENDING;
    return take_result(S, it, est_out, hits_out, info);
}

int mantra_server_wait(mantra_server* srv, uint64_t req_id, double timeout_s, double* est_out, uint64_t* hits_out,
                       mantra_info* info) {
    Server* S = reinterpret_cast<Server*>(srv);
    if (!S) return MANTRA_E_INVAL;
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->reqs.find(req_id);
    if (it == S->reqs.end()) return MANTRA_E_INVAL;
    Request* r = it->second;
    const auto deadline = std::chrono::steady_clock::now() +
                          std::chrono::duration_cast<std::chrono::steady_clock::duration>(
                              std::chrono::duration<double>(timeout_s > 0 ? timeout_s : 1e9));
    while (r->state != 2) {
        if (S->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && r->state != 2) return MANTRA_PENDING;
    }
    return take_result(S, S->reqs.find(req_id), est_out, hits_out, info);
}

int mantra_server_stats(mantra_server* srv, uint64_t* queued, uint64_t* active, uint64_t* finished,
                        uint64_t* ticks, uint64_t* bytes_in_use) {
    Server* S = reinterpret_cast<Server*>(srv);
    if (!S) return MANTRA_E_INVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    if (queued) *queued = S->queue.size();
    if (active) *active = S->active.size();
    if (finished) *finished = S->finished;
    if (ticks) *ticks = S->ticks;
    if (bytes_in_use) *bytes_in_use = S->active.empty() ? 0 : S->used + S->ws_for(nullptr);
    return MANTRA_OK;
}

void mantra_server_destroy(mantra_server* srv) {
    Server* S = reinterpret_cast<Server*>(srv);
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
        // queued requests are dropped; running ones finish
        for (Request* r : S->queue) { S->reqs.erase(r->id); delete r; }
        S->queue.clear();
        S->cv_work.notify_all();
    }
    if (S->th.joinable()) S->th.join();
    for (auto& kv : S->reqs) delete kv.second;
    delete S;
}

}  // extern "C"
