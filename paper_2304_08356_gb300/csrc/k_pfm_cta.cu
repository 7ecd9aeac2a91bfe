// Prefix-foremost search with one CTA per sample (paper Sec. 3 Def. 1(3)).
// The lane-per-sample kernel walks the time-sorted stream serially, so one
// of its launches costs at least one warp's walk however few samples it has;
// this kernel spreads each sample over a CTA instead.  Per sample:
//   arrivals  label-correcting rounds over the out-CSR.  A vertex u whose
//             earliest arrival fa(u) improved is expanded over its out-edges
//             with fa(u) < t <= bound; an edge (u, v, t), v != s, lowers v's
//             arrival to t.  An improvement of fa(u) from a to b only adds the
//             times in (b, a], so every out-edge is expanded at most once.
//             bound = the latest in-edge time of z, then fa(z) once z is
//             reached (later edges reach no vertex earlier than z).
//   counts    pfm paths use the edges (w, v, fa(v)) with fa(w) < fa(v): a DAG.
//             A scan of each reached vertex's arrival-slot in-edges finds them
//             all: pend(v) = their number, and the DAG is stored as out-lists
//             (per-tail counts, a scan, a fill).  A vertex whose in-edges are
//             all counted is expanded (Kahn levels) over its list and adds
//             sigma(u) to sigma(v) (hop(v) = min hop(u) + 1 for the Algorithm 2
//             searches).
//   draw      backward over DAG in-edges by ascending w, weight sigma(w)
//             (App. C path sampler), then the Update step of Algorithm 1.
// Path counts are 64-bit; a sample whose count overflows goes to the
// overflow list for the 128-bit lane kernel.
//
// Arrival state: fsl(v) = the arrival slot of v's earliest arrival (slots of
// one vertex are numbered in time order, so the minimum slot is the earliest
// time), NONE when unreached, SRC for s.  An edge carries the slot of its head
// appearance (out_slot), so expansion never reads edge times, and the DAG
// test of an edge is out_slot(e) == fsl(v).  A round processes its frontier
// in chunks of CHUNK vertices: the out-edge ranges of a chunk go to shared
// memory and every warp walks a contiguous slice of the chunk's edges,
// tracking the owning range with one ballot per 32 edges.  The first usable
// out-edge of each expansion is kept (lo_prev), so a re-expansion and the
// Kahn pass need at most one search of an out-row; searches of several
// vertices run interleaved.
//
// State modes (template FA): 0 -- fsl and the two bitmaps in a global-memory
// region; 1 -- in shared memory; 2 -- in shared memory with fsl(v) kept as
// the 16-bit offset of the slot within v's slots (slot_ptr(v) + offset is
// the slot; 0xFFFF unreached, 0xFFFE the source), which halves the largest
// shared-memory array so that more CTAs, or more L1, fit per SM.  Mode 2
// needs every vertex to have at most 0xFFFE slots; its expansion reads the
// store's per-edge head offsets (out_loff) instead of out_slot, and the
// arrival minimum is a compare-and-swap loop on the 16-bit entry.
#include "mantra_dev.cuh"

#include <mutex>

namespace mantra {

constexpr uint32_t SRC = NONE - 1u;        // fsl of the source
constexpr uint32_t O16_NONE = 0xFFFFu;     // mode 2: unreached
constexpr uint32_t O16_SRC = 0xFFFEu;      // mode 2: the source
constexpr int WALK_K = 2;                  // edge windows with loads in flight per warp
constexpr int CK = 8;                      // vertices with loads in flight per thread in the O(n) passes

template <bool SM>
__device__ __forceinline__ uint32_t ldv(const uint32_t* p) {
    if (SM) return *p;
    return __ldcg(p);
}

// ---- bulk copies (TMA engine) of out-edge tiles into shared memory ----
// One mbarrier per CTA tracks a chunk's copies by their byte count (expect_tx
// by one thread, complete_tx by every copy).  Addresses and sizes are 16-byte
// multiples by construction (see the staged table).
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0u;
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Waits for the mbarrier phase with the given parity, at most about a second
// of polls (each poll may suspend the thread for a while); false on timeout.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
    for (uint32_t it = 0; it < (1u << 22); ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// PC_NT threads per CTA; FA the state mode.  The launch bound asks for
// 1536 / PC_NT CTAs per SM, i.e. at most 40 registers: three 512-thread CTAs
// where shared memory allows (16-bit or global state), and measured 3 %
// faster than the 64-register build even at two CTAs per SM (the 32-bit
// shared state), despite some spilling.
template <int PC_NT, int FA>
__global__ void __launch_bounds__(PC_NT, 1536 / PC_NT) k_pfm_cta(const Task* tasks, const uint64_t* unit_start,
                                                                const uint32_t* ntasks_p, u64* work, const PfmCtaWs ws) {
    constexpr int PC_NW = PC_NT / 32;
    constexpr uint32_t CHUNK = 2 * PC_NT;      // frontier vertices per range table
    constexpr bool FA_SMEM = FA != 0;          // state in shared memory
    constexpr bool W16 = FA == 2;              // fsl as 16-bit slot offsets
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const uint32_t FULL = 0xFFFFFFFFu;
    __shared__ __align__(16) Task sh_task;
    __shared__ int sh_t;
    __shared__ uint64_t sh_q;
    __shared__ u64 sm_scan64[32];
    __shared__ uint32_t sm_scan32[32];
    __shared__ uint32_t sm_wcnt[PC_NW];
    __shared__ uint32_t sh_L, sh_Gc, sh_ovf, sh_err, sh_len;
    __shared__ uint32_t sh_rade[4];
    __shared__ u64 sh_sigma;
    __shared__ uint32_t sh_nt;
    __shared__ uint32_t cs_off[CHUNK + 1], cs_first[CHUNK], cs_u[CHUNK];   // range table of a chunk
    __shared__ __align__(8) uint64_t sh_mbar;     // completion of a chunk's staged edge tiles
    extern __shared__ __align__(128) uint32_t pc_dyn[];
    // global-state variant with staging: out_v and out_slot tiles of a chunk's
    // ranges, ws.stage_cap entries each, filled by bulk copies
    uint32_t* const stg_v = pc_dyn;
    uint32_t* const stg_s = pc_dyn + ws.stage_cap;
    const bool stage = !FA_SMEM && ws.stage_cap > 0;
    uint32_t stage_par = 0;                        // parity of the mbarrier phase to wait for

    char* region = ws.base + (size_t)blockIdx.x * ws.stride;
    uint32_t* fsl = FA == 1 ? pc_dyn : reinterpret_cast<uint32_t*>(region + ws.o_fa);
    unsigned short* const fso = reinterpret_cast<unsigned short*>(pc_dyn);   // mode 2
    const uint32_t fa_words = W16 ? (ws.n_cap + 1) / 2 : ws.n_cap;           // shared words of the state
    uint32_t* NB = FA_SMEM ? pc_dyn + fa_words : reinterpret_cast<uint32_t*>(region + ws.o_bits);  // next frontier
    uint32_t* XB = NB + ws.bits_words;                                                              // expanded before
    uint32_t* lo_prev = reinterpret_cast<uint32_t*>(region + ws.o_exp);  // first out-edge of the last expansion
    uint32_t* fat = reinterpret_cast<uint32_t*>(region + ws.o_fat);      // fa' = fa + 1 (0: s, NONE: unreached)
    u64* sig = reinterpret_cast<u64*>(region + ws.o_sig);
    uint32_t* hop = reinterpret_cast<uint32_t*>(region + ws.o_hop);
    uint32_t* pend = reinterpret_cast<uint32_t*>(region + ws.o_pend);
    uint32_t* Fl = reinterpret_cast<uint32_t*>(region + ws.o_list);      // frontier vertices
    uint32_t* path = reinterpret_cast<uint32_t*>(region + ws.o_path);
    uint32_t* pathe = reinterpret_cast<uint32_t*>(region + ws.o_pathe);   // in-CSR index of path edge k
    u64* dl = reinterpret_cast<u64*>(region + ws.o_dl);                  // ob: continuation counts
    uint32_t* kofs = reinterpret_cast<uint32_t*>(region + ws.o_kofs);    // ob: Kahn round offsets in Fl
    uint32_t* dcnt = reinterpret_cast<uint32_t*>(region + ws.o_dcnt);    // DAG out-list ends per vertex
    uint32_t* dag = reinterpret_cast<uint32_t*>(region + ws.o_dag);      // DAG successors, grouped by tail

    const uint32_t ntasks = *ntasks_p;
    u64* flush_ctr = nullptr;
    u64 my_escan = 0, my_eadd = 0, my_x = 0, my_rounds = 0;   // my_x, my_rounds: thread 0
    // the next-frontier bitmap is all zero between samples (compaction clears what it reads)
    for (uint32_t w = tid; w < ws.bits_words; w += PC_NT) NB[w] = 0u;
    if (tid == 0 && stage) {
        mbar_init(&sh_mbar, 1u);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    // Compacts the next-frontier bitmap (nwords words) into out in vertex order
    // and clears it; returns the number of vertices.  Contains barriers.
    auto compact = [&](uint32_t nwords, uint32_t* out) -> uint32_t {
        const uint32_t per_w = (((nwords + PC_NW - 1) / PC_NW) + 31u) & ~31u;
        const uint32_t w_lo = min((uint32_t)wid * per_w, nwords), w_hi = min(w_lo + per_w, nwords);
        uint32_t cnt = 0;
        for (uint32_t w = w_lo + lane; w < w_hi; w += 32) cnt += __popc(ldv<FA_SMEM>(NB + w));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(FULL, cnt, o);
        if (lane == 0) sm_wcnt[wid] = cnt;
        __syncthreads();
        if (wid == 0) {
            const uint32_t x = (lane < PC_NW) ? sm_wcnt[lane] : 0u;
            uint32_t incl = x;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(FULL, incl, o);
                if (lane >= o) incl += y;
            }
            if (lane < PC_NW) sm_wcnt[lane] = incl - x;
            if (lane == 31) sh_L = incl;
        }
        __syncthreads();
        uint32_t off = sm_wcnt[wid];
        for (uint32_t w0 = w_lo; w0 < w_hi; w0 += 32) {
            const uint32_t w = w0 + lane;
            uint32_t bits = (w < w_hi) ? ldv<FA_SMEM>(NB + w) : 0u;
            if (bits) NB[w] = 0u;
            const uint32_t c = __popc(bits);
            uint32_t incl = c;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(FULL, incl, o);
                if (lane >= o) incl += y;
            }
            uint32_t pos = off + incl - c;
            while (bits) {
                const uint32_t b = __ffs(bits) - 1;
                bits &= bits - 1;
                out[pos++] = w * 32u + b;
            }
            off += __shfl_sync(FULL, incl, 31);
        }
        const uint32_t L = sh_L;
        __syncthreads();
        return L;
    };

    // Writes the range table of this thread's (up to) two ranges [lo_j, hi_j)
    // of vertices u_j; returns the chunk's edge total.  Contains barriers.
    auto table = [&](const uint32_t (&u)[2], const uint32_t (&lo)[2], const uint32_t (&hi)[2]) -> uint32_t {
        const uint32_t c0 = hi[0] > lo[0] ? hi[0] - lo[0] : 0u, c1 = hi[1] > lo[1] ? hi[1] - lo[1] : 0u;
        const uint32_t nr = (c0 > 0) + (c1 > 0);
        u64 tot;
        const u64 ex = block_exclusive_scan64<PC_NT>(((u64)nr << 32) | (c0 + c1), &tot, sm_scan64);
        uint32_t g = (uint32_t)(ex >> 32), e = (uint32_t)ex;
        if (c0 > 0) { cs_first[g] = lo[0]; cs_off[g] = e; cs_u[g] = u[0]; ++g; e += c0; }
        if (c1 > 0) { cs_first[g] = lo[1]; cs_off[g] = e; cs_u[g] = u[1]; }
        const uint32_t Gc = (uint32_t)(tot >> 32), E = (uint32_t)tot;
        if (tid == 0) { cs_off[Gc] = E; sh_Gc = Gc; }
        __syncthreads();
        return E;
    };

    // As table, and with staging on, the ranges' out_v / out_slot entries are
    // copied into the shared tiles by bulk copies when the chunk's tiles fit:
    // a range [lo, hi) is copied as [lo & ~3, (hi + 3) & ~3) (16-byte aligned
    // start, length a multiple of 16 bytes; the store's arrays start 256-byte
    // aligned in one allocation, so the rounded copy stays inside it), and
    // cs_first then indexes the tiles.  *staged tells which.  Barriers inside.
    auto table_staged = [&](const uint32_t (&u)[2], const uint32_t (&lo)[2], const uint32_t (&hi)[2],
                            const uint32_t* g_out_v, const uint32_t* g_out_slot, bool* staged) -> uint32_t {
        const uint32_t c0 = hi[0] > lo[0] ? hi[0] - lo[0] : 0u, c1 = hi[1] > lo[1] ? hi[1] - lo[1] : 0u;
        const uint32_t nr = (c0 > 0) + (c1 > 0);
        const uint32_t a0 = lo[0] & ~3u, a1 = lo[1] & ~3u;
        const uint32_t s0 = c0 > 0 ? ((hi[0] + 3u) & ~3u) - a0 : 0u, s1 = c1 > 0 ? ((hi[1] + 3u) & ~3u) - a1 : 0u;
        u64 tot;
        const u64 ex = block_exclusive_scan64<PC_NT>(((u64)nr << 32) | (c0 + c1), &tot, sm_scan64);
        uint32_t stot;
        const uint32_t so = block_exclusive_scan<PC_NT>(s0 + s1, &stot, sm_scan32);   // tile offsets (entries)
        const bool st = stot > 0 && stot <= ws.stage_cap;                               // block-uniform
        if (st) {
            fence_proxy_async_smem();   // the previous chunk's tile reads (before the scans' barriers) come first
            if (tid == 0) mbar_arrive_expect_tx(&sh_mbar, stot * 8u);
            if (s0) {
                bulk_g2s(stg_v + so, g_out_v + a0, s0 * 4u, &sh_mbar);
                bulk_g2s(stg_s + so, g_out_slot + a0, s0 * 4u, &sh_mbar);
            }
            if (s1) {
                bulk_g2s(stg_v + so + s0, g_out_v + a1, s1 * 4u, &sh_mbar);
                bulk_g2s(stg_s + so + s0, g_out_slot + a1, s1 * 4u, &sh_mbar);
            }
        }
        uint32_t gi = (uint32_t)(ex >> 32), e = (uint32_t)ex;
        if (c0 > 0) { cs_first[gi] = st ? so + (lo[0] - a0) : lo[0]; cs_off[gi] = e; cs_u[gi] = u[0]; ++gi; e += c0; }
        if (c1 > 0) { cs_first[gi] = st ? so + s0 + (lo[1] - a1) : lo[1]; cs_off[gi] = e; cs_u[gi] = u[1]; }
        const uint32_t Gc = (uint32_t)(tot >> 32), E = (uint32_t)tot;
        if (tid == 0) { cs_off[Gc] = E; sh_Gc = Gc; }
        __syncthreads();
        *staged = st;
        return E;
    };

    // Every edge of the range table once: warp w walks a contiguous slice in
    // windows of 32; h is the range holding the window's first edge.  Ends
    // with a barrier.
    // edge(u, v, slot) for every out-edge (u, v) of the table, head's arrival slot
    // loaded; WALK_K windows of loads in flight per warp.
    auto expand = [&](uint32_t E, const uint32_t* out_v, auto out_slot, auto edge) {
        const uint32_t per = ((E + PC_NW * 32u - 1u) / (PC_NW * 32u)) * 32u;
        const uint32_t w_lo = min((uint32_t)wid * per, E), w_hi = min(w_lo + per, E);
        lbs_walk_batched<WALK_K>(cs_off, sh_Gc, cs_first, w_lo, w_hi, out_v, out_slot,
                                 [&](uint32_t r, uint32_t, uint32_t v, uint32_t sl) { edge(cs_u[r], v, sl); });
        __syncthreads();
    };

    for (;;) {
        if (tid == 0) {
            const uint64_t u = atomicAdd(work, 1ull);
            int t = -1;
            if (ntasks > 0 && u < unit_start[ntasks]) {
                t = task_of_unit(unit_start, ntasks, u);
                sh_q = u - unit_start[t];
            }
            sh_t = t;
            sh_ovf = 0; sh_err = 0; sh_len = 0; sh_sigma = 0;
        }
        __syncthreads();
        if (sh_t < 0) break;
        if (wid == 0) {
            const u64* src = reinterpret_cast<const u64*>(tasks + sh_t);
            u64* dst = reinterpret_cast<u64*>(&sh_task);
            for (uint32_t w = lane; w < sizeof(Task) / 8; w += 32) dst[w] = src[w];
        }
        __syncthreads();
        const DevGraph& g = sh_task.g;
        const Job& job = sh_task.job;
        if (job.ctr != flush_ctr) {
            if (flush_ctr) {
                if (my_escan) atomicAdd(flush_ctr + C_ESCAN, my_escan);
                if (my_eadd) atomicAdd(flush_ctr + C_EADD, my_eadd);
                if (my_x) atomicAdd(flush_ctr + C_XEDGE, my_x);
                if (my_rounds) atomicAdd(flush_ctr + C_FSEG, my_rounds);
            }
            my_escan = my_eadd = my_x = my_rounds = 0;
            flush_ctr = job.ctr;
        }
        const uint32_t n = g.n;
        const uint32_t nwords = (n + 31) >> 5;
        const bool stats = job.stats != 0;
        const uint64_t q = sh_q;
        const uint64_t i = job.idx_list ? job.idx_list[q] : job.i0 + q;
        uint32_t s, z;
        bool ok;
        const bool full = stats || job.rtb;   // a source only, untruncated search
        if (full) {
            uint64_t x;
            ok = draw_below64(n, job.seed, i, stats ? DOM_STATS : job.dom_pair, &x);
            s = (uint32_t)x; z = NONE;
        } else {
            ok = draw_pair(n, job.seed, i, job.dom_pair, &s, &z);
        }
        if (!ok) { if (tid == 0) set_status(job.status, ST_RNG); s = 0; z = full ? NONE : 1; }
        bool live = ok && g.out_ptr[s + 1] > g.out_ptr[s];
        if (!full && live && g.slot_ptr[z + 1] == g.slot_ptr[z]) live = false;
        const uint32_t* const out_ptr = g.out_ptr;
        const uint32_t* const out_t = g.out_t;
        const uint32_t* const out_v = g.out_v;
        const uint32_t* const out_slot = g.out_slot;
        const uint32_t* const slot_t = g.slot_t;
        // v's arrival slot (NONE: unreached, SRC: the source), and whether v is reached
        auto slot_of = [&](uint32_t v) -> uint32_t {
            if constexpr (W16) {
                const uint32_t x = fso[v];
                return x >= O16_SRC ? (x == O16_NONE ? NONE : SRC) : __ldg(g.slot_ptr + v) + x;
            } else {
                return ldv<FA_SMEM>(fsl + v);
            }
        };
        auto reached_v = [&](uint32_t v) -> bool {
            if constexpr (W16) return fso[v] != O16_NONE;
            else return ldv<FA_SMEM>(fsl + v) != NONE;
        };

        if constexpr (W16) {
            for (uint32_t w = tid; w < (n + 1) / 2; w += PC_NT) pc_dyn[w] = 0xFFFFFFFFu;
        } else {
            for (uint32_t v = tid; v < n; v += PC_NT) fsl[v] = NONE;
        }
        for (uint32_t w = tid; w < nwords; w += PC_NT) XB[w] = 0u;
        __syncthreads();
        if (tid == 0 && live) {
            if constexpr (W16) fso[s] = (unsigned short)O16_SRC;
            else fsl[s] = SRC;
            NB[s >> 5] |= 1u << (s & 31);
        }
        __syncthreads();

        // ---- earliest arrivals ----
        uint32_t bound = live ? (full ? NONE - 1u : g.tmax_in[z]) : 0u;
        while (live) {
            const uint32_t L = compact(nwords, Fl);
            if (L == 0) break;
            if (tid == 0) ++my_rounds;
            for (uint32_t c0 = 0; c0 < L; c0 += CHUNK) {
                // ranges of this thread's two vertices: lo = first t > fa(u) (search 2j),
                // hi = first t > bound below the previous expansion's lo (search 2j+1)
                uint32_t u[2], lo[4], hi[4], key[4];
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    const uint32_t x = c0 + (uint32_t)tid + (uint32_t)j * PC_NT;
                    lo[2 * j] = hi[2 * j] = lo[2 * j + 1] = hi[2 * j + 1] = 0u;
                    key[2 * j] = key[2 * j + 1] = 0u;
                    u[j] = NONE;
                    if (x < L) {
                        const uint32_t uu = Fl[x];
                        u[j] = uu;
                        const uint32_t r0 = out_ptr[uu], r1 = out_ptr[uu + 1];
                        const bool again = (ldv<FA_SMEM>(XB + (uu >> 5)) >> (uu & 31)) & 1u;
                        const uint32_t cap = again ? lo_prev[uu] : r1;
                        const uint32_t fu = slot_of(uu);
                        // first t > fa(u): the store's per-slot table, no search
                        const uint32_t f0 = (fu != SRC) ? __ldg(g.slot_nout + fu) : r0;
                        lo[2 * j] = hi[2 * j] = f0;
                        lo[2 * j + 1] = min(f0, cap); hi[2 * j + 1] = cap; key[2 * j + 1] = bound;
                    }
                }
                upper_bounds<4>(out_t, lo, hi, key);
                uint32_t rl[2], rh[2];
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    rl[j] = lo[2 * j]; rh[j] = lo[2 * j + 1];
                    if (u[j] != NONE) {
                        lo_prev[u[j]] = rl[j];
                        atomicOr(XB + (u[j] >> 5), 1u << (u[j] & 31));
                    }
                }
                // sl: the head's arrival slot (mode 2: its offset within v's slots)
                auto relax = [&](uint32_t, uint32_t v, uint32_t sl) {
                    if constexpr (W16) {
                        if (v == s) return;
                        uint32_t old = fso[v];
                        while (sl < old) {
                            const uint32_t prev = atomicCAS(fso + v, (unsigned short)old, (unsigned short)sl);
                            if (prev == old) { atomicOr(NB + (v >> 5), 1u << (v & 31)); return; }
                            old = prev;
                        }
                    } else {
                        if (v == s || sl >= ldv<FA_SMEM>(fsl + v)) return;
                        if (sl < atomicMin(fsl + v, sl)) atomicOr(NB + (v >> 5), 1u << (v & 31));
                    }
                };
                if (stage) {
                    bool staged = false;
                    const uint32_t E = table_staged(u, rl, rh, out_v, out_slot, &staged);
                    if (tid == 0) my_x += E;
                    if (!staged) {
                        expand(E, out_v, out_slot, relax);
                    } else {
                        // every thread waits for the chunk's tiles; a wait that runs out
                        // reports a timeout, waits once more for the copies in flight and
                        // ends the CTA (block-uniform)
                        const bool ok = mbar_wait_bounded(&sh_mbar, stage_par);
                        if (__syncthreads_or(!ok)) {
                            if (tid == 0) set_status(job.status, ST_TIMEOUT);
                            mbar_wait_bounded(&sh_mbar, stage_par);
                            __syncthreads();
                            return;
                        }
                        stage_par ^= 1u;
                        const uint32_t per = ((E + PC_NW * 32u - 1u) / (PC_NW * 32u)) * 32u;
                        const uint32_t w_lo = min((uint32_t)wid * per, E), w_hi = min(w_lo + per, E);
                        lbs_walk_batched<WALK_K, false>(cs_off, sh_Gc, cs_first, w_lo, w_hi, stg_v, stg_s,
                                                        [&](uint32_t r, uint32_t, uint32_t v, uint32_t sl) {
                                                            relax(cs_u[r], v, sl);
                                                        });
                        __syncthreads();
                    }
                } else {
                    const uint32_t E = table(u, rl, rh);
                    if (tid == 0) my_x += E;
                    if constexpr (W16) expand(E, out_v, g.out_loff, relax);
                    else expand(E, out_v, out_slot, relax);
                }
            }
            if (!full) {
                const uint32_t fz = slot_of(z);
                if (fz != NONE) bound = min(bound, __ldg(slot_t + fz));
            }
        }
        const bool reached = live && (full || reached_v(z));

        // fa' of every vertex, for the DAG tests of in-edges
        if (live) {
            for (uint32_t v0 = tid; v0 < n; v0 += PC_NT * CK) {   // CK vertices' loads in flight
                uint32_t f[CK], tt[CK];
#pragma unroll
                for (int j = 0; j < CK; ++j) {
                    const uint32_t v = v0 + PC_NT * j;
                    f[j] = v < n ? slot_of(v) : NONE;
                }
#pragma unroll
                for (int j = 0; j < CK; ++j) tt[j] = (f[j] != NONE && f[j] != SRC) ? __ldg(slot_t + f[j]) : 0u;
#pragma unroll
                for (int j = 0; j < CK; ++j) {
                    const uint32_t v = v0 + PC_NT * j;
                    if (v < n) {
                        fat[v] = f[j] == SRC ? 0u : (f[j] == NONE ? NONE : tt[j] + 1u);
                        dcnt[v] = 0u;
                    }
                }
            }
            __syncthreads();
        }

        // edges of the prefix-foremost scan window (same count as the lane kernel):
        // stream edges with tmin_out(s) <= t <= fa(z) (z's latest in-edge time when
        // unreached), not into s
        // (warp 0, warp-wide searches)
        if (wid == 0 && live) {
            const uint32_t ts = g.tmin_out[s];
            const uint32_t te = full ? NONE - 1u : (reached ? bound : g.tmax_in[z]);
            if (ts <= te) {
                const uint32_t a = warp_lower_bound(g.st_t, 0, g.m, ts), b = warp_lower_bound(g.st_t, a, g.m, te + 1u);
                const uint32_t s0 = g.slot_ptr[s], s1 = g.slot_ptr[s + 1];
                const uint32_t sa = warp_lower_bound(g.slot_t, s0, s1, ts);
                const uint32_t sb = warp_lower_bound(g.slot_t, sa, s1, te + 1u);
                if (lane == 0) my_escan += (u64)(b - a) - (u64)(g.slot_in[sb] - g.slot_in[sa]);
            }
        }

        // ---- path counts over the prefix-foremost DAG (Kahn levels) ----
        // pend(v) for every v with fa(v) <= bound; their sum is the scan's number
        // of path-count updates, counted also when z is not reached
        if (live) {
            for (uint32_t v0 = tid; v0 < n; v0 += PC_NT * CK) {   // CK vertices' loads in flight
                uint32_t fvs[CK];
#pragma unroll
                for (int j = 0; j < CK; ++j) {
                    const uint32_t v = v0 + PC_NT * j;
                    fvs[j] = v < n ? __ldcg(fat + v) : NONE;
                }
#pragma unroll
                for (int j = 0; j < CK; ++j) {
                    const uint32_t v = v0 + PC_NT * j;
                    const uint32_t fv = fvs[j];
                    if (fv == NONE || v == s || fv - 1u > bound) continue;
                    const uint32_t a = slot_of(v);
                    const uint32_t e1 = __ldg(g.slot_in + a + 1);
                    uint32_t c = 0;
                    for (uint32_t e = __ldg(g.slot_in + a); e < e1; ++e) {
                        const uint32_t w = __ldg(g.in_u + e);
                        if (__ldcg(fat + w) < fv) {
                            ++c;
                            if (reached) atomicAdd(dcnt + w, 1u);
                        }
                    }
                    my_eadd += c;
                    if (reached) {
                        pend[v] = c;
                        sig[v] = 0ull;
                        hop[v] = NONE;
                    }
                }
            }
        }
        // The prefix-foremost DAG as out-lists (the in-edge scan above found every
        // DAG edge): dcnt holds each vertex's out-degree, then an exclusive scan
        // (a contiguous block of vertices per thread), then the fill advances it
        // to each list's end, so u's successors are dag[(u ? dcnt[u-1] : 0) .. dcnt[u]).
        if (reached) {
            __syncthreads();
            const uint32_t per = (n + PC_NT - 1) / PC_NT;
            const uint32_t v_lo = min((uint32_t)tid * per, n), v_hi = min(v_lo + per, n);
            uint32_t sum = 0;
            for (uint32_t v = v_lo; v < v_hi; ++v) sum += __ldcg(dcnt + v);
            uint32_t tot;
            uint32_t run = block_exclusive_scan<PC_NT>(sum, &tot, sm_scan32);
            for (uint32_t v = v_lo; v < v_hi; ++v) { const uint32_t c = __ldcg(dcnt + v); dcnt[v] = run; run += c; }
            if (tot > ws.dag_cap && tid == 0) { sh_err = 1; set_status(job.status, ST_CHECK); }
            __syncthreads();
            if (tot <= ws.dag_cap) {
                for (uint32_t v = tid; v < n; v += PC_NT) {
                    const uint32_t fv = __ldcg(fat + v);
                    if (fv == NONE || v == s || fv - 1u > bound) continue;
                    const uint32_t a = slot_of(v);
                    const uint32_t e1 = __ldg(g.slot_in + a + 1);
                    for (uint32_t e = __ldg(g.slot_in + a); e < e1; ++e) {
                        const uint32_t w = __ldg(g.in_u + e);
                        if (__ldcg(fat + w) < fv) dag[atomicAdd(dcnt + w, 1u)] = v;
                    }
                }
            }
            __syncthreads();
        }
        // Kahn rounds are appended: round r's vertices are Fl[kofs[r] .. kofs[r+1])
        uint32_t kb = 0, nr = 0;
        if (reached && !sh_err) {
            if (tid == 0) { sig[s] = 1ull; hop[s] = 0u; NB[s >> 5] |= 1u << (s & 31); }
            __syncthreads();
            for (;;) {
                const uint32_t L = compact(nwords, Fl + kb);
                if (L == 0) break;
                if (tid == 0) { ++my_rounds; kofs[nr] = kb; }
                for (uint32_t c0 = 0; c0 < L; c0 += CHUNK) {
                    // u's DAG successors
                    uint32_t u[2], rl[2], rh[2];
#pragma unroll
                    for (int j = 0; j < 2; ++j) {
                        const uint32_t x = c0 + (uint32_t)tid + (uint32_t)j * PC_NT;
                        rl[j] = rh[j] = 0u;
                        u[j] = NONE;
                        if (x < L) {
                            const uint32_t uu = Fl[kb + x];
                            u[j] = uu;
                            rl[j] = uu ? __ldcg(dcnt + uu - 1) : 0u;
                            rh[j] = __ldcg(dcnt + uu);
                        }
                    }
                    const uint32_t E = table(u, rl, rh);
                    if (tid == 0) my_x += E;
                    expand(E, dag, dag, [&](uint32_t uu, uint32_t v, uint32_t) {
                        if (stats) atomicMin(hop + v, __ldcg(hop + uu) + 1u);
                        else if (!SigOps<false>::atomic_add(sig + v, __ldcg(sig + uu))) sh_ovf = 1;
                        if (atomicSub(pend + v, 1u) == 1u) atomicOr(NB + (v >> 5), 1u << (v & 31));
                    });
                }
                kb += L;
                ++nr;
            }
            if (tid == 0) kofs[nr] = kb;
        }

        if (stats) {
            uint32_t dloc = 0;
            if (reached) {
                for (uint32_t v0 = 0; v0 < n; v0 += PC_NT) {
                    const uint32_t v = v0 + tid;
                    const bool r = v < n && v != s && reached_v(v);
                    const uint32_t h = r ? __ldcg(hop + v) : NONE;
                    const unsigned grp = __match_any_sync(FULL, h);
                    if (r && lane == __ffs(grp) - 1) atomicAdd(job.cnt + h, (u64)__popc(grp));
                    if (r && job.clos) atomicAdd(job.clos + v, recip32(h));
                    if (r && h > dloc) dloc = h;
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) dloc = max(dloc, __shfl_xor_sync(FULL, dloc, o));
            if (lane == 0 && dloc) atomicMax(job.dmax, (u64)dloc);
            __syncthreads();
            continue;
        }
        __syncthreads();

        // ---- backward draw (warp 0); ob: sigma_sz and the Rademacher bits only ----
        if (reached && !sh_ovf && !sh_err && wid == 0 && job.ob) {
            if (lane == 0) {
                sh_sigma = __ldcg(sig + z);
                uint32_t w4[4];
                philox_block(job.seed, i, DOM_RADE, 0, w4);
                sh_rade[0] = w4[0]; sh_rade[1] = w4[1]; sh_rade[2] = w4[2]; sh_rade[3] = w4[3];
            }
        } else if (reached && !sh_ovf && !sh_err && wid == 0 && !job.rtb) {
            const u64 tot = __ldcg(sig + z);
            u128 x = 0;
            uint32_t rng_ok = 1;
            if (lane == 0) rng_ok = draw_below128((u128)tot, job.seed, i, job.dom_path, &x) ? 1u : 0u;
            rng_ok = __shfl_sync(FULL, rng_ok, 0);
            u64 xs = shfl_idx_w((u64)x, 0);
            bool err = !rng_ok;
            if (err && lane == 0) set_status(job.status, ST_RNG);
            uint32_t v = z, cnt = 1;
            if (lane == 0) path[0] = z;
            while (!err && v != s) {
                const uint32_t fv = __ldcg(fat + v);
                const uint32_t a = slot_of(v);
                const uint32_t e_lo = g.slot_in[a], e_hi = g.slot_in[a + 1];
                uint32_t nxt = NONE, ech = NONE;
                for (uint32_t e0 = e_lo; e0 < e_hi; e0 += 32) {
                    const uint32_t e = e0 + lane;
                    u64 wt = 0;
                    uint32_t w = 0;
                    if (e < e_hi) {
                        w = g.in_u[e];
                        if (__ldcg(fat + w) < fv) wt = __ldcg(sig + w);
                    }
                    const u64 incl = warp_inclusive_sum(wt);
                    const unsigned msk = __ballot_sync(FULL, xs < incl);
                    if (msk) {
                        const int l = __ffs(msk) - 1;
                        nxt = __shfl_sync(FULL, w, l);
                        ech = e0 + l;
                        xs -= shfl_idx_w(incl - wt, l);
                        break;
                    }
                    xs -= shfl_idx_w(incl, 31);
                }
                if (nxt == NONE || cnt > n) { err = true; break; }
                v = nxt;
                if (lane == 0) { path[cnt] = v; pathe[cnt - 1] = ech; }
                ++cnt;
            }
            if (lane == 0) {
                if (err) {
                    sh_err = 1;
                    set_status(job.status, ST_CHECK);
                } else {
                    for (uint32_t p = 0; p < cnt / 2; ++p) {
                        const uint32_t tmp = path[p]; path[p] = path[cnt - 1 - p]; path[cnt - 1 - p] = tmp;
                    }
                    for (uint32_t p = 0; p < (cnt - 1) / 2; ++p) {
                        const uint32_t tmp = pathe[p]; pathe[p] = pathe[cnt - 2 - p]; pathe[cnt - 2 - p] = tmp;
                    }
                    sh_len = cnt;
                    sh_sigma = tot;
                    uint32_t w4[4];
                    philox_block(job.seed, i, DOM_RADE, 0, w4);
                    sh_rade[0] = w4[0]; sh_rade[1] = w4[1]; sh_rade[2] = w4[2]; sh_rade[3] = w4[3];
                }
            }
        }
        __syncthreads();

        // ---- ob (Sec. 4.1): sigma_sz(v) = sigma(v) * continuations(v), the
        // continuations counted over the prefix-foremost DAG in reverse Kahn
        // order from z (block-uniform condition) ----
        if (job.ob && job.hits && reached && !sh_ovf && !sh_err) {
            for (uint32_t p = tid; p < kb; p += PC_NT) dl[Fl[p]] = 0ull;
            if (tid == 0) sh_nt = 0;
            __syncthreads();
            if (tid == 0) dl[z] = 1ull;
            __syncthreads();
            for (int r = (int)nr - 1; r >= 0; --r) {
                const uint32_t p1 = kofs[r + 1];
                for (uint32_t p = kofs[r] + tid; p < p1; p += PC_NT) {
                    const uint32_t v = Fl[p];
                    if (v == s) continue;
                    const u64 x = __ldcg(dl + v);
                    if (!x) continue;
                    const uint32_t fv = __ldcg(fat + v), a = slot_of(v);
                    const uint32_t e1 = __ldg(g.slot_in + a + 1);
                    for (uint32_t e = __ldg(g.slot_in + a); e < e1; ++e) {
                        const uint32_t w = __ldg(g.in_u + e);
                        if (__ldcg(fat + w) < fv) atomicAdd(dl + w, x);   // <= sigma_sz: no wrap
                    }
                }
                __syncthreads();
            }
            // ob values of the internal vertices, into sig (no longer needed); the
            // nonzero ones listed in path
            u64 my_sum = 0;
            for (uint32_t p = tid; p < kb; p += PC_NT) {
                const uint32_t v = Fl[p];
                if (v == s || v == z) continue;
                const u64 x = __ldcg(dl + v);
                if (!x) continue;
                const uint64_t q = ob_q((u128)__ldcg(sig + v) * x, (u128)sh_sigma);
                sig[v] = q;
                path[atomicAdd(&sh_nt, 1u)] = v;
                my_sum += q;
            }
            __syncthreads();
            const uint32_t T = sh_nt, rows = 2 + (job.S64 ? job.c : 0);
            for (uint32_t it = tid; it < T * rows; it += PC_NT) {
                const uint32_t v = path[it % T];
                ob_term(job, v, sig[v], it / T, sh_rade);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) my_sum += __shfl_xor_sync(FULL, my_sum, o);
            if (lane == 0 && my_sum) atomicAdd(job.ctr + C_SUMINT, my_sum);
        }

        // ---- RTB (App. C): dependency accumulation over the whole prefix-foremost
        // DAG in reverse Kahn order: every reached x != s is its own endpoint
        // (share 1), delta(w) += round(sigma(w) (1 + delta(x)) / sigma(x)) over
        // DAG edges w -> x, w != s; f_v = round(delta(v) / (n-1)), 2^-32 units ----
        if (job.rtb && job.hits && reached && !sh_ovf) {
            for (uint32_t p = tid; p < kb; p += PC_NT) dl[Fl[p]] = 0ull;
            if (tid == 0) {
                sh_nt = 0;
                uint32_t w4[4];
                philox_block(job.seed, i, DOM_RADE, 0, w4);
                sh_rade[0] = w4[0]; sh_rade[1] = w4[1]; sh_rade[2] = w4[2]; sh_rade[3] = w4[3];
            }
            __syncthreads();
            for (int r = (int)nr - 1; r >= 0; --r) {
                const uint32_t p1 = kofs[r + 1];
                for (uint32_t p = kofs[r] + tid; p < p1; p += PC_NT) {
                    const uint32_t x = Fl[p];
                    if (x == s) continue;
                    const u64 X = (1ull << 32) + __ldcg(dl + x), sx = __ldcg(sig + x);
                    const uint32_t fv = __ldcg(fat + x), a = slot_of(x);
                    const uint32_t e1 = __ldg(g.slot_in + a + 1);
                    for (uint32_t e = __ldg(g.slot_in + a); e < e1; ++e) {
                        const uint32_t w = __ldg(g.in_u + e);
                        if (w == s || __ldcg(fat + w) >= fv) continue;
                        const u64 term = muldiv_round((u128)__ldcg(sig + w), X, (u128)sx);
                        if (term) atomicAdd(dl + w, term);
                    }
                }
                __syncthreads();
            }
            u64 my_sum = 0;
            for (uint32_t p = tid; p < kb; p += PC_NT) {
                const uint32_t v = Fl[p];
                if (v == s) continue;
                const u64 d = __ldcg(dl + v);
                if (!d) continue;
                const uint64_t q = muldiv_round(1, d, n - 1);
                if (!q) continue;
                sig[v] = q;
                path[atomicAdd(&sh_nt, 1u)] = v;
                my_sum += q;
            }
            __syncthreads();
            const uint32_t T = sh_nt, rows = 2 + (job.S64 ? job.c : 0);
            for (uint32_t it = tid; it < T * rows; it += PC_NT) {
                const uint32_t v = path[it % T];
                ob_term(job, v, sig[v], it / T, sh_rade);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) my_sum += __shfl_xor_sync(FULL, my_sum, o);
            if (lane == 0 && my_sum) atomicAdd(job.ctr + C_SUMINT, my_sum);
        }

        if (sh_ovf) {
            if (tid == 0) push_overflow(job, i);
        } else if (!sh_err) {
            const uint32_t len = sh_len;
            const uint32_t nint = family_count(job, len);
            if (job.hits && nint > 0) {
                const uint32_t rows = 1 + (job.S ? job.c : 0);
                for (uint32_t it = tid; it < nint * rows; it += PC_NT) {
                    const uint32_t p = it % nint, jrow = it / nint;
                    const uint32_t x = family_item(job, g, path, pathe, p);
                    if (jrow == 0) {
                        atomicAdd(job.hits + x, 1ull);
                    } else {
                        const uint32_t jj = jrow - 1;
                        const int lam = ((sh_rade[jj >> 5] >> (jj & 31)) & 1u) ? 1 : -1;
                        atomicAdd(job.S + (size_t)jj * job.fam + x, lam);
                    }
                }
                if (tid == 0) atomicAdd(job.ctr + C_SUMINT, (u64)nint);
            }
            if (job.rec_len) {
                const uint64_t r = i - job.i0;
                if (tid == 0) {
                    job.rec_s[r] = s; job.rec_z[r] = z;
                    job.rec_sig[2 * r] = sh_sigma; job.rec_sig[2 * r + 1] = 0ull;
                    job.rec_len[r] = len;
                }
                for (uint32_t p = tid; p < len && p < job.rec_cap; p += PC_NT)
                    job.rec_nodes[r * job.rec_cap + p] = path[p];
                if (job.rec_edges)
                    for (uint32_t p = tid; p + 1 < len && p < job.rec_cap; p += PC_NT)
                        job.rec_edges[r * job.rec_cap + p] = pathe[p];
            }
        }
        __syncthreads();
    }
    if (flush_ctr) {
        if (my_escan) atomicAdd(flush_ctr + C_ESCAN, my_escan);
        if (my_eadd) atomicAdd(flush_ctr + C_EADD, my_eadd);
        if (my_x) atomicAdd(flush_ctr + C_XEDGE, my_x);
        if (my_rounds) atomicAdd(flush_ctr + C_FSEG, my_rounds);
    }
}

// Region of one CTA (global memory).  The arrival slots and the two bitmaps
// (next frontier, expanded before) are in shared memory instead when
// fa_in_smem.
size_t pfm_cta_region_bytes(uint32_t n, uint32_t dag_cap, bool fa_in_smem, PfmCtaWs* ws) {
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    size_t o = 0;
    ws->n_cap = n;
    ws->bits_words = (n + 31) / 32;
    ws->fa_in_smem = fa_in_smem ? 1 : 0;
    ws->o_fa = o;    if (!fa_in_smem) o = al(o + (size_t)n * 4);
    ws->o_bits = o;  if (!fa_in_smem) o = al(o + (size_t)ws->bits_words * 8);
    ws->o_exp = o;   o = al(o + (size_t)n * 4);
    ws->o_fat = o;   o = al(o + (size_t)n * 4);
    ws->o_sig = o;   o = al(o + (size_t)n * 8);
    ws->o_hop = o;   o = al(o + (size_t)n * 4);
    ws->o_pend = o;  o = al(o + (size_t)n * 4);
    ws->o_list = o;  o = al(o + (size_t)(n + 1) * 4);
    ws->o_path = o;  o = al(o + (size_t)(n + 2) * 4);
    ws->o_pathe = o; o = al(o + (size_t)(n + 2) * 4);
    ws->o_dl = o;    o = al(o + (size_t)n * 8);
    ws->o_kofs = o;  o = al(o + (size_t)(n + 2) * 4);
    ws->o_dcnt = o;  o = al(o + (size_t)(n + 1) * 4);
    ws->dag_cap = dag_cap;
    ws->o_dag = o;   o = al(o + ((size_t)dag_cap + 1) * 4);
    return o;
}

// Dynamic shared memory of the variants with the arrival state in shared
// memory: 32-bit slots (mode 1) or 16-bit offsets (mode 2), then the bitmaps.
size_t pfm_cta_smem_bytes(uint32_t n, bool w16) {
    return ((size_t)(w16 ? (n + 1) / 2 : n) + 2 * ((n + 31) / 32)) * 4;
}

// Dynamic shared memory of the global-state variant's staged edge tiles
// (out_v and out_slot, cap entries each; cap a multiple of 4).
size_t pfm_cta_stage_bytes(uint32_t cap) { return (size_t)cap * 8; }

// Static shared memory of the kernel (range table, task copy, scratch).
size_t pfm_cta_static_smem(int nt) {
    cudaFuncAttributes a{};
    const cudaError_t e = nt == 256 ? cudaFuncGetAttributes(&a, k_pfm_cta<256, 1>)
                                    : cudaFuncGetAttributes(&a, k_pfm_cta<512, 1>);
    return e == cudaSuccess ? a.sharedSizeBytes : 16384;
}

// Raises (never lowers) the dynamic shared-memory limit of the shared-memory
// variants on the current device (the attribute, and its record, are per device).
cudaError_t pfm_cta_configure(size_t smem) {
    static std::mutex mu;
    static size_t configured[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(mu);
    if (smem <= configured[dev]) return cudaSuccess;
    const void* ks[6] = {(const void*)k_pfm_cta<512, 1>, (const void*)k_pfm_cta<256, 1>,
                         (const void*)k_pfm_cta<512, 2>, (const void*)k_pfm_cta<256, 2>,
                         (const void*)k_pfm_cta<512, 0>, (const void*)k_pfm_cta<256, 0>};
    for (const void* k : ks) {
        e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    configured[dev] = smem;
    return cudaSuccess;
}

// fa: the state mode (0 global, 1 shared 32-bit, 2 shared 16-bit).
cudaError_t pfm_cta_blocks_per_sm(int nt, int fa, size_t smem, int* out) {
    if (nt == 256) {
        if (fa == 1) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, k_pfm_cta<256, 1>, 256, smem);
        if (fa == 2) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, k_pfm_cta<256, 2>, 256, smem);
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, k_pfm_cta<256, 0>, 256, smem);
    }
    if (fa == 1) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, k_pfm_cta<512, 1>, 512, smem);
    if (fa == 2) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, k_pfm_cta<512, 2>, 512, smem);
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, k_pfm_cta<512, 0>, 512, smem);
}

cudaError_t launch_pfm_cta(const Task* tasks, const uint64_t* unit_start, const uint32_t* ntasks, u64* work,
                           const PfmCtaWs& ws, int grid, cudaStream_t st) {
    const int fa = ws.fa_in_smem;
    const size_t smem = fa ? pfm_cta_smem_bytes(ws.n_cap, fa == 2) : pfm_cta_stage_bytes(ws.stage_cap);
    if (ws.nt == 256) {
        if (fa == 1) k_pfm_cta<256, 1><<<grid, 256, smem, st>>>(tasks, unit_start, ntasks, work, ws);
        else if (fa == 2) k_pfm_cta<256, 2><<<grid, 256, smem, st>>>(tasks, unit_start, ntasks, work, ws);
        else k_pfm_cta<256, 0><<<grid, 256, smem, st>>>(tasks, unit_start, ntasks, work, ws);
    } else {
        if (fa == 1) k_pfm_cta<512, 1><<<grid, 512, smem, st>>>(tasks, unit_start, ntasks, work, ws);
        else if (fa == 2) k_pfm_cta<512, 2><<<grid, 512, smem, st>>>(tasks, unit_start, ntasks, work, ws);
        else k_pfm_cta<512, 0><<<grid, 512, smem, st>>>(tasks, unit_start, ntasks, work, ws);
    }
    return cudaGetLastError();
}

}  // namespace mantra
