// Prefix-foremost (pfm) temporal search (paper Sec. 3 Def. 1(3); running-time
// theorem of Sec. 4.4: one pass over the time-sorted edges), the backward
// path draw over earliest-arrival predecessors (App. C, theorem on the path
// sampler) and the Update step of Algorithm 1.  Also the pfm full searches of
// Algorithm 2 (distance = minimum hops among prefix-foremost paths).
//
// One lane owns one sample; a warp walks the time-sorted stream (t, u, v)
// once for its 32 samples.  Per-sample state is laid out [v][lane] so the
// warp's 32 reads of fa(u) for one edge are one 128-byte row:
//   fa'   earliest arrival + 1 (0 for the source, NONE when unreached)
//   sigma number of pfm paths (64-bit, or 128-bit on the wide re-run)
//   hop   minimum hops (Algorithm 2 only)
// An edge (u, v, t) with v != s and fa(u) < t reaches v at t when v is
// unreached, and adds sigma(u) to sigma(v) when fa(v) = t; within one
// timestamp fa(u) < t ignores values set at that timestamp, so edge order
// inside a group does not matter.  A lane is active from its source's
// earliest out-edge time to z's latest in-edge time and stops after the
// group at which z is reached.  fa rows of 8 edges are loaded together; the
// lane's own updates inside those 8 edges are forwarded in registers.
#include "mantra_dev.cuh"

namespace mantra {

constexpr int PFM_NT = 128;
constexpr int PFM_G = 16;      // edges per prefetch group

template <bool WIDE>
__global__ void __launch_bounds__(PFM_NT) k_pfm(const DevGraph g, const Job job, const PfmWs ws) {
    typedef typename SigOps<WIDE>::T Sig;
    const uint32_t FULL = 0xFFFFFFFFu;
    const int lane = threadIdx.x & 31;
    const uint64_t gw = ((uint64_t)blockIdx.x * PFM_NT + threadIdx.x) >> 5;
    const uint32_t n = g.n;
    char* region = ws.base + gw * ws.stride;
    uint32_t* fa = reinterpret_cast<uint32_t*>(region + ws.o_fa) + lane;     // fa[v * 32]
    Sig* sig = reinterpret_cast<Sig*>(region + ws.o_sig) + lane;             // sig[v * 32]
    uint32_t* hop = reinterpret_cast<uint32_t*>(region + ws.o_hop) + lane;   // hop[v * 32]
    uint32_t* path = reinterpret_cast<uint32_t*>(region + ws.o_path) + (size_t)lane * (n + 2);
    const bool stats = job.stats != 0;
    u64 my_escan = 0, my_eadd = 0;
    __shared__ uint4 stage_all[PFM_NT];      // one 32-edge chunk per warp

    for (;;) {
        uint64_t q0 = 0;
        if (lane == 0) q0 = atomicAdd(job.ctr + C_WORK, 32ull);
        q0 = __shfl_sync(FULL, q0, 0);
        if (q0 >= job.count) break;
        const uint64_t q = q0 + lane;
        const bool have = q < job.count;
        const uint64_t i = have ? (job.idx_list ? job.idx_list[q] : job.i0 + q) : 0;

        uint32_t s = 0, z = 1;
        bool ok = true;
        if (have) {
            if (stats) {
                uint64_t x;
                ok = draw_below64(n, job.seed, i, DOM_STATS, &x);
                s = (uint32_t)x; z = NONE;
            } else {
                ok = draw_pair(n, job.seed, i, job.dom_pair, &s, &z);
            }
            if (!ok) { set_status(job.status, ST_RNG); s = 0; z = 1; }
        }
        bool live = have && ok && g.out_ptr[s + 1] > g.out_ptr[s];
        if (!stats && live && g.slot_ptr[z + 1] == g.slot_ptr[z]) live = false;
        const uint32_t ts = live ? g.tmin_out[s] : NONE;
        const uint32_t te = live ? (stats ? NONE - 1 : g.tmax_in[z]) : 0;

        for (uint32_t v = 0; v < n; ++v) fa[(size_t)v * 32] = NONE;
        if (live) { fa[(size_t)s * 32] = 0u; sig[(size_t)s * 32] = (Sig)1; hop[(size_t)s * 32] = 0u; }
        __syncwarp();

        // stream window of the warp: union of the lanes' windows
        uint32_t wlo = ts, whi = te;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            wlo = min(wlo, __shfl_xor_sync(FULL, wlo, o));
            whi = max(whi, __shfl_xor_sync(FULL, whi, o));
        }
        uint32_t e_lo = 0, e_hi = 0;
        if (__any_sync(FULL, live)) {
            if (lane == 0) {
                e_lo = lower_bound_u32(g.st_t, 0, g.m, wlo);
                e_hi = upper_bound_u32(g.st_t, 0, g.m, whi);
            }
            e_lo = __shfl_sync(FULL, e_lo, 0);
            e_hi = __shfl_sync(FULL, e_hi, 0);
        }
        uint32_t fz = NONE;        // fa'(z) once reached
        uint32_t ovf = 0;
        uint4* stage = stage_all + (threadIdx.x >> 5) * 32;
        for (uint32_t base = e_lo; base < e_hi; base += 32) {
            const uint32_t e = base + lane;
            uint4 me = make_uint4(0u, 0u, NONE, 0u);
            if (e < e_hi) { me.x = g.st_u[e]; me.y = g.st_v[e]; me.z = g.st_t[e]; }
            __syncwarp();
            stage[lane] = me;
            __syncwarp();
            // lanes still scanning at this chunk's first time
            const uint32_t t0 = stage[0].z;
            const bool running = live && t0 <= te && t0 < fz;
            if (!__any_sync(FULL, running)) break;
#pragma unroll 1
            for (int h = 0; h < 32; h += PFM_G) {
                // (1) arrival-time rows of both endpoints for PFM_G edges
                uint32_t FU[PFM_G], FV[PFM_G];
                unsigned onm = 0;
                const uint32_t hi_t = min(te, fz - 1u);      // fz = NONE: te
#pragma unroll
                for (int j = 0; j < PFM_G; ++j) {
                    const uint4 E = stage[h + j];
                    const bool on = live && E.z >= ts && E.z <= hi_t && E.y != s;
                    FU[j] = on ? fa[(size_t)E.x * 32] : NONE;
                    FV[j] = on ? fa[(size_t)E.y * 32] : NONE;
                    onm |= on ? (1u << j) : 0u;
                }
                my_escan += __popc(onm);
                // (2) arrival decisions in stream order; this lane's own updates
                //     inside the group are forwarded from registers
                unsigned cm = 0, fm = 0;
                uint32_t uv[4], uf[4];
                int nu = 0;
#pragma unroll
                for (int j = 0; j < PFM_G; ++j) {
                    if (!((onm >> j) & 1u)) continue;
                    const uint4 E = stage[h + j];
                    uint32_t fu = FU[j], fv = FV[j];
                    if (nu > 4) { fu = fa[(size_t)E.x * 32]; fv = fa[(size_t)E.y * 32]; }
                    else {
                        for (int q = 0; q < nu; ++q) {
                            if (uv[q] == E.x) fu = uf[q];
                            if (uv[q] == E.y) fv = uf[q];
                        }
                    }
                    if (E.z < fz && fu <= E.z) {
                        if (fv == NONE) {
                            fa[(size_t)E.y * 32] = E.z + 1u;
                            if (nu < 4) { uv[nu] = E.y; uf[nu] = E.z + 1u; }
                            ++nu;
                            fm |= 1u << j;
                            cm |= 1u << j;
                            if (E.y == z) fz = E.z + 1u;
                        } else if (fv == E.z + 1u) {
                            cm |= 1u << j;
                        }
                    }
                }
                // (3) path counts of the contributing edges, in stream order, up to
                //     4 prefetched at a time; forwarding of this lane's new counts
                my_eadd += __popc(cm);
                while (cm) {
                    int jj[4];
                    Sig SU[4], SV[4];
                    int k = 0;
                    unsigned rest = cm;
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        jj[q] = -1;
                        if (rest) {
                            const int j = __ffs(rest) - 1;
                            rest &= rest - 1;
                            jj[q] = j;
                            const uint4 E = stage[h + j];
                            SU[q] = sig[(size_t)E.x * 32];
                            SV[q] = ((fm >> j) & 1u) ? (Sig)0 : sig[(size_t)E.y * 32];
                            k = q + 1;
                        }
                    }
                    cm = rest;
                    uint32_t wv[4];
                    Sig wsig[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        if (q >= k) break;
                        const uint4 E = stage[h + jj[q]];
                        Sig su = SU[q], sv = SV[q];
#pragma unroll
                        for (int r = 0; r < q; ++r) {
                            if (wv[r] == E.x) su = wsig[r];
                            if (wv[r] == E.y) sv = wsig[r];
                        }
                        Sig nv;
                        if (!SigOps<WIDE>::add(sv, su, &nv) && !stats) ovf = 1;
                        sig[(size_t)E.y * 32] = nv;
                        wv[q] = E.y;
                        wsig[q] = nv;
                        if (stats) {
                            const uint32_t hu = hop[(size_t)E.x * 32] + 1u;
                            if ((fm >> jj[q]) & 1u) hop[(size_t)E.y * 32] = hu;
                            else if (hu < hop[(size_t)E.y * 32]) hop[(size_t)E.y * 32] = hu;
                        }
                    }
                }
            }
            if (__any_sync(FULL, ovf)) break;
        }
        __syncwarp();
        ovf = __any_sync(FULL, ovf) ? 1u : 0u;

        if (stats) {
            uint32_t dloc = 0;
            for (uint32_t v = 0; v < n; ++v) {
                const bool r = live && v != s && fa[(size_t)v * 32] != NONE;
                const uint32_t h = r ? hop[(size_t)v * 32] : NONE;
                const unsigned grp = __match_any_sync(FULL, h);
                if (r && lane == __ffs(grp) - 1) atomicAdd(job.cnt + h, (u64)__popc(grp));
                if (r && h > dloc) dloc = h;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) dloc = max(dloc, __shfl_xor_sync(FULL, dloc, o));
            if (lane == 0 && dloc) atomicMax(job.dmax, (u64)dloc);
            continue;
        }

        // ---------------- path draw, one lane per sample ----------------
        uint32_t len = 0, err = 0;
        u128 sigma_sz = 0;
        if (have && !ovf && live && fz != NONE) {
            const Sig tot = sig[(size_t)z * 32];
            sigma_sz = SigOps<WIDE>::wide(tot);
            u128 x;
            if (!draw_below128(sigma_sz, job.seed, i, job.dom_path, &x)) { err = 1; set_status(job.status, ST_RNG); }
            Sig xs = (Sig)x;
            uint32_t v = z, cnt = 0;
            path[cnt++] = z;
            while (!err && v != s) {
                const uint32_t fv = fa[(size_t)v * 32];
                const uint32_t a = lower_bound_u32(g.slot_t, g.slot_ptr[v], g.slot_ptr[v + 1], fv - 1u);
                Sig cum = 0;
                uint32_t nxt = NONE;
                for (uint32_t e = g.slot_in[a]; e < g.slot_in[a + 1]; ++e) {
                    const uint32_t w = g.in_u[e];
                    if (!(fa[(size_t)w * 32] < fv)) continue;
                    const Sig wt = sig[(size_t)w * 32];
                    if (xs < cum + wt) { xs -= cum; nxt = w; break; }
                    cum += wt;
                }
                if (nxt == NONE || cnt > n) { err = 1; break; }
                v = nxt;
                path[cnt++] = v;
            }
            if (err) set_status(job.status, ST_CHECK);
            else {
                for (uint32_t p = 0; p < cnt / 2; ++p) {
                    const uint32_t tmp = path[p]; path[p] = path[cnt - 1 - p]; path[cnt - 1 - p] = tmp;
                }
                len = cnt;
            }
        }
        if (have && ovf) {
            if (WIDE) set_status(job.status, ST_OVERFLOW);
            else job.ovf_list[atomicAdd(job.ctr + C_NOVF, 1ull)] = i;
        }
        if (have && !ovf && !err) {
            if (job.hits && len >= 3) {
                uint32_t w4[4];
                philox_block(job.seed, i, DOM_RADE, 0, w4);
                for (uint32_t p = 1; p + 1 < len; ++p) {
                    const uint32_t v = path[p];
                    atomicAdd(job.hits + v, 1ull);
                    if (job.S)
                        for (uint32_t jj = 0; jj < job.c; ++jj) {
                            const int lam = ((w4[jj >> 5] >> (jj & 31)) & 1u) ? 1 : -1;
                            atomicAdd(job.S + (size_t)jj * n + v, lam);
                        }
                }
                atomicAdd(job.ctr + C_SUMINT, (u64)(len - 2));
            }
            if (job.rec_len) {
                const uint64_t r = i - job.i0;
                job.rec_s[r] = s; job.rec_z[r] = z;
                job.rec_sig[2 * r] = (u64)sigma_sz; job.rec_sig[2 * r + 1] = (u64)(sigma_sz >> 64);
                job.rec_len[r] = len;
                for (uint32_t p = 0; p < len && p < job.rec_cap; ++p) job.rec_nodes[r * job.rec_cap + p] = path[p];
            }
        }
        __syncwarp();
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        my_escan += __shfl_xor_sync(FULL, my_escan, o);
        my_eadd += __shfl_xor_sync(FULL, my_eadd, o);
    }
    if (lane == 0) {
        if (my_escan) atomicAdd(job.ctr + C_ESCAN, my_escan);
        if (my_eadd) atomicAdd(job.ctr + C_EADD, my_eadd);
    }
}

// ---------------------------------------------------------------------------
// Fast variant (64-bit path counts).  Same search, reorganised so that a
// warp decides the 32 edges of a chunk in parallel:
//   * every lane loads the fa' rows of both endpoints of all 32 edges;
//   * arrival decisions are taken for all edges at once from those values;
//     they equal the in-order decisions unless this lane reaches a vertex at
//     edge k that a later edge j of the chunk touches (v_k in {u_j, v_j}) or
//     reaches z.  A warp-uniform mask per edge k lists those later edges; a lane
//     with such a conflict redoes the chunk in order;
//   * contributing edges (first arrival at v, or a further edge into v at
//     fa(v)) are appended in stream order to the lane's list, and path counts
//     are summed from that list after the scan, 8 entries per batch.
// A lane whose list would exceed its capacity, or whose count exceeds 64 bits,
// is handed to the in-order kernel above (overflow list).
// ---------------------------------------------------------------------------
constexpr uint32_t LIST_FIRST = 0x80000000u;
constexpr size_t PFM_BUF_BYTES = 64 * 32 * 4;                       // one chunk's rows
constexpr size_t PFM_WARP_SMEM = 2 * PFM_BUF_BYTES + 512 + 128;    // two buffers, edges, barriers
constexpr size_t PFM_FAST_SMEM = (PFM_NT / 32) * PFM_WARP_SMEM;

__global__ void __launch_bounds__(PFM_NT) k_pfm_fast(const DevGraph g, const Job job, const PfmWs ws) {
    typedef u64 Sig;
    const uint32_t FULL = 0xFFFFFFFFu;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const uint64_t gw = ((uint64_t)blockIdx.x * PFM_NT + threadIdx.x) >> 5;
    const uint32_t n = g.n;
    char* region = ws.base + gw * ws.stride;
    uint32_t* fa = reinterpret_cast<uint32_t*>(region + ws.o_fa) + lane;
    Sig* sig = reinterpret_cast<Sig*>(region + ws.o_sig) + lane;
    uint32_t* hop = reinterpret_cast<uint32_t*>(region + ws.o_hop) + lane;
    uint32_t* path = reinterpret_cast<uint32_t*>(region + ws.o_path) + (size_t)lane * (n + 2);
    uint32_t* list = reinterpret_cast<uint32_t*>(region + ws.o_list) + lane;      // list[p * 32]
    const uint32_t* fa_rows = reinterpret_cast<const uint32_t*>(region + ws.o_fa);
    const uint32_t cap = ws.list_cap;
    const bool stats = job.stats != 0;
    u64 my_escan = 0, my_eadd = 0;

    // per warp: two row buffers [64 rows][32 lanes] (rows 0..31: fa'(u_j), 32..63: fa'(v_j)),
    // the chunk's edges and one mbarrier per buffer
    extern __shared__ __align__(128) unsigned char pfm_smem[];
    uint32_t* rowbuf = reinterpret_cast<uint32_t*>(pfm_smem + (size_t)wib * PFM_WARP_SMEM);
    uint4* stage = reinterpret_cast<uint4*>(pfm_smem + (size_t)wib * PFM_WARP_SMEM + 2 * PFM_BUF_BYTES);
    uint64_t* bars = reinterpret_cast<uint64_t*>(pfm_smem + (size_t)wib * PFM_WARP_SMEM + 2 * PFM_BUF_BYTES + 512);
    if (lane == 0) { mbar_init(bars, 32); mbar_init(bars + 1, 32); fence_mbar_init(); }
    __syncwarp();
    uint32_t phase = 0;      // bit b: parity of buffer b's next completion

    for (;;) {
        uint64_t q0 = 0;
        if (lane == 0) q0 = atomicAdd(job.ctr + C_WORK, 32ull);
        q0 = __shfl_sync(FULL, q0, 0);
        if (q0 >= job.count) break;
        const uint64_t q = q0 + lane;
        const bool have = q < job.count;
        const uint64_t i = have ? (job.idx_list ? job.idx_list[q] : job.i0 + q) : 0;

        uint32_t s = 0, z = 1;
        bool ok = true;
        if (have) {
            if (stats) {
                uint64_t x;
                ok = draw_below64(n, job.seed, i, DOM_STATS, &x);
                s = (uint32_t)x; z = NONE;
            } else {
                ok = draw_pair(n, job.seed, i, job.dom_pair, &s, &z);
            }
            if (!ok) { set_status(job.status, ST_RNG); s = 0; z = 1; }
        }
        bool live = have && ok && g.out_ptr[s + 1] > g.out_ptr[s];
        if (!stats && live && g.slot_ptr[z + 1] == g.slot_ptr[z]) live = false;
        const uint32_t ts = live ? g.tmin_out[s] : NONE;
        const uint32_t te = live ? (stats ? NONE - 1 : g.tmax_in[z]) : 0;

        for (uint32_t v = 0; v < n; ++v) fa[(size_t)v * 32] = NONE;
        if (live) fa[(size_t)s * 32] = 0u;
        fence_proxy_async();          // these stores before the first row copies
        __syncwarp();

        uint32_t wlo = ts, whi = te;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            wlo = min(wlo, __shfl_xor_sync(FULL, wlo, o));
            whi = max(whi, __shfl_xor_sync(FULL, whi, o));
        }
        uint32_t e_lo = 0, e_hi = 0;
        if (__any_sync(FULL, live)) {
            if (lane == 0) {
                e_lo = lower_bound_u32(g.st_t, 0, g.m, wlo);
                e_hi = upper_bound_u32(g.st_t, 0, g.m, whi);
            }
            e_lo = __shfl_sync(FULL, e_lo, 0);
            e_hi = __shfl_sync(FULL, e_hi, 0);
        }
        const uint32_t nchunks = (e_hi - e_lo + 31) / 32;
        uint32_t fz = NONE;
        uint32_t nlist = 0;
        bool lovf = false;
        bool timed_out = false;
        uint32_t pv[4], pf[4];     // this lane's first arrivals of the previous chunk (patch list)
        int np = 0;
        // edge of lane l in chunk c: e_lo + 32 c + l (sentinel row 0, time NONE past e_hi)
        auto load_edge = [&](uint32_t e) {
            uint4 r = make_uint4(0u, 0u, NONE, 0u);
            if (e < e_hi) { r.x = g.st_u[e]; r.y = g.st_v[e]; r.z = g.st_t[e]; }
            return r;
        };
        // rows of both endpoints of this lane's edge into buffer b
        auto issue = [&](int b, const uint4& me) {
            uint32_t* dst = rowbuf + (size_t)b * (PFM_BUF_BYTES / 4);
            mbar_arrive_expect_tx(bars + b, 256u);
            bulk_copy_g2s(dst + lane * 32, fa_rows + (size_t)me.x * 32, 128u, bars + b);
            bulk_copy_g2s(dst + (32 + lane) * 32, fa_rows + (size_t)me.y * 32, 128u, bars + b);
        };
        uint4 cur = make_uint4(0u, 0u, NONE, 0u);
        if (nchunks > 0) {
            cur = load_edge(e_lo + lane);
            issue(0, cur);
        }
        for (uint32_t c = 0; c < nchunks; ++c) {
            const uint32_t base = e_lo + c * 32;
            const int b = (int)(c & 1u);
            __syncwarp();
            stage[lane] = cur;
            __syncwarp();
            const bool landed = mbar_wait_bounded(bars + b, (phase >> b) & 1u, 1u << 24);
            if (!__all_sync(FULL, landed)) {
                timed_out = true;
                break;
            }
            phase ^= 1u << b;
            const uint32_t t0 = stage[0].z;
            const bool running = live && t0 <= te && t0 < fz;
            if (!__any_sync(FULL, running)) break;
            uint4 nxt = make_uint4(0u, 0u, NONE, 0u);
            if (c + 1 < nchunks) {
                nxt = load_edge(base + 32 + lane);
                issue(b ^ 1, nxt);
            }
            uint32_t* RU = rowbuf + (size_t)b * (PFM_BUF_BYTES / 4) + lane;        // RU[j * 32]: fa'(u_j)
            uint32_t* RV = RU + 32 * 32;                                            // RV[j * 32]: fa'(v_j)
            // rows were copied before the previous chunk's stores: patch them
            if (np > 4) {
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const uint4 E = stage[j];
                    RU[j * 32] = fa[(size_t)E.x * 32];
                    RV[j * 32] = fa[(size_t)E.y * 32];
                }
            } else {
                for (int qq = 0; qq < np; ++qq) {
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        const uint4 E = stage[j];
                        if (E.x == pv[qq]) RU[j * 32] = pf[qq];
                        if (E.y == pv[qq]) RV[j * 32] = pf[qq];
                    }
                }
            }
            np = 0;
            // later edges of the chunk that touch this edge's head
            uint32_t coll = 0;
#pragma unroll
            for (int o = 1; o < 32; ++o) {
                const uint32_t uj = __shfl_down_sync(FULL, cur.x, o);
                const uint32_t vj = __shfl_down_sync(FULL, cur.y, o);
                if (lane + o < 32 && (uj == cur.y || vj == cur.y)) coll |= 1u << (lane + o);
            }
            const uint32_t hi_t = min(te, fz - 1u);
            unsigned onm = 0, fm = 0, am = 0;
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const uint4 E = stage[j];
                const bool on = live && E.z >= ts && E.z <= hi_t && E.y != s;
                const uint32_t fu = RU[j * 32], fv = RV[j * 32];
                const bool act = on && fu <= E.z;
                onm |= on ? (1u << j) : 0u;
                fm |= (act && fv == NONE) ? (1u << j) : 0u;
                am |= (act && fv == E.z + 1u) ? (1u << j) : 0u;
            }
            my_escan += __popc(onm);
            bool conflict = false;
            unsigned rem = fm;
            int rounds = __popc(fm);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) rounds = max(rounds, __shfl_xor_sync(FULL, rounds, o));
            for (int r = 0; r < rounds; ++r) {
                const int k = rem ? __ffs(rem) - 1 : 0;
                const uint32_t ck = __shfl_sync(FULL, coll, k);
                if (rem) {
                    if ((ck & onm) || stage[k].y == z) conflict = true;
                    rem &= rem - 1;
                }
            }
            if (!conflict) {
                unsigned w = fm;
                while (w) {
                    const int k = __ffs(w) - 1;
                    w &= w - 1;
                    const uint4 E = stage[k];
                    fa[(size_t)E.y * 32] = E.z + 1u;
                    if (np < 4) { pv[np] = E.y; pf[np] = E.z + 1u; }
                    ++np;
                }
                w = fm | am;
                my_eadd += __popc(w);
                while (w) {
                    const int k = __ffs(w) - 1;
                    w &= w - 1;
                    if (nlist < cap) list[(size_t)nlist * 32] = (base + k) | (((fm >> k) & 1u) ? LIST_FIRST : 0u);
                    else lovf = true;
                    ++nlist;
                }
            } else {
                // in-order pass of this lane over the chunk
                for (int j = 0; j < 32; ++j) {
                    if (!((onm >> j) & 1u)) continue;
                    const uint4 E = stage[j];
                    uint32_t fu = RU[j * 32], fv = RV[j * 32];
                    if (np > 4) { fu = fa[(size_t)E.x * 32]; fv = fa[(size_t)E.y * 32]; }
                    else {
                        for (int qq = 0; qq < np; ++qq) {
                            if (pv[qq] == E.x) fu = pf[qq];
                            if (pv[qq] == E.y) fv = pf[qq];
                        }
                    }
                    if (!(E.z < fz && fu <= E.z)) continue;
                    bool first = false;
                    if (fv == NONE) {
                        fa[(size_t)E.y * 32] = E.z + 1u;
                        if (np < 4) { pv[np] = E.y; pf[np] = E.z + 1u; }
                        ++np;
                        first = true;
                        if (E.y == z) fz = E.z + 1u;
                    } else if (fv != E.z + 1u) {
                        continue;
                    }
                    ++my_eadd;
                    if (nlist < cap) list[(size_t)nlist * 32] = (base + j) | (first ? LIST_FIRST : 0u);
                    else lovf = true;
                    ++nlist;
                }
            }
            fence_proxy_async();      // this chunk's row stores and buffer reads before later copies
            cur = nxt;
        }
        __syncwarp();
        if (__any_sync(FULL, timed_out)) {
            if (lane == 0) set_status(job.status, ST_TIMEOUT);
            return;
        }

        // path counts (and hops) from the lane's contribution list, in stream order
        uint32_t ovf = lovf ? 1u : 0u;
        if (live && !lovf) {
            sig[(size_t)s * 32] = 1ull;
            if (stats) hop[(size_t)s * 32] = 0u;
            for (uint32_t p0 = 0; p0 < nlist; p0 += 8) {
                uint32_t LU[8], LV[8], LF[8];
                Sig SU[8], SV[8];
                const uint32_t cnt = min(8u, nlist - p0);
#pragma unroll
                for (int b = 0; b < 8; ++b) {
                    LU[b] = 0; LV[b] = 0; LF[b] = 0;
                    if (b < (int)cnt) {
                        const uint32_t ent = list[(size_t)(p0 + b) * 32];
                        const uint32_t ee = ent & ~LIST_FIRST;
                        LF[b] = ent & LIST_FIRST;
                        LU[b] = g.st_u[ee];
                        LV[b] = g.st_v[ee];
                    }
                }
#pragma unroll
                for (int b = 0; b < 8; ++b) {
                    SU[b] = (b < (int)cnt) ? sig[(size_t)LU[b] * 32] : 0ull;
                    SV[b] = (b < (int)cnt && !LF[b]) ? sig[(size_t)LV[b] * 32] : 0ull;
                }
#pragma unroll
                for (int b = 0; b < 8; ++b) {
                    if (b >= (int)cnt) break;
                    Sig su = SU[b], sv = SV[b];
#pragma unroll
                    for (int r = 0; r < b; ++r) {
                        if (LV[r] == LU[b]) su = SV[r];          // SV[r] holds entry r's new count
                        if (LV[r] == LV[b] && !LF[b]) sv = SV[r];
                    }
                    const Sig nv = sv + su;
                    if (nv < sv && !stats) ovf = 1u;
                    SV[b] = nv;
                    sig[(size_t)LV[b] * 32] = nv;
                    if (stats) {
                        const uint32_t hu = hop[(size_t)LU[b] * 32] + 1u;
                        if (LF[b]) hop[(size_t)LV[b] * 32] = hu;
                        else if (hu < hop[(size_t)LV[b] * 32]) hop[(size_t)LV[b] * 32] = hu;
                    }
                }
            }
        }
        __syncwarp();

        if (stats) {
            if (ovf && have) job.ovf_list[atomicAdd(job.ctr + C_NOVF, 1ull)] = i;
            const bool cnt_ok = live && !ovf;
            uint32_t dloc = 0;
            for (uint32_t v = 0; v < n; ++v) {
                const bool r = cnt_ok && v != s && fa[(size_t)v * 32] != NONE;
                const uint32_t h = r ? hop[(size_t)v * 32] : NONE;
                const unsigned grp = __match_any_sync(FULL, h);
                if (r && lane == __ffs(grp) - 1) atomicAdd(job.cnt + h, (u64)__popc(grp));
                if (r && h > dloc) dloc = h;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) dloc = max(dloc, __shfl_xor_sync(FULL, dloc, o));
            if (lane == 0 && dloc) atomicMax(job.dmax, (u64)dloc);
            continue;
        }

        uint32_t len = 0, err = 0;
        u128 sigma_sz = 0;
        if (have && !ovf && live && fz != NONE) {
            const Sig tot = sig[(size_t)z * 32];
            sigma_sz = (u128)tot;
            u128 x;
            if (!draw_below128(sigma_sz, job.seed, i, job.dom_path, &x)) { err = 1; set_status(job.status, ST_RNG); }
            Sig xs = (Sig)x;
            uint32_t v = z, cnt = 0;
            path[cnt++] = z;
            while (!err && v != s) {
                const uint32_t fv = fa[(size_t)v * 32];
                const uint32_t a = lower_bound_u32(g.slot_t, g.slot_ptr[v], g.slot_ptr[v + 1], fv - 1u);
                Sig cum = 0;
                uint32_t nxt = NONE;
                for (uint32_t e = g.slot_in[a]; e < g.slot_in[a + 1]; ++e) {
                    const uint32_t w = g.in_u[e];
                    if (!(fa[(size_t)w * 32] < fv)) continue;
                    const Sig wt = sig[(size_t)w * 32];
                    if (xs < cum + wt) { xs -= cum; nxt = w; break; }
                    cum += wt;
                }
                if (nxt == NONE || cnt > n) { err = 1; break; }
                v = nxt;
                path[cnt++] = v;
            }
            if (err) set_status(job.status, ST_CHECK);
            else {
                for (uint32_t p = 0; p < cnt / 2; ++p) {
                    const uint32_t tmp = path[p]; path[p] = path[cnt - 1 - p]; path[cnt - 1 - p] = tmp;
                }
                len = cnt;
            }
        }
        if (have && ovf) job.ovf_list[atomicAdd(job.ctr + C_NOVF, 1ull)] = i;
        if (have && !ovf && !err) {
            if (job.hits && len >= 3) {
                uint32_t w4[4];
                philox_block(job.seed, i, DOM_RADE, 0, w4);
                for (uint32_t p = 1; p + 1 < len; ++p) {
                    const uint32_t v = path[p];
                    atomicAdd(job.hits + v, 1ull);
                    if (job.S)
                        for (uint32_t jj = 0; jj < job.c; ++jj) {
                            const int lam = ((w4[jj >> 5] >> (jj & 31)) & 1u) ? 1 : -1;
                            atomicAdd(job.S + (size_t)jj * n + v, lam);
                        }
                }
                atomicAdd(job.ctr + C_SUMINT, (u64)(len - 2));
            }
            if (job.rec_len) {
                const uint64_t r = i - job.i0;
                job.rec_s[r] = s; job.rec_z[r] = z;
                job.rec_sig[2 * r] = (u64)sigma_sz; job.rec_sig[2 * r + 1] = (u64)(sigma_sz >> 64);
                job.rec_len[r] = len;
                for (uint32_t p = 0; p < len && p < job.rec_cap; ++p) job.rec_nodes[r * job.rec_cap + p] = path[p];
            }
        }
        __syncwarp();
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        my_escan += __shfl_xor_sync(FULL, my_escan, o);
        my_eadd += __shfl_xor_sync(FULL, my_eadd, o);
    }
    if (lane == 0) {
        if (my_escan) atomicAdd(job.ctr + C_ESCAN, my_escan);
        if (my_eadd) atomicAdd(job.ctr + C_EADD, my_eadd);
    }
}

// Per-warp region: 32 lanes' state rows, one path buffer per lane and the
// fast kernel's contribution lists (list_cap entries per lane).
size_t pfm_region_bytes(uint32_t n, uint32_t list_cap, PfmWs* ws) {
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    size_t o = 0;
    ws->o_fa = o;   o = al(o + (size_t)n * 32 * 4);
    ws->o_sig = o;  o = al(o + (size_t)n * 32 * 16);
    ws->o_hop = o;  o = al(o + (size_t)n * 32 * 4);
    ws->o_path = o; o = al(o + (size_t)32 * (n + 2) * 4);
    ws->o_list = o; o = al(o + (size_t)32 * list_cap * 4);
    ws->list_cap = list_cap;
    return o;
}

int pfm_threads() { return PFM_NT; }

cudaError_t launch_pfm_fast(const DevGraph& g, const Job& job, const PfmWs& ws, int grid, cudaStream_t st) {
    static bool configured = false;
    if (!configured) {
        const cudaError_t e = cudaFuncSetAttribute(k_pfm_fast, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)PFM_FAST_SMEM);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    k_pfm_fast<<<grid, PFM_NT, PFM_FAST_SMEM, st>>>(g, job, ws);
    return cudaGetLastError();
}

cudaError_t launch_pfm(const DevGraph& g, const Job& job, const PfmWs& ws, int grid, bool wide, cudaStream_t st) {
    if (wide) k_pfm<true><<<grid, PFM_NT, 0, st>>>(g, job, ws);
    else k_pfm<false><<<grid, PFM_NT, 0, st>>>(g, job, ws);
    return cudaGetLastError();
}

}  // namespace mantra
