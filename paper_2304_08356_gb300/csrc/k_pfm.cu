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
constexpr int PFM_ILP = 8;

constexpr uint32_t LIST_FIRST = 0x80000000u;

// DEFER (64-bit counts only): arrival decisions in the scan, path counts (and
// hops) afterwards from the lane's ordered list of contributing edges, so the
// scan never waits on a path-count load.  A lane whose list would exceed
// list_cap is handed to the in-order kernel (overflow list).
template <bool WIDE, bool DEFER>
__global__ void __launch_bounds__(PFM_NT) k_pfm(const Task* tasks, const uint64_t* unit_start,
                                                const uint32_t* ntasks_p, u64* work, const PfmWs ws) {
    typedef typename SigOps<WIDE>::T Sig;
    const uint32_t FULL = 0xFFFFFFFFu;
    const int lane = threadIdx.x & 31;
    const uint64_t gw = ((uint64_t)blockIdx.x * PFM_NT + threadIdx.x) >> 5;
    char* region = ws.base + gw * ws.stride;
    uint32_t* fa = reinterpret_cast<uint32_t*>(region + ws.o_fa) + lane;     // fa[v * 32]
    Sig* sig = reinterpret_cast<Sig*>(region + ws.o_sig) + lane;             // sig[v * 32]
    uint32_t* hop = reinterpret_cast<uint32_t*>(region + ws.o_hop) + lane;   // hop[v * 32]
    uint32_t* path = reinterpret_cast<uint32_t*>(region + ws.o_path) + (size_t)lane * (ws.n_cap + 2);
    uint32_t* pathe = reinterpret_cast<uint32_t*>(region + ws.o_pathe) + (size_t)lane * (ws.n_cap + 2);
    uint32_t* list = reinterpret_cast<uint32_t*>(region + ws.o_list) + lane;     // list[p * 32]
    Sig* dl = reinterpret_cast<Sig*>(region + ws.o_dl) + lane;               // ob: dl[v * 32]
    __shared__ __align__(16) Task sh_tasks[PFM_NT / 32];
    Task& T = sh_tasks[threadIdx.x >> 5];
    const uint32_t ntasks = *ntasks_p;

    for (;;) {
        int t = -1;
        uint64_t unit = 0;
        if (lane == 0) {
            const uint64_t u = atomicAdd(work, 1ull);
            if (ntasks > 0 && u < unit_start[ntasks]) {
                t = task_of_unit(unit_start, ntasks, u);
                unit = u - unit_start[t];
            }
        }
        t = __shfl_sync(FULL, t, 0);
        unit = __shfl_sync(FULL, unit, 0);
        if (t < 0) break;
        __syncwarp();
        {
            const u64* src = reinterpret_cast<const u64*>(tasks + t);
            u64* dst = reinterpret_cast<u64*>(&T);
            for (uint32_t w = lane; w < sizeof(Task) / 8; w += 32) dst[w] = src[w];
        }
        __syncwarp();
        const DevGraph& g = T.g;
        const Job& job = T.job;
        const uint32_t n = g.n;
        const uint32_t* const st_u = g.st_u;   // hot pointers in registers
        const uint32_t* const st_v = g.st_v;
        const uint32_t* const st_t = g.st_t;
        const bool stats = job.stats != 0;
        u64 my_escan = 0, my_eadd = 0;
        const uint64_t q0 = unit * 32;
        const uint64_t q = q0 + lane;
        const bool have = q < job.count;
        const uint64_t i = have ? (job.idx_list ? job.idx_list[q] : job.i0 + q) : 0;

        uint32_t s = 0, z = 1;
        bool ok = true;
        if (have) {
            if (stats || job.rtb) {
                uint64_t x;
                ok = draw_below64(n, job.seed, i, stats ? DOM_STATS : job.dom_pair, &x);
                s = (uint32_t)x; z = NONE;
            } else {
                ok = draw_pair(n, job.seed, i, job.dom_pair, &s, &z);
            }
            if (!ok) { set_status(job.status, ST_RNG); s = 0; z = (stats || job.rtb) ? NONE : 1; }
        }
        const bool full = stats || job.rtb;   // a source only, untruncated scan
        bool live = have && ok && g.out_ptr[s + 1] > g.out_ptr[s];
        if (!full && live && g.slot_ptr[z + 1] == g.slot_ptr[z]) live = false;
        const uint32_t ts = live ? g.tmin_out[s] : NONE;
        const uint32_t te = live ? (full ? NONE - 1 : g.tmax_in[z]) : 0;

        for (uint32_t v = 0; v < n; ++v) fa[(size_t)v * 32] = NONE;
        if (job.ob || job.rtb) for (uint32_t v = 0; v < n; ++v) dl[(size_t)v * 32] = (Sig)0;
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
        uint32_t nlist = 0;
        bool lovf = false;
        for (uint32_t base = e_lo; base < e_hi; base += 32) {
            const uint32_t e = base + lane;
            uint32_t eu = 0, ev = 0, et = NONE;
            if (e < e_hi) { eu = st_u[e]; ev = st_v[e]; et = st_t[e]; }
            // lanes still scanning at this chunk's first time
            const uint32_t t0 = __shfl_sync(FULL, et, 0);
            const bool running = live && t0 <= te && t0 < fz;
            if (!__any_sync(FULL, running)) break;
            const uint32_t kmax = min(32u, e_hi - base);
            for (uint32_t k0 = 0; k0 < kmax; k0 += PFM_ILP) {
                uint32_t U[PFM_ILP], Vv[PFM_ILP], T[PFM_ILP], FU[PFM_ILP], FV[PFM_ILP];
                bool on[PFM_ILP];
#pragma unroll
                for (int j = 0; j < PFM_ILP; ++j) {
                    U[j] = __shfl_sync(FULL, eu, (k0 + j) & 31);
                    Vv[j] = __shfl_sync(FULL, ev, (k0 + j) & 31);
                    T[j] = __shfl_sync(FULL, et, (k0 + j) & 31);
                    on[j] = (k0 + j < kmax) && live && T[j] >= ts && T[j] <= te && T[j] < fz && Vv[j] != s;
                    FU[j] = on[j] ? fa[(size_t)U[j] * 32] : NONE;
                    FV[j] = on[j] ? fa[(size_t)Vv[j] * 32] : NONE;
                }
                uint32_t newf[PFM_ILP];
                bool upd[PFM_ILP];
#pragma unroll
                for (int j = 0; j < PFM_ILP; ++j) {
                    uint32_t fu = FU[j], fv = FV[j];
#pragma unroll
                    for (int k = 0; k < j; ++k) {          // this lane's own earlier updates in the group
                        if (upd[k] && Vv[k] == U[j]) fu = newf[k];
                        if (upd[k] && Vv[k] == Vv[j]) fv = newf[k];
                    }
                    upd[j] = false;
                    newf[j] = 0;
                    const uint32_t t = T[j];
                    // fz may have been set by an earlier edge of this group
                    if (DEFER && on[j] && t < fz && fu <= t && (fv == NONE || fv == t + 1u)) {
                        const uint32_t v = Vv[j];
                        const bool first = fv == NONE;
                        if (first) {
                            fa[(size_t)v * 32] = t + 1u;
                            upd[j] = true;
                            newf[j] = t + 1u;
                            if (v == z) fz = t + 1u;
                        }
                        if (nlist < ws.list_cap) list[(size_t)nlist * 32] = (base + k0 + j) | (first ? LIST_FIRST : 0u);
                        else lovf = true;
                        ++nlist;
                        ++my_eadd;
                    } else if (!DEFER && on[j] && t < fz && fu <= t) {
                        const uint32_t u = U[j], v = Vv[j];
                        if (fv == NONE) {
                            fa[(size_t)v * 32] = t + 1u;
                            sig[(size_t)v * 32] = sig[(size_t)u * 32];
                            if (stats) hop[(size_t)v * 32] = hop[(size_t)u * 32] + 1u;
                            upd[j] = true;
                            newf[j] = t + 1u;
                            if (v == z) fz = t + 1u;
                            ++my_eadd;
                        } else if (fv == t + 1u) {
                            Sig nv;
                            if (!SigOps<WIDE>::add(sig[(size_t)v * 32], sig[(size_t)u * 32], &nv) && !stats) ovf = 1;
                            sig[(size_t)v * 32] = nv;
                            if (stats) {
                                const uint32_t hu = hop[(size_t)u * 32] + 1u;
                                if (hu < hop[(size_t)v * 32]) hop[(size_t)v * 32] = hu;
                            }
                            ++my_eadd;
                        }
                    }
                    my_escan += (on[j] && t < fz) ? 1 : 0;     // scan window ends at fa(z)
                }
            }
        }
        __syncwarp();
        if (DEFER) {
            // path counts (and hops) from the contribution list, in stream order,
            // 8 entries per batch; this lane's updates inside a batch are forwarded
            if (lovf) ovf = 1;
            else if (live) {
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
                            LU[b] = st_u[ee];
                            LV[b] = st_v[ee];
                        }
                    }
#pragma unroll
                    for (int b = 0; b < 8; ++b) {
                        SU[b] = (b < (int)cnt) ? sig[(size_t)LU[b] * 32] : (Sig)0;
                        SV[b] = (b < (int)cnt && !LF[b]) ? sig[(size_t)LV[b] * 32] : (Sig)0;
                    }
#pragma unroll
                    for (int b = 0; b < 8; ++b) {
                        if (b >= (int)cnt) break;
                        Sig su = SU[b], sv = SV[b];
#pragma unroll
                        for (int r = 0; r < b; ++r) {
                            if (LV[r] == LU[b]) su = SV[r];          // SV[r] now holds entry r's new count
                            if (LV[r] == LV[b] && !LF[b]) sv = SV[r];
                        }
                        Sig nv;
                        if (!SigOps<WIDE>::add(sv, su, &nv) && !stats) ovf = 1;
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

        if (stats) {
            // a lane whose contribution list overflowed is re-run by the in-order kernel
            if (have && ovf) push_overflow(job, i);
            uint32_t dloc = 0;
            for (uint32_t v = 0; v < n; ++v) {
                const bool r = live && !ovf && v != s && fa[(size_t)v * 32] != NONE;
                const uint32_t h = r ? hop[(size_t)v * 32] : NONE;
                const unsigned grp = __match_any_sync(FULL, h);
                if (r && lane == __ffs(grp) - 1) atomicAdd(job.cnt + h, (u64)__popc(grp));
                if (r && job.clos) atomicAdd(job.clos + v, recip32(h));
                if (r && h > dloc) dloc = h;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) dloc = max(dloc, __shfl_xor_sync(FULL, dloc, o));
            if (lane == 0 && dloc) atomicMax(job.dmax, (u64)dloc);
            continue;
        }

        // ---------------- ob (Sec. 4.1), one lane per sample ----------------
        // continuation counts to z over the DAG edges (w, x, fa(x)), fa(w) < fa(x),
        // by a backward walk of the stream from fa(z) (every edge out of x comes
        // later in time than fa(x)); sigma_sz(v) = sigma(v) * continuations(v)
        if (job.ob && job.hits && have && !ovf && live && fz != NONE) {
            const u128 tot = SigOps<WIDE>::wide(sig[(size_t)z * 32]);
            uint32_t w4[4];
            philox_block(job.seed, i, DOM_RADE, 0, w4);
            dl[(size_t)z * 32] = (Sig)1;
            uint32_t nt = 0;                              // vertices listed in path
            uint32_t e = upper_bound_u32(st_t, 0, g.m, fz - 1u);
            const uint32_t e0 = lower_bound_u32(st_t, 0, g.m, ts);
            while (e > e0) {
                --e;
                const uint32_t x = st_v[e], t = st_t[e];
                if (fa[(size_t)x * 32] != t + 1u) continue;         // not x's earliest arrival
                const Sig dx = dl[(size_t)x * 32];
                if (dx == (Sig)0) continue;
                const uint32_t w = st_u[e];
                if (fa[(size_t)w * 32] > t) continue;               // needs fa(w) < t
                if (dl[(size_t)w * 32] == (Sig)0 && w != s) path[nt++] = w;
                dl[(size_t)w * 32] += dx;                           // <= sigma_sz: no wrap
            }
            u64 sum = 0;
            for (uint32_t k = 0; k < nt; ++k) {
                const uint32_t w = path[k];
                const uint64_t q = ob_q(SigOps<WIDE>::wide((Sig)(sig[(size_t)w * 32] * dl[(size_t)w * 32])), tot);
                dl[(size_t)w * 32] = (Sig)0;
                if (!q) continue;
                sum += q;
                const uint32_t rows = 2 + (job.S64 ? job.c : 0);
                for (uint32_t row = 0; row < rows; ++row) ob_term(job, w, q, row, w4);
            }
            dl[(size_t)z * 32] = (Sig)0;
            dl[(size_t)s * 32] = (Sig)0;
            if (sum) atomicAdd(job.ctr + C_SUMINT, sum);
        }

        // ---------------- RTB (App. C), one lane per sample ----------------
        // dependencies over the whole prefix-foremost DAG by a backward walk of
        // the stream: an edge (w, x, fa(x)), fa(w) < fa(x), w != s, adds
        // round(sigma(w) (1 + delta(x)) / sigma(x)) to delta(w) (x's edges out
        // come later, so delta(x) is final); dl holds delta in 2^-32 units
        if (job.rtb && job.hits && have && !ovf && live) {
            uint32_t w4[4];
            philox_block(job.seed, i, DOM_RADE, 0, w4);
            uint32_t nt = 0;
            uint32_t e = g.m;
            const uint32_t e0 = lower_bound_u32(st_t, 0, g.m, ts);
            while (e > e0) {
                --e;
                const uint32_t x = st_v[e], t = st_t[e];
                if (fa[(size_t)x * 32] != t + 1u) continue;
                const uint32_t w = st_u[e];
                if (w == s || fa[(size_t)w * 32] > t) continue;
                const uint64_t X = (1ull << 32) + (uint64_t)dl[(size_t)x * 32];
                const uint64_t term = muldiv_round(SigOps<WIDE>::wide(sig[(size_t)w * 32]), X,
                                                   SigOps<WIDE>::wide(sig[(size_t)x * 32]));
                if (!term) continue;
                if (dl[(size_t)w * 32] == (Sig)0) path[nt++] = w;
                dl[(size_t)w * 32] += (Sig)term;
            }
            u64 sum = 0;
            for (uint32_t k = 0; k < nt; ++k) {
                const uint32_t w = path[k];
                const uint64_t q = muldiv_round(1, (uint64_t)dl[(size_t)w * 32], n - 1);
                dl[(size_t)w * 32] = (Sig)0;
                if (!q) continue;
                sum += q;
                const uint32_t rows = 2 + (job.S64 ? job.c : 0);
                for (uint32_t row = 0; row < rows; ++row) ob_term(job, w, q, row, w4);
            }
            if (sum) atomicAdd(job.ctr + C_SUMINT, sum);
        }

        // ---------------- path draw, one lane per sample ----------------
        uint32_t len = 0, err = 0;
        u128 sigma_sz = 0;
        if (have && !ovf && live && fz != NONE && !job.ob && !job.rtb) {
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
                uint32_t nxt = NONE, ech = NONE;
                for (uint32_t e = g.slot_in[a]; e < g.slot_in[a + 1]; ++e) {
                    const uint32_t w = g.in_u[e];
                    if (!(fa[(size_t)w * 32] < fv)) continue;
                    const Sig wt = sig[(size_t)w * 32];
                    if (xs < cum + wt) { xs -= cum; nxt = w; ech = e; break; }
                    cum += wt;
                }
                if (nxt == NONE || cnt > n) { err = 1; break; }
                v = nxt;
                pathe[cnt - 1] = ech;
                path[cnt++] = v;
            }
            if (err) set_status(job.status, ST_CHECK);
            else {
                for (uint32_t p = 0; p < cnt / 2; ++p) {
                    const uint32_t tmp = path[p]; path[p] = path[cnt - 1 - p]; path[cnt - 1 - p] = tmp;
                }
                for (uint32_t p = 0; p < (cnt - 1) / 2; ++p) {
                    const uint32_t tmp = pathe[p]; pathe[p] = pathe[cnt - 2 - p]; pathe[cnt - 2 - p] = tmp;
                }
                len = cnt;
            }
        }
        if (have && ovf) {
            if (WIDE) set_status(job.status, ST_OVERFLOW);
            else push_overflow(job, i);
        }
        // ---- hits and Rademacher sums of the warp's 32 samples, warp-aggregated:
        // in step k every lane adds its path's k-th entry; lanes adding to the
        // same entry combine (their count, and per trial the sum of their
        // signs), and one lane issues the atomic ----
        {
            const uint32_t nint = (have && !ovf && !err && job.hits) ? family_count(job, len) : 0u;
            uint32_t w4[4] = {0u, 0u, 0u, 0u};
            if (nint > 0) philox_block(job.seed, i, DOM_RADE, 0, w4);
            const uint32_t kmax = __reduce_max_sync(FULL, nint);
            for (uint32_t k = 0; k < kmax; ++k) {
                const bool act = k < nint;
                const uint32_t x = act ? family_item(job, g, path, pathe, k) : 0u;
                const u64 key = act ? (u64)x : ((1ull << 32) | (u64)lane);   // idle lanes never match
                const unsigned grp = __match_any_sync(FULL, key);
                const bool lead = act && lane == __ffs(grp) - 1;
                if (lead) atomicAdd(job.hits + x, (u64)__popc(grp));
                if (job.S)
                    for (uint32_t jj = 0; jj < job.c; ++jj) {
                        const unsigned plus = __ballot_sync(FULL, act && ((w4[jj >> 5] >> (jj & 31)) & 1u));
                        const int sum = 2 * __popc(grp & plus) - __popc(grp);   // lambda = +1 / -1 per lane
                        if (lead && sum) atomicAdd(job.S + (size_t)jj * job.fam + x, sum);
                    }
            }
            const uint32_t tot = __reduce_add_sync(FULL, nint);
            if (lane == 0 && tot) atomicAdd(job.ctr + C_SUMINT, (u64)tot);
        }
        if (have && !ovf && !err) {
            if (job.rec_len) {
                const uint64_t r = i - job.i0;
                job.rec_s[r] = s; job.rec_z[r] = z;
                job.rec_sig[2 * r] = (u64)sigma_sz; job.rec_sig[2 * r + 1] = (u64)(sigma_sz >> 64);
                job.rec_len[r] = len;
                for (uint32_t p = 0; p < len && p < job.rec_cap; ++p) job.rec_nodes[r * job.rec_cap + p] = path[p];
                if (job.rec_edges)
                    for (uint32_t p = 0; p + 1 < len && p < job.rec_cap; ++p) job.rec_edges[r * job.rec_cap + p] = pathe[p];
            }
        }
        __syncwarp();
    }
}

// Per-warp region: 32 lanes' state rows plus one path buffer per lane.
size_t pfm_region_bytes(uint32_t n, uint32_t list_cap, PfmWs* ws) {
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    ws->n_cap = n;
    ws->list_cap = list_cap;
    size_t o = 0;
    ws->o_fa = o;   o = al(o + (size_t)n * 32 * 4);
    ws->o_sig = o;  o = al(o + (size_t)n * 32 * 16);
    ws->o_hop = o;  o = al(o + (size_t)n * 32 * 4);
    ws->o_path = o; o = al(o + (size_t)32 * (n + 2) * 4);
    ws->o_pathe = o; o = al(o + (size_t)32 * (n + 2) * 4);
    ws->o_list = o; o = al(o + (size_t)32 * list_cap * 4);
    ws->o_dl = o;   o = al(o + (size_t)n * 32 * 16);
    return o;
}

int pfm_threads() { return PFM_NT; }

cudaError_t launch_pfm(const Task* tasks, const uint64_t* unit_start, const uint32_t* ntasks, u64* work,
                       const PfmWs& ws, int grid, bool wide, cudaStream_t st) {
    // narrow launches defer path counts; the 128-bit re-run takes overflowed
    // counts and overflowed contribution lists, in order
    if (wide) k_pfm<true, false><<<grid, PFM_NT, 0, st>>>(tasks, unit_start, ntasks, work, ws);
    else k_pfm<false, true><<<grid, PFM_NT, 0, st>>>(tasks, unit_start, ntasks, work, ws);
    return cudaGetLastError();
}

}  // namespace mantra
