// Prefix-foremost (pfm) temporal search (paper Sec. 3 Def. 1(3); running-time
// theorem of Sec. 4.4: one pass over the time-sorted edges), the backward
// path draw over earliest-arrival predecessors (App. C, theorem on the path
// sampler) and the Update step of Algorithm 1.  Also the pfm full searches of
// Algorithm 2 (distance = minimum hops among prefix-foremost paths).
//
// One warp owns one sample.  Per vertex: fa (earliest arrival, encoded
// fa' = fa + 1, 0 for the source, NONE when unreached), sigma (number of pfm
// paths) and hop (minimum hops).  The warp walks the stream (t, u, v) in
// chunks of 32 edges, from the first edge at the source's earliest out-edge
// time to the last edge at z's latest in-edge time, and stops after the
// timestamp group at which z is reached.  Inside a chunk an edge (u, v, t)
// is live when fa(u) < t; arrival times are settled by a fixpoint of
// atomicMin(fa'(v), t + 1) over live edges (edges in one chunk can chain
// only across different timestamps), then the edges with fa(v) = t add
// sigma(u) to sigma(v) one at a time in stream order.
#include "mantra_dev.cuh"

namespace mantra {

constexpr int PFM_NT = 256;

__device__ __forceinline__ uint32_t ld_fa(const uint32_t* p) { return __ldcg(p); }

template <bool WIDE>
__global__ void __launch_bounds__(PFM_NT) k_pfm(const DevGraph g, const Job job, const PfmWs ws) {
    typedef typename SigOps<WIDE>::T Sig;
    const uint32_t FULL = 0xFFFFFFFFu;
    const int lane = threadIdx.x & 31;
    const uint64_t gw = ((uint64_t)blockIdx.x * PFM_NT + threadIdx.x) >> 5;
    const uint32_t n = g.n;
    char* region = ws.base + gw * ws.stride;
    uint32_t* fa = reinterpret_cast<uint32_t*>(region + ws.o_fa);
    Sig* sig = reinterpret_cast<Sig*>(region + ws.o_sig);
    uint32_t* hop = reinterpret_cast<uint32_t*>(region + ws.o_hop);
    uint32_t* path = reinterpret_cast<uint32_t*>(region + ws.o_path);
    u64 my_escan = 0, my_eadd = 0;
    const bool stats = job.stats != 0;

    for (;;) {
        uint64_t q = 0;
        if (lane == 0) q = atomicAdd(job.ctr + C_WORK, 1ull);
        q = __shfl_sync(FULL, q, 0);
        if (q >= job.count) break;
        const uint64_t i = job.idx_list ? job.idx_list[q] : job.i0 + q;

        uint32_t s, z;
        bool ok;
        if (stats) {
            uint64_t x;
            ok = draw_below64(n, job.seed, i, DOM_STATS, &x);
            s = (uint32_t)x; z = NONE;
        } else {
            ok = draw_pair(n, job.seed, i, job.dom_pair, &s, &z);
        }
        if (!ok) { if (lane == 0) set_status(job.status, ST_RNG); s = 0; z = 1; }

        for (uint32_t v = lane; v < n; v += 32) { fa[v] = NONE; sig[v] = (Sig)0; hop[v] = NONE; }
        __syncwarp();
        if (lane == 0) { fa[s] = 0u; sig[s] = (Sig)1; hop[s] = 0u; }
        __syncwarp();

        bool live = ok && g.out_ptr[s + 1] > g.out_ptr[s];
        if (!stats && g.slot_ptr[z + 1] == g.slot_ptr[z]) live = false;
        uint32_t ovf = 0;
        uint32_t fz = NONE;
        if (live) {
            const uint32_t ts = g.tmin_out[s];
            const uint32_t tz = stats ? (NONE - 1) : g.tmax_in[z];
            uint32_t e_lo = 0, e_hi = 0;
            if (lane == 0) {
                e_lo = lower_bound_u32(g.st_t, 0, g.m, ts);
                e_hi = upper_bound_u32(g.st_t, 0, g.m, tz);
            }
            e_lo = __shfl_sync(FULL, e_lo, 0);
            e_hi = __shfl_sync(FULL, e_hi, 0);
            for (uint32_t base = e_lo; base < e_hi; base += 32) {
                const uint32_t e = base + lane;
                bool valid = e < e_hi;
                uint32_t u = 0, v = 0, t = 0;
                if (valid) { u = g.st_u[e]; v = g.st_v[e]; t = g.st_t[e]; }
                valid = valid && (t < fz);                 // past z's arrival group: nothing left to do
                if (!__any_sync(FULL, valid)) break;
                my_escan += valid ? 1 : 0;
                valid = valid && (v != s);
                // arrival times inside the chunk
                unsigned prev = 0;
                bool act = false;
                for (int rep = 0; rep < 33; ++rep) {
                    act = valid && ld_fa(fa + u) <= t;
                    const unsigned bal = __ballot_sync(FULL, act);
                    if (bal == prev) break;
                    if (act) atomicMin(fa + v, t + 1u);
                    prev = bal;
                    __syncwarp();
                }
                __syncwarp();
                const bool contrib = act && ld_fa(fa + v) == t + 1u;
                unsigned cm = __ballot_sync(FULL, contrib);
                my_eadd += contrib ? 1 : 0;
                while (cm) {
                    const int l = __ffs(cm) - 1;
                    if (lane == l) {
                        Sig nv;
                        if (!SigOps<WIDE>::add(sig[v], sig[u], &nv) && !stats) ovf = 1;
                        sig[v] = nv;
                        const uint32_t hu = hop[u] + 1u;
                        if (hu < hop[v]) hop[v] = hu;
                    }
                    __syncwarp();
                    cm &= cm - 1;
                }
                if (!stats) fz = ld_fa(fa + z);
                if (__any_sync(FULL, ovf)) break;
            }
        }
        ovf = __any_sync(FULL, ovf) ? 1u : 0u;

        if (stats) {
            if (!ovf && live) {
                uint32_t dloc = 0;
                for (uint32_t v0 = 0; v0 < n; v0 += 32) {
                    const uint32_t v = v0 + lane;
                    const bool r = v < n && v != s && ld_fa(fa + v) != NONE;
                    const uint32_t h = r ? hop[v] : NONE;
                    const unsigned grp = __match_any_sync(FULL, h);
                    if (r && lane == __ffs(grp) - 1) atomicAdd(job.cnt + h, (u64)__popc(grp));
                    if (r && h > dloc) dloc = h;
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) dloc = max(dloc, __shfl_xor_sync(FULL, dloc, o));
                if (lane == 0 && dloc) atomicMax(job.dmax, (u64)dloc);
            }
            if (ovf && lane == 0) {
                if (WIDE) set_status(job.status, ST_OVERFLOW);
                else job.ovf_list[atomicAdd(job.ctr + C_NOVF, 1ull)] = i;
            }
            continue;
        }

        // ---------------- path draw (lane 0) ----------------
        uint32_t len = 0, err = 0;
        u128 sigma_sz = 0;
        if (!ovf && lane == 0 && live && fz != NONE) {
            const Sig tot = sig[z];
            sigma_sz = SigOps<WIDE>::wide(tot);
            u128 x;
            if (!draw_below128(sigma_sz, job.seed, i, job.dom_path, &x)) { err = 1; set_status(job.status, ST_RNG); }
            Sig xs = (Sig)x;
            // walk back from z; path[] collects z .. s, reversed below
            uint32_t v = z, cnt = 0;
            path[cnt++] = z;
            while (!err && v != s) {
                const uint32_t fv = ld_fa(fa + v);
                const uint32_t a = lower_bound_u32(g.slot_t, g.slot_ptr[v], g.slot_ptr[v + 1], fv - 1u);
                Sig cum = 0;
                uint32_t nxt = NONE;
                for (uint32_t e = g.slot_in[a]; e < g.slot_in[a + 1]; ++e) {
                    const uint32_t w = g.in_u[e];
                    if (!(ld_fa(fa + w) < fv)) continue;
                    const Sig wt = sig[w];
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
        len = __shfl_sync(FULL, len, 0);
        err = __shfl_sync(FULL, err, 0);
        __syncwarp();

        if (ovf) {
            if (lane == 0) {
                if (WIDE) set_status(job.status, ST_OVERFLOW);
                else job.ovf_list[atomicAdd(job.ctr + C_NOVF, 1ull)] = i;
            }
            continue;
        }
        if (err) continue;
        if (job.hits && len >= 3) {
            uint32_t w4[4];
            philox_block(job.seed, i, DOM_RADE, 0, w4);
            const uint32_t nint = len - 2;
            const uint32_t rows = 1 + (job.S ? job.c : 0);
            for (uint32_t it = lane; it < nint * rows; it += 32) {
                const uint32_t p = it % nint, j = it / nint;
                const uint32_t v = path[1 + p];
                if (j == 0) atomicAdd(job.hits + v, 1ull);
                else {
                    const uint32_t jj = j - 1;
                    const int lam = ((w4[jj >> 5] >> (jj & 31)) & 1u) ? 1 : -1;
                    atomicAdd(job.S + (size_t)jj * n + v, lam);
                }
            }
            if (lane == 0) atomicAdd(job.ctr + C_SUMINT, (u64)nint);
        }
        if (job.rec_len) {
            const uint64_t r = i - job.i0;
            if (lane == 0) {
                job.rec_s[r] = s; job.rec_z[r] = z;
                job.rec_sig[2 * r] = (u64)sigma_sz; job.rec_sig[2 * r + 1] = (u64)(sigma_sz >> 64);
                job.rec_len[r] = len;
            }
            for (uint32_t p = lane; p < len && p < job.rec_cap; p += 32) job.rec_nodes[r * job.rec_cap + p] = path[p];
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

size_t pfm_region_bytes(uint32_t n, PfmWs* ws) {
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    size_t o = 0;
    ws->o_fa = o;   o = al(o + (size_t)n * 4);
    ws->o_sig = o;  o = al(o + (size_t)n * 16);
    ws->o_hop = o;  o = al(o + (size_t)n * 4);
    ws->o_path = o; o = al(o + (size_t)(n + 2) * 4);
    return o;
}

int pfm_threads() { return PFM_NT; }

cudaError_t launch_pfm(const DevGraph& g, const Job& job, const PfmWs& ws, int grid, bool wide, cudaStream_t st) {
    if (wide) k_pfm<true><<<grid, PFM_NT, 0, st>>>(g, job, ws);
    else k_pfm<false><<<grid, PFM_NT, 0, st>>>(g, job, ws);
    return cudaGetLastError();
}

}  // namespace mantra
