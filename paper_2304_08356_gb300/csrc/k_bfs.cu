// (*)-temporal BFS for the shortest (sh) and shortest-foremost (sfm)
// optimalities (paper Sec. 3 Def. 1; running-time theorem of Sec. 4.4), the
// backward path draw of the temporal Riondato-Kornaropoulos estimator
// (App. C, theorem on the path sampler), and the Update step of Algorithm 1
// (hit counts and Rademacher sums).  Also the full searches of Algorithm 2.
//
// One CTA owns one sample at a time (persistent grid, samples taken from an
// atomic counter).  States are arrival appearances (v, t) ("slots"); level 0
// is the source appearance (s, -inf).  Per level k:
//   segments  the level-k frontier F_k is kept sorted by slot id, i.e. grouped
//             by vertex and ascending in time; per vertex u a running sum of
//             sigma over its frontier appearances.
//   pull      before expanding, z's in-edges are checked against F_k: if any
//             reaches z, level k+1 is z's level d and the search stops (the
//             last level is never pushed).
//   push      every out-edge (u, v, t) of a frontier vertex with
//             t_min'(u) < t < tmax_in(z) marks slot (v, t) for level k+1
//             unless that slot already has a level <= k.  Appearances at or
//             after z's latest in-edge time cannot lie on an s-z path; they
//             are not created.
//   compact   the next-level bitmap is compacted in slot order into F_{k+1}.
//   count     each state b = (v, t) of F_{k+1} sums, over its in-edges
//             (w, v, t), the path counts of w's level-k appearances earlier
//             than t (Def. 1: sigma(b) is the number of shortest walks to b),
//             and stores the sum at b's frontier position.
// Path counts therefore live in frontier order (Fs, parallel to F): they are
// written once, read in order by the next level's scan, and never cleared;
// only z's endpoint slots, reached by the pull, keep per-slot counts (zsig).
// The visited bitmap lives in shared memory when it fits (else in per-CTA
// global scratch); the next-level bitmap is in the scratch.
#include "mantra_dev.cuh"

#include <algorithm>
#include <mutex>

namespace mantra {

constexpr int IPT = 4;            // frontier states per thread in a segmented-scan tile
constexpr int WALK_K = 2;         // edge windows with loads in flight per warp in the push
constexpr int CK = 8;             // bitmap words in flight per lane in the compaction and cleanup scans
constexpr int CB = 4;             // new states per thread with loads in flight in the count pass
constexpr uint32_t SUMW = 512;    // words of the next-level bitmap's summary (one bit per 2^sumshift bitmap words)

// Path count of the state at frontier position p, from the running sums
// that the level's scan leaves in place (cum[p] = the sum of sigma over
// p's vertex's states of the level up to p); lv0 is the first position of
// p's level.
template <typename Sig>
__device__ __forceinline__ Sig sigma_at(const Sig* cum, const uint32_t* F, const uint32_t* slot_v, uint32_t p,
                                        uint32_t lv0) {
    const Sig c = cum[p];
    if (p == lv0 || slot_v[F[p - 1]] != slot_v[F[p]]) return c;
    return c - cum[p - 1];
}

// For each j: the first index in [lo[j], hi[j]) whose value is >= key[j]
// (hi[j] if none), left in lo[j]; the K searches advance together so their
// loads overlap.  Plain loads: the array is written by this kernel.
template <int K>
__device__ __forceinline__ void lower_bounds_rw(const uint32_t* a, uint32_t (&lo)[K], uint32_t (&hi)[K],
                                                const uint32_t (&key)[K]) {
    for (;;) {
        bool any = false;
        uint32_t mid[K], val[K];
#pragma unroll
        for (int j = 0; j < K; ++j) {
            const bool act = lo[j] < hi[j];
            any |= act;
            mid[j] = lo[j] + ((hi[j] - lo[j]) >> 1);
            val[j] = act ? a[mid[j]] : 0u;
        }
        if (!any) break;
#pragma unroll
        for (int j = 0; j < K; ++j)
            if (lo[j] < hi[j]) {
                if (val[j] < key[j]) lo[j] = mid[j] + 1u;
                else hi[j] = mid[j];
            }
    }
}

// ob update of one sample (Sec. 4.1), all threads of the CTA: continuation
// counts dl (the number of optimal ways from a state to z's endpoints) per
// frontier position, backward from level d; sigma_sz(v) = sum over v's states
// of sigma * dl (a path visits v once); then every internal v gets its ob
// value.  sig: running sums of the path counts by frontier position (see
// sigma_at); dl: per frontier position (scratch of the ob and RTB updates);
// acc: per-vertex sums (zero on entry and exit); VB: vertex bitmap (zero on
// entry and exit); tl: n entries.
template <bool WIDE, int BFS_NT>
__device__ __forceinline__ void bfs_ob_update(const DevGraph& g, const Job& job, uint32_t z, uint32_t d, uint32_t first,
                                           u128 sigma, const uint32_t* rade, const uint32_t* F, const uint32_t* lev,
                                           const uint32_t* N, const typename SigOps<WIDE>::T* sig,
                                           typename SigOps<WIDE>::T* dl, typename SigOps<WIDE>::T* acc, uint32_t* VB,
                                           uint32_t* tl, uint32_t* sh_nt) {
    typedef typename SigOps<WIDE>::T Sig;
    const int tid = threadIdx.x, lane = tid & 31;
    const uint32_t P0 = lev[1], P1 = lev[d];  // positions of levels 1 .. d-1
    for (uint32_t p = P0 + tid; p < P1; p += BFS_NT) dl[p] = (Sig)0;
    if (tid == 0) *sh_nt = 0;
    __syncthreads();
    // adds x to the states of in-edge e's tail on level lv with times before t
    auto to_preds = [&](uint32_t e, uint32_t t, uint32_t lv, Sig x) {
        const uint32_t w = g.in_u[e];
        const uint32_t* Fp = F + lev[lv];
        const uint32_t Lp = lev[lv + 1] - lev[lv];
        const uint32_t w1 = g.slot_ptr[w + 1];
        for (uint32_t p = lower_bound_u32(Fp, 0, Lp, g.slot_ptr[w]); p < Lp; ++p) {
            const uint32_t a2 = Fp[p];
            if (a2 >= w1 || g.slot_t[a2] >= t) break;
            SigOps<WIDE>::atomic_add(dl + lev[lv] + p, x);
        }
    };
    {   // level d: z's endpoint states (sh: all on level d, sfm: the earliest;
        // fsfm: z's earliest slot, on level d), count 1
        const uint32_t zs = g.slot_ptr[z], ze = g.slot_ptr[z + 1];
        const bool one = job.opt == 1 || job.opt == 3;
        const uint32_t a0 = one ? first : zs, a1 = one ? first + 1 : ze;
        for (uint32_t a = a0; a < a1; ++a) {
            if (job.opt != 3 && !((__ldcg(N + (a >> 5)) >> (a & 31)) & 1u)) continue;
            const uint32_t ta = g.slot_t[a];
            for (uint32_t e = g.slot_in[a] + tid; e < g.slot_in[a + 1]; e += BFS_NT) to_preds(e, ta, d - 1, (Sig)1);
        }
    }
    __syncthreads();
    for (uint32_t lv = d - 1; lv >= 2; --lv) {
        for (uint32_t p = lev[lv] + tid; p < lev[lv + 1]; p += BFS_NT) {
            const Sig x = ldcg_sig(dl + p);
            if (x == (Sig)0) continue;
            const uint32_t b = F[p], tb = g.slot_t[b];
            for (uint32_t e = g.slot_in[b]; e < g.slot_in[b + 1]; ++e) to_preds(e, tb, lv - 1, x);
        }
        __syncthreads();
    }
    // through counts per vertex; the first touch of v lists it (VB marks)
    // (a vertex's states of a level sit on consecutive lanes: one atomic per run)
    for (uint32_t lv = 1; lv < d; ++lv) {
        const uint32_t pe = lev[lv + 1];
        for (uint32_t p0 = lev[lv] + (uint32_t)(tid & ~31); p0 < pe; p0 += BFS_NT) {
            const uint32_t p = p0 + lane;
            uint32_t v = NONE;
            Sig val = (Sig)0;
            if (p < pe) {
                const Sig x = ldcg_sig(dl + p);
                v = g.slot_v[F[p]];
                if (x != (Sig)0) val = (Sig)(sigma_at(sig, F, g.slot_v, p, lev[lv]) * x);   // <= sigma_sz: no wrap
            }
            warp_run_add<Sig>(v, val, [&](uint32_t vv, Sig tot) {
                SigOps<WIDE>::atomic_add(acc + vv, tot);
                const uint32_t bit = 1u << (vv & 31);
                if (!(atomicOr(VB + (vv >> 5), bit) & bit)) tl[atomicAdd(sh_nt, 1u)] = vv;
            });
        }
    }
    __syncthreads();
    const uint32_t T = *sh_nt;
    u64 my_sum = 0;
    for (uint32_t p = tid; p < T; p += BFS_NT) {
        const uint32_t v = tl[p];
        const uint64_t q = ob_q(SigOps<WIDE>::wide(ldcg_sig(acc + v)), sigma);
        acc[v] = (Sig)q;
        atomicAnd(VB + (v >> 5), ~(1u << (v & 31)));
        my_sum += q;
    }
    __syncthreads();
    const uint32_t rows = 2 + (job.S64 ? job.c : 0);
    for (uint32_t it = tid; it < T * rows; it += BFS_NT) {
        const uint32_t p = it % T, row = it / T;
        const uint32_t v = tl[p];
        const uint64_t q = (uint64_t)acc[v];
        if (q) ob_term(job, v, q, row, rade);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) my_sum += __shfl_xor_sync(0xFFFFFFFFu, my_sum, o);
    if (lane == 0 && my_sum) atomicAdd(job.ctr + C_SUMINT, my_sum);
    __syncthreads();
    for (uint32_t p = tid; p < T; p += BFS_NT) acc[tl[p]] = (Sig)0;
}

// RTB update of one sample (App. C), all threads of the CTA, after a full
// search from s with levels 1 .. D in F.  The endpoint states of a vertex v
// are its states on its first level d_v (sfm: the earliest of them; fsfm: its
// earliest state at any level); eps(b) =
// sigma(b) / sigma_{s,v_b} for an endpoint b.  From level D down, every state
// b with X(b) = eps(b) + delta(b) > 0 adds round(sigma(a) X(b) / sigma(b)) to
// delta(a) of each DAG predecessor a; f_v(s) = round(sum of delta over v's
// states / (n-1)), all in 2^-32 units.  sig: running sums of the path counts
// by frontier position (see sigma_at); dl: per frontier position (scratch of
// the ob and RTB updates); sv: sigma_{s,v} (zero on entry and exit); dsum:
// per-vertex sums (zero on entry and exit); dv: first level per vertex (n
// entries, overwritten); VB: vertex bitmap (zero on entry and exit); tl: n
// entries.
template <bool WIDE, int BFS_NT>
__device__ __forceinline__ void bfs_rtb_update(const DevGraph& g, const Job& job, uint32_t s, uint64_t i, uint32_t D,
                                            uint32_t* rade, const uint32_t* F, const uint32_t* lev,
                                            const typename SigOps<WIDE>::T* sig, u64* dl, typename SigOps<WIDE>::T* sv,
                                            u64* dsum, uint32_t* dv, uint32_t* VB, uint32_t* tl, uint32_t* sh_nt) {
    typedef typename SigOps<WIDE>::T Sig;
    const int tid = threadIdx.x, lane = tid & 31;
    const uint32_t n = g.n;
    const bool sfm = job.opt == 1, fsfm = job.opt == 3;
    for (uint32_t v = tid; v < n; v += BFS_NT) dv[v] = NONE;
    if (tid == 0) {
        *sh_nt = 0;
        uint32_t w4[4];
        philox_block(job.seed, i, DOM_RADE, 0, w4);
        rade[0] = w4[0]; rade[1] = w4[1]; rade[2] = w4[2]; rade[3] = w4[3];
    }
    __syncthreads();
    // dv: first level of each vertex (fsfm: its earliest slot, the smallest id)
    for (uint32_t k = 1; k <= D; ++k)
        for (uint32_t p = lev[k] + tid; p < lev[k + 1]; p += BFS_NT) {
            const uint32_t a = F[p], v = g.slot_v[a];
            if (v != s) atomicMin(dv + v, fsfm ? a : k);
        }
    __syncthreads();
    // a level lists a vertex's states together, in time order
    auto is_end = [&](uint32_t p, uint32_t k, uint32_t v) -> bool {
        if (v == s) return false;
        if (fsfm) return F[p] == dv[v];
        if (dv[v] != k) return false;
        return !sfm || p == lev[k] || g.slot_v[F[p - 1]] != v;
    };
    for (uint32_t k = 1; k <= D; ++k) {
        const uint32_t pe = lev[k + 1];
        for (uint32_t p0 = lev[k] + (uint32_t)(tid & ~31); p0 < pe; p0 += BFS_NT) {   // one atomic per run
            const uint32_t p = p0 + lane;
            uint32_t v = NONE;
            Sig val = (Sig)0;
            if (p < pe) {
                v = g.slot_v[F[p]];
                if (is_end(p, k, v)) val = sigma_at(sig, F, g.slot_v, p, lev[k]);
            }
            warp_run_add<Sig>(v, val, [&](uint32_t vv, Sig tot) { SigOps<WIDE>::atomic_add(sv + vv, tot); });
        }
    }
    __syncthreads();
    auto eps_of = [&](uint32_t p, uint32_t k, uint32_t v) -> u64 {
        return is_end(p, k, v) ? ob_q(SigOps<WIDE>::wide(sigma_at(sig, F, g.slot_v, p, lev[k])),
                                      SigOps<WIDE>::wide(ldcg_sig(sv + v))) : 0ull;
    };
    for (uint32_t k = 1; k <= D; ++k)
        for (uint32_t p = lev[k] + tid; p < lev[k + 1]; p += BFS_NT) {
            dl[p] = eps_of(p, k, g.slot_v[F[p]]);
        }
    __syncthreads();
    for (uint32_t k = D; k >= 2; --k) {
        const uint32_t* Fp = F + lev[k - 1];
        const Sig* Sp = sig + lev[k - 1];
        const uint32_t Lp = lev[k] - lev[k - 1];
        for (uint32_t p = lev[k] + tid; p < lev[k + 1]; p += BFS_NT) {
            const u64 X = __ldcg(reinterpret_cast<const unsigned long long*>(dl + p));
            if (!X) continue;
            const uint32_t b = F[p], tb = g.slot_t[b];
            const u128 sb = SigOps<WIDE>::wide(sigma_at(sig, F, g.slot_v, p, lev[k]));
            for (uint32_t e = g.slot_in[b]; e < g.slot_in[b + 1]; ++e) {
                const uint32_t w = g.in_u[e], w1 = g.slot_ptr[w + 1];
                const uint32_t ph = lower_bound_u32(Fp, 0, Lp, g.slot_ptr[w]);   // w's first state on level k-1
                for (uint32_t p2 = ph; p2 < Lp; ++p2) {
                    const uint32_t a2 = Fp[p2];
                    if (a2 >= w1 || g.slot_t[a2] >= tb) break;
                    const Sig s2 = p2 == ph ? Sp[p2] : (Sig)(Sp[p2] - Sp[p2 - 1]);
                    const u64 term = muldiv_round(SigOps<WIDE>::wide(s2), X, sb);
                    if (term) atomicAdd(dl + lev[k - 1] + p2, term);
                }
            }
        }
        __syncthreads();
    }
    // per-vertex dependency sums (X minus the endpoint share)
    for (uint32_t k = 1; k <= D; ++k) {
        const uint32_t pe = lev[k + 1];
        for (uint32_t p0 = lev[k] + (uint32_t)(tid & ~31); p0 < pe; p0 += BFS_NT) {   // one atomic per run
            const uint32_t p = p0 + lane;
            uint32_t v = NONE;
            u64 val = 0;
            if (p < pe) {
                v = g.slot_v[F[p]];
                if (v != s) val = __ldcg(reinterpret_cast<const unsigned long long*>(dl + p)) - eps_of(p, k, v);
            }
            warp_run_add<u64>(v, val, [&](uint32_t vv, u64 tot) {
                atomicAdd(dsum + vv, tot);
                const uint32_t bit = 1u << (vv & 31);
                if (!(atomicOr(VB + (vv >> 5), bit) & bit)) tl[atomicAdd(sh_nt, 1u)] = vv;
            });
        }
    }
    __syncthreads();
    const uint32_t T = *sh_nt;
    u64 my_sum = 0;
    for (uint32_t p = tid; p < T; p += BFS_NT) {
        const uint32_t v = tl[p];
        const uint64_t q = muldiv_round(1, __ldcg(reinterpret_cast<const unsigned long long*>(dsum + v)), n - 1);
        dsum[v] = q;
        atomicAnd(VB + (v >> 5), ~(1u << (v & 31)));
        my_sum += q;
    }
    __syncthreads();
    const uint32_t rows = 2 + (job.S64 ? job.c : 0);
    for (uint32_t it = tid; it < T * rows; it += BFS_NT) {
        const uint32_t v = tl[it % T];
        const uint64_t q = dsum[v];
        if (q) ob_term(job, v, q, it / T, rade);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) my_sum += __shfl_xor_sync(0xFFFFFFFFu, my_sum, o);
    if (lane == 0 && my_sum) atomicAdd(job.ctr + C_SUMINT, my_sum);
    __syncthreads();
    for (uint32_t p = tid; p < T; p += BFS_NT) dsum[tl[p]] = 0ull;
    for (uint32_t v = tid; v < n; v += BFS_NT)
        if (dv[v] != NONE) sv[v] = (Sig)0;
}

// Algorithm 2 reach counts for fsfm after a full search from s with levels
// 1 .. D in F: the distance of v is the level of its earliest state (the
// fewest hops among the foremost paths).  dv: n entries, overwritten.
template <int BFS_NT>
__device__ __forceinline__ void bfs_fsfm_reach(const DevGraph& g, const Job& job, uint32_t s, uint32_t D,
                                               const uint32_t* F, const uint32_t* lev, uint32_t* dv) {
    const int tid = threadIdx.x, lane = tid & 31;
    for (uint32_t v = tid; v < g.n; v += BFS_NT) dv[v] = NONE;
    __syncthreads();
    for (uint32_t k = 1; k <= D; ++k)
        for (uint32_t p = lev[k] + tid; p < lev[k + 1]; p += BFS_NT) {
            const uint32_t a = F[p], v = g.slot_v[a];
            if (v != s) atomicMin(dv + v, a);
        }
    __syncthreads();
    for (uint32_t k = 1; k <= D; ++k) {
        uint32_t cnt = 0;
        for (uint32_t p0 = lev[k]; p0 < lev[k + 1]; p0 += BFS_NT) {
            const uint32_t p = p0 + tid;
            if (p < lev[k + 1]) {
                const uint32_t a = F[p], v = g.slot_v[a];
                if (v != s && dv[v] == a) {
                    ++cnt;
                    if (job.clos) atomicAdd(job.clos + v, recip32(k));
                }
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xFFFFFFFFu, cnt, o);
        if (lane == 0 && cnt) {
            atomicAdd(job.cnt + k, (u64)cnt);
            atomicMax(job.dmax, (u64)k);
        }
    }
    __syncthreads();
}

// Per-sample inputs of the fractional updates (ob, RTB) and the CTA's region
// arrays, kept in shared memory so that the out-of-line call carries two
// arguments.
struct FracCtx {
    const Task* task;
    const BfsWs* ws;
    uint32_t s, z, D, first, nt;
    uint64_t i;
    u128 sigma;
    uint32_t rade[4];
};

// The ob (mode 1) or RTB (mode 2) update of the CTA's current sample, or the
// fsfm reach counts of an Algorithm 2 search (mode 3); the
// region arrays are re-derived from the workspace.  Out of line, so that the
// search's register allocation does not carry it.
template <bool WIDE, int BFS_NT>
__device__ __noinline__ void bfs_frac_update(int mode, FracCtx* x) {
    typedef typename SigOps<WIDE>::T Sig;
    const DevGraph& g = x->task->g;
    const Job& job = x->task->job;
    const BfsWs& ws = *x->ws;
    char* region = ws.base + (size_t)blockIdx.x * ws.stride;
    const uint32_t* F = reinterpret_cast<const uint32_t*>(region + ws.o_f);
    const uint32_t* lev = reinterpret_cast<const uint32_t*>(region + ws.o_lev);
    const uint32_t* N = reinterpret_cast<const uint32_t*>(region + ws.o_nbits);
    uint32_t* seg_b = reinterpret_cast<uint32_t*>(region + ws.o_segb);
    uint32_t* seg_u = reinterpret_cast<uint32_t*>(region + ws.o_segu);
    uint32_t* VB = reinterpret_cast<uint32_t*>(region + ws.o_vb);
    Sig* sig = reinterpret_cast<Sig*>(region + ws.o_sig);
    Sig* Fc = reinterpret_cast<Sig*>(region + ws.o_fc);
    Sig* acc = reinterpret_cast<Sig*>(region + ws.o_acc);
    u64* acc2 = reinterpret_cast<u64*>(region + ws.o_acc2);
    if (mode == 1)
        bfs_ob_update<WIDE, BFS_NT>(g, job, x->z, x->D, x->first, x->sigma, x->rade, F, lev, N, sig, Fc, acc, VB,
                                    seg_u, &x->nt);
    else if (mode == 3)
        bfs_fsfm_reach<BFS_NT>(g, job, x->s, x->D, F, lev, seg_b);
    else
        bfs_rtb_update<WIDE, BFS_NT>(g, job, x->s, x->i, x->D, x->rade, F, lev, sig, reinterpret_cast<u64*>(Fc), acc,
                                     acc2, seg_b, VB, seg_u, &x->nt);
}

// BFS_NT threads per CTA, 1024 / BFS_NT CTAs per SM at 64 registers.  FRAC:
// the instantiation that also runs the ob and RTB updates and fsfm (a tick
// with such a problem launches it); the others report those jobs as a
// consistency error.
template <bool WIDE, int BFS_NT, bool FRAC>
__global__ void __launch_bounds__(BFS_NT, 1024 / BFS_NT) k_bfs(const Task* tasks, const uint64_t* unit_start,
                                                   const uint32_t* ntasks_p, u64* work,
                                                   const __grid_constant__ BfsWs ws) {
    typedef typename SigOps<WIDE>::T Sig;
    constexpr int BFS_NW = BFS_NT / 32;
    // frontier states whose times and running sums fit in shared memory.  Kept
    // small: with the visited bitmap of a 500k-slot graph, two 512-thread CTAs
    // then fit the 164 KB shared-memory carveout and the SM keeps 92 KB of L1
    // (the path-count and graph reads hit it); 4 * BFS_NT needed the 196 KB
    // carveout (60 KB of L1) and measured 4 % slower
    constexpr uint32_t FCAP = BFS_NT * 3 / 2;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    __shared__ __align__(16) Task sh_task;
    __shared__ int sh_t;

    char* region = ws.base + (size_t)blockIdx.x * ws.stride;
    // per frontier position: the state's path count, written by the count pass,
    // then replaced in place by the level's scan with the running sum over the
    // vertex's states of the level up to it (sigma_at recovers the count)
    Sig* Fs = reinterpret_cast<Sig*>(region + ws.o_sig);
    Sig* zsig = reinterpret_cast<Sig*>(region + ws.o_zsig);   // path counts of z's slots reached by the pull
    uint32_t* F = reinterpret_cast<uint32_t*>(region + ws.o_f);
    // per frontier position: the state's time and vertex, written by the count
    // pass with its path count (Algorithm 2 searches: the time by the scan)
    uint32_t* Ft = reinterpret_cast<uint32_t*>(region + ws.o_ft);
    uint32_t* Fu = reinterpret_cast<uint32_t*>(region + ws.o_fu);
    uint32_t* lev = reinterpret_cast<uint32_t*>(region + ws.o_lev);
    uint32_t* seg_b = reinterpret_cast<uint32_t*>(region + ws.o_segb);
    uint32_t* seg_u = reinterpret_cast<uint32_t*>(region + ws.o_segu);
    uint32_t* path = reinterpret_cast<uint32_t*>(region + ws.o_path);
    uint32_t* pathe = reinterpret_cast<uint32_t*>(region + ws.o_pathe);   // in-CSR index of path edge k
    uint32_t* VB = reinterpret_cast<uint32_t*>(region + ws.o_vb);   // vertex bitmap (stats)
    u64* segmap = reinterpret_cast<u64*>(region + ws.o_segmap);      // vertex -> (level stamp, frontier segment)
    Sig* acc = reinterpret_cast<Sig*>(region + ws.o_acc);             // ob: through counts per vertex
    u64* acc2 = reinterpret_cast<u64*>(region + ws.o_acc2);           // RTB: dependency sums per vertex
    uint32_t* stamp_p = reinterpret_cast<uint32_t*>(region + ws.o_stamp);

    extern __shared__ uint32_t dyn_smem[];
    uint32_t* V = ws.bits_in_smem ? dyn_smem : reinterpret_cast<uint32_t*>(region + ws.o_bits);   // visited
    uint32_t* N = reinterpret_cast<uint32_t*>(region + ws.o_nbits);   // next level (written by fire-and-forget atomics)

    __shared__ uint32_t sm_scan[32];
    __shared__ u64 sm_scan64[32];
    __shared__ Sig sm_segx[32];
    __shared__ uint32_t sm_segf[32];
    __shared__ Sig sh_carry;
    __shared__ Sig sm_lastx[BFS_NW];
    __shared__ Sig sh_cin;
    __shared__ uint32_t sh_scan_ovf;
    __shared__ uint32_t sm_wcnt[BFS_NW];
    __shared__ uint64_t sh_q;
    __shared__ uint32_t sh_found, sh_ovf, sh_err;
    __shared__ uint32_t sh_rade[4];
    __shared__ uint32_t sh_d, sh_len;
    __shared__ u128 sh_sigma;
    __shared__ uint32_t sh_first;
    __shared__ uint32_t sh_zbest, sh_zmin, sh_zlev;   // fsfm: earliest slot of z so far, and its level
    __shared__ FracCtx sh_fx;
    __shared__ uint32_t cs_off[BFS_NT + 1], cs_first[BFS_NT];   // range table
    __shared__ uint32_t sh_stamp, sh_wrap;
    __shared__ uint32_t sm_Ft[WIDE ? 1 : FCAP];   // level times and running sums (64-bit counts, L <= FCAP)
    __shared__ u64 sm_Fc[WIDE ? 1 : FCAP];
    // summary of the next-level bitmap: bit i is set when bitmap words
    // [i << sumshift, (i + 1) << sumshift) may hold a bit; the push marks it, the
    // compaction loads only marked words and clears it
    __shared__ uint32_t sm_nsum[SUMW];

    if (ws.bits_in_smem) {
        for (uint32_t w = tid; w < ws.bits_words; w += BFS_NT) V[w] = 0u;
    }
    for (uint32_t w = tid; w < SUMW; w += BFS_NT) sm_nsum[w] = 0u;
    if (tid == 0) sh_stamp = *stamp_p;
    // Next level stamp (segmap entries of older levels never match it) and the
    // level's scan scratch; on wrap-around the map is cleared once.
    auto advance_stamp = [&]() {
        if (tid == 0) {
            const uint32_t st = sh_stamp + 1u;
            sh_wrap = st == 0u;
            sh_stamp = st == 0u ? 1u : st;
            sh_carry = (Sig)0; sh_scan_ovf = 0;
        }
        __syncthreads();
        if (sh_wrap) {
            for (uint32_t v = tid; v < ws.n_cap; v += BFS_NT) segmap[v] = 0ull;
            __syncthreads();
        }
    };
    const uint32_t ntasks = *ntasks_p;
    // per-thread work counters, added to the current task's counters when the
    // CTA moves to another task and at exit
    u64* flush_ctr = nullptr;
    u64 my_escan = 0, my_eadd = 0, my_snew = 0, my_fseg = 0;
    auto flush = [&]() {
        if (!flush_ctr) return;
        if (my_escan) atomicAdd(flush_ctr + C_ESCAN, my_escan);
        if (my_eadd) atomicAdd(flush_ctr + C_EADD, my_eadd);
        if (my_snew) atomicAdd(flush_ctr + C_SNEW, my_snew);
        if (my_fseg) atomicAdd(flush_ctr + C_FSEG, my_fseg);
        my_escan = my_eadd = my_snew = my_fseg = 0;
    };
    __syncthreads();

    for (;;) {
        if (tid == 0) {
            const uint64_t u = atomicAdd(work, 1ull);
            int t = -1;
            if (ntasks > 0 && u < unit_start[ntasks]) {
                t = task_of_unit(unit_start, ntasks, u);
                sh_q = u - unit_start[t];
            }
            sh_t = t;
            sh_found = 0; sh_ovf = 0; sh_err = 0; sh_d = 0; sh_len = 0; sh_sigma = 0;
            sh_zbest = NONE; sh_zmin = NONE; sh_zlev = 0;
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
        const uint32_t n = g.n;
        const uint32_t words = (g.A + 31) >> 5;
        uint32_t sumshift = 0;             // smallest shift with every bitmap word covered by the summary
        while ((((words + (1u << sumshift) - 1u) >> sumshift) + 31u) / 32u > SUMW) ++sumshift;
        if (job.ctr != flush_ctr) { flush(); flush_ctr = job.ctr; }
        const uint64_t q = sh_q;
        const uint64_t i = job.idx_list ? job.idx_list[q] : job.i0 + q;

        uint32_t s, z;
        bool ok;
        if (job.stats || job.rtb) {       // a source only: Algorithm 2, or the RTB sample space V
            uint64_t x;
            ok = draw_below64(n, job.seed, i, job.stats ? DOM_STATS : job.dom_pair, &x);
            s = (uint32_t)x; z = NONE;
        } else {
            ok = draw_pair(n, job.seed, i, job.dom_pair, &s, &z);
        }
        if (!ok) { if (tid == 0) set_status(job.status, ST_RNG); s = 0; z = 1; }
        const bool stats = job.stats != 0;
        const bool full = stats || job.rtb;   // untruncated search (no target)
        // fsfm (foremost first, then fewest hops): no stop at z's first level;
        // every state up to z's latest in-edge time, the endpoint is z's
        // earliest slot found at any level (FRAC instantiation only)
        const bool fsfm = FRAC && job.opt == 3 && !full;
        const uint32_t tz = full ? NONE : g.tmax_in[z];
        const uint32_t zlo = fsfm ? g.slot_ptr[z] : 0u, zhi = fsfm ? g.slot_ptr[z + 1] : 0u;
        bool live = ok && (g.out_ptr[s + 1] > g.out_ptr[s]);
        if (!full && (g.slot_ptr[z + 1] == g.slot_ptr[z])) live = false;   // z has no in-edges

        // ---------------- level loop ----------------
        uint32_t k = 0;
        uint32_t L = 1;                 // |F_k| (level 0: the virtual source)
        uint32_t Fend = 0;              // end of the frontier lists (states of levels 1 .. k+1)
        if (tid == 0) { lev[0] = 0; lev[1] = 0; }
        __syncthreads();
        while (live) {
            // ---- segments of level k ----
            uint32_t G;
            // this level's frontier times and running sums: shared memory when they
            // fit (always for level 0, the virtual source, which has no position)
            const bool fsm = k == 0 || (!WIDE && L <= FCAP);
            uint32_t* const FtL = fsm ? sm_Ft : Ft + lev[k];
            Sig* const FsL = Fs + lev[k];
            Sig* const FcL = fsm ? reinterpret_cast<Sig*>(sm_Fc) : FsL;
            advance_stamp();
            const uint32_t stamp = sh_stamp;
            if (k == 0) {
                if (tid == 0) {
                    seg_b[0] = 0; seg_u[0] = s; FcL[0] = (Sig)1; FtL[0] = 0; my_fseg += 1;
                    segmap[s] = ((u64)stamp << 32);
                }
                __syncthreads();
                G = 1;
            } else {
                const uint32_t* Fk = F + lev[k];
                // B1: frontier attributes, segment heads and per-vertex running sums
                // of sigma.  Each thread takes IPT consecutive states of a tile: a
                // thread-local segmented scan, one block-wide segmented scan of the
                // thread aggregates, and the value carried into each thread.
                // The count pass left each state's vertex and time beside its count
                // (coalesced loads; large levels use the times in place); Algorithm 2
                // searches have no count pass and look them up from the slot ids.
                uint32_t gbase = 0;
                const uint32_t* const g_slot_v = g.slot_v;
                const uint32_t* const g_slot_t = g.slot_t;
                const uint32_t* const FuK = Fu + lev[k];
                const uint32_t* const FtK = Ft + lev[k];
                for (uint32_t it = 0; it < L; it += BFS_NT * IPT) {
                    const uint32_t i0 = it + (uint32_t)tid * IPT;
                    uint32_t uq[IPT];
                    Sig vq[IPT];
                    uint32_t uprev;
                    if (!stats) {
#pragma unroll
                        for (int q = 0; q < IPT; ++q) {
                            uq[q] = 0u; vq[q] = (Sig)0;
                            if (i0 + q < L) {
                                uq[q] = FuK[i0 + q];
                                if (fsm) FtL[i0 + q] = FtK[i0 + q];
                                vq[q] = FsL[i0 + q];
                            }
                        }
                        uprev = (i0 > 0 && i0 < L) ? FuK[i0 - 1] : NONE;
                    } else {
                        uint32_t aq[IPT];
#pragma unroll
                        for (int q = 0; q < IPT; ++q) aq[q] = (i0 + q < L) ? Fk[i0 + q] : 0u;
#pragma unroll
                        for (int q = 0; q < IPT; ++q) {
                            uq[q] = 0u; vq[q] = (Sig)0;
                            if (i0 + q < L) {
                                uq[q] = g_slot_v[aq[q]];
                                FtL[i0 + q] = g_slot_t[aq[q]];
                                vq[q] = FsL[i0 + q];
                            }
                        }
                        uprev = (i0 > 0 && i0 < L) ? g_slot_v[Fk[i0 - 1]] : NONE;
                    }
                    // heads (bit q): a state whose vertex differs from the previous state's
                    // (states past L are heads of value 0); agg = the thread's running sum
                    // since its last head
                    uint32_t hm = 0, nh = 0;
                    bool bad = false;
                    Sig agg = 0;
#pragma unroll
                    for (int q = 0; q < IPT; ++q) {
                        const uint32_t idx = i0 + q;
                        const uint32_t up = q == 0 ? uprev : uq[q - 1];
                        const bool h = (idx >= L) || idx == 0 || up != uq[q];
                        if (h) { hm |= 1u << q; agg = vq[q]; }
                        else { const Sig sm = agg + vq[q]; bad |= sm < agg; agg = sm; }
                        if (idx < L && h) ++nh;
                    }
                    if (tid == 0) sh_cin = sh_carry;          // carried into the tile
                    const Sig incl = block_segmented_scan<BFS_NT, Sig>(agg, hm != 0u, sm_segx, sm_segf, &sh_carry,
                                                                        &sh_scan_ovf);
                    // value carried into this thread: the previous thread's inclusive value
                    Sig run = shfl_up_w(incl, 1);
                    if (lane == 31) sm_lastx[wid] = incl;
                    __syncthreads();
                    if (lane == 0) run = wid ? sm_lastx[wid - 1] : sh_cin;
#pragma unroll
                    for (int q = 0; q < IPT; ++q) {
                        const uint32_t idx = i0 + q;
                        if ((hm >> q) & 1u) run = vq[q];
                        else { const Sig sm = run + vq[q]; bad |= sm < run; run = sm; }
                        if (idx < L) {
                            FcL[idx] = run;
                            if (fsm) FsL[idx] = run;   // the running sums stay in place for the draw and the updates
                        }
                    }
                    if (bad) sh_scan_ovf = 1u;
                    uint32_t tot;
                    uint32_t ex = block_exclusive_scan<BFS_NT>(nh, &tot, sm_scan);
#pragma unroll
                    for (int q = 0; q < IPT; ++q) {
                        const uint32_t idx = i0 + q;
                        if (idx < L && ((hm >> q) & 1u)) {
                            seg_b[gbase + ex] = idx; seg_u[gbase + ex] = uq[q];
                            segmap[uq[q]] = ((u64)stamp << 32) | (gbase + ex);
                            ++ex;
                        }
                    }
                    gbase += tot;
                }
                G = gbase;
                if (tid == 0) {
                    my_fseg += G;
                    if (sh_scan_ovf && !stats) sh_ovf = 1;
                }
                __syncthreads();
            }
            if (sh_ovf) break;

            // ---- pull: does level k reach z?  (z's slots keep their counts in zsig) ----
            if (!full && !fsfm) {
                const uint32_t zs = g.slot_ptr[z], ze = g.slot_ptr[z + 1];
                const uint32_t e_lo = g.slot_in[zs], e_hi = g.slot_in[ze];
                const uint32_t* const g_in_u = g.in_u;
                const uint32_t* const g_in_slot = g.in_slot;
                const uint32_t* const g_slot_t = g.slot_t;
                for (uint32_t e = e_lo + tid; e < e_hi; e += BFS_NT) {
                    const uint32_t w = g_in_u[e];
                    const uint32_t a = g_in_slot[e];
                    const uint32_t t = g_slot_t[a];
                    // frontier segment of w, if w is on this level
                    const u64 mw = __ldcg(segmap + w);
                    if ((uint32_t)(mw >> 32) == stamp) {
                        const uint32_t lo = (uint32_t)mw;
                        const uint32_t fb = seg_b[lo], fe = (lo + 1 < G) ? seg_b[lo + 1] : L;
                        bool have = true;
                        uint32_t idx = fb;
                        if (k > 0) {
                            const uint32_t c = lower_bound_u32(FtL, fb, fe, t);   // first Ft >= t
                            if (c == fb) have = false; else idx = c - 1;
                        }
                        if (have) {
                            if (!SigOps<WIDE>::atomic_add(zsig + (a - zs), FcL[idx])) sh_ovf = 1;
                            atomicOr(N + (a >> 5), 1u << (a & 31));
                            sh_found = 1;
                        }
                    }
                    ++my_escan;
                }
                __syncthreads();
                if (sh_found || sh_ovf) break;
            }

            // ---- push expansion of level k, BFS_NT segments per range table ----
            // candidate out-edges of segment gi (vertex u): first t > u's earliest
            // frontier time (every out-edge of s at level 0) up to the first t >= tz
            const uint32_t* const g_out_ptr = g.out_ptr;
            const uint32_t* const g_out_t = g.out_t;
            const uint32_t* const g_out_slot = g.out_slot;
            for (uint32_t c0 = 0; c0 < G; c0 += BFS_NT) {
                const uint32_t gi = c0 + tid;
                uint32_t lo2[2] = {0u, 0u}, hi2[2] = {0u, 0u}, key2[2] = {0u, 0u};
                if (gi < G) {
                    const uint32_t fb = seg_b[gi];
                    const uint32_t u = seg_u[gi];
                    const uint32_t r0 = g_out_ptr[u], r1 = g_out_ptr[u + 1];
                    lo2[0] = r0; hi2[0] = (k == 0) ? r0 : r1; key2[0] = (k == 0) ? 0u : FtL[fb];
                    lo2[1] = r0;
                    if (fsfm) { hi2[1] = r1; key2[1] = tz; }          // z's own appearances come from the push
                    else { hi2[1] = (tz == 0) ? r0 : r1; key2[1] = tz - 1u; }
                }
                upper_bounds<2>(g_out_t, lo2, hi2, key2);
                const uint32_t first = lo2[0], last = lo2[1];
                const uint32_t cand = (gi < G && last > first) ? last - first : 0u;
                u64 tot;
                const u64 ex = block_exclusive_scan64<BFS_NT>(((u64)(cand > 0 ? 1u : 0u) << 32) | cand, &tot,
                                                              sm_scan64);
                if (cand > 0) {
                    const uint32_t x = (uint32_t)(ex >> 32);
                    cs_first[x] = first; cs_off[x] = (uint32_t)ex;
                }
                const uint32_t Gc = (uint32_t)(tot >> 32), E = (uint32_t)tot;
                if (tid == 0) cs_off[Gc] = E;
                __syncthreads();
                const uint32_t per = ((E + BFS_NW * 32u - 1u) / (BFS_NW * 32u)) * 32u;
                const uint32_t w_lo = min((uint32_t)wid * per, E), w_hi = min(w_lo + per, E);
                lbs_walk_batched<WALK_K>(cs_off, Gc, cs_first, w_lo, w_hi, g_out_slot, g_out_t,
                                         [&](uint32_t, uint32_t, uint32_t a, uint32_t) {
                    ++my_escan;
                    if (!((V[a >> 5] >> (a & 31)) & 1u)) {
                        atomicOr(N + (a >> 5), 1u << (a & 31));
                        const uint32_t sb = (a >> 5) >> sumshift, m = 1u << (sb & 31);
                        if (!(sm_nsum[sb >> 5] & m)) atomicOr(sm_nsum + (sb >> 5), m);
                        ++my_eadd;
                    }
                });
                __syncthreads();
            }

            // ---- compact the next-level bitmap into F_{k+1} ----
            // Thread t owns the summary words [t q, (t + 1) q); only the bitmap
            // words that their set bits cover are loaded (CK loads in flight),
            // once to count and once to write.  Thread order is slot order, so
            // a block scan of the counts gives every thread its output offset.
            const uint32_t nsw = (((words + (1u << sumshift) - 1u) >> sumshift) + 31u) >> 5;
            const uint32_t q = (nsw + BFS_NT - 1) / BFS_NT;
            const uint32_t s_lo = min((uint32_t)tid * q, nsw), s_hi = min(s_lo + q, nsw);
            // body(w, N[w]) for every bitmap word w of this thread's marked groups, in order
            auto for_marked = [&](auto&& body) {
                for (uint32_t sw = s_lo; sw < s_hi; ++sw) {
                    uint32_t m = sm_nsum[sw];
                    if (sumshift == 0) {            // one bitmap word per summary bit
                        while (m) {
                            uint32_t w[CK], x[CK];
#pragma unroll
                            for (int j = 0; j < CK; ++j) {
                                w[j] = NONE;
                                if (m) { w[j] = (sw << 5) + (uint32_t)(__ffs(m) - 1); m &= m - 1; }
                            }
#pragma unroll
                            for (int j = 0; j < CK; ++j) x[j] = (w[j] != NONE) ? __ldcg(N + w[j]) : 0u;
#pragma unroll
                            for (int j = 0; j < CK; ++j) if (w[j] != NONE) body(w[j], x[j]);
                        }
                    } else {                        // 2^sumshift consecutive bitmap words per summary bit
                        while (m) {
                            const uint32_t g0 = ((sw << 5) + (uint32_t)(__ffs(m) - 1)) << sumshift;
                            m &= m - 1;
                            const uint32_t g1 = min(g0 + (1u << sumshift), words);
                            for (uint32_t w0 = g0; w0 < g1; w0 += CK) {
                                uint32_t x[CK];
#pragma unroll
                                for (int j = 0; j < CK; ++j) x[j] = (w0 + j < g1) ? __ldcg(N + w0 + j) : 0u;
#pragma unroll
                                for (int j = 0; j < CK; ++j) if (w0 + j < g1) body(w0 + j, x[j]);
                            }
                        }
                    }
                }
            };
            uint32_t cnt = 0;
            for_marked([&](uint32_t, uint32_t x) { cnt += __popc(x); });
            uint32_t Lnext;
            const uint32_t fbase = lev[k + 1];
            uint32_t off = fbase + block_exclusive_scan<BFS_NT>(cnt, &Lnext, sm_scan);
            uint32_t newv = 0;
            const uint32_t* const g_slot_v2 = g.slot_v;
            for_marked([&](uint32_t w, uint32_t bits) {
                if (!bits) return;
                V[w] |= bits;
                N[w] = 0u;
                while (bits) {
                    const uint32_t b = __ffs(bits) - 1;
                    bits &= bits - 1;
                    const uint32_t a = w * 32u + b;
                    F[off++] = a;
                    if (fsfm && a >= zlo && a < zhi) atomicMin(&sh_zmin, a);
                    if (stats && job.opt != 3) {
                        const uint32_t v = g_slot_v2[a];
                        if (v != s) {
                            const uint32_t old = atomicOr(VB + (v >> 5), 1u << (v & 31));
                            if (!(old & (1u << (v & 31)))) {
                                ++newv;
                                if (job.clos) atomicAdd(job.clos + v, recip32(k + 1));
                            }
                        }
                    }
                }
            });
            for (uint32_t sw = s_lo; sw < s_hi; ++sw) sm_nsum[sw] = 0u;   // read again by the next push, after barriers
            if (stats) {
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) newv += __shfl_xor_sync(0xFFFFFFFFu, newv, o);
                if (lane == 0 && newv) {
                    atomicAdd(job.cnt + (k + 1), (u64)newv);
                    atomicMax(job.dmax, (u64)(k + 1));
                }
            }
            if (tid == 0) lev[k + 2] = fbase + Lnext;
            if (tid == 0) my_snew += Lnext;
            Fend = fbase + Lnext;
            __syncthreads();
            if (fsfm && tid == 0 && sh_zmin < sh_zbest) { sh_zbest = sh_zmin; sh_zlev = k + 1; }
            if (Lnext == 0) break;

            // ---- count: sigma of each new state b = (v, t) is the sum, over its
            // in-edges (w, v, t) from level-k vertices, of the path counts of w's
            // level-k appearances earlier than t (the running sum up to the last
            // of them); stored at b's frontier position ----
            if (!stats) {
                const uint32_t* const c_slot_t = g.slot_t;
                const uint32_t* const c_slot_v = g.slot_v;
                const uint32_t* const c_slot_in = g.slot_in;
                const uint32_t* const c_in_u = g.in_u;
                // the count one in-edge (tail w, head time ta, w's map entry mw) adds
                auto term = [&](uint32_t ta, u64 mw, Sig* x) -> bool {
                    if ((uint32_t)(mw >> 32) != stamp) return false;         // w is not on level k
                    uint32_t idx = 0;                                        // level 0: the source, count 1
                    if (k > 0) {
                        const uint32_t lo = (uint32_t)mw;
                        const uint32_t fb = seg_b[lo], fe = (lo + 1 < G) ? seg_b[lo + 1] : L;
                        const uint32_t c = lower_bound_u32(FtL, fb, fe, ta);  // first Ft >= ta
                        if (c == fb) return false;                           // none earlier than ta
                        idx = c - 1;
                    }
                    *x = FcL[idx];
                    return true;
                };
                const uint32_t fend = fbase + Lnext;
                bool bad = false;
                // CB states per thread, each stage's loads issued for all of them
                // before any is used; a new state has at least one in-edge
                for (uint32_t p0 = fbase + tid; p0 < fend; p0 += BFS_NT * CB) {
                    uint32_t ta[CB], e0[CB], e1[CB], fb[CB], lo[CB], hi[CB], uv[CB];
                    u64 mw[CB];
                    // the state's slot, its time and in-edge range, the first
                    // in-edge's tail and its map entry
#pragma unroll
                    for (int j = 0; j < CB; ++j) {
                        const uint32_t p = p0 + (uint32_t)j * BFS_NT;
                        lo[j] = p < fend ? F[p] : NONE;
                    }
#pragma unroll
                    for (int j = 0; j < CB; ++j) {
                        ta[j] = e0[j] = e1[j] = uv[j] = 0u;
                        if (lo[j] != NONE) {
                            ta[j] = c_slot_t[lo[j]]; uv[j] = c_slot_v[lo[j]];
                            e0[j] = c_slot_in[lo[j]]; e1[j] = c_slot_in[lo[j] + 1];
                        }
                    }
#pragma unroll
                    for (int j = 0; j < CB; ++j) {
                        const uint32_t p = p0 + (uint32_t)j * BFS_NT;
                        if (p < fend) { Ft[p] = ta[j]; Fu[p] = uv[j]; }
                    }
#pragma unroll
                    for (int j = 0; j < CB; ++j) hi[j] = (e1[j] > e0[j]) ? c_in_u[e0[j]] : 0u;
#pragma unroll
                    for (int j = 0; j < CB; ++j) mw[j] = (e1[j] > e0[j]) ? __ldcg(segmap + hi[j]) : 0ull;
                    // the tail's segment on level k, then the first of its times >= ta
#pragma unroll
                    for (int j = 0; j < CB; ++j) {
                        const bool on = e1[j] > e0[j] && (uint32_t)(mw[j] >> 32) == stamp;
                        fb[j] = lo[j] = hi[j] = 0u;
                        if (on) {
                            if (k > 0) {
                                const uint32_t sg = (uint32_t)mw[j];
                                fb[j] = lo[j] = seg_b[sg];
                                hi[j] = (sg + 1 < G) ? seg_b[sg + 1] : L;
                            } else {
                                hi[j] = 1u;               // level 0: the source, count 1 (FcL[0])
                            }
                        }
                    }
                    if (k > 0) lower_bounds_rw<CB>(FtL, lo, hi, ta);
#pragma unroll
                    for (int j = 0; j < CB; ++j) {
                        if (e1[j] <= e0[j]) continue;
                        Sig sum = (Sig)0, x;
                        if (k == 0) { if (hi[j]) sum = FcL[0]; }
                        else if (lo[j] > fb[j]) sum = FcL[lo[j] - 1];
                        for (uint32_t e = e0[j] + 1; e < e1[j]; ++e) {
                            if (!term(ta[j], __ldcg(segmap + c_in_u[e]), &x)) continue;
                            const Sig s2 = sum + x;
                            bad |= s2 < sum;
                            sum = s2;
                        }
                        Fs[p0 + (uint32_t)j * BFS_NT] = sum;
                    }
                }
                if (bad) sh_ovf = 1;
                __syncthreads();
                if (sh_ovf) break;
            }
            k += 1;
            L = Lnext;
        }
        if (fsfm && tid == 0 && sh_zbest != NONE) sh_found = 1;
        __syncthreads();

        // ---------------- path draw (warp 0) ----------------
        const bool found = sh_found && !sh_ovf;
        if (found && wid == 0) {
            const uint32_t FULL = 0xFFFFFFFFu;
            const uint32_t d = fsfm ? sh_zlev : k + 1;
            const uint32_t zs = g.slot_ptr[z], ze = g.slot_ptr[z + 1];
            bool bad = false, err = false;
            // endpoints: z's slots on level d, ascending in time (sfm: the first
            // only; fsfm: z's earliest slot, on its own level d)
            uint32_t first = fsfm ? sh_zbest : NONE;
            for (uint32_t a0 = zs; a0 < ze && first == NONE; a0 += 32) {
                const uint32_t a = a0 + lane;
                const bool b = a < ze && ((__ldcg(N + (a >> 5)) >> (a & 31)) & 1u);
                const unsigned msk = __ballot_sync(FULL, b);
                if (msk) first = a0 + __ffs(msk) - 1;
            }
            // path count of an endpoint slot: sh / sfm from the pull's per-slot
            // counts; fsfm's endpoint is a frontier state of level d
            Sig zfs = 0;
            if (fsfm) {
                const uint32_t zpos = lev[d] + lower_bound_u32(F + lev[d], 0, lev[d + 1] - lev[d], first);
                zfs = sigma_at(Fs, F, g.slot_v, zpos, lev[d]);
            }
            auto end_sig = [&](uint32_t a) -> Sig { return fsfm ? zfs : ldcg_sig(zsig + (a - zs)); };
            Sig tot = 0;
            if (job.opt == 1 || fsfm) tot = end_sig(first);
            else {
                for (uint32_t a = zs + lane; a < ze; a += 32)
                    if ((__ldcg(N + (a >> 5)) >> (a & 31)) & 1u) { const Sig sm = tot + end_sig(a); bad |= sm < tot; tot = sm; }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const Sig y = shfl_xor_w(tot, o);
                    const Sig sm = tot + y;
                    bad |= sm < tot;
                    tot = sm;
                }
            }
            if (__any_sync(FULL, bad)) {
                if (lane == 0) sh_ovf = 1;
            } else if (job.ob) {
                // ob (Sec. 4.1): no draw; sigma_sz and the endpoints go to the ob update
                if (lane == 0) {
                    sh_d = d;
                    sh_first = first;
                    sh_sigma = SigOps<WIDE>::wide(tot);
                    uint32_t w4[4];
                    philox_block(job.seed, i, DOM_RADE, 0, w4);
                    sh_rade[0] = w4[0]; sh_rade[1] = w4[1]; sh_rade[2] = w4[2]; sh_rade[3] = w4[3];
                }
            } else {
                u128 x = 0;
                uint32_t rng_ok = 1;
                if (lane == 0) rng_ok = draw_below128(SigOps<WIDE>::wide(tot), job.seed, i, job.dom_path, &x) ? 1u : 0u;
                rng_ok = __shfl_sync(FULL, rng_ok, 0);
                Sig xs = shfl_idx_w((Sig)x, 0);
                if (!rng_ok) { err = true; if (lane == 0) set_status(job.status, ST_RNG); }
                uint32_t cur = NONE;
                const bool one = job.opt == 1 || fsfm;
                const uint32_t ze_end = one ? first + 1 : ze;
                for (uint32_t a0 = (one ? first : zs); !err && a0 < ze_end && cur == NONE; a0 += 32) {
                    const uint32_t a = a0 + lane;
                    const Sig wt = (a < ze_end && (fsfm || ((__ldcg(N + (a >> 5)) >> (a & 31)) & 1u))) ? end_sig(a) : (Sig)0;
                    const Sig incl = warp_inclusive_sum(wt);
                    const unsigned msk = __ballot_sync(FULL, xs < incl);
                    if (msk) {
                        const int l = __ffs(msk) - 1;
                        const Sig before = shfl_idx_w(incl - wt, l);
                        cur = a0 + l;
                        xs -= before;
                    } else {
                        xs -= shfl_idx_w(incl, 31);
                    }
                }
                if (cur == NONE) err = true;
                if (lane == 0) path[d] = z;
                uint32_t lvl = d;
                while (!err && lvl > 1) {
                    const uint32_t tv = g.slot_t[cur];
                    const uint32_t* Fp = F + lev[lvl - 1];
                    const Sig* Sp = Fs + lev[lvl - 1];
                    const uint32_t Lp = lev[lvl] - lev[lvl - 1];
                    const uint32_t e_lo = g.slot_in[cur], e_hi = g.slot_in[cur + 1];
                    uint32_t nxt = NONE;
                    for (uint32_t e0 = e_lo; e0 < e_hi && nxt == NONE; e0 += 32) {
                        const uint32_t e = e0 + lane;
                        // w's states on level lvl-1 earlier than tv are positions
                        // [p0, p1) from w's first (Sp: running sums from p0)
                        Sig wt = 0;
                        uint32_t p0 = 0, p1 = 0;
                        if (e < e_hi) {
                            const uint32_t w = g.in_u[e];
                            const uint32_t ws1 = g.slot_ptr[w + 1];
                            p0 = p1 = lower_bound_u32(Fp, 0, Lp, g.slot_ptr[w]);
                            while (p1 < Lp) {
                                const uint32_t a2 = Fp[p1];
                                if (a2 >= ws1 || g.slot_t[a2] >= tv) break;
                                ++p1;
                            }
                            if (p1 > p0) wt = Sp[p1 - 1];
                        }
                        const Sig incl = warp_inclusive_sum(wt);
                        const unsigned msk = __ballot_sync(FULL, xs < incl);
                        if (msk) {
                            const int l = __ffs(msk) - 1;
                            uint32_t pick = NONE;
                            Sig xr = xs - (incl - wt);
                            if (lane == l) {
                                for (uint32_t p = p0; p < p1; ++p) {
                                    if (xr < Sp[p]) {
                                        pick = Fp[p];
                                        if (p > p0) xr -= Sp[p - 1];
                                        break;
                                    }
                                }
                            }
                            nxt = __shfl_sync(FULL, pick, l);
                            xs = shfl_idx_w(xr, l);
                            if (nxt == NONE) err = true;
                            else if (lane == 0) pathe[lvl - 1] = e0 + l;
                            break;
                        }
                        xs -= shfl_idx_w(incl, 31);
                    }
                    if (nxt == NONE) { err = true; break; }
                    cur = nxt;
                    lvl -= 1;
                    if (lane == 0) path[lvl] = g.slot_v[cur];
                }
                if (lane == 0) {
                    path[0] = s;
                    if (!err) {   // the first edge: s's in-edge of the level-1 slot
                        const uint32_t e = lower_bound_u32(g.in_u, g.slot_in[cur], g.slot_in[cur + 1], s);
                        if (e < g.slot_in[cur + 1] && g.in_u[e] == s) pathe[0] = e;
                        else err = true;
                    }
                    if (err) { sh_err = 1; set_status(job.status, ST_CHECK); }
                    sh_d = d;
                    sh_len = d + 1;
                    sh_sigma = SigOps<WIDE>::wide(tot);
                    uint32_t w4[4];
                    philox_block(job.seed, i, DOM_RADE, 0, w4);
                    sh_rade[0] = w4[0]; sh_rade[1] = w4[1]; sh_rade[2] = w4[2]; sh_rade[3] = w4[3];
                }
            }
        }
        __syncthreads();

        if (sh_ovf) {
            if (tid == 0) {
                if (WIDE) set_status(job.status, ST_OVERFLOW);
                else push_overflow(job, i);
            }
        } else if (!sh_err) {
            const bool drawn = found && sh_len > 0 && !job.ob;
            // ---------------- hits and Rademacher sums ----------------
            const uint32_t nint = drawn ? family_count(job, sh_len) : 0u;
            if (job.hits && nint > 0) {
                const uint32_t rows = 1 + (job.S ? job.c : 0);
                for (uint32_t it = tid; it < nint * rows; it += BFS_NT) {
                    const uint32_t p = it % nint, j = it / nint;
                    const uint32_t x = family_item(job, g, path, pathe, p);
                    if (j == 0) atomicAdd(job.hits + x, 1ull);
                    else {
                        const uint32_t jj = j - 1;
                        const int lam = ((sh_rade[jj >> 5] >> (jj & 31)) & 1u) ? 1 : -1;
                        atomicAdd(job.S + (size_t)jj * job.fam + x, lam);
                    }
                }
                if (tid == 0) atomicAdd(job.ctr + C_SUMINT, (u64)nint);
            }
            // ---------------- per-sample record ----------------
            if (job.rec_len) {
                const uint64_t r = i - job.i0;
                const uint32_t len = drawn ? sh_len : 0;
                if (tid == 0) {
                    job.rec_s[r] = s; job.rec_z[r] = z;
                    job.rec_sig[2 * r] = (u64)sh_sigma; job.rec_sig[2 * r + 1] = (u64)(sh_sigma >> 64);
                    job.rec_len[r] = len;
                }
                for (uint32_t p = tid; p < len && p < job.rec_cap; p += BFS_NT)
                    job.rec_nodes[r * job.rec_cap + p] = path[p];
                if (job.rec_edges)
                    for (uint32_t p = tid; p + 1 < len && p < job.rec_cap; p += BFS_NT)
                        job.rec_edges[r * job.rec_cap + p] = pathe[p];
            }
        }

        // ---------------- ob (Sec. 4.1) and RTB (App. C) updates (block-uniform conditions) ----------------
        if constexpr (!FRAC) {
            if ((job.ob || job.rtb || job.opt == 3) && tid == 0) set_status(job.status, ST_CHECK);
        } else {
            const int mode = (job.ob && job.hits && found && !sh_ovf && !sh_err && sh_d >= 2) ? 1
                           : (job.rtb && job.hits && live && !sh_ovf && k >= 2) ? 2
                           : (stats && job.opt == 3 && live && k >= 1) ? 3 : 0;
            if ((mode == 1 || mode == 2) && !ws.has_dl) {
                if (tid == 0) set_status(job.status, ST_CHECK);   // a workspace without the updates' scratch
            } else if (mode) {
                if (tid == 0) {
                    FracCtx& x = sh_fx;
                    x.task = &sh_task; x.ws = &ws;
                    x.s = s; x.z = z; x.i = i; x.D = mode == 1 ? sh_d : k; x.first = sh_first; x.sigma = sh_sigma;
                    x.rade[0] = sh_rade[0]; x.rade[1] = sh_rade[1]; x.rade[2] = sh_rade[2]; x.rade[3] = sh_rade[3];
                }
                __syncthreads();
                bfs_frac_update<WIDE, BFS_NT>(mode, &sh_fx);
            }
        }

        // ---------------- cleanup: z's slot counts, the bitmaps ----------------
        // Every compaction cleared the next-level bitmap, so only the pull's bits
        // (z's slots) can be left in it; the visited bitmap holds exactly the
        // states of F[0 .. Fend).
        if (live && !full && !fsfm) {
            const uint32_t zs = g.slot_ptr[z], ze = g.slot_ptr[z + 1];   // ze > zs: z has an in-edge
            for (uint32_t w = (zs >> 5) + tid; w <= ((ze - 1) >> 5); w += BFS_NT) {
                uint32_t bits = __ldcg(N + w);
                if (!bits) continue;
                N[w] = 0u;
                while (bits) {
                    const uint32_t b = __ffs(bits) - 1;
                    bits &= bits - 1;
                    const uint32_t a = w * 32u + b;
                    if (a >= zs && a < ze) zsig[a - zs] = (Sig)0;
                }
            }
        }
        if (ws.bits_in_smem || Fend >= words) {
            for (uint32_t w = tid; w < words; w += BFS_NT) V[w] = 0u;
        } else {
            for (uint32_t p = tid; p < Fend; p += BFS_NT) V[F[p] >> 5] = 0u;
        }
        if (stats) {
            for (uint32_t w = tid; w < (n + 31) / 32; w += BFS_NT) VB[w] = 0u;
        }
        __syncthreads();
    }
    flush();
    if (tid == 0) *stamp_p = sh_stamp;
}

// Host-side launch helpers -------------------------------------------------

// Region of one CTA.  The visited bitmap is in shared memory when
// bits_in_smem; the next-level bitmap is always in the region.  The path
// counts take one entry per frontier position (at most A states per search)
// plus one per slot of z (at most zcap, the largest slot count of a vertex).
// With dl, the scratch of the ob and RTB updates (one entry per position and
// two per vertex) is added.
size_t bfs_region_bytes(uint32_t n, uint32_t A, uint32_t zcap, bool bits_in_smem, bool dl, BfsWs* ws) {
    ws->bits_words = (A + 31) / 32;
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    size_t o = 0;
    ws->o_sig = o;     o = al(o + (size_t)A * 16);
    ws->o_zsig = o;    o = al(o + (size_t)std::max<uint32_t>(zcap, 1) * 16);
    ws->o_fc = ws->o_acc = ws->o_acc2 = 0;
    ws->has_dl = dl ? 1 : 0;
    if (dl) {
        ws->o_fc = o;      o = al(o + (size_t)(A + 1) * 16);
        ws->o_acc = o;     o = al(o + (size_t)n * 16);
        ws->o_acc2 = o;    o = al(o + (size_t)n * 8);
    }
    ws->o_f = o;       o = al(o + (size_t)(A + 1) * 4);
    ws->o_ft = o;      o = al(o + (size_t)(A + 1) * 4);
    ws->o_fu = o;      o = al(o + (size_t)(A + 1) * 4);
    ws->o_lev = o;     o = al(o + (size_t)(n + 3) * 4);
    ws->o_segb = o;    o = al(o + (size_t)(n + 2) * 4);
    ws->o_segu = o;    o = al(o + (size_t)(n + 2) * 4);
    ws->o_path = o;    o = al(o + (size_t)(n + 2) * 4);
    ws->o_pathe = o;   o = al(o + (size_t)(n + 2) * 4);
    ws->o_vb = o;      o = al(o + (size_t)((n + 31) / 32 + 1) * 4);
    ws->o_segmap = o;  o = al(o + (size_t)n * 8);
    ws->o_stamp = o;   o = al(o + 4);
    ws->o_nbits = o;   o = al(o + (size_t)ws->bits_words * 4);
    ws->n_cap = n;
    ws->o_bits = o;
    if (!bits_in_smem) o = al(o + (size_t)ws->bits_words * 4);
    ws->bits_in_smem = bits_in_smem ? 1 : 0;
    return o;
}

size_t bfs_smem_bytes(uint32_t A) { return (size_t)((A + 31) / 32) * 4; }

// Static shared memory of the nt-thread kernels (range table, task copy,
// level scratch).
size_t bfs_static_smem(int nt) {
    cudaFuncAttributes a{}, b{}, c{};
    const cudaError_t e1 = nt == 1024 ? cudaFuncGetAttributes(&a, k_bfs<false, 1024, false>)
                         : nt == 256  ? cudaFuncGetAttributes(&a, k_bfs<false, 256, false>)
                                      : cudaFuncGetAttributes(&a, k_bfs<false, 512, false>);
    const cudaError_t e2 = nt == 1024 ? cudaFuncGetAttributes(&b, k_bfs<true, 1024, true>)
                         : nt == 256  ? cudaFuncGetAttributes(&b, k_bfs<true, 256, true>)
                                      : cudaFuncGetAttributes(&b, k_bfs<true, 512, true>);
    const cudaError_t e3 = nt == 1024 ? cudaFuncGetAttributes(&c, k_bfs<false, 1024, true>)
                         : nt == 256  ? cudaFuncGetAttributes(&c, k_bfs<false, 256, true>)
                                      : cudaFuncGetAttributes(&c, k_bfs<false, 512, true>);
    if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess) return 96 * 1024;
    return std::max(std::max(a.sharedSizeBytes, b.sharedSizeBytes), c.sharedSizeBytes);
}

// Raises (never lowers) the kernels' dynamic shared-memory limit on the
// current device, so callers with different graph sizes do not undo each
// other's setting.  The attribute is per device, so is the record of it.
cudaError_t bfs_configure(size_t smem) {
    static std::mutex mu;
    static size_t configured[64] = {};
    int dev = 0;
    const cudaError_t ed = cudaGetDevice(&dev);
    if (ed != cudaSuccess) return ed;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(mu);
    if (smem <= configured[dev]) return cudaSuccess;
    const void* ks[9] = {(const void*)k_bfs<false, 512, false>, (const void*)k_bfs<false, 512, true>,
                         (const void*)k_bfs<true, 512, true>, (const void*)k_bfs<false, 1024, false>,
                         (const void*)k_bfs<false, 1024, true>, (const void*)k_bfs<true, 1024, true>,
                         (const void*)k_bfs<false, 256, false>, (const void*)k_bfs<false, 256, true>,
                         (const void*)k_bfs<true, 256, true>};
    for (const void* k : ks) {
        const cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    configured[dev] = smem;
    return cudaSuccess;
}

cudaError_t bfs_blocks_per_sm(int nt, size_t smem, int* out) {
    if (nt == 1024) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, k_bfs<false, 1024, false>, 1024, smem);
    if (nt == 256) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, k_bfs<false, 256, false>, 256, smem);
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, k_bfs<false, 512, false>, 512, smem);
}

cudaError_t launch_bfs(const Task* tasks, const uint64_t* unit_start, const uint32_t* ntasks, u64* work,
                       const BfsWs& ws, int grid, size_t smem, bool wide, bool frac, cudaStream_t st) {
    // the 128-bit re-run always takes the FRAC instantiation
    if (ws.nt == 1024) {
        if (wide) k_bfs<true, 1024, true><<<grid, 1024, smem, st>>>(tasks, unit_start, ntasks, work, ws);
        else if (frac) k_bfs<false, 1024, true><<<grid, 1024, smem, st>>>(tasks, unit_start, ntasks, work, ws);
        else k_bfs<false, 1024, false><<<grid, 1024, smem, st>>>(tasks, unit_start, ntasks, work, ws);
    } else if (ws.nt == 256) {
        if (wide) k_bfs<true, 256, true><<<grid, 256, smem, st>>>(tasks, unit_start, ntasks, work, ws);
        else if (frac) k_bfs<false, 256, true><<<grid, 256, smem, st>>>(tasks, unit_start, ntasks, work, ws);
        else k_bfs<false, 256, false><<<grid, 256, smem, st>>>(tasks, unit_start, ntasks, work, ws);
    } else {
        if (wide) k_bfs<true, 512, true><<<grid, 512, smem, st>>>(tasks, unit_start, ntasks, work, ws);
        else if (frac) k_bfs<false, 512, true><<<grid, 512, smem, st>>>(tasks, unit_start, ntasks, work, ws);
        else k_bfs<false, 512, false><<<grid, 512, smem, st>>>(tasks, unit_start, ntasks, work, ws);
    }
    return cudaGetLastError();
}

}  // namespace mantra
