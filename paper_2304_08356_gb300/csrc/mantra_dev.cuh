// Internal device-side declarations of the MANTRA GB300 library.
//
// Graph store (built once at load, resident in HBM):
//   out-CSR  by (u, t, v): out_ptr[n+1], out_v[m], out_t[m], out_slot[m]
//   slots    distinct arrival appearances (v, t) sorted by (v, t):
//            slot_ptr[n+1], slot_t[A], slot_v[A], slot_in[A+1]
//   in-CSR   by (v, t, u): in_u[m], in_slot[m]  (slot a's in-edges are
//            in_u[slot_in[a] .. slot_in[a+1]), ascending u); the in-CSR index
//            of an edge is its temporal-edge id, in_uedge[m] the id of its
//            underlying edge (u, v) (rank of (v, u) among the distinct pairs)
//   stream   by (t, u, v): st_u[m], st_v[m], st_t[m]
//   tmax_in[n]  latest in-edge time of v (valid when v has a slot)
//   tmin_out[n] earliest out-edge time of u (valid when u has out-edges)
//   slot_nout[A] first out-edge of v later than slot (v, t): out-row index
//   out_loff[m]  16-bit: out_slot[e] - slot_ptr[out_v[e]] (clamped to 0xFFFF)
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace mantra {

typedef unsigned long long u64;
typedef unsigned __int128 u128;

// Random-stream domains: word 2 of the Philox counter.
enum : uint32_t { DOM_PAIR = 0, DOM_PATH = 1, DOM_RADE = 2, DOM_BOOT_PAIR = 3, DOM_BOOT_PATH = 4, DOM_STATS = 5 };
constexpr uint32_t RNG_MAX_ATTEMPTS = 1u << 16;
constexpr uint32_t NONE = 0xFFFFFFFFu;

// Device status word values (same numbers as the public error codes).
enum : int { ST_OK = 0, ST_OVERFLOW = 3, ST_TIMEOUT = 5, ST_CHECK = 6, ST_RNG = 7 };

// Counter slots of a launch (u64 each).
// C_FSEG: sh/sfm frontier vertices; CTA pfm kernel: frontier rounds.
// C_XEDGE: CTA pfm kernel, out-edges of the arrival expansions plus the DAG
// edges of the Kahn pass; diagnostics only.
enum : int { C_WORK = 0, C_SUMINT = 1, C_ESCAN = 2, C_EADD = 3, C_SNEW = 4, C_NOVF = 5, C_FSEG = 6, C_XEDGE = 7,
             C_NCOUNT = 8 };

struct DevGraph {
    uint32_t n;
    uint32_t A;       // number of arrival slots
    uint32_t m;       // deduplicated temporal edges
    const uint32_t* out_ptr;
    const uint32_t* out_v;
    const uint32_t* out_t;
    const uint32_t* out_slot;
    const uint32_t* slot_ptr;
    const uint32_t* slot_t;
    const uint32_t* slot_v;
    const uint32_t* slot_in;
    const uint32_t* in_u;
    const uint32_t* in_slot;
    const uint32_t* st_u;
    const uint32_t* st_v;
    const uint32_t* st_t;
    const uint32_t* tmax_in;
    const uint32_t* tmin_out;
    uint32_t cbound;  // sum over v of the largest in-edge count of v's slots: bounds the
                      // path-count additions of one prefix-foremost search
    uint32_t max_slot_in;   // largest in-edge count of one arrival slot
    const uint32_t* in_uedge;
    uint32_t n_uedge;       // distinct ordered pairs (u, v) with a temporal edge
    uint32_t max_vslots;    // largest number of arrival slots of one vertex
    const uint32_t* slot_nout;   // per arrival slot (v, t): first index of v's out-row with time > t
    const unsigned short* out_loff;   // per out-edge: its head's slot offset within the head's slots
                                      // (out_slot - slot_ptr[out_v], 0xFFFF when above)
};

// Largest number of arrival slots of one vertex for the CTA pfm kernel's
// 16-bit state (offsets 0xFFFE and 0xFFFF are reserved).
constexpr uint32_t PFM_W16_MAX_VSLOTS = 0xFFFEu;

// One launch over a range (or list) of sample indices.
struct Job {
    uint64_t seed;
    uint64_t i0;               // sample index of position 0
    uint64_t count;            // number of samples in this launch
    const uint64_t* idx_list;  // optional: explicit sample indices (count entries)
    uint32_t dom_pair, dom_path;
    int opt;                   // 0 sh, 1 sfm, 2 pfm
    uint32_t c;                // Rademacher trials (S updated when S != nullptr)
    int target;                // estimated family: 0 nodes, 1 underlying edges, 2 temporal edges
    uint32_t fam;              // its size F (n, n_uedge or m)
    u64* hits;                 // F, or nullptr: no accumulation
    int* S;                    // c*F, row j at S + j*F, or nullptr
    // ob estimator (Sec. 4.1; nodes only): instead of the drawn path's hits,
    // every internal vertex v of an optimal path gets q = 2^32 sigma_sz(v) /
    // sigma_sz rounded to nearest (ties up): hits[v] += q, wsq[v] += q^2 / 2^32
    // (rounded the same way), S64[j][v] += lambda_j q.  No path is drawn.
    int ob;
    // RTB estimator (App. C; nodes only): sample i is a source s (uniform over
    // the n vertices, pair domain); a full search and a backward dependency
    // accumulation give f_v(s) = 1/(n-1) sum_z sigma_sz(v) / sigma_sz, added
    // like the ob values (every term in 2^-32 units).
    int rtb;
    u64* wsq;                  // F (ob, RTB)
    long long* S64;            // c*F (ob, RTB), or nullptr
    u64* ctr;                  // C_NCOUNT counters
    uint64_t* ovf_list;        // sample indices whose 64-bit path counts overflowed
    int* status;
    // optional per-sample records, indexed by (sample index - i0)
    uint32_t* rec_s;
    uint32_t* rec_z;
    u64* rec_sig;              // 2 per sample: low, high 64 bits of sigma_sz
    uint32_t* rec_len;         // number of path vertices (0 if unreachable)
    uint32_t* rec_nodes;       // rec_cap per sample, s .. z
    uint32_t* rec_edges;       // optional: rec_cap per sample, the path's temporal-edge ids from s
    uint32_t rec_cap;
    // Algorithm 2 mode: full searches from sources, reach histogram per hop
    int stats;
    u64* cnt;                  // n+1
    u64* dmax;
    u64* clos;                 // or nullptr: n, per vertex sum over the searches of recip32(distance)
};

// One entry of a launch's task table: a graph and a range of its samples.
struct Task {
    DevGraph g;
    Job job;
};
static_assert(sizeof(Task) % 8 == 0, "Task is copied as 8-byte words");

// Task of work unit u: the last t with unit_start[t] <= u (unit_start ascending,
// ntasks + 1 entries).
__device__ __forceinline__ int task_of_unit(const uint64_t* unit_start, uint32_t ntasks, uint64_t u) {
    uint32_t lo = 0, hi = ntasks;          // unit_start[lo] <= u < unit_start[hi]
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (unit_start[mid] <= u) lo = mid; else hi = mid;
    }
    return (int)lo;
}

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), device side.
// Counter (i_lo, i_hi, domain, attempt), key (seed_lo, seed_hi).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void philox_block(uint64_t seed, uint64_t i, uint32_t dom, uint32_t attempt,
                                             uint32_t out[4]) {
    uint32_t x0 = (uint32_t)i, x1 = (uint32_t)(i >> 32), x2 = dom, x3 = attempt;
    uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t a = 0xD2511F53u * x0, ah = __umulhi(0xD2511F53u, x0);
        const uint32_t b = 0xCD9E8D57u * x2, bh = __umulhi(0xCD9E8D57u, x2);
        const uint32_t y0 = bh ^ x1 ^ k0, y2 = ah ^ x3 ^ k1;
        x0 = y0; x1 = b; x2 = y2; x3 = a;
        k0 += 0x9E3779B9u; k1 += 0xBB67AE85u;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

// Uniform in [0, N) (N >= 1): low 64 bits of a block masked to the smallest
// all-ones value >= N-1, rejected when >= N (next attempt counter).
__device__ __forceinline__ bool draw_below64(uint64_t N, uint64_t seed, uint64_t i, uint32_t dom, uint64_t* x) {
    const uint64_t span = N - 1;
    const uint64_t mask = span ? (~0ull >> __clzll((long long)span)) : 0ull;
    for (uint32_t att = 0; att < RNG_MAX_ATTEMPTS; ++att) {
        uint32_t w[4];
        philox_block(seed, i, dom, att, w);
        const uint64_t val = (((uint64_t)w[1] << 32) | w[0]) & mask;
        if (val < N) { *x = val; return true; }
    }
    return false;
}

// Same over all 128 bits of the block.
__device__ __forceinline__ bool draw_below128(u128 N, uint64_t seed, uint64_t i, uint32_t dom, u128* x) {
    const u128 span = N - 1;
    const uint64_t sh = (uint64_t)(span >> 64), sl = (uint64_t)span;
    u128 mask;
    if (sh) mask = ((u128)(~0ull >> __clzll((long long)sh)) << 64) | (u128)~0ull;
    else mask = sl ? (u128)(~0ull >> __clzll((long long)sl)) : (u128)0;
    for (uint32_t att = 0; att < RNG_MAX_ATTEMPTS; ++att) {
        uint32_t w[4];
        philox_block(seed, i, dom, att, w);
        const u128 val = (((u128)w[3] << 96) | ((u128)w[2] << 64) | ((u128)w[1] << 32) | (u128)w[0]) & mask;
        if (val < N) { *x = val; return true; }
    }
    return false;
}

// Ordered pair (s, z), s != z, uniform over the n(n-1) choices.
__device__ __forceinline__ bool draw_pair(uint32_t n, uint64_t seed, uint64_t i, uint32_t dom, uint32_t* s,
                                          uint32_t* z) {
    uint64_t x;
    if (!draw_below64((uint64_t)n * (uint64_t)(n - 1), seed, i, dom, &x)) return false;
    const uint64_t a = x / (uint64_t)(n - 1), b = x - a * (uint64_t)(n - 1);
    *s = (uint32_t)a;
    *z = (uint32_t)(b + (b >= a ? 1 : 0));
    return true;
}

// ---------------------------------------------------------------------------
// Path-count arithmetic: 64-bit fast path and 128-bit wide path.
// ---------------------------------------------------------------------------
template <bool WIDE> struct SigOps;

template <> struct SigOps<false> {
    typedef u64 T;
    __device__ static __forceinline__ bool add(T a, T b, T* r) { *r = a + b; return *r >= a; }
    // atomic sig[a] += v; returns false when the true sum no longer fits
    __device__ static __forceinline__ bool atomic_add(T* p, T v) {
        const T old = atomicAdd(p, v);
        return old + v >= old;
    }
    __device__ static __forceinline__ u128 wide(T a) { return (u128)a; }
};

template <> struct SigOps<true> {
    typedef u128 T;
    __device__ static __forceinline__ bool add(T a, T b, T* r) { *r = a + b; return *r >= a; }
    __device__ static __forceinline__ bool atomic_add(T* p, T v) {
        u64* w = reinterpret_cast<u64*>(p);
        const u64 lo = (u64)v, hi = (u64)(v >> 64);
        const u64 old_lo = atomicAdd(w, lo);
        const u64 carry = (old_lo + lo < old_lo) ? 1ull : 0ull;
        const u64 add_hi = hi + carry;
        if (add_hi == 0) return !(hi == ~0ull && carry);   // hi + carry wrapped to 0 only if hi was all ones
        const u64 old_hi = atomicAdd(w + 1, add_hi);
        return old_hi + add_hi >= old_hi;
    }
    __device__ static __forceinline__ u128 wide(T a) { return a; }
};

// Block-wide exclusive scan of one uint32 per thread.  NT threads; `scratch`
// holds 32 words of shared memory.  Every thread gets its prefix and the
// total.  Contains barriers: call from block-uniform control flow only.
template <int NT>
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* total, uint32_t* scratch) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) scratch[wid] = x;
    __syncthreads();
    if (wid == 0) {
        uint32_t w = (lane < NT / 32) ? scratch[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, w, o);
            if (lane >= o) w += y;
        }
        scratch[lane] = w;
    }
    __syncthreads();
    const uint32_t before = wid ? scratch[wid - 1] : 0u;
    *total = scratch[NT / 32 - 1];
    __syncthreads();
    return before + x - v;
}

// Loads through L2 (skipping L1) of path counts written by atomics.
__device__ __forceinline__ u64 ldcg_sig(const u64* p) { return __ldcg(reinterpret_cast<const unsigned long long*>(p)); }
__device__ __forceinline__ u128 ldcg_sig(const u128* p) {
    const unsigned long long* w = reinterpret_cast<const unsigned long long*>(p);
    return ((u128)__ldcg(w + 1) << 64) | (u128)__ldcg(w);
}

// Warp shuffles of 64- and 128-bit path counts.
__device__ __forceinline__ u64 shfl_up_w(u64 x, int o) { return __shfl_up_sync(0xFFFFFFFFu, x, o); }
__device__ __forceinline__ u128 shfl_up_w(u128 x, int o) {
    const u64 lo = __shfl_up_sync(0xFFFFFFFFu, (u64)x, o), hi = __shfl_up_sync(0xFFFFFFFFu, (u64)(x >> 64), o);
    return ((u128)hi << 64) | lo;
}
__device__ __forceinline__ u64 shfl_idx_w(u64 x, int l) { return __shfl_sync(0xFFFFFFFFu, x, l); }
__device__ __forceinline__ u128 shfl_idx_w(u128 x, int l) {
    const u64 lo = __shfl_sync(0xFFFFFFFFu, (u64)x, l), hi = __shfl_sync(0xFFFFFFFFu, (u64)(x >> 64), l);
    return ((u128)hi << 64) | lo;
}
__device__ __forceinline__ u64 shfl_down_w(u64 x, int o) { return __shfl_down_sync(0xFFFFFFFFu, x, o); }
__device__ __forceinline__ u128 shfl_down_w(u128 x, int o) {
    const u64 lo = __shfl_down_sync(0xFFFFFFFFu, (u64)x, o), hi = __shfl_down_sync(0xFFFFFFFFu, (u64)(x >> 64), o);
    return ((u128)hi << 64) | lo;
}
__device__ __forceinline__ u64 shfl_xor_w(u64 x, int o) { return __shfl_xor_sync(0xFFFFFFFFu, x, o); }
__device__ __forceinline__ u128 shfl_xor_w(u128 x, int o) {
    const u64 lo = __shfl_xor_sync(0xFFFFFFFFu, (u64)x, o), hi = __shfl_xor_sync(0xFFFFFFFFu, (u64)(x >> 64), o);
    return ((u128)hi << 64) | lo;
}

// Warp-aggregated addition for runs of lanes: consecutive lanes holding the
// same key form a run (a frontier lists a vertex's states next to each other),
// a segmented reduction over each run sums their values, and the run's first
// lane calls add(key, total) -- one atomic per run instead of one per lane.
// Lanes with nothing to add pass x = 0 (whatever their key, they change no
// total).  Every lane of the warp calls it.
template <typename T, typename AddF>
__device__ __forceinline__ void warp_run_add(uint32_t key, T x, AddF add) {
    const int lane = threadIdx.x & 31;
    T sum = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const T y = shfl_down_w(sum, o);
        const uint32_t ky = __shfl_down_sync(0xFFFFFFFFu, key, o);
        if (lane + o < 32 && ky == key) sum += y;
    }
    const uint32_t kp = __shfl_up_sync(0xFFFFFFFFu, key, 1);
    if ((lane == 0 || kp != key) && sum != (T)0) add(key, sum);
}

// Inclusive warp scan of unsigned path counts (callers guarantee no wrap).
template <typename T>
__device__ __forceinline__ T warp_inclusive_sum(T x) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const T y = shfl_up_w(x, o);
        if (lane >= o) x += y;
    }
    return x;
}

// Block-wide exclusive scan of one uint64 per thread (same contract as the
// 32-bit scan; `scratch` holds 32 uint64 of shared memory).
template <int NT>
__device__ __forceinline__ u64 block_exclusive_scan64(u64 v, u64* total, u64* scratch) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    u64 x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const u64 y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) scratch[wid] = x;
    __syncthreads();
    if (wid == 0) {
        u64 w = (lane < NT / 32) ? scratch[lane] : 0ull;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const u64 y = __shfl_up_sync(0xFFFFFFFFu, w, o);
            if (lane >= o) w += y;
        }
        scratch[lane] = w;
    }
    __syncthreads();
    const u64 before = wid ? scratch[wid - 1] : 0ull;
    *total = scratch[NT / 32 - 1];
    __syncthreads();
    return before + x - v;
}

// Block-wide inclusive segmented scan: f = 1 starts a new segment at this
// thread; the running sum continues across calls through *carry (the value
// entering thread 0 when its f = 0).  Any wrapped addition sets *ovf (exact:
// every partial sum is a sum inside one segment).  wx / wf: 32 entries of
// shared memory.  Contains barriers.
template <int NT, typename T>
__device__ __forceinline__ T block_segmented_scan(T x, uint32_t f, T* wx, uint32_t* wf, T* carry, uint32_t* ovf) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    bool bad = false;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const T y = shfl_up_w(x, o);
        const uint32_t g = __shfl_up_sync(0xFFFFFFFFu, f, o);
        if (lane >= o) {
            if (!f) { const T sm = x + y; bad |= sm < x; x = sm; }
            f |= g;
        }
    }
    if (lane == 31) { wx[wid] = x; wf[wid] = f; }
    __syncthreads();
    if (wid == 0) {
        T X = (lane < NT / 32) ? wx[lane] : (T)0;
        uint32_t F = (lane < NT / 32) ? wf[lane] : 1u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const T y = shfl_up_w(X, o);
            const uint32_t g = __shfl_up_sync(0xFFFFFFFFu, F, o);
            if (lane >= o) {
                if (!F) { const T sm = X + y; bad |= sm < X; X = sm; }
                F |= g;
            }
        }
        const T Xp = shfl_up_w(X, 1);
        const uint32_t Fp = __shfl_up_sync(0xFFFFFFFFu, F, 1);
        const T c = *carry;
        T P = c;
        if (lane > 0) {
            if (Fp) P = Xp;
            else { P = c + Xp; bad |= P < c; }
        }
        if (lane < NT / 32) wx[lane] = P;
    }
    __syncthreads();
    if (!f) { const T sm = x + wx[wid]; bad |= sm < x; x = sm; }
    if (bad) *ovf = 1u;
    __syncthreads();
    if (threadIdx.x == NT - 1) *carry = x;
    return x;
}

// First index in [lo, hi) with a[idx] > key (a ascending).
__device__ __forceinline__ uint32_t upper_bound_u32(const uint32_t* a, uint32_t lo, uint32_t hi, uint32_t key) {
    while (lo < hi) {
        const uint32_t mid = lo + ((hi - lo) >> 1);
        if (a[mid] <= key) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// First index in [lo, hi) with a[idx] >= key.
__device__ __forceinline__ uint32_t lower_bound_u32(const uint32_t* a, uint32_t lo, uint32_t hi, uint32_t key) {
    while (lo < hi) {
        const uint32_t mid = lo + ((hi - lo) >> 1);
        if (a[mid] < key) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// First index in [lo, hi) with a[idx] >= key, by the whole warp (same
// arguments on every lane): each step every lane probes one of 32 evenly
// spaced positions and a ballot narrows the range 32-fold, so a search costs
// about log32 of the range in dependent loads instead of log2.
__device__ __forceinline__ uint32_t warp_lower_bound(const uint32_t* __restrict__ a, uint32_t lo, uint32_t hi,
                                                     uint32_t key) {
    const uint32_t lane = threadIdx.x & 31;
    while (hi - lo > 32u) {
        const uint32_t step = (hi - lo + 31u) / 32u;
        const uint32_t idx = lo + lane * step;
        const bool lt = idx < hi && __ldg(a + idx) < key;
        const uint32_t c = __popc(__ballot_sync(0xFFFFFFFFu, lt));   // probes below key: a prefix
        if (c == 0) return lo;
        const uint32_t nlo = lo + (c - 1u) * step + 1u;
        const uint32_t nhi = lo + c * step;
        lo = nlo;
        hi = min(hi, nhi);
    }
    const uint32_t idx = lo + lane;
    const bool lt = idx < hi && __ldg(a + idx) < key;
    return lo + __popc(__ballot_sync(0xFFFFFFFFu, lt));
}

// For each k: the first index in [lo[k], hi[k]) whose value exceeds key[k]
// (hi[k] if none), left in lo[k].  The K searches advance together so their
// loads overlap.
template <int K>
__device__ __forceinline__ void upper_bounds(const uint32_t* __restrict__ a, uint32_t (&lo)[K], uint32_t (&hi)[K],
                                             const uint32_t (&key)[K]) {
    for (;;) {
        bool any = false;
        uint32_t mid[K], val[K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const bool act = lo[k] < hi[k];
            any |= act;
            mid[k] = lo[k] + ((hi[k] - lo[k]) >> 1);
            val[k] = act ? __ldg(a + mid[k]) : 0u;
        }
        if (!any) break;
#pragma unroll
        for (int k = 0; k < K; ++k)
            if (lo[k] < hi[k]) {
                if (val[k] <= key[k]) lo[k] = mid[k] + 1u;
                else hi[k] = mid[k];
            }
    }
}

// Walks the edges [w_lo, w_hi) of a range table -- Gc ranges, range g owns
// the edges [off[g], off[g+1]), off[Gc] = the edge total -- in windows of 32
// consecutive edges, calling edge(g, j) for every edge j.  The window's range
// starts are found with one reduce-or over the next 32 offsets (every range
// is non-empty, so at most 32 start inside a window).  Called by a whole warp
// with warp-uniform bounds.
template <typename F>
__device__ __forceinline__ void lbs_walk(const uint32_t* off, uint32_t Gc, uint32_t w_lo, uint32_t w_hi, F edge) {
    const uint32_t lane = threadIdx.x & 31;
    if (w_lo >= w_hi) return;
    uint32_t lo = 0, hi = Gc;                 // off[lo] <= w_lo < off[hi]
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (off[mid] <= w_lo) lo = mid; else hi = mid;
    }
    uint32_t h = lo;
    for (uint32_t base = w_lo; base < w_hi; base += 32u) {
        const uint32_t k = h + 1u + lane;
        const uint32_t o = (k <= Gc) ? off[k] : 0xFFFFFFFFu;   // > base for every k
        const uint32_t d = o - base;
        const uint32_t mask = __reduce_or_sync(0xFFFFFFFFu, d < 32u ? (1u << d) : 0u);
        const uint32_t g = h + __popc(mask & ((2u << lane) - 1u));
        const uint32_t j = base + lane;
        if (j < w_hi) edge(g, j);
        h += __popc(__ballot_sync(0xFFFFFFFFu, o <= base + 32u));
    }
}

// lbs_walk over K windows at a time with the edge loads batched: the range
// and edge index of every edge of the K windows come from the table first
// (shared memory), then pa[e] and pb[e] are loaded for all of them, then
// edge(g, e, pa[e], pb[e]) runs for each valid edge -- K times the loads in
// flight per warp.  first[g] is the first edge of range g.  RO: pa and pb
// are read-only for the kernel's lifetime (read-only data path); otherwise
// plain loads (e.g. shared-memory tiles).  pb holds 32-bit or 16-bit
// entries (TB).
template <int K, bool RO = true, typename TB = uint32_t, typename F>
__device__ __forceinline__ void lbs_walk_batched(const uint32_t* off, uint32_t Gc, const uint32_t* first, uint32_t w_lo,
                                                 uint32_t w_hi, const uint32_t* __restrict__ pa,
                                                 const TB* __restrict__ pb, F edge) {
    const uint32_t lane = threadIdx.x & 31;
    if (w_lo >= w_hi) return;
    uint32_t lo = 0, hi = Gc;                 // off[lo] <= w_lo < off[hi]
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (off[mid] <= w_lo) lo = mid; else hi = mid;
    }
    uint32_t h = lo;
    for (uint32_t base = w_lo; base < w_hi; base += 32u * K) {
        uint32_t rr[K], ee[K];
        bool ok[K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const uint32_t b = base + 32u * k;
            ok[k] = false; rr[k] = 0u; ee[k] = 0u;
            if (b < w_hi) {                       // the same for the whole warp
                const uint32_t kk = h + 1u + lane;
                const uint32_t o = (kk <= Gc) ? off[kk] : 0xFFFFFFFFu;   // > b for every kk
                const uint32_t d = o - b;
                const uint32_t mask = __reduce_or_sync(0xFFFFFFFFu, d < 32u ? (1u << d) : 0u);
                const uint32_t g = h + __popc(mask & ((2u << lane) - 1u));
                const uint32_t j = b + lane;
                ok[k] = j < w_hi;
                if (ok[k]) { rr[k] = g; ee[k] = first[g] + (j - off[g]); }
                h += __popc(__ballot_sync(0xFFFFFFFFu, o <= b + 32u));
            }
        }
        uint32_t va[K], vb[K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            if constexpr (RO) {
                va[k] = ok[k] ? __ldg(pa + ee[k]) : 0u;
                vb[k] = ok[k] ? __ldg(pb + ee[k]) : 0u;
            } else {
                va[k] = ok[k] ? pa[ee[k]] : 0u;
                vb[k] = ok[k] ? pb[ee[k]] : 0u;
            }
        }
#pragma unroll
        for (int k = 0; k < K; ++k)
            if (ok[k]) edge(rr[k], ee[k], va[k], vb[k]);
    }
}

__device__ __forceinline__ void set_status(int* status, int code) { atomicCAS(status, ST_OK, code); }

// ob value of a vertex: the integer nearest to 2^32 * thr / sig (ties up),
// 0 <= thr <= sig, sig >= 1.  Counts below 2^64 take one 128-by-64-bit
// division of thr * 2^32 + floor(sig / 2); wider counts a restoring division
// of the 160-bit numerator, one quotient bit per step (the quotient has at
// most 33 bits).
__device__ __forceinline__ uint64_t ob_q(u128 thr, u128 sig) {
    if ((uint64_t)(sig >> 64) == 0) {
        const u128 num = (thr << 32) + (sig >> 1);
        return (uint64_t)(num / (uint64_t)sig);
    }
    // numerator N = thr * 2^32 + floor(sig/2) as (nh : bits 128..159, nl : bits 0..127)
    const u128 half = sig >> 1;
    u128 nl = thr << 32;
    uint64_t nh = (uint64_t)(thr >> 96);
    nl += half;
    if (nl < half) nh += 1;
    // long division over the 33 low-order quotient positions: the partial
    // remainder starts as N >> 32 (< 2 sig)
    u128 rem = ((u128)nh << 96) | (nl >> 32);
    uint64_t q = 0;
    if (rem >= sig) { rem -= sig; q = 1; }
    for (int b = 31; b >= 0; --b) {
        const bool top = (uint64_t)(rem >> 127) != 0;
        rem = (rem << 1) | (u128)((uint64_t)(nl >> b) & 1u);
        q <<= 1;
        if (top || rem >= sig) { rem -= sig; q |= 1u; }
    }
    return q;
}

// floor(a * x / d + 1/2) for 0 <= a <= d (d >= 1), x < 2^64 (the result is at
// most x + 1): the RTB dependency terms.  A 64-bit a and d take one 128-by-64
// division; otherwise the 192-bit product is divided by a restoring division
// over the 64 low quotient positions (the quotient fits 64 bits).
__device__ __forceinline__ uint64_t muldiv_round(u128 a, uint64_t x, u128 d) {
    if ((uint64_t)(a >> 64) == 0 && (uint64_t)(d >> 64) == 0) {
        const u128 p = a * (u128)x;
        const uint64_t dd = (uint64_t)d;
        const uint64_t q = (uint64_t)(p / dd), r = (uint64_t)(p - (u128)q * dd);
        return q + (r >= dd - r ? 1u : 0u);
    }
    // p = a * x as (ph : 64 high bits, pl : 128 low bits)
    const u128 mlo = (u128)(uint64_t)a * x, mhi = (u128)(uint64_t)(a >> 64) * x;
    const u128 pl = mlo + (mhi << 64);
    const uint64_t ph = (uint64_t)(mhi >> 64) + (pl < mlo ? 1u : 0u);
    // partial remainder p >> 64 (< d, as the quotient is below 2^64), then one
    // low bit of p per quotient position
    u128 rem = ((u128)ph << 64) | (pl >> 64);
    uint64_t q = 0;
    for (int b = 63; b >= 0; --b) {
        const bool top = (uint64_t)(rem >> 127) != 0;
        rem = (rem << 1) | (u128)((uint64_t)(pl >> b) & 1u);
        q <<= 1;
        if (top || rem >= d) { rem -= d; q |= 1u; }
    }
    const bool top = (uint64_t)(rem >> 127) != 0;
    return q + ((top || (rem << 1) >= d) ? 1u : 0u);
}

// 2^32 / d rounded to nearest (ties up), d >= 1: the closeness term of a
// vertex at hop distance d.
__device__ __forceinline__ u64 recip32(uint32_t d) { return ((1ull << 33) + d) / (2ull * d); }

// q^2 / 2^32 rounded to nearest (ties up): the ob value of f^2 (wimpy variance).
__device__ __forceinline__ uint64_t ob_sq(uint64_t q) { return (uint64_t)(((u128)q * q + (1ull << 31)) >> 32); }

// One (vertex, row) term of the ob update: row 0 hits, row 1 wsq, row 2 + j
// the Rademacher sum of trial j.
__device__ __forceinline__ void ob_term(const Job& job, uint32_t v, uint64_t q, uint32_t row, const uint32_t rade[4]) {
    if (row == 0) atomicAdd(job.hits + v, (u64)q);
    else if (row == 1) atomicAdd(job.wsq + v, (u64)ob_sq(q));
    else if (job.S64) {
        const uint32_t jj = row - 2;
        const long long lq = ((rade[jj >> 5] >> (jj & 31)) & 1u) ? (long long)q : -(long long)q;
        atomicAdd(reinterpret_cast<u64*>(job.S64 + (size_t)jj * job.fam + v), (u64)lq);
    }
}

// Records sample i for the 128-bit / in-order re-run (a job without a list
// reports a consistency error instead).
__device__ __forceinline__ void push_overflow(const Job& job, uint64_t i) {
    if (job.ovf_list) job.ovf_list[atomicAdd(job.ctr + C_NOVF, 1ull)] = i;
    else set_status(job.status, ST_CHECK);
}

// Entries of the estimated family that a drawn path of len vertices adds one
// hit to: its len-2 internal vertices (Sec. 3) or its len-1 edges (App. A).
__device__ __forceinline__ uint32_t family_count(const Job& job, uint32_t len) {
    if (len < 2) return 0;
    return job.target == 0 ? len - 2 : len - 1;
}

// The k-th of them; path holds the vertices s .. z, pe the in-CSR indices of
// the edges (path[k] -> path[k+1]).
__device__ __forceinline__ uint32_t family_item(const Job& job, const DevGraph& g, const uint32_t* path,
                                                const uint32_t* pe, uint32_t k) {
    if (job.target == 0) return path[1 + k];
    return job.target == 2 ? pe[k] : g.in_uedge[pe[k]];
}


// Per-CTA scratch of the sh/sfm search kernel (one region per CTA).
struct BfsWs {
    char* base;          // CTA b uses base + b * stride
    size_t stride;
    size_t o_sig, o_fc, o_f, o_ft, o_lev, o_segb, o_segu, o_path, o_pathe, o_bits, o_vb, o_segmap, o_stamp, o_nbits;
    size_t o_fu;         // per frontier position: the state's vertex (written by the count pass)
    int bits_in_smem;    // visited bitmap in dynamic shared memory (the next-level bitmap is in the region)
    uint32_t bits_words; // capacity of each bitmap (words): ceil(A_max / 32)
    uint32_t n_cap;      // node capacity of a region
    int nt;              // threads per CTA (512 or 1024)
    size_t o_acc;        // ob: per-vertex sums of through counts; RTB: sigma_{s,v}
    size_t o_acc2;       // RTB: per-vertex dependency sums
    size_t o_zsig;       // path counts of z's slots reached by the pull (sh / sfm endpoints)
    int has_dl;          // the ob / RTB scratch (o_fc, o_acc, o_acc2) is allocated
};

// Per-warp scratch of the pfm search kernel.
struct PfmWs {
    char* base;          // warp w uses base + w * stride
    size_t stride;
    size_t o_fa, o_sig, o_hop, o_path, o_pathe, o_list, o_dl;   // o_dl: ob continuation counts
    uint32_t n_cap;      // node capacity of a region (largest graph of the launch)
    uint32_t list_cap;   // contributing-edge entries per lane (deferred path counts)
};

// Per-CTA scratch of the pfm search kernel with one CTA per sample.
struct PfmCtaWs {
    char* base;          // CTA b uses base + b * stride
    size_t stride;
    size_t o_fa, o_bits, o_exp, o_fat, o_sig, o_hop, o_pend, o_list, o_path, o_pathe;
    size_t o_dl, o_kofs; // ob: continuation counts per vertex, Kahn round offsets
    size_t o_dcnt, o_dag;// the prefix-foremost DAG as out-lists: per-vertex ends, successors
    uint32_t dag_cap;    // capacity of the successor array (>= cbound of every graph)
    uint32_t n_cap;      // node capacity of a region
    uint32_t bits_words; // words of each bitmap: ceil(n_cap / 32)
    int fa_in_smem;      // state mode: 0 global region; arrival state and bitmaps in dynamic shared
                         // memory, 1 as 32-bit slots, 2 as 16-bit offsets within each vertex's slots
    int nt;              // threads per CTA (256 or 512)
    uint32_t stage_cap;  // global-state variant: out-edges per chunk staged in shared memory by bulk copies (0: none)
};

size_t bfs_region_bytes(uint32_t n, uint32_t A, uint32_t zcap, bool bits_in_smem, bool dl, BfsWs* ws);
size_t bfs_smem_bytes(uint32_t A);
size_t bfs_static_smem(int nt);
cudaError_t bfs_blocks_per_sm(int nt, size_t smem, int* out);
cudaError_t bfs_configure(size_t smem);
// Task-table launches: work unit u of the launch belongs to task
// task_of_unit(unit_start, *ntasks, u); the first unused unit ends a CTA/warp.
// sh/sfm: one unit per sample; pfm: one unit per 32 consecutive samples of a task.
cudaError_t launch_bfs(const Task* tasks, const uint64_t* unit_start, const uint32_t* ntasks, u64* work,
                       const BfsWs& ws, int grid, size_t smem, bool wide, bool frac, cudaStream_t st);
size_t pfm_region_bytes(uint32_t n, uint32_t list_cap, PfmWs* ws);
int pfm_threads();
cudaError_t launch_pfm(const Task* tasks, const uint64_t* unit_start, const uint32_t* ntasks, u64* work,
                       const PfmWs& ws, int grid, bool wide, cudaStream_t st);
size_t pfm_cta_region_bytes(uint32_t n, uint32_t dag_cap, bool fa_in_smem, PfmCtaWs* ws);
size_t pfm_cta_smem_bytes(uint32_t n, bool w16);
size_t pfm_cta_stage_bytes(uint32_t cap);
size_t pfm_cta_static_smem(int nt);
cudaError_t pfm_cta_configure(size_t smem);
cudaError_t pfm_cta_blocks_per_sm(int nt, int fa, size_t smem, int* out);
cudaError_t launch_pfm_cta(const Task* tasks, const uint64_t* unit_start, const uint32_t* ntasks, u64* work,
                           const PfmCtaWs& ws, int grid, cudaStream_t st);
// One problem of a multi-problem round reduction.
struct ReduceItem {
    const int* S;        // c rows of n (unused when c = 0)
    const long long* S64;// instead of S when set (ob sums)
    const u64* hits;     // n: hits, or the ob wimpy sums
    uint32_t n, c;       // n: the family size (0: every maximum is 0)
    long long* rowmax;   // c results: max_v S[j][v]
    u64* hmax;           // max_v hits[v]
};
cudaError_t launch_round_reduce(const ReduceItem* items, const uint32_t* row_start, const uint32_t* np, int grid,
                                cudaStream_t st);
cudaError_t launch_normalise(const u64* hits, uint32_t n, double denom, double* est, cudaStream_t st);

}  // namespace mantra
