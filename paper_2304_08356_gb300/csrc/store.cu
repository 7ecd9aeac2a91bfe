// Host construction of the temporal-edge store (paper Sec. 3; the arrays are
// listed in store.h).  A team of host threads runs every step in SPMD style:
// the stream order (t, u, v) comes from stable least-significant-digit radix
// passes (digits of at most 16 bits over v, then u, then t), the in-CSR
// (v, t, u) and out-CSR (u, t, v) orders from one more stable pass by v or u
// each, and the underlying-edge order (v, u, t) from a pass by v over the
// out-CSR order.  Boundaries (distinct triples, arrival slots, distinct
// ordered pairs) are counted per thread chunk, offset by the chunk counts
// before it and written in parallel; row pointers are filled from sorted keys.
#include "store.h"
#include "mantra.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdlib>
#include <thread>
#include <vector>

namespace mantra {
namespace {

constexpr size_t kCacheCap = (size_t)256 << 20;   // buffers at most this large stay cached
constexpr unsigned kMaxThreads = 16;
constexpr uint32_t kDigitBits = 16;                // widest radix digit
constexpr uint32_t kMaxKeys = 1u << kDigitBits;

struct Rec { uint32_t t, u, v, id; };              // id: index in the deduplicated stream

// Part x of T near-equal contiguous parts of [0, len).
struct Range { uint64_t lo, hi; };
inline Range part(uint64_t len, unsigned T, unsigned x) {
    const uint64_t q = len / T, r = len % T;
    const uint64_t lo = q * x + std::min<uint64_t>(x, r);
    return {lo, lo + q + (x < r ? 1 : 0)};
}

// A team of host threads running one body in SPMD style; sync() is a barrier
// among all of them (every member reaches the same barriers in the same order).
class Team {
public:
    unsigned size() const { return T_; }

    void sync() {
        if (T_ == 1) return;
        const uint32_t g = gen_.load(std::memory_order_acquire);
        if (arrived_.fetch_add(1, std::memory_order_acq_rel) + 1 == T_) {
            arrived_.store(0, std::memory_order_relaxed);
            gen_.store(g + 1, std::memory_order_release);
            return;
        }
        for (unsigned k = 0; gen_.load(std::memory_order_acquire) == g; ++k)
            if (k >= 256) std::this_thread::yield();
    }

    // Runs body(team, x) for x = 0 .. T-1, x = 0 on the calling thread.  T is
    // `want`, or fewer when the system refuses a thread; it is fixed before
    // any member starts.
    template <class F>
    static void run(unsigned want, F&& body) {
        Team tm;
        std::vector<std::thread> th;
        th.reserve(want);
        for (unsigned x = 1; x < want; ++x) {
            try {
                th.emplace_back([&tm, &body, x] {
                    while (!tm.go_.load(std::memory_order_acquire)) std::this_thread::yield();
                    body(tm, x);
                });
            } catch (...) {
                break;
            }
        }
        tm.T_ = (unsigned)th.size() + 1;
        tm.go_.store(true, std::memory_order_release);
        body(tm, 0u);
        for (auto& h : th) h.join();
    }

private:
    unsigned T_ = 1;
    std::atomic<uint32_t> arrived_{0}, gen_{0};
    std::atomic<bool> go_{false};
};

enum Field { F_T, F_U, F_V };
template <Field F>
inline uint32_t fval(const Rec& r) { return F == F_T ? r.t : (F == F_U ? r.u : r.v); }

// State shared by the team during one build.
struct Ctx {
    const uint32_t *u = nullptr, *v = nullptr, *t = nullptr;
    uint64_t m = 0;
    uint32_t n = 0;
    uint64_t p0[kMaxThreads] = {}, p1[kMaxThreads] = {}, p2[kMaxThreads] = {}, p3[kMaxThreads] = {},
             psum[kMaxThreads] = {};
    std::atomic<int> bad{0};
    int rc = MANTRA_OK;
    uint64_t m1 = 0, loops = 0, tmax = 0;   // triples without self loops, self loops, largest time
    Rec* rb[3] = {};
    uint32_t* inpos = nullptr;              // inpos[id]: in-CSR index of stream edge id
    uint32_t* cnt = nullptr;                // kMaxThreads x K digit counts of a pass
    uint32_t* a[SA_COUNT] = {};
    uint32_t M = 0, A = 0;
};

// Sum of p[0 .. x).
inline uint64_t before(const uint64_t* p, unsigned x) {
    uint64_t s = 0;
    for (unsigned y = 0; y < x; ++y) s += p[y];
    return s;
}

// Read position and the two buffers a sequence of radix passes alternates between.
struct PingPong {
    const Rec* cur;
    Rec* buf[2];
    int next;
};

// One stable counting pass of len records from pp.cur into the next buffer by
// key(rec) in [0, K): per-thread digit counts over the thread's chunk, global
// offsets in (digit, thread) order, per-thread scatter.  pos (or null)
// receives each record's new index at pos[rec.id].
template <class Key>
void pass(Team& tm, unsigned x, Ctx& c, PingPong& pp, uint32_t len, uint32_t K, Key key, uint32_t* pos) {
    const unsigned T = tm.size();
    const Rec* src = pp.cur;
    Rec* dst = pp.buf[pp.next];
    uint32_t* my = c.cnt + (size_t)x * K;
    std::fill(my, my + K, 0u);
    const Range r = part(len, T, x);
    for (uint64_t i = r.lo; i < r.hi; ++i) ++my[key(src[i])];
    tm.sync();
    const Range kr = part(K, T, x);
    uint64_t s = 0;
    for (uint64_t d = kr.lo; d < kr.hi; ++d)
        for (unsigned y = 0; y < T; ++y) s += c.cnt[(size_t)y * K + d];
    c.psum[x] = s;
    tm.sync();
    uint64_t acc = before(c.psum, x);
    for (uint64_t d = kr.lo; d < kr.hi; ++d)
        for (unsigned y = 0; y < T; ++y) {
            uint32_t& e = c.cnt[(size_t)y * K + d];
            const uint32_t k = e;
            e = (uint32_t)acc;
            acc += k;
        }
    tm.sync();
    if (pos) {
        for (uint64_t i = r.lo; i < r.hi; ++i) {
            const uint32_t k = my[key(src[i])]++;
            dst[k] = src[i];
            pos[src[i].id] = k;
        }
    } else {
        for (uint64_t i = r.lo; i < r.hi; ++i) dst[my[key(src[i])]++] = src[i];
    }
    tm.sync();
    pp.cur = dst;
    pp.next ^= 1;
}

// Stable sort of the records by field F, whose values are < R: one pass when
// R <= 2^16, else passes of equal digit widths of at most 16 bits, low first.
// pos (or null): the last pass stores each record's final index at pos[id].
template <Field F>
void sort_field(Team& tm, unsigned x, Ctx& c, PingPong& pp, uint32_t len, uint64_t R, uint32_t* pos = nullptr) {
    uint32_t bits = 0;
    while (bits < 32 && ((R - 1) >> bits) != 0) ++bits;
    if (bits == 0) return;
    if (bits <= kDigitBits) {
        pass(tm, x, c, pp, len, (uint32_t)R, [](const Rec& r) { return fval<F>(r); }, pos);
        return;
    }
    const uint32_t np = (bits + kDigitBits - 1) / kDigitBits;
    const uint32_t w = (bits + np - 1) / np;
    for (uint32_t j = 0; j < np; ++j) {
        const uint32_t sh = j * w, wb = std::min(w, bits - sh), mask = (1u << wb) - 1;
        pass(tm, x, c, pp, len, 1u << wb, [sh, mask](const Rec& r) { return (fval<F>(r) >> sh) & mask; },
             j + 1 == np ? pos : nullptr);
    }
}

// ptr[y] = the first index i of the sorted key sequence with key(i) >= y, for
// y in [0, nk]; every entry is written by exactly one thread.
template <class Key>
void fill_ptr(unsigned T, unsigned x, uint32_t* ptr, uint32_t len, uint32_t nk, Key key) {
    const Range r = part(len, T, x);
    for (uint64_t i = r.lo; i < r.hi; ++i) {
        const uint64_t from = i == 0 ? 0 : (uint64_t)key(i - 1) + 1;
        for (uint64_t y = from; y <= key(i); ++y) ptr[y] = (uint32_t)i;
    }
    if (x == T - 1)
        for (uint64_t y = len == 0 ? 0 : (uint64_t)key(len - 1) + 1; y <= nk; ++y) ptr[y] = len;
}

inline bool same_tuv(const Rec& a, const Rec& b) { return a.t == b.t && a.u == b.u && a.v == b.v; }

}  // namespace

StoreBuilder::~StoreBuilder() {
    release(out_);
    release(work_);
    release(cnt_);
}

void StoreBuilder::release(Buf& b) {
    if (b.p) {
        if (b.pinned) cudaFreeHost(b.p);
        else std::free(b.p);
    }
    b = Buf{};
}

bool StoreBuilder::reserve(Buf& b, size_t bytes, bool want_pinned) {
    if (b.p && b.bytes >= bytes) return true;
    release(b);
    const size_t want = bytes + bytes / 8;
    if (want_pinned && want <= kCacheCap && cudaHostAlloc(&b.p, want, cudaHostAllocDefault) == cudaSuccess) {
        b.bytes = want;
        b.pinned = true;
        return true;
    }
    cudaGetLastError();
    b.p = std::malloc(want);
    if (!b.p) return false;
    b.bytes = want;
    return true;
}

void StoreBuilder::trim() {
    if (out_.bytes > kCacheCap) release(out_);
    if (work_.bytes > kCacheCap) release(work_);
}

int StoreBuilder::build(const uint32_t* u, const uint32_t* v, const uint32_t* t, uint64_t m, uint32_t n,
                        StoreHost* out) {
    *out = StoreHost{};
    if (!reserve(cnt_, (size_t)kMaxThreads * kMaxKeys * 4, false)) return MANTRA_E_NOMEM;
    unsigned want = std::min(kMaxThreads, std::max(1u, std::thread::hardware_concurrency()));
    if (m < ((uint64_t)1 << 16)) want = 1;
    // MANTRA_STORE_THREADS=k: exactly k threads (1 .. 16), whatever the size
    if (const char* env = std::getenv("MANTRA_STORE_THREADS"))
        want = (unsigned)std::min<long>(kMaxThreads, std::max<long>(1, std::atol(env)));

    Ctx c;
    c.u = u; c.v = v; c.t = t; c.m = m; c.n = n;
    c.cnt = (uint32_t*)cnt_.p;
    size_t cap[SA_COUNT] = {};

    Team::run(want, [&](Team& tm, unsigned x) {
        const unsigned T = tm.size();
        // -- n from the ids when not given
        const Range ri = part(c.m, T, x);
        if (n == 0) {
            uint32_t mx = 0;
            for (uint64_t e = ri.lo; e < ri.hi; ++e) mx = std::max(mx, std::max(c.u[e], c.v[e]));
            c.p0[x] = mx;
            tm.sync();
            uint64_t all = 0;
            for (unsigned y = 0; y < T; ++y) all = std::max(all, c.p0[y]);
            if (all >= 0xFFFFFFFFull) c.bad.store(1);
            else if (x == 0) c.n = (uint32_t)all + 1;
            tm.sync();
        }
        // -- validation, self loops, largest time
        uint64_t loops = 0, tmx = 0;
        const uint32_t N = c.n;
        for (uint64_t e = ri.lo; e < ri.hi; ++e) {
            if (c.u[e] >= N || c.v[e] >= N || c.t[e] > 0xFFFFFFFDu) { c.bad.store(1, std::memory_order_relaxed); break; }
            if (c.u[e] == c.v[e]) ++loops;
            else tmx = std::max<uint64_t>(tmx, c.t[e]);
        }
        c.p0[x] = (ri.hi - ri.lo) - loops;
        c.p1[x] = loops;
        c.p2[x] = tmx;
        tm.sync();
        if (x == 0) {
            for (unsigned y = 0; y < T; ++y) {
                c.m1 += c.p0[y];
                c.loops += c.p1[y];
                c.tmax = std::max(c.tmax, c.p2[y]);
            }
            if (c.bad.load() || N < 2 || c.m1 >= 0xFFFFFFF0ull) {
                c.rc = MANTRA_E_INVAL;
            } else {
                const uint64_t m1 = c.m1;
                const size_t lens[SA_COUNT] = {(size_t)N + 1, m1, m1, m1, (size_t)N + 1, m1, m1, m1 + 1, m1,
                                               m1, m1, m1, m1, N, N, m1, m1, (m1 + 1) / 2};
                size_t total = 0;
                for (int k = 0; k < SA_COUNT; ++k) { cap[k] = (lens[k] + 64) & ~(size_t)63; total += cap[k]; }
                const size_t recs = std::max<uint64_t>(m1, 1);
                if (!reserve(out_, total * 4, true) || !reserve(work_, recs * (3 * sizeof(Rec) + 4), false)) {
                    c.rc = MANTRA_E_NOMEM;
                } else {
                    uint32_t* p = (uint32_t*)out_.p;
                    for (int k = 0; k < SA_COUNT; ++k) { c.a[k] = p; p += cap[k]; }
                    Rec* r = (Rec*)work_.p;
                    c.rb[0] = r; c.rb[1] = r + recs; c.rb[2] = r + 2 * recs;
                    c.inpos = (uint32_t*)(r + 3 * recs);
                }
            }
        }
        tm.sync();
        if (c.rc != MANTRA_OK) return;
        const uint32_t m1 = (uint32_t)c.m1;

        // -- copy the triples without self loops, in input order
        {
            Rec* dst = c.rb[0] + before(c.p0, x);
            for (uint64_t e = ri.lo; e < ri.hi; ++e)
                if (c.u[e] != c.v[e]) *dst++ = Rec{c.t[e], c.u[e], c.v[e], 0u};
        }
        tm.sync();

        // -- (t, u, v) order: stable passes by v, then u, then t
        PingPong pp{c.rb[0], {c.rb[1], c.rb[0]}, 0};
        sort_field<F_V>(tm, x, c, pp, m1, N);
        sort_field<F_U>(tm, x, c, pp, m1, N);
        sort_field<F_T>(tm, x, c, pp, m1, c.tmax + 1);
        const Rec* S = pp.cur;

        // -- deduplicate into D, numbering the stream
        Rec* D = S == c.rb[0] ? c.rb[1] : c.rb[0];
        Rec* X = S == c.rb[0] ? c.rb[0] : c.rb[1];
        Rec* Y = c.rb[2];
        const Range rs = part(m1, T, x);
        {
            uint64_t k = 0;
            for (uint64_t e = rs.lo; e < rs.hi; ++e) k += (e == 0 || !same_tuv(S[e], S[e - 1]));
            c.p0[x] = k;
        }
        tm.sync();
        {
            uint64_t j = before(c.p0, x);
            uint32_t *su = c.a[SA_ST_U], *sv = c.a[SA_ST_V], *st = c.a[SA_ST_T];
            for (uint64_t e = rs.lo; e < rs.hi; ++e) {
                if (e != 0 && same_tuv(S[e], S[e - 1])) continue;
                D[j] = Rec{S[e].t, S[e].u, S[e].v, (uint32_t)j};
                su[j] = S[e].u; sv[j] = S[e].v; st[j] = S[e].t;
                ++j;
            }
        }
        const uint32_t M = (uint32_t)before(c.p0, T);
        if (x == 0) c.M = M;
        tm.sync();
        const Range rm = part(M, T, x);

        // -- in-CSR (v, t, u): a stable pass by v of the stream; arrival slots
        PingPong pi{D, {X, Y}, 0};
        sort_field<F_V>(tm, x, c, pi, M, N, c.inpos);
        const Rec* I = pi.cur;
        {
            uint32_t* in_u = c.a[SA_IN_U];
            uint64_t k = 0;
            for (uint64_t e = rm.lo; e < rm.hi; ++e) {
                k += (e == 0 || I[e].v != I[e - 1].v || I[e].t != I[e - 1].t);
                in_u[e] = I[e].u;
            }
            c.p0[x] = k;
        }
        tm.sync();
        {
            uint32_t *in_slot = c.a[SA_IN_SLOT], *sl_t = c.a[SA_SLOT_T], *sl_v = c.a[SA_SLOT_V],
                     *sl_in = c.a[SA_SLOT_IN];
            uint64_t a = before(c.p0, x);   // slots started before this chunk
            for (uint64_t e = rm.lo; e < rm.hi; ++e) {
                if (e == 0 || I[e].v != I[e - 1].v || I[e].t != I[e - 1].t) {
                    sl_t[a] = I[e].t; sl_v[a] = I[e].v; sl_in[a] = (uint32_t)e;
                    ++a;
                }
                in_slot[e] = (uint32_t)(a - 1);
            }
        }
        const uint32_t A = (uint32_t)before(c.p0, T);
        if (x == 0) { c.A = A; c.a[SA_SLOT_IN][A] = M; }
        tm.sync();
        {
            const uint32_t* sl_v = c.a[SA_SLOT_V];
            fill_ptr(T, x, c.a[SA_SLOT_PTR], A, N, [sl_v](uint64_t i) { return sl_v[i]; });
        }

        // -- out-CSR (u, t, v): a stable pass by u of the stream
        PingPong po{D, {X, Y}, 0};
        sort_field<F_U>(tm, x, c, po, M, N);
        const Rec* O = po.cur;
        {
            uint32_t *o_v = c.a[SA_OUT_V], *o_t = c.a[SA_OUT_T], *o_s = c.a[SA_OUT_SLOT];
            const uint32_t* in_slot = c.a[SA_IN_SLOT];
            for (uint64_t e = rm.lo; e < rm.hi; ++e) {
                o_v[e] = O[e].v; o_t[e] = O[e].t;
                o_s[e] = in_slot[c.inpos[O[e].id]];
            }
            fill_ptr(T, x, c.a[SA_OUT_PTR], M, N, [O](uint64_t i) { return O[i].u; });
        }
        tm.sync();

        // -- per slot: first out-edge of v later than the slot's time; per
        //    vertex: latest arrival, earliest departure, largest slot in-count
        {
            const uint32_t *o_ptr = c.a[SA_OUT_PTR], *o_t = c.a[SA_OUT_T], *sl_t = c.a[SA_SLOT_T],
                           *sl_ptr = c.a[SA_SLOT_PTR], *sl_in = c.a[SA_SLOT_IN];
            uint32_t* nout = c.a[SA_SLOT_NOUT];
            uint32_t *tmax_in = c.a[SA_TMAX_IN], *tmin_out = c.a[SA_TMIN_OUT];
            const uint32_t *o_v = c.a[SA_OUT_V], *o_s = c.a[SA_OUT_SLOT];
            uint16_t* loff = reinterpret_cast<uint16_t*>(c.a[SA_OUT_LOFF]);
            // vertices split by their slot + out-edge counts (a monotone prefix);
            // each vertex merges its slot times with its out-row times
            const uint64_t tot = (uint64_t)A + M;
            auto first_w = [&](uint64_t target) {
                uint64_t lo = 0, hi = N;
                while (lo < hi) {
                    const uint64_t mid = (lo + hi) / 2;
                    if ((uint64_t)sl_ptr[mid] + o_ptr[mid] < target) lo = mid + 1;
                    else hi = mid;
                }
                return lo;
            };
            const uint64_t wlo = x == 0 ? 0 : first_w(tot * x / T);
            const uint64_t whi = x == T - 1 ? N : first_w(tot * (x + 1) / T);
            uint64_t cb = 0, mxs = 0, mxv = 0;
            for (uint64_t w = wlo; w < whi; ++w) {
                const uint32_t a0 = sl_ptr[w], a1 = sl_ptr[w + 1], q1 = o_ptr[w + 1];
                mxv = std::max<uint64_t>(mxv, a1 - a0);
                uint32_t q = o_ptr[w], mx = 0;
                for (uint32_t a = a0; a < a1; ++a) {
                    const uint32_t ta = sl_t[a];
                    while (q < q1 && o_t[q] <= ta) ++q;
                    nout[a] = q;
                    mx = std::max(mx, sl_in[a + 1] - sl_in[a]);
                }
                for (uint32_t e = o_ptr[w]; e < q1; ++e)   // heads' slot offsets (16-bit entries)
                    loff[e] = (uint16_t)std::min<uint32_t>(o_s[e] - sl_ptr[o_v[e]], 0xFFFFu);
                tmax_in[w] = a1 > a0 ? sl_t[a1 - 1] : 0;
                tmin_out[w] = q1 > o_ptr[w] ? o_t[o_ptr[w]] : 0;
                cb += mx;
                mxs = std::max<uint64_t>(mxs, mx);
            }
            c.p1[x] = cb;
            c.p2[x] = mxs;
            c.p3[x] = mxv;
        }

        // -- underlying edges (App. A): a stable pass by v of the out-CSR order
        //    lists the edges by (v, u, t); ids rank the distinct (v, u) pairs
        PingPong pw{O, {D, O == X ? Y : X}, 0};
        sort_field<F_V>(tm, x, c, pw, M, N);
        const Rec* W = pw.cur;
        {
            uint64_t k = 0;
            for (uint64_t e = rm.lo; e < rm.hi; ++e) k += (e > 0 && (W[e].v != W[e - 1].v || W[e].u != W[e - 1].u));
            c.p0[x] = k;
        }
        tm.sync();
        {
            uint32_t* ue = c.a[SA_IN_UEDGE];
            uint64_t k = before(c.p0, x);
            for (uint64_t e = rm.lo; e < rm.hi; ++e) {
                k += (e > 0 && (W[e].v != W[e - 1].v || W[e].u != W[e - 1].u));
                ue[c.inpos[W[e].id]] = (uint32_t)k;
            }
        }
        tm.sync();
    });
    if (c.rc != MANTRA_OK) return c.rc;

    const uint32_t N = c.n, M = c.M, A = c.A;
    out->n = N; out->m = M; out->A = A;
    out->self_loops = c.loops;
    out->duplicates = c.m1 - M;
    uint64_t n_ue = 0, cb = 0, mxs = 0, mxv = 0;
    for (unsigned y = 0; y < kMaxThreads; ++y) {
        n_ue += c.p0[y]; cb += c.p1[y]; mxs = std::max(mxs, c.p2[y]); mxv = std::max(mxv, c.p3[y]);
    }
    out->n_uedge = M > 0 ? (uint32_t)(n_ue + 1) : 0;
    out->cbound = (uint32_t)std::min<uint64_t>(cb, 0xFFFFFFFFull);
    out->max_slot_in = (uint32_t)mxs;
    out->max_vslots = (uint32_t)mxv;
    if (M & 1) reinterpret_cast<uint16_t*>(c.a[SA_OUT_LOFF])[M] = 0;
    const size_t lens[SA_COUNT] = {(size_t)N + 1, M, M, M, (size_t)N + 1, A, A, (size_t)A + 1, M, M, M, M, M,
                                   N, N, M, A, ((size_t)M + 1) / 2};
    for (int k = 0; k < SA_COUNT; ++k) { out->arr[k] = c.a[k]; out->len[k] = lens[k]; }
    return MANTRA_OK;
}

}  // namespace mantra
