// Host construction of the temporal-edge store (paper Sec. 3, the temporal
// graph G = (V, E) with E a set of triples (u, v, t)): the edge stream in
// (t, u, v) order, the arrival slots (v, t), the in-CSR by (v, t, u), the
// out-CSR by (u, t, v) and the underlying-edge ids of App. A, built by a team
// of host threads with stable radix passes into host buffers laid out for one
// upload per array.
#pragma once

#include <cstddef>
#include <cstdint>

namespace mantra {

// The store's arrays, in the order of the device block.
enum StoreArr : int {
    SA_OUT_PTR, SA_OUT_V, SA_OUT_T, SA_OUT_SLOT, SA_SLOT_PTR, SA_SLOT_T, SA_SLOT_V, SA_SLOT_IN, SA_IN_U,
    SA_IN_SLOT, SA_ST_U, SA_ST_V, SA_ST_T, SA_TMAX_IN, SA_TMIN_OUT, SA_IN_UEDGE, SA_SLOT_NOUT, SA_OUT_LOFF, SA_COUNT
};
// SA_OUT_LOFF holds 16-bit entries, two per uint32 word (entry e in the low
// half of word e / 2 when e is even): per out-edge, the offset of its head's
// arrival slot within the head's slots, min(out_slot - slot_ptr[out_v],
// 0xFFFF); a trailing odd half is 0.

// Result of a build: sizes, counters and the host arrays (each len[k] uint32
// entries, owned by the builder).
struct StoreHost {
    uint32_t n = 0, m = 0, A = 0, n_uedge = 0, cbound = 0, max_slot_in = 0;
    uint32_t max_vslots = 0;   // largest number of arrival slots of one vertex
    uint64_t self_loops = 0, duplicates = 0;
    const uint32_t* arr[SA_COUNT] = {};
    size_t len[SA_COUNT] = {};
};

// Reusable host memory of the store build: the output arrays (page-locked
// while they fit under a cap, so that the uploads are DMA transfers from
// them) and the radix passes' record buffers.  One builder serves one caller
// at a time.
class StoreBuilder {
public:
    StoreBuilder() = default;
    StoreBuilder(const StoreBuilder&) = delete;
    StoreBuilder& operator=(const StoreBuilder&) = delete;
    ~StoreBuilder();

    // Builds the store of the m triples (u[e], v[e], t[e]); n = 0 takes the
    // largest id + 1.  Self loops are dropped and duplicate triples kept once.
    // Threads: up to 16 (one below 2^16 triples); the environment variable
    // MANTRA_STORE_THREADS=k sets k (1 .. 16) for any size.
    // Returns MANTRA_OK, MANTRA_E_INVAL (an id >= n, a time above 2^32 - 3,
    // n < 2, or 2^32 - 16 or more triples left after dropping self loops) or
    // MANTRA_E_NOMEM.  The arrays of *out stay valid until the next build() or
    // trim().
    int build(const uint32_t* u, const uint32_t* v, const uint32_t* t, uint64_t m, uint32_t n, StoreHost* out);

    // Releases buffers above the caching cap (call once the arrays are uploaded).
    void trim();

private:
    struct Buf {
        void* p = nullptr;
        size_t bytes = 0;
        bool pinned = false;
    };
    bool reserve(Buf& b, size_t bytes, bool want_pinned);
    static void release(Buf& b);

    Buf out_, work_, cnt_;
};

}  // namespace mantra
