// Test driver for the host store builder (store.cu), run without a GPU.
// Reads one graph (uint64 m, uint32 n, then u[m], v[m], t[m] as uint32),
// builds the store twice with one builder (the second build reuses its
// buffers) and writes: int32 rc; uint32 n, m, A, n_uedge, cbound,
// max_slot_in, max_vslots, pad; uint64 self_loops, duplicates; then per array in the order
// of the device block a uint64 length and the uint32 entries.
#include "store.h"

#include <cstdio>
#include <cstdint>
#include <cstring>
#include <vector>

int main(int argc, char** argv) {
    if (argc != 3) return 2;
    FILE* f = std::fopen(argv[1], "rb");
    if (!f) return 2;
    uint64_t m = 0;
    uint32_t n = 0;
    if (std::fread(&m, 8, 1, f) != 1 || std::fread(&n, 4, 1, f) != 1) return 2;
    std::vector<uint32_t> buf(3 * m + 1);
    if (m && std::fread(buf.data(), 4, 3 * m, f) != 3 * m) return 2;
    std::fclose(f);
    mantra::StoreBuilder B;
    mantra::StoreHost H;
    int rc = 0;
    for (int k = 0; k < 2; ++k) rc = B.build(buf.data(), buf.data() + m, buf.data() + 2 * m, m, n, &H);
    FILE* o = std::fopen(argv[2], "wb");
    if (!o) return 2;
    const int32_t rc32 = rc;
    const uint32_t sc[8] = {H.n, H.m, H.A, H.n_uedge, H.cbound, H.max_slot_in, H.max_vslots, 0u};
    const uint64_t cn[2] = {H.self_loops, H.duplicates};
    std::fwrite(&rc32, 4, 1, o);
    std::fwrite(sc, 4, 8, o);
    std::fwrite(cn, 8, 2, o);
    for (int k = 0; k < mantra::SA_COUNT; ++k) {
        const uint64_t len = rc == 0 ? H.len[k] : 0;
        std::fwrite(&len, 8, 1, o);
        if (len) std::fwrite(H.arr[k], 4, len, o);
    }
    std::fclose(o);
    return 0;
}
