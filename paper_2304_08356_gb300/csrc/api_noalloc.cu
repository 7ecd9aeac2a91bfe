// Allocation-free variant of mantra_sample_paths for the sh and sfm
// optimalities.  The paper has no counterpart: this exists for callers that
// cannot call cudaMalloc once they are running -- a process whose device
// memory is fixed after start-up (a pre-sized serving process, an embedded or
// sandboxed host that gets no allocator on its hot path) or code that must not
// pay an allocator's latency or risk its failure between requests.
//
// The search scratch (per-CTA path counts, frontier lists, bitmaps) and the
// launch counters live in one file-scope __device__ array of a fixed size,
// kScratchBytes, which every GPU that loads the library holds until exit.  The
// graph (loaded earlier with mantra_graph_load) and the output buffers are the
// caller's.  Host code gets the array's device address with
// cudaGetSymbolAddress, once per device, on the first call made with that
// device current.
#include "mantra.h"
#include "mantra_dev.cuh"

#include <algorithm>
#include <mutex>

namespace mantra {
int graph_view(const mantra_graph* g, const DevGraph** dg, int* device, uint32_t* n, uint32_t* A, int* num_sms,
               size_t* smem_optin, std::mutex** mu);
}
using namespace mantra;

namespace {

constexpr size_t kScratchBytes = (size_t)64 << 20;     // 64 MiB per device
constexpr size_t kCtrBytes = 256;                       // launch counters + status word
constexpr size_t kTaskOff = kCtrBytes;                  // one-entry task table
constexpr size_t kUnitOff = kTaskOff + ((sizeof(Task) + 255) / 256) * 256;   // unit starts, task count, work counter
constexpr size_t kHeadBytes = kUnitOff + 256;
constexpr int kMaxDevices = 64;

}  // namespace

// The shared scratch.  In host code this name is only a host-side stand-in;
// its device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

namespace {

std::mutex g_setup_mu;
void* g_scratch_dev[kMaxDevices];   // device address of g_noalloc_scratch per device, nullptr until set up

// Device address of the scratch on the current device (set up on first use).
int scratch_address(void** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return MANTRA_E_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return MANTRA_E_CUDA;
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_scratch_dev[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) return MANTRA_E_CUDA;
        g_scratch_dev[dev] = p;
    }
    *out = g_scratch_dev[dev];
    return MANTRA_OK;
}

size_t round256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

extern "C" int mantra_sample_paths_noalloc(const mantra_graph* g, mantra_opt opt, uint64_t seed, uint32_t dom_pair,
                                           uint32_t dom_path, uint64_t i0, uint64_t count, uint32_t* s_dev,
                                           uint32_t* z_dev, uint64_t* sigma_dev, uint32_t* len_dev,
                                           uint32_t* nodes_dev, uint32_t cap, void* stream) {
    if (!g || !s_dev || !z_dev || !sigma_dev || !len_dev || (cap > 0 && !nodes_dev)) return MANTRA_E_INVAL;
    if (opt != MANTRA_SH && opt != MANTRA_SFM) return MANTRA_E_INVAL;
    if (dom_pair > 5 || dom_path > 5) return MANTRA_E_INVAL;
    if (count == 0) return MANTRA_OK;

    uint32_t n = 0, A = 0;
    int num_sms = 0, gdev = -1, cur = -1;
    size_t smem_optin = 0;
    std::mutex* gmu = nullptr;
    const DevGraph* dg = nullptr;
    const int vrc = graph_view(g, &dg, &gdev, &n, &A, &num_sms, &smem_optin, &gmu);
    if (vrc != MANTRA_OK) return vrc;
    // the scratch address, the launch and the stream all belong to the current
    // device; the graph's store must live on that same device
    if (cudaGetDevice(&cur) != cudaSuccess) return MANTRA_E_CUDA;
    if (cur != gdev) return MANTRA_E_INVAL;

    // layout: [counters | task table (one task) | overflow list (count entries) | per-CTA search regions]
    const size_t smem = bfs_smem_bytes(A);
    const bool in_smem = smem + bfs_static_smem(512) + 1024 <= smem_optin;
    BfsWs ws{};
    const size_t region = bfs_region_bytes(n, A, dg->max_vslots, in_smem, false, &ws);
    ws.nt = 512;
    const size_t head = kHeadBytes + round256(count * 8);
    if (head >= kScratchBytes || region > kScratchBytes - head) return MANTRA_E_INVAL;   // exceeds the fixed scratch
    int grid = (int)std::min<size_t>((size_t)num_sms, (kScratchBytes - head) / region);
    if (grid < 1) return MANTRA_E_INVAL;

    void* base = nullptr;
    int rc = scratch_address(&base);
    if (rc != MANTRA_OK) return rc;
    char* scratch = (char*)base;
    cudaStream_t st = (cudaStream_t)stream;

    std::lock_guard<std::mutex> lock(*gmu);
    // counters, path counts and global bitmaps must start at zero
    const size_t used = head + (size_t)grid * region;
    if (cudaMemsetAsync(scratch, 0, used, st) != cudaSuccess) return MANTRA_E_CUDA;
    if (bfs_configure(in_smem ? smem : 0) != cudaSuccess) return MANTRA_E_CUDA;

    Task task{};
    task.g = *dg;
    Job& j = task.job;
    j.seed = seed; j.i0 = i0; j.count = count; j.dom_pair = dom_pair; j.dom_path = dom_path; j.opt = (int)opt;
    j.ctr = (u64*)scratch;
    j.status = (int*)(scratch + 64);
    j.ovf_list = (uint64_t*)(scratch + kHeadBytes);
    j.rec_s = s_dev; j.rec_z = z_dev; j.rec_sig = (u64*)sigma_dev; j.rec_len = len_dev;
    j.rec_nodes = nodes_dev; j.rec_cap = cap;
    struct { uint64_t unit_start[2]; uint32_t ntasks; uint32_t pad; u64 work; } units = {{0, count}, 1u, 0u, 0ull};
    if (cudaMemcpyAsync(scratch + kTaskOff, &task, sizeof(Task), cudaMemcpyHostToDevice, st) != cudaSuccess)
        return MANTRA_E_CUDA;
    if (cudaMemcpyAsync(scratch + kUnitOff, &units, sizeof(units), cudaMemcpyHostToDevice, st) != cudaSuccess)
        return MANTRA_E_CUDA;
    ws.base = scratch + head;
    ws.stride = region;
    char* ub = scratch + kUnitOff;
    if (launch_bfs((const Task*)(scratch + kTaskOff), (const uint64_t*)ub, (const uint32_t*)(ub + 16), (u64*)(ub + 24),
                   ws, grid, in_smem ? smem : 0, false, false, st) != cudaSuccess)
        return MANTRA_E_CUDA;

    u64 h[9];
    if (cudaMemcpyAsync(h, scratch, 72, cudaMemcpyDeviceToHost, st) != cudaSuccess) return MANTRA_E_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return MANTRA_E_CUDA;
    const int status = (int)(h[8] & 0xFFFFFFFFu);
    if (status != 0) return status;
    if (h[C_NOVF] != 0) return MANTRA_E_OVERFLOW;     // this variant has no 128-bit re-run
    return MANTRA_OK;
}
