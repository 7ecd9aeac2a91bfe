// Round reduction (Algorithm 1, UpdateEstimates and the c-MCERA sup) and the
// final normalisation of the estimates.
#include "mantra_dev.cuh"

namespace mantra {

constexpr int RED_NT = 1024;

// Block j < c: rowmax[j] = max_v S[j][v] (the sup over all nodes, nodes never
// hit contribute 0; no absolute value -- paper Sec. 3 c-MCERA).
// Block c: out_hmax = max_v hits[v] (empirical wimpy variance numerator).
__global__ void __launch_bounds__(RED_NT) k_round_reduce(const int* S, const u64* hits, uint32_t n, uint32_t c,
                                                          long long* rowmax, u64* hmax) {
    __shared__ long long red_i[RED_NT / 32];
    __shared__ u64 red_u[RED_NT / 32];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const uint32_t j = blockIdx.x;
    if (j < c) {
        const int* row = S + (size_t)j * n;
        int mx = INT_MIN;
        for (uint32_t v = tid; v < n; v += RED_NT) mx = max(mx, row[v]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xFFFFFFFFu, mx, o));
        if (lane == 0) red_i[wid] = mx;
        __syncthreads();
        if (wid == 0) {
            long long x = (lane < RED_NT / 32) ? red_i[lane] : (long long)INT_MIN;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) x = max(x, __shfl_xor_sync(0xFFFFFFFFu, x, o));
            if (lane == 0) rowmax[j] = x;
        }
    } else {
        u64 mx = 0;
        for (uint32_t v = tid; v < n; v += RED_NT) mx = max(mx, hits[v]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xFFFFFFFFu, mx, o));
        if (lane == 0) red_u[wid] = mx;
        __syncthreads();
        if (wid == 0) {
            u64 x = (lane < RED_NT / 32) ? red_u[lane] : 0ull;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) x = max(x, __shfl_xor_sync(0xFFFFFFFFu, x, o));
            if (lane == 0) *hmax = x;
        }
    }
}

// est_v = hits_v / r (Algorithm 1's return value), IEEE double division.
__global__ void k_normalise(const u64* hits, uint32_t n, uint64_t r, double* est) {
    const uint32_t v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v < n) est[v] = (double)hits[v] / (double)r;
}

cudaError_t launch_round_reduce(const int* S, const u64* hits, uint32_t n, uint32_t c, long long* rowmax, u64* hmax,
                                cudaStream_t st) {
    k_round_reduce<<<c + 1, RED_NT, 0, st>>>(S, hits, n, c, rowmax, hmax);
    return cudaGetLastError();
}

cudaError_t launch_normalise(const u64* hits, uint32_t n, uint64_t r, double* est, cudaStream_t st) {
    k_normalise<<<(n + 255) / 256, 256, 0, st>>>(hits, n, r, est);
    return cudaGetLastError();
}

}  // namespace mantra
