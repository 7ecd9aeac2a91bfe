// Round reduction (Algorithm 1, UpdateEstimates and the c-MCERA sup) and the
// final normalisation of the estimates.
#include "mantra_dev.cuh"

#include <climits>

namespace mantra {

constexpr int RED_NT = 512;

// One reduction row: rows 0..c-1 are S[j][*] (max over all n nodes -- nodes
// never hit contribute 0, no absolute value: the sup of the c-MCERA, paper
// Sec. 3); row c is hits[*] (its max is the empirical wimpy variance's
// numerator).  row_start[p] is the first row of problem p (np + 1 entries).
__global__ void __launch_bounds__(RED_NT) k_round_reduce(const ReduceItem* items, const uint32_t* row_start,
                                                          const uint32_t* np_p) {
    __shared__ long long red_i[RED_NT / 32];
    __shared__ u64 red_u[RED_NT / 32];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const uint32_t np = *np_p;
    const uint32_t rows = np ? row_start[np] : 0;
    for (uint32_t row = blockIdx.x; row < rows; row += gridDim.x) {
        uint32_t lo = 0, hi = np;                       // row_start[lo] <= row < row_start[hi]
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (row_start[mid] <= row) lo = mid; else hi = mid;
        }
        const ReduceItem it = items[lo];
        const uint32_t j = row - row_start[lo];
        if (j < it.c) {
            long long mx = LLONG_MIN;
            if (it.S64) {
                const long long* r = it.S64 + (size_t)j * it.n;
                for (uint32_t v = tid; v < it.n; v += RED_NT) mx = max(mx, r[v]);
            } else {
                const int* r = it.S + (size_t)j * it.n;
                for (uint32_t v = tid; v < it.n; v += RED_NT) mx = max(mx, (long long)r[v]);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xFFFFFFFFu, mx, o));
            if (lane == 0) red_i[wid] = mx;
            __syncthreads();
            if (wid == 0) {
                long long x = (lane < RED_NT / 32) ? red_i[lane] : LLONG_MIN;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) x = max(x, __shfl_xor_sync(0xFFFFFFFFu, x, o));
                if (lane == 0) it.rowmax[j] = it.n ? x : 0;     // an empty family: 0
            }
        } else {
            u64 mx = 0;
            for (uint32_t v = tid; v < it.n; v += RED_NT) mx = max(mx, it.hits[v]);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xFFFFFFFFu, mx, o));
            if (lane == 0) red_u[wid] = mx;
            __syncthreads();
            if (wid == 0) {
                u64 x = (lane < RED_NT / 32) ? red_u[lane] : 0ull;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) x = max(x, __shfl_xor_sync(0xFFFFFFFFu, x, o));
                if (lane == 0) *it.hmax = x;
            }
        }
        __syncthreads();
    }
}

// est_v = hits_v / denom (Algorithm 1's return value), IEEE double division;
// denom = r, or r 2^32 for the ob sums (exact in double).
__global__ void k_normalise(const u64* hits, uint32_t n, double denom, double* est) {
    const uint32_t v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v < n) est[v] = (double)hits[v] / denom;
}

cudaError_t launch_round_reduce(const ReduceItem* items, const uint32_t* row_start, const uint32_t* np, int grid,
                                cudaStream_t st) {
    k_round_reduce<<<grid, RED_NT, 0, st>>>(items, row_start, np);
    return cudaGetLastError();
}

cudaError_t launch_normalise(const u64* hits, uint32_t n, double denom, double* est, cudaStream_t st) {
    k_normalise<<<(n + 255) / 256, 256, 0, st>>>(hits, n, denom, est);
    return cudaGetLastError();
}

}  // namespace mantra
