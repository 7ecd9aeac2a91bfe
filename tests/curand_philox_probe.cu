// Test helper: four outputs of curand's Philox4_32_10 device generator after
// curand_init(seed, subsequence, offset), for cross-checking the oracle's
// Philox4x32-10 (test infrastructure; built by tests/test_gpu_philox.py).
#include <curand_kernel.h>

__global__ void philox_probe_kernel(unsigned long long seed, unsigned long long subsequence,
                                    unsigned long long offset, unsigned int* out) {
    curandStatePhilox4_32_10_t st;
    curand_init(seed, subsequence, offset, &st);
    const uint4 r = curand4(&st);
    out[0] = r.x; out[1] = r.y; out[2] = r.z; out[3] = r.w;
}

extern "C" int philox_probe(unsigned long long seed, unsigned long long subsequence, unsigned long long offset,
                            unsigned int* host_out) {
    unsigned int* d = nullptr;
    if (cudaMalloc(&d, 16) != cudaSuccess) return 1;
    philox_probe_kernel<<<1, 1>>>(seed, subsequence, offset, d);
    cudaError_t e = cudaMemcpy(host_out, d, 16, cudaMemcpyDeviceToHost);
    cudaFree(d);
    return e == cudaSuccess ? 0 : 2;
}
