// Test helper: cuRAND's device Philox4_32_10 evaluated at given (counter, key)
// pairs, an independent implementation of the generator the library and the
// oracle use.  curand_init(seed, subsequence, offset) with subsequence = the
// counter's high 64 bits and offset = 4 x its low 64 bits makes the next
// curand4() return the block at exactly that counter.
#include <cstdint>

#include <cuda_runtime.h>
#include <curand_kernel.h>

__global__ void k_curand_philox(const uint4 *ctr, const uint2 *key, uint4 *out, long long n) {
    const long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
    if (i >= n) return;
    const unsigned long long seed = key[i].x | (static_cast<unsigned long long>(key[i].y) << 32);
    const unsigned long long sub = ctr[i].z | (static_cast<unsigned long long>(ctr[i].w) << 32);
    const unsigned long long off = ctr[i].x | (static_cast<unsigned long long>(ctr[i].y) << 32);
    curandStatePhilox4_32_10_t st;
    curand_init(seed, sub, 4ull * off, &st);
    out[i] = curand4(&st);
}

extern "C" int curand_philox(const uint32_t *ctr, const uint32_t *key, uint32_t *out, long long n) {
    uint4 *dc = nullptr, *dout = nullptr;
    uint2 *dk = nullptr;
    const size_t b4 = sizeof(uint4) * n, b2 = sizeof(uint2) * n;
    if (cudaMalloc(&dc, b4) || cudaMalloc(&dk, b2) || cudaMalloc(&dout, b4)) return 1;
    cudaMemcpy(dc, ctr, b4, cudaMemcpyHostToDevice);
    cudaMemcpy(dk, key, b2, cudaMemcpyHostToDevice);
    k_curand_philox<<<static_cast<unsigned>((n + 255) / 256), 256>>>(dc, dk, dout, n);
    const cudaError_t e = cudaMemcpy(out, dout, b4, cudaMemcpyDeviceToHost);
    cudaFree(dc);
    cudaFree(dk);
    cudaFree(dout);
    return e == cudaSuccess ? 0 : 2;
}
