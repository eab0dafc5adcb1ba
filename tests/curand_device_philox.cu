// Test infrastructure: outputs of cuRAND's device-API Philox4_32_10 generator
// (a library routine, called, not reimplemented), used to pin the oracle's
// Philox4x32-10 on counters whose words 2 and 3 are non-zero: the purpose and
// colour word of every real draw, which cuRAND's host generator never sets.
// Each query i runs curand_init(seed, subsequence[i], offset[i]) and returns
// the next curand4() block.
#include <cuda_runtime.h>
#include <curand_kernel.h>

__global__ void philox_blocks(unsigned long long seed, const unsigned long long* subseq,
                              const unsigned long long* offset, int n, uint4* out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    curandStatePhilox4_32_10_t st;
    curand_init(seed, subseq[i], offset[i], &st);
    out[i] = curand4(&st);
}

extern "C" int curand_device_philox(unsigned long long seed, const unsigned long long* subseq,
                                    const unsigned long long* offset, int n, unsigned* out)
{
    if (n <= 0) return 0;
    unsigned long long *d_sub = nullptr, *d_off = nullptr;
    uint4* d_out = nullptr;
    cudaError_t e = cudaMalloc(&d_sub, n * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMalloc(&d_off, n * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMalloc(&d_out, n * sizeof(uint4));
    if (e == cudaSuccess)
        e = cudaMemcpy(d_sub, subseq, n * sizeof(unsigned long long), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(d_off, offset, n * sizeof(unsigned long long), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        philox_blocks<<<(n + 127) / 128, 128>>>(seed, d_sub, d_off, n, d_out);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(out, d_out, n * sizeof(uint4), cudaMemcpyDeviceToHost);
    cudaFree(d_sub);
    cudaFree(d_off);
    cudaFree(d_out);
    return (int)e;
}
