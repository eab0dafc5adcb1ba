// Throughput microbenchmarks of the units the sweeps lean on, so that a
// measured compute ceiling stands beside the one derived from unit counts and
// the clock: Philox4x32-10 calls (the random numbers of every update rule,
// with the sweep kernels' own code), 32-bit integer multiplies (the pipe
// those calls load), FP32 fused multiply-adds and the hardware exp2 of the
// special-function unit (the continuous-spin arithmetic).  Every thread of a
// full-occupancy grid runs independent chains and folds its results into one
// output word, so nothing is optimised away; the caller times the launch.
#include "internal.h"

namespace spinmc {
namespace {

constexpr int kMbBlock = 256;
constexpr int kMbBlocksPerSm = 8;  // 2048 threads per SM
constexpr int kMbChains = 8;

// Philox4x32-10, key 1: thread g makes the calls with counters
// (g * iters + i, 7, 0, 0), i < iters, and xors all their outputs.
__global__ void __launch_bounds__(kMbBlock) mb_philox(RoundKeys rk, int iters, uint32_t* out)
{
    const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t acc = 0u;
    for (int i = 0; i < iters; ++i) {
        const uint4 r = philox4x32_10(make_uint4(g * (uint32_t)iters + (uint32_t)i, 7u, 0u, 0u), rk);
        acc ^= r.x ^ r.y ^ r.z ^ r.w;
    }
    out[g] = acc;
}

// Integer multiplies: kMbChains chains a <- mulhi(a, M0) + a * M1, two
// multiplies per step.
__global__ void __launch_bounds__(kMbBlock) mb_imad(int iters, uint32_t* out)
{
    const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t a[kMbChains];
#pragma unroll
    for (int k = 0; k < kMbChains; ++k) a[k] = g * 0x9E3779B9u + (uint32_t)k;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kMbChains; ++k) a[k] = __umulhi(a[k], 0xD2511F53u) + a[k] * 0xCD9E8D57u;
    }
    uint32_t acc = 0u;
#pragma unroll
    for (int k = 0; k < kMbChains; ++k) acc ^= a[k];
    out[g] = acc;
}

// FP32 fused multiply-adds: kMbChains chains x <- x * 0.9999999 + 1e-7.
__global__ void __launch_bounds__(kMbBlock) mb_ffma(int iters, float* out)
{
    const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    float x[kMbChains];
#pragma unroll
    for (int k = 0; k < kMbChains; ++k) x[k] = 1.0f + 1e-3f * (float)((g + k) & 1023);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kMbChains; ++k) x[k] = fmaf(x[k], 0.9999999f, 1e-7f);
    }
    float acc = 0.f;
#pragma unroll
    for (int k = 0; k < kMbChains; ++k) acc += x[k];
    out[g] = acc;
}

// Special-function unit: kMbChains chains x <- 2^(-x / 2) with the hardware
// exp2 (ex2.approx), which keeps x in (0.7, 1].
__global__ void __launch_bounds__(kMbBlock) mb_mufu(int iters, float* out)
{
    const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    float x[kMbChains];
#pragma unroll
    for (int k = 0; k < kMbChains; ++k) x[k] = 0.5f + 1e-3f * (float)((g + k) & 255);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kMbChains; ++k) {
            float y;
            asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(-0.5f * x[k]));
            x[k] = y;
        }
    }
    float acc = 0.f;
#pragma unroll
    for (int k = 0; k < kMbChains; ++k) acc += x[k];
    out[g] = acc;
}

int mb_blocks(int* blocks)
{
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail(e, "multiprocessor count");
    *blocks = sms * kMbBlocksPerSm;
    return SL_OK;
}

}  // namespace
}  // namespace spinmc

using namespace spinmc;

extern "C" int sl_microbench_threads(int* threads)
{
    if (!threads) return fail(SL_EINVAL, "threads is NULL");
    int blocks = 0;
    const int st = mb_blocks(&blocks);
    if (st != SL_OK) return st;
    *threads = blocks * kMbBlock;
    return SL_OK;
}

extern "C" int sl_microbench(int kind, int iterations, void* dev_out, size_t out_bytes,
                             void* stream, double* ops)
{
    if (kind < SL_MB_PHILOX || kind > SL_MB_MUFU) return fail(SL_EINVAL, "unknown microbenchmark %d", kind);
    if (iterations < 1) return fail(SL_EINVAL, "iterations must be >= 1");
    if (!dev_out || !ops) return fail(SL_EINVAL, "dev_out and ops must not be NULL");
    int blocks = 0;
    const int st = mb_blocks(&blocks);
    if (st != SL_OK) return st;
    const double threads = (double)blocks * kMbBlock;
    if (out_bytes < (size_t)blocks * kMbBlock * 4)
        return fail(SL_EINVAL, "dev_out needs %zu bytes", (size_t)blocks * kMbBlock * 4);
    if (kind == SL_MB_PHILOX && (double)iterations * threads > 4294967295.0)
        return fail(SL_EINVAL, "Philox counters would exceed 32 bits");
    cudaStream_t s = (cudaStream_t)stream;
    switch (kind) {
    case SL_MB_PHILOX:
        mb_philox<<<blocks, kMbBlock, 0, s>>>(make_round_keys(1), iterations, (uint32_t*)dev_out);
        *ops = threads * iterations;
        break;
    case SL_MB_IMAD:
        mb_imad<<<blocks, kMbBlock, 0, s>>>(iterations, (uint32_t*)dev_out);
        *ops = threads * iterations * kMbChains * 2.0;
        break;
    case SL_MB_FFMA:
        mb_ffma<<<blocks, kMbBlock, 0, s>>>(iterations, (float*)dev_out);
        *ops = threads * iterations * kMbChains;
        break;
    default:
        mb_mufu<<<blocks, kMbBlock, 0, s>>>(iterations, (float*)dev_out);
        *ops = threads * iterations * kMbChains;
        break;
    }
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? SL_OK : cuda_fail(e, "microbenchmark launch");
}
