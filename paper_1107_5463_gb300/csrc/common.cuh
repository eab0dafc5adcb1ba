// Device-side building blocks shared by the spinmc kernels (sm_103a):
// Philox4x32-10, the device control block, and the fixed-order reduction of
// per-block partial sums that finishes every sweep's observables.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace spinmc {

// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11).  The ten round keys are
// precomputed on the host (key + r * Weyl constant) so that a kernel reads
// them straight from its parameter bank.
struct RoundKeys {
    uint32_t k0[10];
    uint32_t k1[10];
};

__host__ inline RoundKeys make_round_keys(uint64_t seed)
{
    RoundKeys rk;
    uint32_t k0 = (uint32_t)(seed & 0xffffffffu), k1 = (uint32_t)(seed >> 32);
    for (int r = 0; r < 10; ++r) {
        rk.k0[r] = k0;
        rk.k1[r] = k1;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return rk;
}

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, const RoundKeys& rk)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = c.x * 0xD2511F53u;
        const uint32_t hi0 = __umulhi(c.x, 0xD2511F53u);
        const uint32_t lo1 = c.z * 0xCD9E8D57u;
        const uint32_t hi1 = __umulhi(c.z, 0xCD9E8D57u);
        c = make_uint4(hi1 ^ c.y ^ rk.k0[r], lo1, hi0 ^ c.w ^ rk.k1[r], lo0);
    }
    return c;
}

enum Purpose : uint32_t { kSweep = 0, kInit = 1, kCoupling = 2, kExchange = 3 };

// Device control block: one per lattice, inside the caller's buffer.
struct Ctrl {
    unsigned long long t;      // index of the sweep in progress
    long long series_base;     // sweep index written to series[0]
    double* series_E;          // per-sweep energy, or null
    double* series_absm;       // per-sweep |m|, or null
    unsigned int done;         // blocks finished in the measuring pass
    unsigned int error;        // bit 0: a bounded device-side wait ran out (sticky)
    double obs[4];             // E, Mx, My, Mz after the last measured pass
};

// Partial sums one block contributes to a measured pass.  Ising passes use
// the integer members (exact), continuous spins the double members.
struct Partial {
    long long i0, i1;
    double f[4];
};

// Fold one value across a warp (any type with operator+).
template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block-wide sum, result valid in thread 0.  `scratch` holds >= 32 T.
template <typename T>
__device__ __forceinline__ T block_sum(T v, T* scratch)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) scratch[warp] = v;
    __syncthreads();
    T r = T(0);
    if (warp == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        r = lane < nw ? scratch[lane] : T(0);
        r = warp_sum(r);
    }
    return r;
}

// Called by every thread of every block at the end of a measured pass with
// the block's partial (valid in thread 0).  The last block to arrive adds all
// partials: thread k takes blocks k, k + blockDim, ... in order and the block
// tree-sums the threads, a fixed order for a given grid, so FP64 totals are
// reproducible.  Thread 0 of that block passes the totals to `finish` and
// resets the arrival count.
template <typename Finish>
__device__ __forceinline__ void finish_pass(Ctrl* ctrl, Partial* partials, const Partial& mine,
                                            Finish finish)
{
    __shared__ bool last;
    __shared__ long long red_i[32];
    __shared__ double red_f[32];
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = mine;
        __threadfence();
        const unsigned prev = atomicAdd(&ctrl->done, 1u);
        last = (prev == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    long long i0 = 0, i1 = 0;
    double f[4] = {0.0, 0.0, 0.0, 0.0};
    for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x) {
        const Partial* p = partials + b;
        i0 += __ldcg(&p->i0);
        i1 += __ldcg(&p->i1);
#pragma unroll
        for (int k = 0; k < 4; ++k) f[k] += __ldcg(&p->f[k]);
    }
    Partial tot;
    tot.i0 = block_sum(i0, red_i);
    tot.i1 = block_sum(i1, red_i);
#pragma unroll
    for (int k = 0; k < 4; ++k) tot.f[k] = block_sum(f[k], red_f);
    if (threadIdx.x == 0) {
        finish(tot);
        ctrl->done = 0;
        __threadfence();
    }
}

// Deferred finishing.  A measuring pass of thousands of short blocks loses
// several percent of its time if every block ends with the fence and the
// arrival atomic above while its SM slot waits.  Instead each block stores
// its partial (no fence, no atomic) and a one-block kernel launched right
// after the pass on the same stream adds them; the kernel boundary orders the
// stores before the loads.  Thread k adds blocks k, k + kFinishThreads, ...
// in order and the block tree-sums the threads: a fixed order for a given
// grid, so FP64 totals stay reproducible.
constexpr int kFinishThreads = 512;

__device__ __forceinline__ void store_partial(Partial* partials, const Partial& mine)
{
    if (threadIdx.x == 0) partials[blockIdx.x] = mine;
}

// Total of the first nblocks partials (FP: also the four double members),
// valid in thread 0.
template <bool FP>
__device__ __forceinline__ Partial sum_partials(const Partial* partials, unsigned nblocks)
{
    __shared__ long long red_i[32];
    __shared__ double red_f[32];
    long long i0 = 0, i1 = 0;
    double f[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll 4
    for (unsigned b = threadIdx.x; b < nblocks; b += blockDim.x) {
        i0 += partials[b].i0;
        i1 += partials[b].i1;
        if (FP) {
#pragma unroll
            for (int k = 0; k < 4; ++k) f[k] += partials[b].f[k];
        }
    }
    Partial tot;
    tot.i0 = block_sum(i0, red_i);
    tot.i1 = block_sum(i1, red_i);
#pragma unroll
    for (int k = 0; k < 4; ++k) tot.f[k] = FP ? block_sum(f[k], red_f) : 0.0;
    return tot;
}

}  // namespace spinmc
