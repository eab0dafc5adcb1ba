// Batched Edwards-Anderson +-J Ising spin glass with replica exchange
// (Weigel & Yavors'kii 2011, Section 2: "trivial parallelization over disorder
// realizations on top of the domain decomposition"; multi-spin coding).
//
// One CTA owns one disorder sample for a whole run: its couplings and the
// spins of all its replicas stay in shared memory, so sweeps make no HBM
// traffic.  Replicas are multispin-coded across a word: bit r of the word of
// a site is slot r's spin (1 = down), so one XOR per bond gives the
// unsatisfied-bond indicator of all replicas and a bitsliced adder their
// counts.  Every (site, slot) still draws its own Philox output (counter
// (j >> 2, t, sample * ntemps + slot, colour), output j & 3) and is accepted
// with the exact integer thresholds of its slot's current temperature, so the
// trajectory equals the oracle's per-replica sweeps bit for bit.  After each
// sweep the per-slot energies are reduced in the CTA and one warp performs
// the exchange step with exact integer thresholds.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <functional>
#include <new>
#include <vector>

#include "internal.h"

namespace spinmc {
namespace {

constexpr int kMaxTemps = 32;

struct PairMeta {
    int sign;        // sign of beta_k - beta_{k+1}
    int m1;          // table entries m < m1 hold ceil(exp(-|db| 2m) 2^32) - 1
    long long m0;    // m1 <= m < m0: accept iff U == 0; m >= m0: never
    int off;         // offset of the pair's table
};

// A queue entry: `count` samples of side L (class_samples[first ...]) run
// side by side, one per sub-group of blockDim / k threads, `stride` bytes of
// shared memory each.
struct WorkItem {
    int first, count, L, k, stride;
};

struct BatchArgs {
    uint32_t* spins;
    uint8_t* bonds;
    int32_t* perm;  // [sample][kMaxTemps] slot holding temperature k
    const int* class_samples;   // samples grouped by size
    const WorkItem* items;      // the work queue
    int nitems;
    unsigned* counter;          // next queue entry
    const long long* word_off;  // per sample: first spin word (colour 0), colour 1 at + H
    int d, ntemps;
    uint32_t sample0;  // global index of sample 0 (Philox counters use global indices)
    long long t0;
    int nsweeps;
    RoundKeys rk;
    const uint32_t* thr_temp;  // [ntemps][4]
    const uint32_t* pt_tab;
    const PairMeta* pt_meta;
    double* E_out;
};

__device__ __forceinline__ void fadd(uint32_t a, uint32_t b, uint32_t c, uint32_t& s, uint32_t& k)
{
    s = a ^ b ^ c;
    k = (a & b) | (c & (a ^ b));
}

// Per-thread bitsliced counter (8 planes, 0..255 per replica).
__device__ __forceinline__ void counter_add(uint32_t (&cnt)[8], uint32_t c0, uint32_t c1, uint32_t c2)
{
    uint32_t s, k;
    fadd(cnt[0], c0, 0u, s, k);
    cnt[0] = s;
    fadd(cnt[1], c1, k, s, k);
    cnt[1] = s;
    fadd(cnt[2], c2, k, s, k);
    cnt[2] = s;
#pragma unroll
    for (int b = 3; b < 8; ++b) {
        s = cnt[b] ^ k;
        k = cnt[b] & k;
        cnt[b] = s;
    }
}

template <int D>
__device__ __forceinline__ void count_planes(const uint32_t (&u)[6], uint32_t& b0, uint32_t& b1,
                                             uint32_t& b2)
{
    if (D == 2) {
        uint32_t s1, c1;
        fadd(u[0], u[1], u[2], s1, c1);
        b0 = s1 ^ u[3];
        const uint32_t k = s1 & u[3];
        b1 = c1 ^ k;
        b2 = c1 & k;
    } else {
        uint32_t s1, c1, s2, c2;
        fadd(u[0], u[1], u[2], s1, c1);
        fadd(u[3], u[4], u[5], s2, c2);
        b0 = s1 ^ s2;
        const uint32_t k = s1 & s2;
        fadd(c1, c2, k, b1, b2);
    }
}

// floor(n / L) for n < 2^26 from M = floor((2^32 - 1) / L) + 1: M L = 2^32 + e
// with 0 <= e < L, so n M / 2^32 exceeds n / L by n e / (L 2^32) < 1 / L,
// which never reaches the next integer
__device__ __forceinline__ int div_small(int n, uint32_t M)
{
    return (int)__umulhi((uint32_t)n, M);
}

// Append the comparison u > th to the low end of a plane word (pl = 2 pl +
// [u > th]) given nth = ~th: u + ~th = u - th - 1 + 2^32 carries out iff
// u > th, and the doubling adds that carry in.
__device__ __forceinline__ uint32_t push_gt(uint32_t pl, uint32_t u, uint32_t nth)
{
    uint32_t d, r;
    asm("add.cc.u32 %0, %2, %3;\n\taddc.u32 %1, %4, %4;"
        : "=r"(d), "=r"(r)
        : "r"(u), "r"(nth), "r"(pl));
    return r;
}

// A barrier over the nthr threads of one sample's sub-group: the whole CTA
// (barrier 0) or named barrier `bar` (1..15) of nthr threads.
__device__ __forceinline__ void group_sync(int bar, int nthr)
{
    if (bar == 0) __syncthreads();
    else asm volatile("bar.sync %0, %1;" ::"r"(bar), "r"(nthr) : "memory");
}

// All sweeps of one sample by a sub-group of nthr threads (local index tid)
// whose shared memory starts at base; the sample's couplings and the spins of
// all its replicas stay in shared memory for the whole run.
template <int D>
__device__ void run_sample(const BatchArgs& a, int s, int L, unsigned char* base, int tid,
                           int nthr, int bar)
{
    uint4* smem_u4 = reinterpret_cast<uint4*>(base);
    const int nt = a.ntemps;
    const int N = D == 3 ? L * L * L : L * L;
    const int H = N / 2, G = H / 4;
    uint32_t* S0 = reinterpret_cast<uint32_t*>(smem_u4);
    uint32_t* S1 = S0 + H;
    uint8_t* B0 = reinterpret_cast<uint8_t*>(S1 + H);
    uint8_t* B1 = B0 + H;
    // complemented thresholds (~th) of each slot's current temperature
    uint4* thr_slot = reinterpret_cast<uint4*>(B0 + ((2 * H + 15) / 16) * 16);
    long long* E_slot = reinterpret_cast<long long*>(thr_slot + kMaxTemps);
    int* unsat = reinterpret_cast<int*>(E_slot + kMaxTemps);
    int* sot = unsat + kMaxTemps;  // slot of temperature
    const int lane = tid & 31, warp = tid >> 5;
    const uint32_t active = nt == 32 ? 0xFFFFFFFFu : ((1u << nt) - 1u);
    const uint32_t gs = a.sample0 + (uint32_t)s;  // the sample's global index
    const uint32_t Minv = 0xFFFFFFFFu / (uint32_t)L + 1u;  // for div_small by L

    // load the sample
    const long long w0 = a.word_off[s];
    for (int q = tid; q < 2 * H; q += nthr) {
        S0[q] = a.spins[w0 + q];
        B0[q] = a.bonds[w0 + q];
    }
    if (tid < kMaxTemps) {
        unsat[tid] = 0;
        sot[tid] = tid < nt ? a.perm[s * kMaxTemps + tid] : tid;
    }
    group_sync(bar, nthr);
    if (tid < nt) {
        const uint4 th = reinterpret_cast<const uint4*>(a.thr_temp)[tid];
        thr_slot[sot[tid]] = make_uint4(~th.x, ~th.y, ~th.z, ~th.w);
    }
    group_sync(bar, nthr);

    for (int step = 0; step < a.nsweeps; ++step) {
        const long long t = a.t0 + step;
        uint32_t cnt[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        for (int c = 0; c < 2; ++c) {
            uint32_t* Sc = c ? S1 : S0;
            const uint32_t* So = c ? S0 : S1;
            const uint8_t* Bc = c ? B1 : B0;
            const uint8_t* Bo = c ? B0 : B1;
            const uint32_t ctr_w = (kSweep << 1) | (uint32_t)c;
            for (int g = tid; g < G; g += nthr) {
                // planes g_k[b]: bit r set iff slot r's u at site 4g+b exceeds
                // threshold k of its temperature
                // (slots from the highest down, each comparison pushed in at
                // bit 0, so slot r ends at bit r)
                uint32_t pl[4][3];
#pragma unroll
                for (int b = 0; b < 4; ++b) pl[b][0] = pl[b][1] = pl[b][2] = 0u;
                auto draw = [&](int r) {
                    const uint4 rnd = philox4x32_10(
                        make_uint4((uint32_t)g, (uint32_t)t, gs * (uint32_t)nt + (uint32_t)r, ctr_w), a.rk);
                    const uint4 nth = thr_slot[r];
                    const uint32_t u[4] = {rnd.x, rnd.y, rnd.z, rnd.w};
#pragma unroll
                    for (int b = 0; b < 4; ++b) {
                        pl[b][0] = push_gt(pl[b][0], u[b], nth.x);
                        pl[b][1] = push_gt(pl[b][1], u[b], nth.y);
                        if (D == 3) pl[b][2] = push_gt(pl[b][2], u[b], nth.z);
                    }
                };
                if (D == 3 && nt == kMaxTemps) {
                    // no branch between the draws, so the scheduler can
                    // interleave several Philox blocks
#pragma unroll
                    for (int r = kMaxTemps - 1; r >= 0; --r) draw(r);
                } else if (nt == kMaxTemps) {
                    // (2D: eight at a time, which keeps the registers in bounds)
#pragma unroll 8
                    for (int r = kMaxTemps - 1; r >= 0; --r) draw(r);
                } else {
#pragma unroll
                    for (int r = kMaxTemps - 1; r >= 0; --r)
                        if (r < nt) draw(r);
                }
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    const int j = 4 * g + b;
                    const int i0 = 2 * j;
                    const int rr = div_small(i0, Minv);
                    int x = i0 - rr * L;
                    const int z = div_small(rr, Minv);
                    const int y = rr - z * L;
                    x += (c + y + z) & 1;
                    int nm[3], np[3];
                    {
                        const int xm = x == 0 ? L - 1 : x - 1, xp = x == L - 1 ? 0 : x + 1;
                        const int ym = y == 0 ? L - 1 : y - 1, yp = y == L - 1 ? 0 : y + 1;
                        const int base = L * (y + L * z);
                        nm[0] = (base + xm) >> 1;
                        np[0] = (base + xp) >> 1;
                        nm[1] = (x + L * (ym + L * z)) >> 1;
                        np[1] = (x + L * (yp + L * z)) >> 1;
                        if (D == 3) {
                            const int zm = z == 0 ? L - 1 : z - 1, zp = z == L - 1 ? 0 : z + 1;
                            nm[2] = (x + L * (y + L * zm)) >> 1;
                            np[2] = (x + L * (y + L * zp)) >> 1;
                        }
                    }
                    const uint32_t Sv = Sc[j];
                    const uint32_t own_b = Bc[j];
                    uint32_t u[6];
#pragma unroll
                    for (int mu = 0; mu < D; ++mu) {
                        const uint32_t jm = (Bo[nm[mu]] >> mu) & 1u ? 0xFFFFFFFFu : 0u;
                        const uint32_t jp = (own_b >> mu) & 1u ? 0xFFFFFFFFu : 0u;
                        u[2 * mu] = Sv ^ So[nm[mu]] ^ jm;
                        u[2 * mu + 1] = Sv ^ So[np[mu]] ^ jp;
                    }
                    uint32_t b0, b1, b2;
                    count_planes<D>(u, b0, b1, b2);
                    const uint32_t ge1 = b0 | b1 | b2, ge2 = b1 | b2, ge3 = b2 | (b1 & b0);
                    uint32_t acc = (~pl[b][0] | ge1) & (~pl[b][1] | ge2);
                    if (D == 3) acc &= ~pl[b][2] | ge3;
                    acc &= active;
                    Sc[j] = Sv ^ acc;
                    if (c == 1) {
#pragma unroll
                        for (int q = 0; q < 2 * D; ++q) u[q] ^= acc;
                        count_planes<D>(u, b0, b1, b2);
                        counter_add(cnt, b0, b1, b2);
                    }
                }
            }
            group_sync(bar, nthr);
        }
        // per-slot unsatisfied bonds: the warp's counters are summed slot by
        // slot in bitsliced form, by a butterfly of bitsliced adds over the
        // lanes (five rounds; a sum of 32 counters below 256 needs 13
        // planes), after which lane r reads slot r's total from bit r
        {
            uint32_t w[13];
#pragma unroll
            for (int b = 0; b < 13; ++b) w[b] = b < 8 ? cnt[b] : 0u;
#pragma unroll
            for (int lvl = 0; lvl < 5; ++lvl) {
                const int nb = 9 + lvl;  // planes that can be set after this round
                uint32_t c = 0u;
#pragma unroll
                for (int b = 0; b < 13; ++b) {
                    if (b < nb) {
                        const uint32_t x =
                            b < nb - 1 ? __shfl_xor_sync(0xFFFFFFFFu, w[b], 16 >> lvl) : 0u;
                        const uint32_t sum = w[b] ^ x ^ c;
                        c = (w[b] & x) | (c & (w[b] ^ x));
                        w[b] = sum;
                    }
                }
            }
            int mine = 0;
#pragma unroll
            for (int b = 0; b < 13; ++b) mine |= (int)((w[b] >> lane) & 1u) << b;
            atomicAdd(&unsat[lane], mine);
        }
        group_sync(bar, nthr);
        if (warp == 0) {
            const int k = lane;
            // energy of every slot: E = -(dN - 2 unsat)
            E_slot[lane] = -(long long)(D * N) + 2LL * unsat[lane];
            __syncwarp();
            if (a.E_out && k < nt)
                a.E_out[((long long)s * a.nsweeps + step) * nt + k] = (double)E_slot[sot[k]];
            if (k + 1 < nt && (k & 1) == (int)(t & 1)) {
                const int ra = sot[k], rb = sot[k + 1];
                const long long dE = E_slot[ra] - E_slot[rb];
                const PairMeta pm = a.pt_meta[k];
                const int sg = pm.sign * (dE > 0 ? 1 : (dE < 0 ? -1 : 0));
                bool accept = sg >= 0;
                if (!accept) {
                    const long long m = (dE < 0 ? -dE : dE) >> 1;
                    const uint4 rnd = philox4x32_10(
                        make_uint4((uint32_t)k, (uint32_t)t, gs, kExchange << 1), a.rk);
                    if (m < pm.m1) accept = rnd.x <= a.pt_tab[pm.off + m];
                    else if (m < pm.m0) accept = rnd.x == 0u;
                }
                if (accept) {
                    sot[k] = rb;
                    sot[k + 1] = ra;
                }
            }
            __syncwarp();
            if (k < nt) {
                const uint4 th = reinterpret_cast<const uint4*>(a.thr_temp)[k];
                thr_slot[sot[k]] = make_uint4(~th.x, ~th.y, ~th.z, ~th.w);
            }
            unsat[lane] = 0;
        }
        group_sync(bar, nthr);
    }
    // write the sample back
    for (int q = tid; q < 2 * H; q += nthr) a.spins[w0 + q] = S0[q];
    if (tid < nt) a.perm[s * kMaxTemps + tid] = sot[tid];
}

// One persistent launch for the whole batch: every CTA takes work items
// (packs of k samples of one size, k sub-groups of blockDim / k threads, each
// with its own named barrier and shared-memory slice) from a queue ordered
// largest first, until the queue is empty.
template <int D>
__global__ void __launch_bounds__(1024) ea_pt_persistent(const BatchArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int item;
    while (true) {
        if (threadIdx.x == 0) item = (int)atomicAdd(a.counter, 1u);
        __syncthreads();
        const int it = item;
        if (it >= a.nitems) break;
        const WorkItem w = a.items[it];
        const int nthr = blockDim.x / w.k;
        const int g = threadIdx.x / nthr;
        if (g < w.count)
            run_sample<D>(a, a.class_samples[w.first + g], w.L, smem_raw + (size_t)g * w.stride,
                          threadIdx.x - g * nthr, nthr, w.k == 1 ? 0 : g + 1);
        __syncthreads();
    }
}

__global__ void batch_init_kernel(uint32_t* spins, uint8_t* bonds, int32_t* perm,
                                  const int* Ls, const long long* word_off, int d, int ntemps,
                                  uint32_t sample0, RoundKeys rk)
{
    const int s = blockIdx.x;
    const uint32_t gs = sample0 + (uint32_t)s;
    const int L = Ls[s];
    const int N = d == 3 ? L * L * L : L * L;
    const int H = N / 2;
    uint32_t* S = spins + word_off[s];
    uint8_t* B = bonds + word_off[s];
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        const int x = i % L, y = (i / L) % L, z = i / (L * L);
        const int c = (x + y + z) & 1;
        uint8_t bits = 0;
        for (int mu = 0; mu < d; ++mu) {
            const uint4 r = philox4x32_10(
                make_uint4((uint32_t)i, (uint32_t)mu, gs, kCoupling << 1), rk);
            if (!(r.x >> 31)) bits |= (uint8_t)(1u << mu);
        }
        B[c * H + (i >> 1)] = bits;
    }
    for (int q = threadIdx.x; q < 2 * (H / 4); q += blockDim.x) {
        const int c = q / (H / 4), g = q % (H / 4);
        uint32_t w[4] = {0, 0, 0, 0};
        for (int r = 0; r < ntemps; ++r) {
            const uint4 o = philox4x32_10(
                make_uint4((uint32_t)g, 0u, gs * (uint32_t)ntemps + (uint32_t)r,
                           (kInit << 1) | (uint32_t)c),
                rk);
            const uint32_t u[4] = {o.x, o.y, o.z, o.w};
            for (int b = 0; b < 4; ++b)
                if (!(u[b] >> 31)) w[b] |= 1u << r;
        }
        for (int b = 0; b < 4; ++b) S[c * H + 4 * g + b] = w[b];
    }
    if (threadIdx.x < kMaxTemps) perm[s * kMaxTemps + threadIdx.x] = threadIdx.x;
}

__global__ void batch_gather_kernel(const uint32_t* spins, const uint8_t* bonds, int8_t* out,
                                    long long w0, int L, int d, int slot, int want_bonds)
{
    const int N = d == 3 ? L * L * L : L * L;
    const int H = N / 2;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        const int x = i % L, y = (i / L) % L, z = i / (L * L);
        const int c = (x + y + z) & 1;
        if (!want_bonds) {
            const uint32_t w = spins[w0 + c * H + (i >> 1)];
            out[i] = ((w >> slot) & 1u) ? (int8_t)-1 : (int8_t)1;
        } else {
            const uint8_t b = bonds[w0 + c * H + (i >> 1)];
            for (int mu = 0; mu < d; ++mu)
                out[(long long)mu * N + i] = ((b >> mu) & 1u) ? (int8_t)-1 : (int8_t)1;
        }
    }
}

// Sets bit `slot` of every site word of one sample from a natural-order
// +-1 configuration (1 = down); the other slots' bits are kept.
__global__ void batch_scatter_kernel(uint32_t* spins, const int8_t* nat, long long w0, int L,
                                     int d, int slot)
{
    const int N = d == 3 ? L * L * L : L * L;
    const int H = N / 2;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        const int x = i % L, y = (i / L) % L, z = i / (L * L);
        const int c = (x + y + z) & 1;
        uint32_t* w = spins + w0 + c * H + (i >> 1);
        *w = (*w & ~(1u << slot)) | ((nat[i] < 0 ? 1u : 0u) << slot);
    }
}

size_t smem_bytes(int d, int L)
{
    const int N = d == 3 ? L * L * L : L * L;
    const int H = N / 2;
    return (size_t)2 * H * 4 + ((size_t)(2 * H + 15) / 16) * 16 + kMaxTemps * 16 +
           kMaxTemps * 8 + 2 * kMaxTemps * 4;
}


}  // namespace
}  // namespace spinmc

using namespace spinmc;

struct sl_batch {
    int d, nsamples, ntemps;
    uint32_t sample0;  // global index of the batch's first sample
    std::vector<int> L;
    std::vector<long long> word_off;
    std::vector<int> class_L;                 // distinct sizes, largest first
    std::vector<std::vector<int>> class_ids;  // samples of each size
    std::vector<int> class_dev_off;           // offset of each class in dev class list
    double betas[kMaxTemps];
    uint64_t seed;
    int64_t sweeps_done;
    cudaStream_t stream;
    uint32_t* spins;
    uint8_t* bonds;
    int32_t* perm;
    int* Ls_dev;
    long long* word_off_dev;
    int* class_dev;
    uint32_t* thr_temp;
    uint32_t* pt_tab;
    PairMeta* pt_meta;
    int8_t* staging;
    long long total_words;
    void* owned_buf;
    // persistent launch: work queue, per-class pack sizes, graph
    WorkItem* items_dev;
    unsigned* counter;
    uint32_t* backup_spins;
    int32_t* backup_perm;
    std::vector<int> class_k;        // samples per CTA for each size class
    std::vector<double> class_cost;  // measured SM-milliseconds per sample-sweep (0: untimed)
    int nitems, grid;
    size_t smem_dyn;
    int autotune, force_k, tuned;
    cudaStream_t cap_stream;
    cudaGraph_t graph_def;       // kept alive: kernel_node belongs to it
    cudaGraphExec_t graph;
    cudaGraphNode_t kernel_node;
};

namespace {

struct BatchLayout {
    size_t off_spins, off_bonds, off_perm, off_Ls, off_woff, off_class, off_thr, off_meta,
        off_tab, off_staging, off_items, off_counter, off_backup, off_backup_perm, total;
    long long total_words;
    int tab_entries;
};

int batch_check(int d, const int* Ls, int nsamples, int ntemps, const double* betas = nullptr)
{
    if (betas)
        for (int k = 0; k < ntemps && k < kMaxTemps; ++k)
            if (!(betas[k] >= 0.0) || !std::isfinite(betas[k]))
                return fail(SL_EINVAL, "betas must be finite and >= 0");
    if (d != 2 && d != 3) return fail(SL_EINVAL, "d must be 2 or 3");
    if (!Ls || nsamples < 1) return fail(SL_EINVAL, "need at least one sample");
    if (ntemps < 2 || ntemps > kMaxTemps) return fail(SL_EINVAL, "ntemps must be in [2, 32]");
    for (int s = 0; s < nsamples; ++s) {
        const int L = Ls[s];
        if (L < 4 || L > 32 || L % 4) return fail(SL_EINVAL, "sample %d: L must be a multiple of 4 in [4, 32]", s);
        if (smem_bytes(d, L) > 220 * 1024) return fail(SL_EINVAL, "sample %d: L too large", s);
    }
    return SL_OK;
}

// Exchange tables for the pairs of a beta ladder (see PairMeta).  The values
// are u <= ceil(exp(-|db| 2m) 2^32) - 1 <=> u < exp(Delta) 2^32 for integer u.
void build_pt(const double* betas, int nt, long long max_m, std::vector<PairMeta>& meta,
              std::vector<uint32_t>& tab)
{
    meta.assign(kMaxTemps, PairMeta{0, 0, 0, 0});
    tab.clear();
    for (int k = 0; k + 1 < nt; ++k) {
        const double db = betas[k] - betas[k + 1];
        PairMeta pm;
        pm.sign = db > 0.0 ? 1 : (db < 0.0 ? -1 : 0);
        pm.off = (int)tab.size();
        pm.m1 = 0;
        pm.m0 = 0;
        if (pm.sign != 0) {
            const double a = std::fabs(db);
            long long m = 0;
            for (;; ++m) {
                const double x = std::exp(-(a * (double)(2 * m))) * 4294967296.0;
                if (!(x > 1.0) || m > max_m) break;
                double T = std::ceil(x) - 1.0;
                if (T > 4294967295.0) T = 4294967295.0;
                tab.push_back((uint32_t)T);
            }
            pm.m1 = (int)m;
            // first m with exp(...) == 0 in FP64
            long long lo = m, hi = m;
            while (hi <= max_m && std::exp(-(a * (double)(2 * hi))) > 0.0) hi = hi * 2 + 1;
            if (hi > max_m) {
                pm.m0 = max_m + 1;
            } else {
                while (lo < hi) {
                    const long long mid = (lo + hi) / 2;
                    if (std::exp(-(a * (double)(2 * mid))) > 0.0) lo = mid + 1;
                    else hi = mid;
                }
                pm.m0 = lo;
            }
        }
        meta[k] = pm;
    }
}

BatchLayout batch_layout(int d, const int* Ls, int nsamples, int ntemps, const double* betas)
{
    BatchLayout y;
    long long words = 0, max_m = 0;
    for (int s = 0; s < nsamples; ++s) {
        const long long N = (long long)Ls[s] * Ls[s] * (d == 3 ? Ls[s] : 1);
        words += N;  // 2 colours x N/2 words
        max_m = std::max(max_m, (long long)d * N);
    }
    y.total_words = words;
    y.tab_entries = 0;
    {
        std::vector<PairMeta> meta;
        std::vector<uint32_t> tab;
        build_pt(betas, ntemps, max_m, meta, tab);
        y.tab_entries = (int)tab.size();
    }
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off += align_up(bytes);
        return o;
    };
    y.off_spins = take((size_t)words * 4);
    y.off_bonds = take((size_t)words);
    y.off_perm = take((size_t)nsamples * kMaxTemps * 4);
    y.off_Ls = take((size_t)nsamples * 4);
    y.off_woff = take((size_t)nsamples * 8);
    y.off_class = take((size_t)nsamples * 4);
    y.off_thr = take((size_t)kMaxTemps * 16);
    y.off_meta = take(sizeof(PairMeta) * kMaxTemps);
    y.off_tab = take((size_t)(y.tab_entries + 1) * 4);
    long long maxN = 0;
    for (int s = 0; s < nsamples; ++s)
        maxN = std::max(maxN, (long long)Ls[s] * Ls[s] * (d == 3 ? Ls[s] : 1));
    y.off_staging = take((size_t)d * maxN);
    y.off_items = take((size_t)nsamples * sizeof(WorkItem));
    y.off_counter = take(sizeof(unsigned));
    y.off_backup = take((size_t)words * 4);
    y.off_backup_perm = take((size_t)nsamples * kMaxTemps * 4);
    y.total = off;
    return y;
}

int dev_attr(cudaDeviceAttr attr, int fallback)
{
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&v, attr, dev) != cudaSuccess)
        return fallback;
    return v;
}

size_t pack_stride(int d, int L) { return (smem_bytes(d, L) + 127) / 128 * 128; }

// packs of k samples for class ci appended to items
void class_items(const sl_batch* b, int ci, int k, std::vector<WorkItem>& items)
{
    const int n = (int)b->class_ids[ci].size();
    for (int q = 0; q < n; q += k) {
        WorkItem w;
        w.first = b->class_dev_off[ci] + q;
        w.count = std::min(k, n - q);
        w.L = b->class_L[ci];
        w.k = k;
        w.stride = (int)pack_stride(b->d, w.L);
        items.push_back(w);
    }
}

template <int D>
cudaError_t launch_persistent(const BatchArgs& a, int grid, size_t smem, cudaStream_t st)
{
    cudaError_t e = cudaFuncSetAttribute(ea_pt_persistent<D>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(a.counter, 0, sizeof(unsigned), st);
    if (e != cudaSuccess) return e;
    ea_pt_persistent<D><<<grid, 1024, smem, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_any(const sl_batch* b, const BatchArgs& a, int grid, size_t smem, cudaStream_t st)
{
    return b->d == 3 ? launch_persistent<3>(a, grid, smem, st) : launch_persistent<2>(a, grid, smem, st);
}

BatchArgs base_args(const sl_batch* b)
{
    BatchArgs a;
    std::memset(&a, 0, sizeof a);
    a.spins = b->spins;
    a.bonds = b->bonds;
    a.perm = b->perm;
    a.word_off = b->word_off_dev;
    a.class_samples = b->class_dev;
    a.items = b->items_dev;
    a.counter = b->counter;
    a.d = b->d;
    a.ntemps = b->ntemps;
    a.sample0 = b->sample0;
    a.thr_temp = b->thr_temp;
    a.pt_tab = b->pt_tab;
    a.pt_meta = b->pt_meta;
    return a;
}

// The largest pack size k in {1, 2, 4, 8} whose shared memory fits one CTA.
int max_pack(const sl_batch* b, int ci)
{
    const size_t limit = (size_t)dev_attr(cudaDevAttrMaxSharedMemoryPerBlockOptin, 227 * 1024);
    const size_t st = pack_stride(b->d, b->class_L[ci]);
    int k = 8;
    while (k > 1 && (size_t)k * st > limit) k /= 2;
    return k;
}

// Makespan of the work queue for pack sizes ks (one per class) when every
// pack of class ci takes item_ms[ci][log2 k] and nctas CTAs take packs in the
// queue's order (largest first), each the next one as it frees up.
double simulate(const sl_batch* b, const std::vector<int>& ks,
                const std::vector<std::vector<double>>& item_ms, int nctas)
{
    std::vector<double> cost;
    for (size_t ci = 0; ci < ks.size(); ++ci) {
        int lk = 0;
        while ((1 << lk) < ks[ci]) ++lk;
        const int n = (int)b->class_ids[ci].size();
        for (int q = 0; q < n; q += ks[ci]) cost.push_back(item_ms[ci][lk]);
    }
    std::sort(cost.begin(), cost.end(), [](double p, double q) { return p > q; });
    std::vector<double> busy(std::max(1, nctas), 0.0);  // min-heap of finish times
    for (double c : cost) {
        std::pop_heap(busy.begin(), busy.end(), std::greater<double>());
        busy.back() += c;
        std::push_heap(busy.begin(), busy.end(), std::greater<double>());
    }
    return *std::max_element(busy.begin(), busy.end());
}

// Autotuner: for every size class, time `trial` sweeps of one pack per CTA
// for each pack size that fits, on a copy of the state that is restored
// afterwards (the chain does not depend on the pack size); then choose the
// pack size of every class that minimises the simulated makespan of the
// whole queue (coarse packs can leave the last CTAs running alone).
int autotune(sl_batch* b)
{
    const int nsm = dev_attr(cudaDevAttrMultiProcessorCount, 152);
    const int trial = 2;
    cudaError_t e = cudaMemcpyAsync(b->backup_spins, b->spins, (size_t)b->total_words * 4,
                                    cudaMemcpyDeviceToDevice, b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->backup_perm, b->perm, (size_t)b->nsamples * kMaxTemps * 4,
                            cudaMemcpyDeviceToDevice, b->stream);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    const int nc = (int)b->class_L.size();
    std::vector<std::vector<double>> item_ms(nc, std::vector<double>(4, -1.0));
    for (int ci = 0; ci < nc && e == cudaSuccess; ++ci) {
        for (int k = 1; k <= max_pack(b, ci) && e == cudaSuccess; k *= 2) {
            if (k > 1 && (int)b->class_ids[ci].size() < k) break;
            std::vector<WorkItem> items;
            class_items(b, ci, k, items);
            const int used = std::min((int)items.size(), nsm);
            items.resize(used);  // one pack per CTA
            int samples = 0;
            for (const WorkItem& w : items) samples += w.count;
            e = cudaMemcpyAsync(b->items_dev, items.data(), items.size() * sizeof(WorkItem),
                                cudaMemcpyHostToDevice, b->stream);
            BatchArgs a = base_args(b);
            a.nitems = used;
            a.nsweeps = trial;
            a.rk = make_round_keys(b->seed);
            const size_t smem = (size_t)k * pack_stride(b->d, b->class_L[ci]);
            for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {  // the first run warms up
                if (e == cudaSuccess) e = cudaEventRecord(e0, b->stream);
                if (e == cudaSuccess) e = launch_any(b, a, used, smem, b->stream);
                if (e == cudaSuccess) e = cudaEventRecord(e1, b->stream);
                if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            }
            float ms = 0.0f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            int lk = 0;
            while ((1 << lk) < k) ++lk;
            item_ms[ci][lk] = (double)ms / trial;
            (void)samples;
        }
    }
    if (e == cudaSuccess) {
        // exhaustive search over the timed pack sizes (at most 4^classes)
        const int nsm = dev_attr(cudaDevAttrMultiProcessorCount, 152);
        std::vector<int> ks(nc, 1), best_ks(nc, 1);
        double best = 1e300;
        std::function<void(int)> rec = [&](int ci) {
            if (ci == nc) {
                const double m = simulate(b, ks, item_ms, nsm);
                if (m < best) {
                    best = m;
                    best_ks = ks;
                }
                return;
            }
            for (int lk = 0; lk < 4; ++lk) {
                if (item_ms[ci][lk] < 0.0) continue;
                ks[ci] = 1 << lk;
                rec(ci + 1);
            }
        };
        rec(0);
        for (int ci = 0; ci < nc; ++ci) {
            int lk = 0;
            while ((1 << lk) < best_ks[ci]) ++lk;
            b->class_k[ci] = best_ks[ci];
            b->class_cost[ci] = item_ms[ci][lk] / best_ks[ci];  // ms per sample-sweep on one CTA
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->spins, b->backup_spins, (size_t)b->total_words * 4,
                            cudaMemcpyDeviceToDevice, b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->perm, b->backup_perm, (size_t)b->nsamples * kMaxTemps * 4,
                            cudaMemcpyDeviceToDevice, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    return e == cudaSuccess ? SL_OK : cuda_fail(e, "batch autotune");
}

// Work queue from the chosen pack sizes, most expensive packs first, and the
// graph of one launch (queue reset + persistent kernel).
int build_queue(sl_batch* b)
{
    const int nc = (int)b->class_L.size();
    std::vector<WorkItem> items;
    std::vector<double> cost;
    for (int ci = 0; ci < nc; ++ci) {
        const int k = b->force_k > 0 ? std::min(b->force_k, max_pack(b, ci)) : b->class_k[ci];
        const size_t before = items.size();
        class_items(b, ci, k, items);
        // a pack's measured time (class_cost is per sample of a pack of k);
        // without a timing, a pack costs its sites (the work is per site)
        const double per_sample = b->class_cost[ci] > 0.0 && b->force_k <= 0
                                      ? b->class_cost[ci]
                                      : (double)b->class_L[ci] * b->class_L[ci] *
                                            (b->d == 3 ? b->class_L[ci] : 1);
        for (size_t q = before; q < items.size(); ++q) cost.push_back(per_sample * k);
    }
    std::vector<int> order(items.size());
    for (size_t q = 0; q < order.size(); ++q) order[q] = (int)q;
    std::stable_sort(order.begin(), order.end(), [&](int p, int q) { return cost[p] > cost[q]; });
    std::vector<WorkItem> sorted;
    size_t smem = 0;
    for (int q : order) {
        sorted.push_back(items[q]);
        smem = std::max(smem, (size_t)items[q].k * items[q].stride);
    }
    const int nsm = dev_attr(cudaDevAttrMultiProcessorCount, 152);
    const size_t per_sm = (size_t)dev_attr(cudaDevAttrMaxSharedMemoryPerMultiprocessor, 228 * 1024);
    const int per = std::max(1, std::min(2, (int)(per_sm / (smem + 1024))));  // 1024 threads: <= 2
    b->grid = std::min((int)sorted.size(), nsm * per);
    b->nitems = (int)sorted.size();
    b->smem_dyn = smem;
    cudaError_t e = cudaMemcpyAsync(b->items_dev, sorted.data(), sorted.size() * sizeof(WorkItem),
                                    cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return cuda_fail(e, "batch work queue");
    if (b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
    if (b->graph_def) {
        cudaGraphDestroy(b->graph_def);
        b->graph_def = nullptr;
    }
    BatchArgs a = base_args(b);
    a.nitems = b->nitems;
    a.rk = make_round_keys(b->seed);
    a.nsweeps = 1;
    e = cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamBeginCapture");
    const cudaError_t el = launch_any(b, a, b->grid, b->smem_dyn, b->cap_stream);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(b->cap_stream, &g);
    if (el != cudaSuccess || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return cuda_fail(el != cudaSuccess ? el : e, "batch graph capture");
    }
    size_t nnodes = 0;
    e = cudaGraphGetNodes(g, nullptr, &nnodes);
    std::vector<cudaGraphNode_t> nodes(nnodes);
    if (e == cudaSuccess) e = cudaGraphGetNodes(g, nodes.data(), &nnodes);
    b->kernel_node = nullptr;
    for (size_t q = 0; q < nnodes && e == cudaSuccess; ++q) {
        cudaGraphNodeType t;
        e = cudaGraphNodeGetType(nodes[q], &t);
        if (e == cudaSuccess && t == cudaGraphNodeTypeKernel) b->kernel_node = nodes[q];
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->graph, g, 0);
    if (e != cudaSuccess || !b->kernel_node) {
        cudaGraphDestroy(g);
        b->graph = nullptr;
        return cuda_fail(e != cudaSuccess ? e : cudaErrorUnknown, "batch graph");
    }
    b->graph_def = g;
    return SL_OK;
}

}  // namespace

extern "C" {

int sl_batch_required_bytes(int d, const int* L_per_sample, int nsamples, int ntemps,
                            const double* betas, size_t* bytes)
{
    if (!bytes || !betas) return fail(SL_EINVAL, "NULL argument");
    int st = batch_check(d, L_per_sample, nsamples, ntemps, betas);
    if (st != SL_OK) return st;
    *bytes = batch_layout(d, L_per_sample, nsamples, ntemps, betas).total;
    return SL_OK;
}

int sl_batch_create(int d, const int* L_per_sample, int nsamples, int ntemps, const double* betas,
                    uint64_t seed, uint32_t first_sample, void* dev_buf, size_t dev_buf_bytes,
                    void* stream, sl_batch** out)
{
    if (!out) return fail(SL_EINVAL, "out is NULL");
    *out = nullptr;
    if (!betas) return fail(SL_EINVAL, "betas is NULL");
    int st = batch_check(d, L_per_sample, nsamples, ntemps, betas);
    if (st != SL_OK) return st;
    if (((uint64_t)first_sample + (uint64_t)nsamples) * (uint64_t)ntemps > 4294967296ULL)
        return fail(SL_EINVAL, "global replica ids (first_sample + nsamples) * ntemps exceed 2^32");
    const BatchLayout y = batch_layout(d, L_per_sample, nsamples, ntemps, betas);
    void* owned = nullptr;
    if (!dev_buf) {
        const cudaError_t e = cudaMalloc(&owned, y.total);
        if (e != cudaSuccess) return fail(SL_ENOMEM, "cudaMalloc(%zu) failed", y.total);
        dev_buf = owned;
        dev_buf_bytes = y.total;
    }
    if ((uintptr_t)dev_buf % kAlign) return fail(SL_EINVAL, "dev_buf must be 256-byte aligned");
    if (dev_buf_bytes < y.total) {
        if (owned) cudaFree(owned);
        return fail(SL_ENOMEM, "dev_buf holds %zu bytes, %zu needed", dev_buf_bytes, y.total);
    }
    sl_batch* b = new (std::nothrow) sl_batch();
    if (!b) {
        if (owned) cudaFree(owned);
        return fail(SL_ENOMEM, "host allocation failed");
    }
    char* base = (char*)dev_buf;
    b->d = d;
    b->nsamples = nsamples;
    b->ntemps = ntemps;
    b->sample0 = first_sample;
    b->L.assign(L_per_sample, L_per_sample + nsamples);
    b->word_off.resize(nsamples);
    long long w = 0;
    for (int s = 0; s < nsamples; ++s) {
        b->word_off[s] = w;
        w += (long long)b->L[s] * b->L[s] * (d == 3 ? b->L[s] : 1);
    }
    b->total_words = w;
    for (int k = 0; k < ntemps; ++k) b->betas[k] = betas[k];
    b->seed = seed;
    b->sweeps_done = 0;
    b->stream = (cudaStream_t)stream;
    b->spins = (uint32_t*)(base + y.off_spins);
    b->bonds = (uint8_t*)(base + y.off_bonds);
    b->perm = (int32_t*)(base + y.off_perm);
    b->Ls_dev = (int*)(base + y.off_Ls);
    b->word_off_dev = (long long*)(base + y.off_woff);
    b->class_dev = (int*)(base + y.off_class);
    b->thr_temp = (uint32_t*)(base + y.off_thr);
    b->pt_meta = (PairMeta*)(base + y.off_meta);
    b->pt_tab = (uint32_t*)(base + y.off_tab);
    b->staging = (int8_t*)(base + y.off_staging);
    b->owned_buf = owned;
    b->items_dev = (WorkItem*)(base + y.off_items);
    b->counter = (unsigned*)(base + y.off_counter);
    b->backup_spins = (uint32_t*)(base + y.off_backup);
    b->backup_perm = (int32_t*)(base + y.off_backup_perm);
    b->nitems = 0;
    b->grid = 0;
    b->smem_dyn = 0;
    b->autotune = 1;
    b->force_k = 0;
    b->tuned = 0;
    b->cap_stream = nullptr;
    b->graph_def = nullptr;
    b->graph = nullptr;
    b->kernel_node = nullptr;
    // size classes, largest first
    std::vector<int> sizes(b->L);
    std::sort(sizes.begin(), sizes.end(), [](int p, int q) { return p > q; });
    sizes.erase(std::unique(sizes.begin(), sizes.end()), sizes.end());
    std::vector<int> class_list;
    for (int L : sizes) {
        std::vector<int> ids;
        for (int s = 0; s < nsamples; ++s)
            if (b->L[s] == L) ids.push_back(s);
        b->class_L.push_back(L);
        b->class_dev_off.push_back((int)class_list.size());
        class_list.insert(class_list.end(), ids.begin(), ids.end());
        b->class_ids.push_back(ids);
    }
    b->class_k.assign(b->class_L.size(), 1);
    b->class_cost.assign(b->class_L.size(), 0.0);
    for (size_t ci = 0; ci < b->class_L.size(); ++ci) b->class_k[ci] = max_pack(b, (int)ci);
    // thresholds of every temperature (Ising classes of the +-1 spin glass)
    std::vector<uint32_t> thr(kMaxTemps * 4, 0xFFFFFFFFu);
    for (int k = 0; k < ntemps; ++k)
        for (int q = 0; q < d; ++q) {
            const int sh = 2 * d - 2 * q;  // s_i h_i with q unsatisfied bonds
            const double dE = 2.0 * 1.0 * (double)sh;
            const double x = std::exp(-betas[k] * dE) * 4294967296.0;
            if (!(x > 0.0)) {
                sl_batch_destroy(b);
                return fail(SL_EINVAL, "beta = %g too large: exp(-beta dE) underflows", betas[k]);
            }
            double T = std::ceil(x) - 1.0;
            if (T > 4294967295.0) T = 4294967295.0;
            thr[k * 4 + q] = (uint32_t)T;
        }
    long long max_m = 0;
    for (int s = 0; s < nsamples; ++s)
        max_m = std::max(max_m, (long long)d * b->L[s] * b->L[s] * (d == 3 ? b->L[s] : 1));
    std::vector<PairMeta> meta;
    std::vector<uint32_t> tab;
    build_pt(betas, ntemps, max_m, meta, tab);
    cudaError_t e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking);
    cudaStream_t s0 = b->stream;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->Ls_dev, b->L.data(), sizeof(int) * nsamples, cudaMemcpyHostToDevice, s0);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->word_off_dev, b->word_off.data(), sizeof(long long) * nsamples,
                            cudaMemcpyHostToDevice, s0);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->class_dev, class_list.data(), sizeof(int) * nsamples,
                            cudaMemcpyHostToDevice, s0);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->thr_temp, thr.data(), thr.size() * 4, cudaMemcpyHostToDevice, s0);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->pt_meta, meta.data(), sizeof(PairMeta) * kMaxTemps,
                            cudaMemcpyHostToDevice, s0);
    if (e == cudaSuccess && !tab.empty())
        e = cudaMemcpyAsync(b->pt_tab, tab.data(), tab.size() * 4, cudaMemcpyHostToDevice, s0);
    if (e == cudaSuccess) {
        batch_init_kernel<<<nsamples, 256, 0, s0>>>(b->spins, b->bonds, b->perm, b->Ls_dev,
                                                   b->word_off_dev, d, ntemps, first_sample,
                                                   make_round_keys(seed));
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s0);
    if (e != cudaSuccess) {
        st = cuda_fail(e, "sl_batch_create");
        sl_batch_destroy(b);
        return st;
    }
    *out = b;
    return SL_OK;
}

int sl_batch_run(sl_batch* b, int64_t nsweeps, uint64_t seed, double* dev_E)
{
    if (!b) return fail(SL_EINVAL, "batch is NULL");
    if (nsweeps < 0 || nsweeps > (1 << 30)) return fail(SL_EINVAL, "nsweeps out of range");
    if (b->sweeps_done + nsweeps > 4294967296LL) return fail(SL_EINVAL, "sweep index would exceed 2^32");
    if (nsweeps == 0) return SL_OK;
    if (!b->tuned) {
        int st = SL_OK;
        if (b->autotune && b->force_k <= 0) st = autotune(b);
        if (st == SL_OK) st = build_queue(b);
        if (st != SL_OK) return st;
        b->tuned = 1;
    }
    BatchArgs a = base_args(b);
    a.nitems = b->nitems;
    a.t0 = b->sweeps_done;
    a.nsweeps = (int)nsweeps;
    a.rk = make_round_keys(seed);
    a.E_out = dev_E;
    // one launch: replay the captured graph with this run's arguments
    cudaKernelNodeParams kp = {};
    void* args[1] = {&a};
    kp.func = b->d == 3 ? (void*)ea_pt_persistent<3> : (void*)ea_pt_persistent<2>;
    kp.gridDim = dim3((unsigned)b->grid);
    kp.blockDim = dim3(1024);
    kp.sharedMemBytes = (unsigned)b->smem_dyn;
    kp.kernelParams = args;
    kp.extra = nullptr;
    cudaError_t e = cudaGraphExecKernelNodeSetParams(b->graph, b->kernel_node, &kp);
    if (e == cudaSuccess) e = cudaGraphLaunch(b->graph, b->stream);
    if (e != cudaSuccess) return cuda_fail(e, "sl_batch_run");
    b->sweeps_done += nsweeps;
    return SL_OK;
}

int sl_batch_set_option(sl_batch* b, int option, int64_t value)
{
    if (!b) return fail(SL_EINVAL, "batch is NULL");
    switch (option) {
    case SL_BOPT_AUTOTUNE:
        if (value != 0 && value != 1) return fail(SL_EINVAL, "autotune must be 0 or 1");
        b->autotune = (int)value;
        b->tuned = 0;
        return SL_OK;
    case SL_BOPT_PACK:
        if (value != 0 && value != 1 && value != 2 && value != 4 && value != 8)
            return fail(SL_EINVAL, "pack must be 0 (tuned) or 1, 2, 4, 8");
        b->force_k = (int)value;
        b->tuned = 0;
        return SL_OK;
    default:
        return fail(SL_EINVAL, "unknown batch option %d", option);
    }
}

int sl_batch_tuning(sl_batch* b, int cls, int* L, int* pack, double* ms_per_sample_sweep)
{
    if (!b) return fail(SL_EINVAL, "batch is NULL");
    if (cls < 0 || cls >= (int)b->class_L.size()) return fail(SL_EINVAL, "class out of range");
    if (L) *L = b->class_L[cls];
    if (pack) *pack = b->force_k > 0 ? std::min(b->force_k, max_pack(b, cls)) : b->class_k[cls];
    if (ms_per_sample_sweep) *ms_per_sample_sweep = b->class_cost[cls];
    return (int)b->class_L.size();
}

int sl_batch_get(sl_batch* b, int sample, int slot, int8_t* dst, int* temp_index)
{
    if (!b || !dst) return fail(SL_EINVAL, "NULL argument");
    if (sample < 0 || sample >= b->nsamples || slot < 0 || slot >= b->ntemps)
        return fail(SL_EINVAL, "sample or slot out of range");
    const int L = b->L[sample];
    const long long N = (long long)L * L * (b->d == 3 ? L : 1);
    batch_gather_kernel<<<(int)((N + 255) / 256), 256, 0, b->stream>>>(
        b->spins, b->bonds, b->staging, b->word_off[sample], L, b->d, slot, 0);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(dst, b->staging, N, cudaMemcpyDefault, b->stream);
    int32_t perm[kMaxTemps];
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(perm, b->perm + sample * kMaxTemps, sizeof perm, cudaMemcpyDeviceToHost,
                            b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return cuda_fail(e, "sl_batch_get");
    if (temp_index) {
        *temp_index = -1;
        for (int k = 0; k < b->ntemps; ++k)
            if (perm[k] == slot) *temp_index = k;
    }
    return SL_OK;
}

int sl_batch_get_bonds(sl_batch* b, int sample, int8_t* dst)
{
    if (!b || !dst) return fail(SL_EINVAL, "NULL argument");
    if (sample < 0 || sample >= b->nsamples) return fail(SL_EINVAL, "sample out of range");
    const int L = b->L[sample];
    const long long N = (long long)L * L * (b->d == 3 ? L : 1);
    batch_gather_kernel<<<(int)((N + 255) / 256), 256, 0, b->stream>>>(
        b->spins, b->bonds, b->staging, b->word_off[sample], L, b->d, 0, 1);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(dst, b->staging, b->d * N, cudaMemcpyDefault, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return cuda_fail(e, "sl_batch_get_bonds");
    return SL_OK;
}

int sl_batch_sweeps_done(sl_batch* b, int64_t* sweeps_done)
{
    if (!b || !sweeps_done) return fail(SL_EINVAL, "NULL argument");
    *sweeps_done = b->sweeps_done;
    return SL_OK;
}

int sl_batch_set(sl_batch* b, int sample, const int8_t* spins, const int32_t* slot_of_temp)
{
    if (!b || !spins || !slot_of_temp) return fail(SL_EINVAL, "NULL argument");
    if (sample < 0 || sample >= b->nsamples) return fail(SL_EINVAL, "sample out of range");
    const int nt = b->ntemps;
    unsigned seen = 0;
    for (int k = 0; k < nt; ++k) {
        const int r = slot_of_temp[k];
        if (r < 0 || r >= nt || (seen >> r) & 1u)
            return fail(SL_EINVAL, "slot_of_temp is not a permutation of 0..%d", nt - 1);
        seen |= 1u << r;
    }
    int32_t perm[kMaxTemps];
    for (int k = 0; k < kMaxTemps; ++k) perm[k] = k < nt ? slot_of_temp[k] : k;
    const int L = b->L[sample];
    const long long N = (long long)L * L * (b->d == 3 ? L : 1);
    cudaError_t e = cudaSuccess;
    for (int r = 0; r < nt && e == cudaSuccess; ++r) {
        e = cudaMemcpyAsync(b->staging, spins + (size_t)r * N, (size_t)N, cudaMemcpyDefault,
                            b->stream);
        if (e == cudaSuccess) {
            batch_scatter_kernel<<<(int)((N + 255) / 256), 256, 0, b->stream>>>(
                b->spins, b->staging, b->word_off[sample], L, b->d, r);
            e = cudaGetLastError();
        }
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->perm + sample * kMaxTemps, perm, sizeof perm,
                            cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return cuda_fail(e, "sl_batch_set");
    return SL_OK;
}

int sl_batch_set_sweeps_done(sl_batch* b, int64_t sweeps_done)
{
    if (!b) return fail(SL_EINVAL, "batch is NULL");
    if (sweeps_done < 0 || sweeps_done > 4294967296LL)
        return fail(SL_EINVAL, "sweeps_done out of range");
    b->sweeps_done = sweeps_done;
    return SL_OK;
}

void sl_batch_destroy(sl_batch* b)
{
    if (!b) return;
    cudaStreamSynchronize(b->stream);
    if (b->graph) cudaGraphExecDestroy(b->graph);
    if (b->graph_def) cudaGraphDestroy(b->graph_def);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    if (b->owned_buf) cudaFree(b->owned_buf);
    delete b;
}

}  // extern "C"
