// Windowed multicanonical (MUCA) and Wang-Landau (WL) walkers of the 2D Ising
// model (Weigel & Yavors'kii 2011, Section 4: one copy of the system per
// thread in a fixed energy window, the threads of a block sharing a window,
// histograms and S(E) estimates in shared memory, windows glued afterwards).
//
// Energies are levels k = (E + 2N) / 4 of the L x L torus (J = 1, L a power
// of two); a walker's arrays are indexed by k - klo of its window.
//
// Storage: a warp is 32 walkers of one window.  Their lattices are
// interleaved bitwise: word q of warp g holds site q of each of its walkers,
// bit l = walker 32 g + l, set for spin down; global layout [warp][site]
// (64 MB for 131072 walkers of 64 x 64 sites, resident in L2).  All 32 lanes
// read the same word (a broadcast) and lane 0 writes back the ballot of
// flips; by default the words are used in place, optionally a warp's N words
// are kept in shared memory for the run (fewer warps fit per SM).  Per walker
// ln g (64-bit fixed point, units of 2^-32) and the histogram live in shared
// memory as [level][lane] (no bank conflicts).
//
// Every sweep visits each site once, all walkers in the same order: step q of
// sweep t takes site (a q + b) mod N, a = (x mod N) | 1, b = y mod N from
// outputs 0, 1 of Philox(0, t, 0, 11 << 1).  Step q draws output q & 3 of
// Philox(q >> 2, t, walker, purpose << 1), purpose 9 (WL) or 10 (MUCA).  A
// move that leaves the window is rejected.
//   MUCA: accept iff u <= T[k][dk], thresholds built on the host from the
//         FP64 weights ln W (u < exp(lnW(k) - lnW(k')) 2^32 as an exact
//         integer test); H counts the level after every attempt.
//   WL:   accept iff D >= 0 or u < exp(D 2^-32) 2^32, D = S(k) - S(k'): an
//         FP32 expf decides unless u lies within 2^-14 (relative) of the
//         threshold, where FP64 exp decides; after every attempt
//         S(k) += 2^(32 - stage), H(k) += 1, level k is marked visited;
//         after every sweep a walker whose visited levels all have
//         H(k) * nvisited * 100 >= flat_percent * sum H moves to the next
//         stage (H = 0, S lowered by its minimum over the visited levels);
//         a walker past final_stage makes no more moves.
// Start states: a ferromagnetic (window middle <= N/2) or Neel ground state,
// the one with spin 0 down iff the top bit of output 0 of
// Philox(0, 1, walker, 8 << 1) is set, then attempt a flips site
// (u N) >> 32, u = output 0 of Philox(a, 0, walker, 8 << 1), iff that moves
// the energy towards the window without passing its far edge; 1000 N
// attempts at most.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>

#include "internal.h"

namespace spinmc {
namespace {

constexpr uint32_t kWalkInit = 8, kWL = 9, kMUCA = 10, kOrder = 11;
constexpr int kKMax = 64;

struct WalkArgs {
    uint32_t* spins;      // [warp][site] words
    int32_t* level;       // [walker]
    int32_t* stage;       // [walker]
    uint64_t* visited;    // [walker]
    int64_t* S;           // [kmax][walker]
    uint32_t* H;          // [kmax][walker]
    const int32_t* klo;   // [window]
    const int32_t* khi;   // [window]
    const int64_t* thr;   // MUCA: [window][kmax][4] thresholds for dk = -2, -1, +1, +2
                          // (accept iff u <= T; -1 never)
    unsigned* error;
    int L, log2L, kmax, wpw, nwalk;
    long long N;
    uint32_t t0;
    long long nsweeps;
    int final_stage, flat_percent;
    int spins_smem;       // keep each warp's lattice in shared memory during a run
    RoundKeys rk;
};

__device__ __forceinline__ void sweep_order(const WalkArgs& a, uint32_t t, uint32_t& oa, uint32_t& ob)
{
    const uint4 r = philox4x32_10(make_uint4(0u, t, 0u, kOrder << 1), a.rk);
    const uint32_t m = (uint32_t)(a.N - 1);  // N is a power of two
    oa = (r.x & m) | 1u;
    ob = r.y & m;
}

// unlike neighbours of site i for this lane, from the warp's words (ld
// reads one word)
template <typename Ld>
__device__ __forceinline__ int unlike(Ld ld, uint32_t i, int L, int log2L, int lane, uint32_t& own)
{
    const uint32_t xmask = (uint32_t)(L - 1), nmask = (1u << (2 * log2L)) - 1u;
    const uint32_t row = i & ~xmask;
    const uint32_t xm = row | ((i - 1) & xmask), xp = row | ((i + 1) & xmask);
    const uint32_t ym = (i - (uint32_t)L) & nmask, yp = (i + (uint32_t)L) & nmask;
    own = ld(i);
    const uint32_t d = ((own ^ ld(xm)) >> lane & 1u) + ((own ^ ld(xp)) >> lane & 1u) +
                       ((own ^ ld(ym)) >> lane & 1u) + ((own ^ ld(yp)) >> lane & 1u);
    return (int)d;
}

// ---------------------------------------------------------------- init ----

__global__ void __launch_bounds__(128) walk_init_kernel(WalkArgs a)
{
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x);
    const int lane = threadIdx.x & 31;
    if (gw - lane >= a.nwalk) return;  // whole warps only (nwalk % 32 == 0)
    const uint32_t walker = (uint32_t)gw;
    const int win = gw / a.wpw;
    const int klo = a.klo[win], khi = a.khi[win];
    const long long N = a.N;
    const int L = a.L;
    uint32_t* col = a.spins + (size_t)(gw >> 5) * (size_t)N;
    const uint4 r0 = philox4x32_10(make_uint4(0u, 1u, walker, kWalkInit << 1), a.rk);
    const bool down0 = (r0.x >> 31) != 0;
    const bool ferro = 2LL * ((klo + khi) / 2) <= N;
    for (long long i = 0; i < N; ++i) {
        const int x = (int)(i & (L - 1)), y = (int)(i >> a.log2L);
        bool up = ferro ? true : ((x + y) % 2 == 0);
        if (down0) up = !up;
        const uint32_t w = __ballot_sync(0xFFFFFFFFu, !up);
        if (lane == 0) col[i] = w;
    }
    __syncwarp();
    int k = ferro ? 0 : (int)N;
    const long long cap = 1000LL * N;
    for (long long at = 0; at < cap && (k < klo || k > khi); ++at) {
        const uint4 r = philox4x32_10(make_uint4((uint32_t)at, 0u, walker, kWalkInit << 1), a.rk);
        const uint32_t i = (uint32_t)(((unsigned long long)r.x * (unsigned long long)N) >> 32);
        // other lanes flip their own bits of these words by atomics, so the
        // words are read from L2 (the lane's own bits are current there)
        uint32_t own;
        const int nu = unlike([&](uint32_t q) { return __ldcg(col + q); }, i, L, a.log2L, lane, own);
        const int dk = 2 - nu;
        const int k2 = k + dk;
        if ((k < klo && dk > 0 && k2 <= khi) || (k > khi && dk < 0 && k2 >= klo)) {
            atomicXor(col + i, 1u << lane);
            k = k2;
        }
    }
    if (k < klo || k > khi) atomicOr(a.error, 1u);
    a.level[gw] = k;
    a.stage[gw] = 0;
    a.visited[gw] = 0ull;
    for (int q = 0; q < a.kmax; ++q) {
        a.S[(size_t)q * a.nwalk + gw] = 0;
        a.H[(size_t)q * a.nwalk + gw] = 0u;
    }
}

// ------------------------------------------------------------ WL / MUCA ----

// Wang-Landau decision for D < 0 (see the file comment).  The FP32 filter
// builds x = D 2^-32 from the two 32-bit halves of D with FP32 instructions
// only (relative error below 2^-22, plus the argument error |x| 2^-24 that
// keeps the filter's 2^-14 margin safe for |x| < 100; beyond, exp(x) < 2^-144
// and only u = 0 reaches the FP64 test).
__device__ __forceinline__ bool wl_accept(int64_t D, uint32_t u)
{
    const float xf = (float)(int32_t)(D >> 32) + (float)(uint32_t)D * (1.0f / 4294967296.0f);
    const float pf = expf(xf);
    const float uf = (float)u * (1.0f / 4294967296.0f);
    const float m = 1.0f / 16384.0f;
    if (uf < pf * (1.0f - m)) return true;
    if (uf > pf * (1.0f + m)) return false;
    return (double)u * (1.0 / 4294967296.0) < exp((double)D * (1.0 / 4294967296.0));
}

template <int KT, bool WL, bool SPINS_SMEM>
__global__ void __launch_bounds__(32) walk_kernel(const WalkArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const size_t colb = SPINS_SMEM ? 4 * (size_t)a.N : 0;
    int64_t* S = reinterpret_cast<int64_t*>(smem + colb);                 // [KT][32]
    uint32_t* H = reinterpret_cast<uint32_t*>(smem + colb + 8 * KT * 32);  // [KT][32]
    int64_t* T = reinterpret_cast<int64_t*>(H + KT * 32);                 // MUCA [KT][4]
    const int lane = threadIdx.x;
    const int warp = blockIdx.x;
    const int gw = warp * 32 + lane;
    const uint32_t walker = (uint32_t)gw;
    const int win = gw / a.wpw;  // the whole warp shares it (wpw % 32 == 0)
    const int klo = a.klo[win];
    const int K = a.khi[win] - klo + 1;
    const long long N = a.N;
    const int L = a.L;
    uint32_t* gcol = a.spins + (size_t)warp * (size_t)N;
    // the warp's lattice column: in shared memory for the run, or read in
    // place from global memory (L2)
    uint32_t* col = SPINS_SMEM ? reinterpret_cast<uint32_t*>(smem) : gcol;
    if (SPINS_SMEM)
        for (long long i = lane; i < N; i += 32) col[i] = gcol[i];
    for (int q = 0; q < KT; ++q) {
        S[q * 32 + lane] = q < a.kmax ? a.S[(size_t)q * a.nwalk + gw] : 0;
        H[q * 32 + lane] = q < a.kmax && WL ? a.H[(size_t)q * a.nwalk + gw] : 0u;
    }
    if (!WL)
        for (int q = lane; q < 4 * KT; q += 32)
            T[q] = q < 4 * a.kmax ? a.thr[((size_t)win * a.kmax) * 4 + q] : -1;
    int kr = a.level[gw] - klo;
    int stage = a.stage[gw];
    uint64_t vis = a.visited[gw];
    __syncwarp();

    for (long long s = 0; s < a.nsweeps; ++s) {
        const uint32_t t = a.t0 + (uint32_t)s;
        const bool active = !WL || stage <= a.final_stage;
        if (!__any_sync(0xFFFFFFFFu, active)) break;
        uint32_t oa, ob;
        sweep_order(a, t, oa, ob);
        const int64_t inc = WL && active ? ((int64_t)1 << (32 - stage)) : 0;
        const uint32_t nmask = (uint32_t)(N - 1);
        const uint32_t purpose = (WL ? kWL : kMUCA) << 1;
        // the block of the next four attempts is drawn while the current four
        // run (the attempts depend on each other, the draws do not; N is a
        // multiple of 4, and the draw after the last block goes unused)
        uint4 rnd_nx = philox4x32_10(make_uint4(0u, t, walker, purpose), a.rk);
        // one attempt at position q of the sweep with uniform u
        auto attempt = [&](uint32_t q, uint32_t u) {
            const uint32_t i = (oa * q + ob) & nmask;  // N divides 2^32
            uint32_t own;
            const int nu = unlike([&](uint32_t w) { return col[w]; }, i, L, a.log2L, lane, own);
            const int dk = 2 - nu;
            const int k2 = kr + dk;
            bool acc = false;
            if (active && k2 >= 0 && k2 < K) {
                if (WL) {
                    const int64_t D = S[kr * 32 + lane] - S[k2 * 32 + lane];
                    acc = D >= 0 || wl_accept(D, u);
                } else {
                    acc = dk == 0 || (int64_t)u <= T[kr * 4 + (dk < 0 ? dk + 2 : dk + 1)];
                }
            }
            const uint32_t flips = __ballot_sync(0xFFFFFFFFu, acc);
            if (lane == 0 && flips) col[i] = own ^ flips;
            if (acc) kr = k2;
            if (active) {
                if (WL) {
                    S[kr * 32 + lane] += inc;
                    vis |= 1ull << kr;
                }
                H[kr * 32 + lane] += 1u;
            }
            __syncwarp();
        };
        for (uint32_t q = 0; q < (uint32_t)N; q += 4) {
            const uint4 rnd = rnd_nx;
            rnd_nx = philox4x32_10(make_uint4((q >> 2) + 1u, t, walker, purpose), a.rk);
            attempt(q, rnd.x);
            attempt(q + 1, rnd.y);
            attempt(q + 2, rnd.z);
            attempt(q + 3, rnd.w);
        }
        if (WL && active) {
            int nv = 0;
            unsigned long long sum = 0;
            for (int q = 0; q < KT; ++q)
                if ((vis >> q) & 1ull) {
                    ++nv;
                    sum += H[q * 32 + lane];
                }
            bool flat = nv > 0;
            for (int q = 0; q < KT; ++q)
                if (((vis >> q) & 1ull) &&
                    (unsigned long long)H[q * 32 + lane] * (unsigned long long)nv * 100ull <
                        (unsigned long long)a.flat_percent * sum)
                    flat = false;
            if (flat) {
                int64_t mn = INT64_MAX;
                for (int q = 0; q < KT; ++q)
                    if (((vis >> q) & 1ull) && S[q * 32 + lane] < mn) mn = S[q * 32 + lane];
                for (int q = 0; q < KT; ++q) {
                    if ((vis >> q) & 1ull) S[q * 32 + lane] -= mn;
                    H[q * 32 + lane] = 0u;
                }
                ++stage;
            }
        }
    }
    __syncwarp();
    if (SPINS_SMEM)
        for (long long i = lane; i < N; i += 32) gcol[i] = col[i];
    for (int q = 0; q < a.kmax && q < KT; ++q) {
        if (WL) a.S[(size_t)q * a.nwalk + gw] = S[q * 32 + lane];
        a.H[(size_t)q * a.nwalk + gw] = H[q * 32 + lane];
    }
    a.level[gw] = kr + klo;
    a.stage[gw] = stage;
    a.visited[gw] = vis;
}

__global__ void walk_gather_kernel(const uint32_t* spins, long long N, int walker, int8_t* nat)
{
    const uint32_t* col = spins + (size_t)(walker >> 5) * (size_t)N;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
         i += (long long)gridDim.x * blockDim.x)
        nat[i] = ((col[i] >> (walker & 31)) & 1u) ? (int8_t)-1 : (int8_t)1;
}

// Writes one walker's bit of every site word from a natural-order +-1
// configuration (1 = down; the other walkers' bits are kept) and sets the
// walker's level to k = (E + 2N) / 4 of that configuration (one block).
__global__ void __launch_bounds__(256) walk_scatter_kernel(uint32_t* spins, const int8_t* nat,
                                                           long long N, int L, int log2L,
                                                           int walker, int32_t* level)
{
    __shared__ long long red[32];
    uint32_t* col = spins + (size_t)(walker >> 5) * (size_t)N;
    const uint32_t bit = 1u << (walker & 31);
    long long bond = 0;
    for (long long i = threadIdx.x; i < N; i += blockDim.x) {
        col[i] = (col[i] & ~bit) | (nat[i] < 0 ? bit : 0u);
        const int x = (int)(i & (L - 1)), y = (int)(i >> log2L);
        const long long xp = (long long)y * L + ((x + 1) & (L - 1));
        const long long yp = (long long)((y + 1) & (L - 1)) * L + x;
        bond += (long long)nat[i] * (nat[xp] + nat[yp]);
    }
    const long long tot = block_sum(bond, red);
    if (threadIdx.x == 0) level[walker] = (int32_t)((-tot + 2 * N) / 4);
}

struct WalkLayout {
    size_t off_spins, off_level, off_stage, off_visited, off_S, off_H, off_klo, off_khi, off_thr,
        off_err, off_nat, total;
};

WalkLayout walk_layout(int L, int nwin, int wpw, int kmax)
{
    WalkLayout y;
    const size_t N = (size_t)L * L, nwalk = (size_t)nwin * wpw;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off += align_up(bytes);
        return o;
    };
    y.off_spins = take(N * (nwalk / 32) * 4);
    y.off_level = take(nwalk * 4);
    y.off_stage = take(nwalk * 4);
    y.off_visited = take(nwalk * 8);
    y.off_S = take((size_t)kmax * nwalk * 8);
    y.off_H = take((size_t)kmax * nwalk * 4);
    y.off_klo = take((size_t)nwin * 4);
    y.off_khi = take((size_t)nwin * 4);
    y.off_thr = take((size_t)nwin * kmax * 4 * 8);
    y.off_err = take(sizeof(unsigned));
    y.off_nat = take(N);
    y.total = off;
    return y;
}

int check_walk_config(int L, int nwin, const int* klo, const int* khi, int wpw, int* kmax)
{
    if (L < 4 || L > 128 || (L & (L - 1)))
        return fail(SL_EINVAL, "walkers need L a power of two in [4, 128] (got %d)", L);
    if (nwin < 1) return fail(SL_EINVAL, "need at least one window");
    if (wpw < 32 || wpw % 32) return fail(SL_EINVAL, "walkers per window must be a multiple of 32");
    if ((long long)nwin * wpw > (1LL << 30)) return fail(SL_EINVAL, "too many walkers");
    const int N = L * L;
    int km = 1;
    if (klo && khi) {
        for (int w = 0; w < nwin; ++w) {
            if (klo[w] < 0 || khi[w] > N || khi[w] - klo[w] < 2)
                return fail(SL_EINVAL, "window %d = [%d, %d] must lie in [0, %d] and span >= 3 "
                                       "levels", w, klo[w], khi[w], N);
            if (khi[w] - klo[w] + 1 > kKMax)
                return fail(SL_EINVAL, "window %d spans more than %d levels", w, kKMax);
            if (khi[w] - klo[w] + 1 > km) km = khi[w] - klo[w] + 1;
        }
    }
    *kmax = km;
    return SL_OK;
}

int kt_for(int kmax)
{
    int kt = 8;
    while (kt < kmax) kt *= 2;
    return kt;
}

template <int KT, bool WL, bool SM>
cudaError_t launch_walk_res(const WalkArgs& a, cudaStream_t s)
{
    const size_t smem = (SM ? 4 * (size_t)a.N : 0) + (size_t)KT * 32 * 12 + (size_t)KT * 4 * 8;
    cudaError_t e = cudaFuncSetAttribute(walk_kernel<KT, WL, SM>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    walk_kernel<KT, WL, SM><<<a.nwalk / 32, 32, smem, s>>>(a);
    return cudaGetLastError();
}

template <int KT, bool WL>
cudaError_t launch_walk(const WalkArgs& a, cudaStream_t s)
{
    return a.spins_smem ? launch_walk_res<KT, WL, true>(a, s) : launch_walk_res<KT, WL, false>(a, s);
}

template <bool WL>
cudaError_t launch_walk_kt(const WalkArgs& a, cudaStream_t s)
{
    switch (kt_for(a.kmax)) {
    case 8: return launch_walk<8, WL>(a, s);
    case 16: return launch_walk<16, WL>(a, s);
    case 32: return launch_walk<32, WL>(a, s);
    default: return launch_walk<64, WL>(a, s);
    }
}

}  // namespace
}  // namespace spinmc

using namespace spinmc;

struct sl_walkers {
    int L, log2L, nwin, wpw, nwalk, kmax;
    int spins_smem;  // SL_WOPT_SPINS_SMEM
    long long N;
    uint64_t seed;
    int64_t sweeps_done;
    cudaStream_t stream;
    WalkLayout y;
    char* base;
    void* owned;
    int* klo_host;
    int* khi_host;
};

namespace {

WalkArgs walk_args(const sl_walkers* w)
{
    WalkArgs a;
    std::memset(&a, 0, sizeof a);
    a.spins = (uint32_t*)(w->base + w->y.off_spins);
    a.level = (int32_t*)(w->base + w->y.off_level);
    a.stage = (int32_t*)(w->base + w->y.off_stage);
    a.visited = (uint64_t*)(w->base + w->y.off_visited);
    a.S = (int64_t*)(w->base + w->y.off_S);
    a.H = (uint32_t*)(w->base + w->y.off_H);
    a.klo = (const int32_t*)(w->base + w->y.off_klo);
    a.khi = (const int32_t*)(w->base + w->y.off_khi);
    a.thr = (const int64_t*)(w->base + w->y.off_thr);
    a.error = (unsigned*)(w->base + w->y.off_err);
    a.L = w->L;
    a.log2L = w->log2L;
    a.kmax = w->kmax;
    a.wpw = w->wpw;
    a.nwalk = w->nwalk;
    a.N = w->N;
    a.spins_smem = w->spins_smem;
    return a;
}

int walk_sync(sl_walkers* w)
{
    cudaError_t e = cudaStreamSynchronize(w->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    unsigned err = 0;
    e = cudaMemcpy(&err, w->base + w->y.off_err, sizeof err, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "read walker error word");
    if (err & 1u) return fail(SL_EDEVICE, "a walker did not reach its window in 1000 N attempts");
    return SL_OK;
}

}  // namespace

extern "C" {

int sl_walkers_required_bytes(int L, int nwin, const int* klo, const int* khi, int wpw,
                              size_t* bytes)
{
    if (!bytes) return fail(SL_EINVAL, "bytes is NULL");
    int kmax = 0;
    const int st = check_walk_config(L, nwin, klo, khi, wpw, &kmax);
    if (st != SL_OK) return st;
    if (!klo || !khi) return fail(SL_EINVAL, "window bounds are NULL");
    *bytes = walk_layout(L, nwin, wpw, kmax).total;
    return SL_OK;
}

int sl_walkers_create(int L, int nwin, const int* klo, const int* khi, int wpw, uint64_t seed,
                      void* dev_buf, size_t dev_buf_bytes, void* stream, sl_walkers** out)
{
    if (!out) return fail(SL_EINVAL, "out is NULL");
    *out = nullptr;
    if (!klo || !khi) return fail(SL_EINVAL, "window bounds are NULL");
    int kmax = 0;
    int st = check_walk_config(L, nwin, klo, khi, wpw, &kmax);
    if (st != SL_OK) return st;
    const WalkLayout y = walk_layout(L, nwin, wpw, kmax);
    void* owned = nullptr;
    if (!dev_buf) {
        const cudaError_t e = cudaMalloc(&owned, y.total);
        if (e != cudaSuccess)
            return fail(SL_ENOMEM, "cudaMalloc(%zu): %s", y.total, cudaGetErrorString(e));
        dev_buf = owned;
        dev_buf_bytes = y.total;
    }
    if ((uintptr_t)dev_buf % kAlign) {
        if (owned) cudaFree(owned);
        return fail(SL_EINVAL, "dev_buf must be %zu-byte aligned", kAlign);
    }
    if (dev_buf_bytes < y.total) {
        if (owned) cudaFree(owned);
        return fail(SL_ENOMEM, "dev_buf holds %zu bytes, %zu needed", dev_buf_bytes, y.total);
    }
    sl_walkers* w = new (std::nothrow) sl_walkers();
    int* kl = new (std::nothrow) int[nwin];
    int* kh = new (std::nothrow) int[nwin];
    if (!w || !kl || !kh) {
        delete w;
        delete[] kl;
        delete[] kh;
        if (owned) cudaFree(owned);
        return fail(SL_ENOMEM, "host allocation failed");
    }
    std::memcpy(kl, klo, sizeof(int) * nwin);
    std::memcpy(kh, khi, sizeof(int) * nwin);
    w->L = L;
    w->log2L = 0;
    while ((1 << w->log2L) < L) ++w->log2L;
    w->nwin = nwin;
    w->wpw = wpw;
    w->nwalk = nwin * wpw;
    w->kmax = kmax;
    w->spins_smem = 0;  // measured on GB300: 48% faster in place (L2) than in shared memory
    w->N = (long long)L * L;
    w->seed = seed;
    w->sweeps_done = 0;
    w->stream = (cudaStream_t)stream;
    w->y = y;
    w->base = (char*)dev_buf;
    w->owned = owned;
    w->klo_host = kl;
    w->khi_host = kh;
    cudaError_t e = cudaMemcpyAsync(w->base + y.off_klo, klo, sizeof(int) * nwin,
                                    cudaMemcpyHostToDevice, w->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(w->base + y.off_khi, khi, sizeof(int) * nwin, cudaMemcpyHostToDevice,
                            w->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(w->base + y.off_err, 0, sizeof(unsigned), w->stream);
    if (e == cudaSuccess) {
        WalkArgs a = walk_args(w);
        a.rk = make_round_keys(seed);
        walk_init_kernel<<<(w->nwalk + 127) / 128, 128, 0, w->stream>>>(a);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        st = cuda_fail(e, "sl_walkers_create");
        sl_walkers_destroy(w);
        return st;
    }
    st = walk_sync(w);
    if (st != SL_OK) {
        sl_walkers_destroy(w);
        return st;
    }
    *out = w;
    return SL_OK;
}

int sl_wl_run(sl_walkers* w, int64_t nsweeps, int final_stage, int flat_percent, uint64_t seed)
{
    if (!w) return fail(SL_EINVAL, "walkers handle is NULL");
    if (nsweeps < 0) return fail(SL_EINVAL, "nsweeps must be >= 0");
    if (final_stage < 0 || final_stage > 32) return fail(SL_EINVAL, "final_stage must be in [0, 32]");
    if (flat_percent < 0) return fail(SL_EINVAL, "flat_percent must be >= 0");
    if (w->sweeps_done + nsweeps > 4294967296LL) return fail(SL_EINVAL, "sweep index would exceed 2^32");
    if (nsweeps == 0) return SL_OK;
    WalkArgs a = walk_args(w);
    a.rk = make_round_keys(seed);
    a.t0 = (uint32_t)w->sweeps_done;
    a.nsweeps = nsweeps;
    a.final_stage = final_stage;
    a.flat_percent = flat_percent;
    const cudaError_t e = launch_walk_kt<true>(a, w->stream);
    if (e != cudaSuccess) return cuda_fail(e, "sl_wl_run");
    w->sweeps_done += nsweeps;
    return SL_OK;
}

int sl_muca_run(sl_walkers* w, const double* lnW, int64_t nsweeps, uint64_t seed)
{
    if (!w || !lnW) return fail(SL_EINVAL, "NULL argument");
    if (nsweeps < 0) return fail(SL_EINVAL, "nsweeps must be >= 0");
    if (w->sweeps_done + nsweeps > 4294967296LL) return fail(SL_EINVAL, "sweep index would exceed 2^32");
    // exact integer thresholds: a move k -> k + dk is accepted iff
    // u < exp(lnW(k) - lnW(k + dk)) 2^32, i.e. u <= ceil(x) - 1 (-1: never)
    const size_t nthr = (size_t)w->nwin * w->kmax * 4;
    int64_t* thr = new (std::nothrow) int64_t[nthr];
    if (!thr) return fail(SL_ENOMEM, "host allocation failed");
    for (int win = 0; win < w->nwin; ++win) {
        const int K = w->khi_host[win] - w->klo_host[win] + 1;
        const double* W = lnW + (size_t)win * w->kmax;
        for (int k = 0; k < w->kmax; ++k) {
            static const int dks[4] = {-2, -1, 1, 2};
            for (int c = 0; c < 4; ++c) {
                const int k2 = k + dks[c];
                int64_t T = -1;
                if (k < K && k2 >= 0 && k2 < K) {
                    if (!std::isfinite(W[k]) || !std::isfinite(W[k2])) {
                        delete[] thr;
                        return fail(SL_EINVAL, "weights of window %d are not finite", win);
                    }
                    const double d = W[k] - W[k2];
                    if (d >= 0.0) {
                        T = 4294967295LL;
                    } else {
                        const double x = std::exp(d) * 4294967296.0;
                        double c1 = std::ceil(x) - 1.0;  // -1 when exp underflows to 0
                        if (c1 > 4294967295.0) c1 = 4294967295.0;
                        T = (int64_t)c1;
                    }
                }
                thr[((size_t)win * w->kmax + k) * 4 + c] = T;
            }
        }
    }
    cudaError_t e = cudaMemcpyAsync(w->base + w->y.off_thr, thr, nthr * sizeof(int64_t),
                                    cudaMemcpyHostToDevice, w->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(w->stream);
    delete[] thr;
    if (e != cudaSuccess) return cuda_fail(e, "upload thresholds");
    if (nsweeps == 0) return SL_OK;
    WalkArgs a = walk_args(w);
    a.rk = make_round_keys(seed);
    a.t0 = (uint32_t)w->sweeps_done;
    a.nsweeps = nsweeps;
    e = launch_walk_kt<false>(a, w->stream);
    if (e != cudaSuccess) return cuda_fail(e, "sl_muca_run");
    w->sweeps_done += nsweeps;
    return SL_OK;
}

int sl_walkers_read(sl_walkers* w, int64_t* S, uint32_t* H, int32_t* level, int32_t* stage,
                    uint64_t* visited)
{
    if (!w) return fail(SL_EINVAL, "walkers handle is NULL");
    int st = walk_sync(w);
    if (st != SL_OK) return st;
    const size_t nw = (size_t)w->nwalk, km = (size_t)w->kmax;
    cudaError_t e = cudaSuccess;
    if (level) e = cudaMemcpy(level, w->base + w->y.off_level, nw * 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && stage)
        e = cudaMemcpy(stage, w->base + w->y.off_stage, nw * 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && visited)
        e = cudaMemcpy(visited, w->base + w->y.off_visited, nw * 8, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && (S || H)) {
        // device arrays are [level][walker]; the caller gets [walker][level]
        char* tmp = new (std::nothrow) char[km * nw * 8];
        if (!tmp) return fail(SL_ENOMEM, "host allocation failed");
        if (S) {
            e = cudaMemcpy(tmp, w->base + w->y.off_S, km * nw * 8, cudaMemcpyDeviceToHost);
            const int64_t* src = (const int64_t*)tmp;
            for (size_t q = 0; q < km && e == cudaSuccess; ++q)
                for (size_t j = 0; j < nw; ++j) S[j * km + q] = src[q * nw + j];
        }
        if (e == cudaSuccess && H) {
            e = cudaMemcpy(tmp, w->base + w->y.off_H, km * nw * 4, cudaMemcpyDeviceToHost);
            const uint32_t* src = (const uint32_t*)tmp;
            for (size_t q = 0; q < km && e == cudaSuccess; ++q)
                for (size_t j = 0; j < nw; ++j) H[j * km + q] = src[q * nw + j];
        }
        delete[] tmp;
    }
    if (e != cudaSuccess) return cuda_fail(e, "sl_walkers_read");
    return SL_OK;
}

int sl_walkers_get_spins(sl_walkers* w, int walker, int8_t* dst)
{
    if (!w || !dst) return fail(SL_EINVAL, "NULL argument");
    if (walker < 0 || walker >= w->nwalk) return fail(SL_EINVAL, "walker %d out of range", walker);
    int8_t* nat = (int8_t*)(w->base + w->y.off_nat);
    walk_gather_kernel<<<(int)((w->N + 255) / 256), 256, 0, w->stream>>>(
        (const uint32_t*)(w->base + w->y.off_spins), w->N, walker, nat);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(dst, nat, (size_t)w->N, cudaMemcpyDefault, w->stream);
    if (e != cudaSuccess) return cuda_fail(e, "sl_walkers_get_spins");
    return walk_sync(w);
}

int sl_walkers_set_spins(sl_walkers* w, int walker, const int8_t* src)
{
    if (!w || !src) return fail(SL_EINVAL, "NULL argument");
    if (walker < 0 || walker >= w->nwalk) return fail(SL_EINVAL, "walker %d out of range", walker);
    int8_t* nat = (int8_t*)(w->base + w->y.off_nat);
    int32_t* level = (int32_t*)(w->base + w->y.off_level);
    cudaError_t e = cudaMemcpyAsync(nat, src, (size_t)w->N, cudaMemcpyDefault, w->stream);
    if (e == cudaSuccess) {
        walk_scatter_kernel<<<1, 256, 0, w->stream>>>((uint32_t*)(w->base + w->y.off_spins), nat,
                                                       w->N, w->L, w->log2L, walker, level);
        e = cudaGetLastError();
    }
    int32_t k = -1;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&k, level + walker, sizeof k, cudaMemcpyDeviceToHost, w->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(w->stream);
    if (e != cudaSuccess) return cuda_fail(e, "sl_walkers_set_spins");
    const int win = walker / w->wpw;
    if (k < w->klo_host[win] || k > w->khi_host[win])
        return fail(SL_EINVAL, "walker %d: the configuration's level %d lies outside its window "
                               "[%d, %d]", walker, k, w->klo_host[win], w->khi_host[win]);
    return SL_OK;
}

int sl_walkers_write(sl_walkers* w, const int64_t* S, const uint32_t* H, const int32_t* stage,
                     const uint64_t* visited)
{
    if (!w) return fail(SL_EINVAL, "walkers handle is NULL");
    int st = walk_sync(w);
    if (st != SL_OK) return st;
    const size_t nw = (size_t)w->nwalk, km = (size_t)w->kmax;
    cudaError_t e = cudaSuccess;
    if (stage) e = cudaMemcpy(w->base + w->y.off_stage, stage, nw * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && visited)
        e = cudaMemcpy(w->base + w->y.off_visited, visited, nw * 8, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && (S || H)) {
        // the caller's arrays are [walker][level]; the device keeps [level][walker]
        char* tmp = new (std::nothrow) char[km * nw * 8];
        if (!tmp) return fail(SL_ENOMEM, "host allocation failed");
        if (S) {
            int64_t* dst = (int64_t*)tmp;
            for (size_t q = 0; q < km; ++q)
                for (size_t j = 0; j < nw; ++j) dst[q * nw + j] = S[j * km + q];
            e = cudaMemcpy(w->base + w->y.off_S, tmp, km * nw * 8, cudaMemcpyHostToDevice);
        }
        if (e == cudaSuccess && H) {
            uint32_t* dst = (uint32_t*)tmp;
            for (size_t q = 0; q < km; ++q)
                for (size_t j = 0; j < nw; ++j) dst[q * nw + j] = H[j * km + q];
            e = cudaMemcpy(w->base + w->y.off_H, tmp, km * nw * 4, cudaMemcpyHostToDevice);
        }
        delete[] tmp;
    }
    if (e != cudaSuccess) return cuda_fail(e, "sl_walkers_write");
    return SL_OK;
}

int sl_walkers_set_sweeps_done(sl_walkers* w, int64_t sweeps_done)
{
    if (!w) return fail(SL_EINVAL, "walkers handle is NULL");
    if (sweeps_done < 0 || sweeps_done > 4294967295LL)
        return fail(SL_EINVAL, "sweeps_done out of range");
    w->sweeps_done = sweeps_done;
    return SL_OK;
}

int sl_walkers_set_option(sl_walkers* w, int option, int64_t value)
{
    if (!w) return fail(SL_EINVAL, "walkers handle is NULL");
    switch (option) {
    case SL_WOPT_SPINS_SMEM:
        if (value != 0 && value != 1) return fail(SL_EINVAL, "spins_smem must be 0 or 1");
        w->spins_smem = (int)value;
        return SL_OK;
    default:
        return fail(SL_EINVAL, "unknown walker option %d", option);
    }
}

int sl_walkers_info(const sl_walkers* w, int* nwalk, int* kmax, int64_t* sweeps_done)
{
    if (!w) return fail(SL_EINVAL, "walkers handle is NULL");
    if (nwalk) *nwalk = w->nwalk;
    if (kmax) *kmax = w->kmax;
    if (sweeps_done) *sweeps_done = w->sweeps_done;
    return SL_OK;
}

void sl_walkers_destroy(sl_walkers* w)
{
    if (!w) return;
    cudaStreamSynchronize(w->stream);
    if (w->owned) cudaFree(w->owned);
    delete[] w->klo_host;
    delete[] w->khi_host;
    delete w;
}

int sl_dos_glue(int L, int nwin, const int* klo, const int* khi, const double* S, int stride,
                const uint64_t* visited, double* out)
{
    if (!klo || !khi || !S || !visited || !out) return fail(SL_EINVAL, "NULL argument");
    const int N = L * L;
    for (int k = 0; k <= N; ++k) out[k] = NAN;
    double shift = 0.0;
    for (int w = 0; w < nwin; ++w) {
        const double* Sw = S + (size_t)w * stride;
        if (klo[w] < 0 || khi[w] > N || khi[w] < klo[w] || khi[w] - klo[w] >= stride)
            return fail(SL_EINVAL, "window %d is out of range", w);
        if (w > 0) {
            if (klo[w] != khi[w - 1])
                return fail(SL_EINVAL, "windows %d and %d do not share an edge level", w - 1, w);
            const double* Sp = S + (size_t)(w - 1) * stride;
            const int qp = khi[w - 1] - klo[w - 1];
            if (!((visited[w - 1] >> qp) & 1u) || !(visited[w] & 1u))
                return fail(SL_EINVAL, "shared level of windows %d and %d was not visited", w - 1,
                            w);
            shift += Sp[qp] - Sw[0];
        }
        for (int k = klo[w]; k <= khi[w]; ++k)
            if ((visited[w] >> (k - klo[w])) & 1u) out[k] = Sw[k - klo[w]] + shift;
    }
    return SL_OK;
}

}  // extern "C"
