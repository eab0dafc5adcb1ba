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

struct BatchArgs {
    uint32_t* spins;
    uint8_t* bonds;
    int32_t* perm;  // [sample][kMaxTemps] slot holding temperature k
    const int* class_samples;
    const long long* word_off;  // per sample: first spin word (colour 0), colour 1 at + H
    int d, L, ntemps;
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

template <int D>
__global__ void __launch_bounds__(1024) ea_pt_kernel(const BatchArgs a)
{
    extern __shared__ uint4 smem_u4[];
    const int s = a.class_samples[blockIdx.x];
    const int L = a.L, nt = a.ntemps;
    const int N = D == 3 ? L * L * L : L * L;
    const int H = N / 2, G = H / 4;
    uint32_t* S0 = reinterpret_cast<uint32_t*>(smem_u4);
    uint32_t* S1 = S0 + H;
    uint8_t* B0 = reinterpret_cast<uint8_t*>(S1 + H);
    uint8_t* B1 = B0 + H;
    uint4* thr_slot = reinterpret_cast<uint4*>(B0 + ((2 * H + 15) / 16) * 16);
    long long* E_slot = reinterpret_cast<long long*>(thr_slot + kMaxTemps);
    int* unsat = reinterpret_cast<int*>(E_slot + kMaxTemps);
    int* sot = unsat + kMaxTemps;  // slot of temperature
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nthr = blockDim.x;
    const uint32_t active = nt == 32 ? 0xFFFFFFFFu : ((1u << nt) - 1u);

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
    __syncthreads();
    if (tid < nt) {
        const uint4 th = reinterpret_cast<const uint4*>(a.thr_temp)[tid];
        thr_slot[sot[tid]] = th;
    }
    __syncthreads();

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
                uint32_t pl[4][3];
#pragma unroll
                for (int b = 0; b < 4; ++b) pl[b][0] = pl[b][1] = pl[b][2] = 0u;
#pragma unroll
                for (int r = 0; r < kMaxTemps; ++r) {
                    if (r < nt) {
                        const uint4 rnd = philox4x32_10(
                            make_uint4((uint32_t)g, (uint32_t)t, (uint32_t)(s * nt + r), ctr_w), a.rk);
                        const uint4 th = thr_slot[r];
                        const uint32_t u[4] = {rnd.x, rnd.y, rnd.z, rnd.w};
#pragma unroll
                        for (int b = 0; b < 4; ++b) {
                            if (u[b] > th.x) pl[b][0] |= 1u << r;
                            if (u[b] > th.y) pl[b][1] |= 1u << r;
                            if (D == 3 && u[b] > th.z) pl[b][2] |= 1u << r;
                        }
                    }
                }
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    const int j = 4 * g + b;
                    const int i0 = 2 * j;
                    int x = i0 % L;
                    const int rr = i0 / L;
                    const int y = rr % L, z = rr / L;
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
            __syncthreads();
        }
        // per-slot unsatisfied bonds: column sums of the counters
        {
            int mine = 0;
#pragma unroll
            for (int b = 0; b < 8; ++b)
#pragma unroll
                for (int r = 0; r < 32; ++r) {
                    const unsigned v = __ballot_sync(0xFFFFFFFFu, (cnt[b] >> r) & 1u);
                    if (lane == r) mine += __popc(v) << b;
                }
            atomicAdd(&unsat[lane], mine);
        }
        __syncthreads();
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
                        make_uint4((uint32_t)k, (uint32_t)t, (uint32_t)s, kExchange << 1), a.rk);
                    if (m < pm.m1) accept = rnd.x <= a.pt_tab[pm.off + m];
                    else if (m < pm.m0) accept = rnd.x == 0u;
                }
                if (accept) {
                    sot[k] = rb;
                    sot[k + 1] = ra;
                }
            }
            __syncwarp();
            if (k < nt) thr_slot[sot[k]] = reinterpret_cast<const uint4*>(a.thr_temp)[k];
            unsat[lane] = 0;
        }
        __syncthreads();
    }
    // write the sample back
    for (int q = tid; q < 2 * H; q += nthr) a.spins[w0 + q] = S0[q];
    if (tid < nt) a.perm[s * kMaxTemps + tid] = sot[tid];
}

__global__ void batch_init_kernel(uint32_t* spins, uint8_t* bonds, int32_t* perm,
                                  const int* Ls, const long long* word_off, int d, int ntemps,
                                  RoundKeys rk)
{
    const int s = blockIdx.x;
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
                make_uint4((uint32_t)i, (uint32_t)mu, (uint32_t)s, kCoupling << 1), rk);
            if (!(r.x >> 31)) bits |= (uint8_t)(1u << mu);
        }
        B[c * H + (i >> 1)] = bits;
    }
    for (int q = threadIdx.x; q < 2 * (H / 4); q += blockDim.x) {
        const int c = q / (H / 4), g = q % (H / 4);
        uint32_t w[4] = {0, 0, 0, 0};
        for (int r = 0; r < ntemps; ++r) {
            const uint4 o = philox4x32_10(
                make_uint4((uint32_t)g, 0u, (uint32_t)(s * ntemps + r), (kInit << 1) | (uint32_t)c),
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

size_t smem_bytes(int d, int L)
{
    const int N = d == 3 ? L * L * L : L * L;
    const int H = N / 2;
    return (size_t)2 * H * 4 + ((size_t)(2 * H + 15) / 16) * 16 + kMaxTemps * 16 +
           kMaxTemps * 8 + 2 * kMaxTemps * 4;
}

int threads_for(int d, int L)
{
    const int N = d == 3 ? L * L * L : L * L;
    const int G = N / 8;
    int t = (G + 31) / 32 * 32;
    return t > 1024 ? 1024 : t;
}

}  // namespace
}  // namespace spinmc

using namespace spinmc;

struct sl_batch {
    int d, nsamples, ntemps;
    std::vector<int> L;
    std::vector<long long> word_off;
    std::vector<int> class_L;                 // distinct sizes, largest first
    std::vector<std::vector<int>> class_ids;  // samples of each size
    std::vector<int> class_dev_off;           // offset of each class in dev class list
    double betas[kMaxTemps];
    uint64_t seed;
    int64_t sweeps_done;
    cudaStream_t stream;
    cudaStream_t side[8];
    cudaEvent_t ev_fork, ev_join[8];
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
};

namespace {

struct BatchLayout {
    size_t off_spins, off_bonds, off_perm, off_Ls, off_woff, off_class, off_thr, off_meta,
        off_tab, off_staging, total;
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
    y.total = off;
    return y;
}

template <int D>
cudaError_t launch_class(const sl_batch* b, int ci, BatchArgs a, cudaStream_t st)
{
    const int L = b->class_L[ci];
    const size_t sm = smem_bytes(b->d, L);
    cudaError_t e = cudaFuncSetAttribute(ea_pt_kernel<D>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sm);
    if (e != cudaSuccess) return e;
    a.L = L;
    a.class_samples = b->class_dev + b->class_dev_off[ci];
    ea_pt_kernel<D><<<(int)b->class_ids[ci].size(), threads_for(b->d, L), sm, st>>>(a);
    return cudaGetLastError();
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
                    uint64_t seed, void* dev_buf, size_t dev_buf_bytes, void* stream,
                    sl_batch** out)
{
    if (!out) return fail(SL_EINVAL, "out is NULL");
    *out = nullptr;
    if (!betas) return fail(SL_EINVAL, "betas is NULL");
    int st = batch_check(d, L_per_sample, nsamples, ntemps, betas);
    if (st != SL_OK) return st;
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
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < 8 && e == cudaSuccess; ++k) {
        e = cudaStreamCreateWithFlags(&b->side[k], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_join[k], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming);
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
                                                   b->word_off_dev, d, ntemps,
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
    BatchArgs a;
    std::memset(&a, 0, sizeof a);
    a.spins = b->spins;
    a.bonds = b->bonds;
    a.perm = b->perm;
    a.word_off = b->word_off_dev;
    a.d = b->d;
    a.ntemps = b->ntemps;
    a.t0 = b->sweeps_done;
    a.nsweeps = (int)nsweeps;
    a.rk = make_round_keys(seed);
    a.thr_temp = b->thr_temp;
    a.pt_tab = b->pt_tab;
    a.pt_meta = b->pt_meta;
    a.E_out = dev_E;
    // fork one stream per sample size so the sizes run side by side
    cudaError_t e = cudaEventRecord(b->ev_fork, b->stream);
    const int nc = (int)b->class_L.size();
    for (int ci = 0; ci < nc && e == cudaSuccess; ++ci) {
        cudaStream_t st = b->side[ci % 8];
        e = cudaStreamWaitEvent(st, b->ev_fork, 0);
        if (e == cudaSuccess) e = b->d == 3 ? launch_class<3>(b, ci, a, st) : launch_class<2>(b, ci, a, st);
        if (e == cudaSuccess) e = cudaEventRecord(b->ev_join[ci % 8], st);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->ev_join[ci % 8], 0);
    }
    if (e != cudaSuccess) return cuda_fail(e, "sl_batch_run");
    b->sweeps_done += nsweeps;
    return SL_OK;
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

void sl_batch_destroy(sl_batch* b)
{
    if (!b) return;
    cudaStreamSynchronize(b->stream);
    for (int k = 0; k < 8; ++k) {
        if (b->side[k]) cudaStreamDestroy(b->side[k]);
        if (b->ev_join[k]) cudaEventDestroy(b->ev_join[k]);
    }
    if (b->ev_fork) cudaEventDestroy(b->ev_fork);
    if (b->owned_buf) cudaFree(b->owned_buf);
    delete b;
}

}  // extern "C"
