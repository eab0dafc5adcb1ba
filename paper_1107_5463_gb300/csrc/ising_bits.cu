// Ising model (n = 1) with one bit per site: multispin coding (Weigel &
// Yavors'kii 2011, Section 2, last paragraph: many spins in one machine word,
// updated with bitwise logic), for the ferromagnet with a uniform coupling.
//
// Storage: per colour, each row (fixed y, z) of W = L/2 sites is W/32 32-bit
// words; bit b of word w is colour column k = 32 w + b, set for spin -1.
// The random stream and every decision are those of the byte kernels
// (Philox per 4 colour indices, exact integer thresholds), so the two
// storages give bit-identical trajectories.
//
// Per word of 32 sites: the unsatisfied-bond indicators of the 2d neighbours
// are word XORs; a bitsliced adder turns them into the count na (bit planes
// b0, b1, b2); the Philox outputs of the 32 sites are compared with the d
// thresholds into planes g_k = [u > T_k]; the move is accepted where
// na >= k + 1 for every k with g_k set, which equals u <= T[na].
//
// Slabs (a lattice split along its slowest axis) are handled as in the byte
// kernels: Lz local planes between halo planes, global Philox groups and
// colour parity.
#include "internal.h"

namespace spinmc {
namespace {

struct BitArgs {
    uint32_t* own;
    const uint32_t* oth;
    int d, L, W, c, R;
    long long H, N;
    uint32_t replica;
    IsingTable tab;
    RoundKeys rk;
    Ctrl* ctrl;
    Partial* partials;
    double J;
    int measure, update;
    int Lz;          // planes along the slowest axis (L, or the slab's planes)
    int wrap;        // 1: periodic along the slowest axis; 0: halo planes at -1 and Lz
    int par;         // parity of the first plane's global index
    long long gofs;  // global colour index of local colour entry 0
};

__device__ __forceinline__ void bits_finish(const BitArgs& a, const Partial& tot)
{
    Ctrl* C = a.ctrl;
    const double E = -a.J * (double)tot.i0;
    const double M = (double)(a.N - 2 * tot.i1);
    C->obs[0] = E;
    C->obs[1] = M;
    C->obs[2] = 0.0;
    C->obs[3] = 0.0;
    if (a.update) {
        const long long k = (long long)C->t - C->series_base;
        if (C->series_E) C->series_E[k] = E;
        // a slab records its own M (summed over slabs, |M| / N is |m|)
        if (C->series_absm) C->series_absm[k] = a.wrap ? fabs(M) / (double)a.N : M;
        C->t = C->t + 1;
    }
}

// full adder on bit planes
__device__ __forceinline__ void fadd(uint32_t a, uint32_t b, uint32_t c, uint32_t& s, uint32_t& k)
{
    s = a ^ b ^ c;
    k = (a & b) | (c & (a ^ b));
}

// MEAS: the measuring (colour-1) pass, whose blocks add their integer totals
// into the accumulator after the block partials for bits_finish_kernel; the
// other pass is compiled without the counters.
// SLAB: a slab of a split lattice (halo planes, global offsets).
template <int D, int JNEG, bool MEAS, bool SLAB = false>
__global__ void __launch_bounds__(128) bits_stream(const BitArgs a)
{
    __shared__ long long red[32];
    const uint32_t t = (uint32_t)a.ctrl->t;
    const int L = a.L, R = a.R, Lz = SLAB ? a.Lz : a.L;
    const int WW = a.W >> 5;  // words per row
    const long long nseg = Lz / R;
    const int spar = SLAB ? a.par : 0;
    const long long gofs = SLAB ? a.gofs : 0;
    // neighbouring plane along the slowest axis: periodic, or a halo plane
    auto zprev = [&](int m) { return m == 0 ? (SLAB ? -1 : Lz - 1) : m - 1; };
    auto znext = [&](int m) { return m == Lz - 1 ? (SLAB ? Lz : 0) : m + 1; };
    const long long nitems = (long long)WW * (D == 3 ? L : 1) * nseg;
    const uint32_t ctr_w = (kSweep << 1) | (uint32_t)a.c;
    const uint32_t inv = JNEG ? 0xFFFFFFFFu : 0u;
    unsigned long long s_na = 0, s_flip = 0, s_flipna = 0, down = 0, nsite = 0;

    for (long long it = (long long)blockIdx.x * blockDim.x + threadIdx.x; it < nitems;
         it += (long long)gridDim.x * blockDim.x) {
        const int w = (int)(it % WW);
        const long long rest = it / WW;
        const int y3 = D == 3 ? (int)(rest % L) : 0;
        const int seg = D == 3 ? (int)(rest / L) : (int)rest;
        const int m0 = seg * R;
        auto row = [&](int yy, int zz) -> long long { return (long long)zz * L + yy; };
        auto mrow = [&](int m) -> long long { return D == 3 ? row(y3, m) : row(m, 0); };
        const int mprev = zprev(m0);
        uint32_t prev = __ldg(a.oth + mrow(mprev) * WW + w);
        uint32_t cur = __ldg(a.oth + mrow(m0) * WW + w);
        const int wl = w == 0 ? WW - 1 : w - 1, wr = w == WW - 1 ? 0 : w + 1;
        const int y_m = y3 == 0 ? L - 1 : y3 - 1, y_p = y3 == L - 1 ? 0 : y3 + 1;
        uint32_t i_na = 0, i_flip = 0, i_flipna = 0, i_down = 0;
        // software pipeline: the next row of the other colour, the own word,
        // the x-neighbour word and (3D) the y -/+ 1 words are loaded one row ahead
        auto rowof = [&](int m) -> long long { return D == 3 ? row(y3, m) : row(m, 0); };
        auto par = [&](int m) -> int { return ((D == 3 ? y3 + m : m) + a.c + spar) & 1; };
        uint32_t next_nx = __ldg(a.oth + mrow(znext(m0)) * WW + w);
        uint32_t A_nx = a.own[rowof(m0) * WW + w];
        uint32_t hw_nx = __ldg(a.oth + rowof(m0) * WW + (par(m0) ? wr : wl));
        uint32_t ym_nx = 0, yp_nx = 0;
        if (D == 3) {
            ym_nx = __ldg(a.oth + row(y_m, m0) * WW + w);
            yp_nx = __ldg(a.oth + row(y_p, m0) * WW + w);
        }
        // two rows per loop pass, so their Philox blocks interleave
#pragma unroll 2
        for (int r = 0; r < R; ++r) {
            const int m = m0 + r;
            const int yy = D == 3 ? y3 : m;
            const int zz = D == 3 ? m : 0;
            const int p = (yy + zz + a.c + spar) & 1;
            const long long rr = row(yy, zz);
            const uint32_t next = next_nx, A = A_nx, hw = hw_nx, ym = ym_nx, yp = yp_nx;
            if (r + 1 < R) {
                const int m1 = m + 1, m2 = znext(m1);
                next_nx = __ldg(a.oth + mrow(m2) * WW + w);
                A_nx = a.own[rowof(m1) * WW + w];
                hw_nx = __ldg(a.oth + rowof(m1) * WW + (par(m1) ? wr : wl));
                if (D == 3) {
                    ym_nx = __ldg(a.oth + row(y_m, m1) * WW + w);
                    yp_nx = __ldg(a.oth + row(y_p, m1) * WW + w);
                }
            }
            // -x / +x neighbours of column k are other-colour columns
            // k-1 / k (p = 0) or k / k+1 (p = 1)
            const uint32_t S = p ? __funnelshift_r(cur, hw, 1) : __funnelshift_l(hw, cur, 1);
            uint32_t b0, b1, b2;
            if (D == 2) {
                uint32_t s1, c1;
                fadd(A ^ S ^ inv, A ^ cur ^ inv, A ^ prev ^ inv, s1, c1);
                const uint32_t u4 = A ^ next ^ inv;
                b0 = s1 ^ u4;
                const uint32_t k = s1 & u4;
                b1 = c1 ^ k;
                b2 = c1 & k;
            } else {
                uint32_t s1, c1, s2, c2;
                fadd(A ^ S ^ inv, A ^ cur ^ inv, A ^ prev ^ inv, s1, c1);
                fadd(A ^ next ^ inv, A ^ ym ^ inv, A ^ yp ^ inv, s2, c2);
                b0 = s1 ^ s2;
                const uint32_t k = s1 & s2;
                fadd(c1, c2, k, b1, b2);
            }
            uint32_t flip = 0;
            if (a.update) {
                const uint32_t ge1 = b0 | b1 | b2, ge2 = b1 | b2, ge3 = b2 | (b1 & b0);
                uint32_t g0 = 0, g1 = 0, g2 = 0;
                const uint32_t grp = (uint32_t)((rr * a.W + gofs + 32 * w) >> 2);
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const uint4 rnd = philox4x32_10(make_uint4(grp + q, t, a.replica, ctr_w), a.rk);
                    const uint32_t u[4] = {rnd.x, rnd.y, rnd.z, rnd.w};
#pragma unroll
                    for (int b = 0; b < 4; ++b) {
                        const uint32_t bit = 1u << (4 * q + b);
                        if (u[b] > a.tab.thr[0]) g0 |= bit;
                        if (u[b] > a.tab.thr[1]) g1 |= bit;
                        if (D == 3 && u[b] > a.tab.thr[2]) g2 |= bit;
                    }
                }
                flip = (~g0 | ge1) & (~g1 | ge2);
                if (D == 3) flip &= ~g2 | ge3;
            }
            const uint32_t An = A ^ flip;
            if (a.update) a.own[rr * WW + w] = An;
            if (MEAS) {
                i_na += __popc(b0) + 2 * __popc(b1) + 4 * __popc(b2);
                i_flip += __popc(flip);
                i_flipna += __popc(flip & b0) + 2 * __popc(flip & b1) + 4 * __popc(flip & b2);
                i_down += __popc(An) + __popc(cur);
            }
            prev = cur;
            cur = next;
        }
        if (MEAS) {
            s_na += i_na;
            s_flip += i_flip;
            s_flipna += i_flipna;
            down += i_down;
            nsite += 32 * R;
        }
    }
    if (!MEAS) return;
    const long long na_after = (long long)s_na + 2 * D * (long long)s_flip - 2 * (long long)s_flipna;
    long long bond = (long long)(2 * D) * (long long)nsite - 2 * na_after;
    if (JNEG) bond = -bond;
    Partial mine;
    mine.i0 = block_sum(bond, red);
    mine.i1 = block_sum((long long)down, red);
    // integer totals: the order of the additions does not matter
    if (threadIdx.x == 0) {
        Partial* acc = a.partials + kMaxBlocks;
        atomicAdd(reinterpret_cast<unsigned long long*>(&acc->i0), (unsigned long long)mine.i0);
        atomicAdd(reinterpret_cast<unsigned long long*>(&acc->i1), (unsigned long long)mine.i1);
    }
}

// Closes a measuring pass from the totals its blocks added into the
// accumulator, and clears the accumulator for the next pass (one thread; the
// kernel boundary orders it after the pass).
__global__ void bits_finish_kernel(const BitArgs a)
{
    Partial* acc = a.partials + kMaxBlocks;
    Partial tot = *acc;
    acc->i0 = 0;
    acc->i1 = 0;
    bits_finish(a, tot);
}

// wofs: global index of local word 0 (the global colour index of entry 0 / 32)
__global__ void bits_init_kernel(uint32_t* s0, uint32_t* s1, long long nwords, uint32_t replica,
                                 RoundKeys rk, long long wofs)
{
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < 2 * nwords;
         q += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(q / nwords);
        const long long w = q % nwords;
        uint32_t word = 0;
#pragma unroll
        for (int g = 0; g < 8; ++g) {
            const uint4 r = philox4x32_10(
                make_uint4((uint32_t)(8 * (w + wofs) + g), 0u, replica, (kInit << 1) | (uint32_t)c),
                rk);
            const uint32_t o[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
            for (int b = 0; b < 4; ++b)
                if (!(o[b] >> 31)) word |= 1u << (4 * g + b);
        }
        (c ? s1 : s0)[w] = word;
    }
}

// natural +-1 bytes -> bit words: word (row r, w) of colour c holds natural
// sites r L + 64 w + 2 b + p, p = (y + z + c) & 1
__global__ void bits_scatter_kernel(uint32_t* s0, uint32_t* s1, const int8_t* nat, long long nwords,
                                    int L, int WW, int par)
{
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < 2 * nwords;
         q += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(q / nwords);
        const long long wi = q % nwords;
        const long long r = wi / WW;
        const int w = (int)(wi % WW);
        const int y = (int)(r % L), z = (int)(r / L);
        const int p = (y + z + c + par) & 1;
        const long long base = r * L + 64LL * w + p;
        uint32_t word = 0;
        for (int b = 0; b < 32; ++b)
            if (nat[base + 2 * b] < 0) word |= 1u << b;
        (c ? s1 : s0)[wi] = word;
    }
}

__global__ void bits_gather_kernel(const uint32_t* s0, const uint32_t* s1, int8_t* nat, long long N,
                                   int L, int par)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % L);
        const long long r = i / L;
        const int y = (int)(r % L), z = (int)(r / L);
        const int c = (x + y + z + par) & 1;
        const long long j = i >> 1;  // = r W + (x >> 1)
        const uint32_t word = (c ? s1 : s0)[j >> 5];
        nat[i] = ((word >> (j & 31)) & 1u) ? (int8_t)-1 : (int8_t)1;
    }
}

int grid_for(long long work, int block)
{
    long long g = (work + block - 1) / block;
    if (g < 1) g = 1;
    if (g > kMaxBlocks) g = kMaxBlocks;
    return (int)g;
}

int pick_rows(const sl_lattice* h)
{
    if (h->rows > 0) return h->rows;
    // measured on GB300: 8 rows per thread in 2D (1147 flips/ns at L = 16384),
    // 4 in 3D (903 at L = 512, against 891-897 for 8 and 16)
    const long long WW = h->W / 32;
    const long long cross = h->d == 3 ? h->L : 1;
    int R = h->d == 3 ? 4 : 8;
    while (R > 1 && (h->Lz % R != 0 || WW * cross * (h->Lz / R) < (long long)h->sms * 512))
        R >>= 1;
    return R;
}

BitArgs make_args(const sl_lattice* h, int c)
{
    BitArgs a;
    a.own = (uint32_t*)h->spins[c];
    a.oth = (const uint32_t*)h->spins[1 - c];
    a.d = h->d;
    a.L = h->L;
    a.W = h->W;
    a.c = c;
    a.R = pick_rows(h);
    a.H = h->H;
    a.N = h->N;
    a.replica = h->replica;
    a.ctrl = h->ctrl;
    a.partials = h->partials;
    a.J = h->J;
    a.measure = c == 1;
    a.update = 1;
    a.Lz = h->Lz;
    a.wrap = !h->slab;
    a.par = h->z0 & 1;
    a.gofs = (long long)h->z0 * h->P;
    return a;
}

cudaError_t launch(const sl_lattice* h, const BitArgs& a, cudaStream_t s)
{
    const long long items = (long long)(h->W / 32) * (h->d == 3 ? h->L : 1) * (h->Lz / a.R);
    int grid = grid_for(items, 128);
    if (h->blocks_per_sm > 0 && grid > h->sms * h->blocks_per_sm) grid = h->sms * h->blocks_per_sm;
    const bool jneg = a.tab.sigma_neg != 0;
#define SPINMC_BITS(D, N)                                                          \
    do {                                                                           \
        if (h->slab) {                                                             \
            if (a.measure) bits_stream<D, N, true, true><<<grid, 128, 0, s>>>(a);  \
            else bits_stream<D, N, false, true><<<grid, 128, 0, s>>>(a);           \
        } else {                                                                   \
            if (a.measure) bits_stream<D, N, true><<<grid, 128, 0, s>>>(a);        \
            else bits_stream<D, N, false><<<grid, 128, 0, s>>>(a);                 \
        }                                                                          \
    } while (0)
    if (h->d == 2) {
        if (jneg) SPINMC_BITS(2, 1);
        else SPINMC_BITS(2, 0);
    } else {
        if (jneg) SPINMC_BITS(3, 1);
        else SPINMC_BITS(3, 0);
    }
#undef SPINMC_BITS
    if (a.measure) {
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        bits_finish_kernel<<<1, 1, 0, s>>>(a);
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t ising_bits_init(const sl_lattice* h, cudaStream_t s)
{
    const long long nwords = h->H / 32;
    bits_init_kernel<<<grid_for(2 * nwords, 256), 256, 0, s>>>(
        (uint32_t*)h->spins[0], (uint32_t*)h->spins[1], nwords, h->replica,
        make_round_keys(h->init_seed), (long long)h->z0 * h->P / 32);
    return cudaGetLastError();
}

cudaError_t ising_bits_scatter(const sl_lattice* h, const int8_t* nat, cudaStream_t s)
{
    const long long nwords = h->H / 32;
    bits_scatter_kernel<<<grid_for(2 * nwords, 256), 256, 0, s>>>(
        (uint32_t*)h->spins[0], (uint32_t*)h->spins[1], nat, nwords, h->L, h->W / 32, h->z0 & 1);
    return cudaGetLastError();
}

cudaError_t ising_bits_gather(const sl_lattice* h, int8_t* nat, cudaStream_t s)
{
    bits_gather_kernel<<<grid_for(h->N, 256), 256, 0, s>>>(
        (const uint32_t*)h->spins[0], (const uint32_t*)h->spins[1], nat, h->N, h->L, h->z0 & 1);
    return cudaGetLastError();
}

cudaError_t ising_bits_sweeps(const sl_lattice* h, const SweepParams& p, int64_t count,
                              cudaStream_t s)
{
    for (int64_t k = 0; k < count; ++k)
        for (int c = 0; c < 2; ++c) {
            BitArgs a = make_args(h, c);
            a.tab = p.tab;
            a.rk = p.rk;
            const cudaError_t e = launch(h, a, s);
            if (e != cudaSuccess) return e;
        }
    return cudaSuccess;
}

cudaError_t ising_bits_pass(const sl_lattice* h, const SweepParams& p, int c, cudaStream_t s)
{
    BitArgs a = make_args(h, c);
    a.tab = p.tab;
    a.rk = p.rk;
    return launch(h, a, s);
}

cudaError_t ising_bits_measure(const sl_lattice* h, cudaStream_t s)
{
    BitArgs a = make_args(h, 1);
    a.update = 0;
    a.measure = 1;
    memset(&a.tab, 0, sizeof a.tab);
    a.tab.sigma_neg = h->J < 0.0;
    memset(&a.rk, 0, sizeof a.rk);
    return launch(h, a, s);
}

}  // namespace spinmc
