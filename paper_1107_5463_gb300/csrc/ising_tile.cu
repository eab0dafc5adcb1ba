// k-fold multi-hit Ising sweeps in big tiles (Weigel & Yavors'kii 2011,
// Section 2, two-level decomposition: "all spins of one of the big tiles plus
// some boundary layer are collaboratively loaded into shared memory", and "a
// number k of updates of all spins of all big tiles of one color is performed
// before updating the second" colour; Table 1 uses k = 100).
//
// The lattice is cut into tiles of side T (T % 8 == 0, L % 2T == 0) coloured
// like a checkerboard.  One launch handles the tiles of one colour: a CTA per
// tile loads the tile and a one-site halo of both colours into shared memory
// (kept split by colour, rows of T/2 bytes plus halo bytes, so four
// same-colour sites are one aligned 32-bit word), performs k inner
// checkerboard passes (site colour 0, barrier, site colour 1, barrier) with
// the same byte logic and exact thresholds as the streaming kernel, and writes
// the tile back.  Hit h of sweep t draws output j & 3 of Philox(j >> 2,
// t*k + h, replica, 4 << 1 | colour).  The halo belongs to tiles of the other
// colour, which do not change during the launch.
#include "internal.h"

namespace spinmc {
namespace {

constexpr uint32_t kMultihit = 4;

struct TileArgs {
    int8_t* s[2];  // colour arrays in global memory (0 = up, 1 = down)
    int L, W, T, k, tile_colour;
    uint32_t replica;
    IsingTable tab;
    RoundKeys rk;
    Ctrl* ctrl;
    int sigma_neg;
};

template <int NCMP>
__device__ __forceinline__ uint32_t q_bias_tile(const uint4& r, const IsingTable& tab)
{
    uint32_t acc = 0x80808080u;
    const uint32_t u[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
        for (int q = 0; q < NCMP; ++q) acc -= (u[b] > tab.thr[q]) ? (1u << (8 * b)) : 0u;
    return acc;
}

template <int D, int T>
__global__ void __launch_bounds__(D == 3 ? T * T * T / 8 : T * T / 8)
    ising_tile_kernel(const TileArgs a)
{
    constexpr int RS = T / 2 + 8;                        // bytes per shared row
    constexpr int ROWS = (T + 2) * (D == 3 ? T + 2 : 1);  // rows incl. halo
    constexpr int WPR = T / 8;                            // words (4 sites) per row
    __shared__ __align__(16) uint8_t sm[2][ROWS * RS];
    const int L = a.L, W = a.W;
    const int tpd = L / T;  // tiles per dimension
    // this CTA's tile: the blockIdx.x-th tile of colour tile_colour
    int tx, ty, tz = 0;
    {
        const long long q = blockIdx.x;  // tiles of one colour, two per pair along x
        const long long per_row = tpd / 2;
        long long rest = q / per_row;
        const int xpair = (int)(q % per_row);
        ty = (int)(rest % tpd);
        if (D == 3) tz = (int)(rest / tpd);
        const int par = (ty + tz + a.tile_colour) & 1;
        tx = 2 * xpair + par;
    }
    const int x0 = tx * (T / 2);  // first colour column of the tile
    auto srow = [&](int y, int z) -> int { return ((D == 3 ? z + 1 : 0) * (T + 2) + (y + 1)); };
    auto grow = [&](int y, int z) -> long long {
        const int Y = (ty * T + y + L) % L;
        const int Z = D == 3 ? (tz * T + z + L) % L : 0;
        return ((long long)Z * L + Y) * W;
    };
    // load the tile and its halo (no corners)
    const int ncell = 2 * ROWS * (T / 2 + 2);
    for (int q = threadIdx.x; q < ncell; q += blockDim.x) {
        const int c = q / (ROWS * (T / 2 + 2));
        const int rem = q % (ROWS * (T / 2 + 2));
        const int r = rem / (T / 2 + 2);
        const int kk = rem % (T / 2 + 2) - 1;  // -1 .. T/2
        const int y = (D == 3 ? r % (T + 2) : r) - 1;
        const int z = D == 3 ? r / (T + 2) - 1 : 0;
        const int outside = (y < 0 || y >= T) + (D == 3 && (z < 0 || z >= T)) + (kk < 0 || kk >= T / 2);
        if (outside > 1) continue;
        const int K = (x0 + kk + W) % W;
        sm[c][r * RS + 4 + kk] = (uint8_t)a.s[c][grow(y, z) + K];
    }
    __syncthreads();

    const uint32_t two_d = 0x01010101u * (uint32_t)(2 * D);
    const int g = threadIdx.x;
    const int m = g % WPR;
    const int rowlin = g / WPR;
    const int y = D == 3 ? rowlin % T : rowlin;
    const int z = D == 3 ? rowlin / T : 0;
    const int so = srow(y, z) * RS + 4 + 4 * m;  // own word in shared memory
    const long long grp0 = (grow(y, z) + x0 + 4 * m) >> 2;
    const uint32_t t = (uint32_t)a.ctrl->t;
    for (int h = 0; h < a.k; ++h) {
        const uint32_t ctr_t = t * (uint32_t)a.k + (uint32_t)h;
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const uint8_t* O = sm[1 - c];
            const int p = (y + z + c) & 1;
            const uint32_t A = *reinterpret_cast<const uint32_t*>(&sm[c][so]);
            const uint32_t cur = *reinterpret_cast<const uint32_t*>(&O[so]);
            const uint32_t S = p ? __funnelshift_r(cur, *reinterpret_cast<const uint32_t*>(&O[so + 4]), 8)
                                 : __funnelshift_l(*reinterpret_cast<const uint32_t*>(&O[so - 4]), cur, 8);
            uint32_t nd = cur + S + *reinterpret_cast<const uint32_t*>(&O[so - RS]) +
                          *reinterpret_cast<const uint32_t*>(&O[so + RS]);
            if (D == 3)
                nd += *reinterpret_cast<const uint32_t*>(&O[so - (T + 2) * RS]) +
                      *reinterpret_cast<const uint32_t*>(&O[so + (T + 2) * RS]);
            uint32_t na = (nd ^ (A * 7u)) - A * (uint32_t)(7 - 2 * D);
            if (a.sigma_neg) na = two_d - na;
            const uint4 rnd = philox4x32_10(
                make_uint4((uint32_t)grp0, ctr_t, a.replica, (kMultihit << 1) | (uint32_t)c), a.rk);
            const uint32_t flip = ((na + q_bias_tile<D>(rnd, a.tab)) & 0x80808080u) >> 7;
            *reinterpret_cast<uint32_t*>(&sm[c][so]) = A ^ flip;
            __syncthreads();
        }
    }
    // write the tile back
    for (int q = threadIdx.x; q < 2 * (ROWS - 0) * (T / 2); q += blockDim.x) {
        const int c = q / (ROWS * (T / 2));
        const int rem = q % (ROWS * (T / 2));
        const int r = rem / (T / 2);
        const int kk = rem % (T / 2);
        const int yy = (D == 3 ? r % (T + 2) : r) - 1;
        const int zz = D == 3 ? r / (T + 2) - 1 : 0;
        if (yy < 0 || yy >= T || (D == 3 && (zz < 0 || zz >= T))) continue;
        a.s[c][grow(yy, zz) + x0 + kk] = (int8_t)sm[c][r * RS + 4 + kk];
    }
}

template <int D, int T>
cudaError_t launch_tile(const TileArgs& a, cudaStream_t s)
{
    const int tpd = a.L / T;
    const long long ntiles = (long long)tpd * tpd * (D == 3 ? tpd : 1) / 2;
    ising_tile_kernel<D, T><<<(unsigned)ntiles, D == 3 ? T * T * T / 8 : T * T / 8, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

bool tile_size_ok(int d, int L, int T)
{
    if (d == 2) return (T == 8 || T == 16 || T == 32 || T == 64) && L % (2 * T) == 0;
    return (T == 8 || T == 16) && L % (2 * T) == 0;
}

cudaError_t ising_tile_sweep(const sl_lattice* h, const SweepParams& p, cudaStream_t s)
{
    TileArgs a;
    a.s[0] = (int8_t*)h->spins[0];
    a.s[1] = (int8_t*)h->spins[1];
    a.L = h->L;
    a.W = h->W;
    a.T = h->tile;
    a.k = h->multihit;
    a.replica = h->replica;
    a.tab = p.tab;
    a.rk = p.rk;
    a.ctrl = h->ctrl;
    a.sigma_neg = p.tab.sigma_neg;
    for (int tc = 0; tc < 2; ++tc) {
        a.tile_colour = tc;
        cudaError_t e = cudaErrorInvalidValue;
        if (h->d == 2) {
            switch (h->tile) {
            case 8: e = launch_tile<2, 8>(a, s); break;
            case 16: e = launch_tile<2, 16>(a, s); break;
            case 32: e = launch_tile<2, 32>(a, s); break;
            case 64: e = launch_tile<2, 64>(a, s); break;
            }
        } else {
            switch (h->tile) {
            case 8: e = launch_tile<3, 8>(a, s); break;
            case 16: e = launch_tile<3, 16>(a, s); break;
            }
        }
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace spinmc
