// Swendsen-Wang cluster updates of the Ising model on byte storage
// (Weigel & Yavors'kii 2011, Section 3: activate bonds between like spins with
// p = 1 - exp(-2 beta J), build the clusters joined by active bonds, flip each
// cluster with probability 1/2; cluster identification in tiles first, then
// amalgamation of the tiles through a union-and-find structure).
//
// One update is five kernels:
//   sw_local    one CTA per tile (64 x 32 sites in 2D, 64 x 16 x 8 in 3D):
//               loads the tile's spins and a one-site halo on its +x/+y/+z
//               faces into shared memory (one warp per row, one lane per site
//               pair), draws the bond uniforms, joins each row's x-runs of
//               active bonds through warp ballots, then joins the runs along
//               y and z by a lock-free union-find in shared memory (the
//               larger root linked below the smaller by compare-and-swap),
//               which names every tile cluster by its smallest site (a y/z
//               bond is skipped when the bond beside it already joins the
//               same two runs), writes every site's label (the natural index
//               of its tile root, the smallest site of its tile cluster),
//               one bit per active bond that leaves the tile, and appends
//               its tile roots to a list;
//   sw_merge    one thread per tile-face bond: unites the two labels of each
//               active face bond in global memory (same hooking rule);
//               afterwards the root of every cluster is its smallest site;
//   sw_resolve  one thread per listed tile root: follows the parents to the
//               cluster root g and rewrites the tile root's word as g with
//               g's flip bit (drawn from g's Philox output);
//   sw_flip     every site reads its tile root's word (its own word if it is
//               one) for the flip bit and flips;
//   sw_measure  E and M of the new configuration, closing the sweep.
// Label words: bits 0-29 the parent (a site index, N <= 2^30), bit 31 marks
// a tile root; after sw_resolve bit 30 of a tile root's word is its
// cluster's flip bit.  Every parent is a smaller or equal index and, beyond
// a site's first step, a tile root.
// Random numbers: the forward bond (i, i + e_mu) draws output 2 (i & 1) + mu
// of Philox(i >> 1, t, replica, 5 << 1) in 2D, output mu of
// Philox(i, t, replica, 5 << 1) in 3D; the cluster rooted at r flips iff the
// top bit of output 0 of Philox(r, t, replica, 6 << 1) is set.  Because the
// root is the smallest site whatever order the unions run in, the result does
// not depend on scheduling.
#include <cuda/atomic>

#include "internal.h"

namespace spinmc {
namespace {

constexpr uint32_t kSwBond = 5, kSwFlip = 6;
constexpr uint32_t kMask = 0x3FFFFFFFu;     // parent index
constexpr uint32_t kTileRoot = 0x80000000u;  // the site is a tile root
constexpr uint32_t kFlipBit = 0x40000000u;   // the cluster rooted here flips
constexpr int kSwThreads = 512;

template <int D>
struct SwTile;
template <>
struct SwTile<2> {
    static constexpr int TX = 64, TY = 32, TZ = 1;
};
template <>
struct SwTile<3> {
    static constexpr int TX = 64, TY = 16, TZ = 8;
};

template <int D>
struct SwFace {
    static constexpr int TX = SwTile<D>::TX, TY = SwTile<D>::TY, TZ = SwTile<D>::TZ;
    // face bits: +x face (TY x TZ), +y face (TX x TZ), +z face (TX x TY, 3D)
    static constexpr int BITS = TY * TZ + TX * TZ + (D == 3 ? TX * TY : 0);
    static constexpr int WORDS = BITS / 32;
};

struct SwArgs {
    int8_t* s[2];     // colour arrays (0 = up, 1 = down)
    uint32_t* lab;    // N labels, natural order
    uint32_t* face;   // WORDS per tile
    uint32_t* roots;  // the tile roots of an update (at most N), in no fixed order
    unsigned* nroots; // their number
    int L;
    int ntx, nty, ntz;
    long long N, ntiles;
    uint32_t thr;     // a satisfied bond is active iff u <= thr
    int never;        // no bond can be active (beta = 0)
    int anti;         // J < 0: unlike spins satisfy a bond
    uint32_t replica;
    RoundKeys rk;
    Ctrl* ctrl;
};

int grid_for(long long work, int block)
{
    long long g = (work + block - 1) / block;
    if (g < 1) g = 1;
    if (g > kMaxBlocks) g = kMaxBlocks;
    return (int)g;
}

using gref = cuda::atomic_ref<uint32_t, cuda::thread_scope_device>;

__device__ __forceinline__ uint32_t gload(uint32_t* p)
{
    return gref(*p).load(cuda::memory_order_relaxed);
}

__device__ __forceinline__ void gstore(uint32_t* p, uint32_t v)
{
    gref(*p).store(v, cuda::memory_order_relaxed);
}

// global find with path halving (the same argument as in shared memory); a
// halving store keeps the entry's tile-root bit
__device__ __forceinline__ uint32_t gfind(uint32_t* lab, uint32_t x)
{
    uint32_t w = gload(lab + x);
    uint32_t p = w & kMask;
    while (p != x) {
        const uint32_t g = gload(lab + p) & kMask;
        if (g == p) return p;
        gstore(lab + x, g | (w & kTileRoot));
        x = g;
        w = gload(lab + x);
        p = w & kMask;
    }
    return x;
}

// roots are tile roots, so a root's word is r | kTileRoot
__device__ __forceinline__ void gunion(uint32_t* lab, uint32_t a, uint32_t b)
{
    a = gfind(lab, a);
    b = gfind(lab, b);
    while (a != b) {
        if (a < b) {
            const uint32_t t = a;
            a = b;
            b = t;
        }
        uint32_t expect = a | kTileRoot;
        if (gref(lab[a]).compare_exchange_strong(expect, b | kTileRoot,
                                                 cuda::memory_order_relaxed))
            return;
        a = gfind(lab, expect & kMask);
        b = gfind(lab, b);
    }
}


template <int D>
__device__ __forceinline__ void tile_origin(const SwArgs& a, long long b, int& X0, int& Y0, int& Z0,
                                            int& nx, int& ny, int& nz)
{
    constexpr int TX = SwTile<D>::TX, TY = SwTile<D>::TY, TZ = SwTile<D>::TZ;
    const int bx = (int)(b % a.ntx);
    const int by = (int)((b / a.ntx) % a.nty);
    const int bz = (int)(b / ((long long)a.ntx * a.nty));
    X0 = bx * TX;
    Y0 = by * TY;
    Z0 = bz * TZ;
    nx = min(TX, a.L - X0);
    ny = min(TY, a.L - Y0);
    nz = D == 3 ? min(TZ, a.L - Z0) : 1;
}

// position of the q-th (from 0) set bit of m; q < popc(m)
__device__ __forceinline__ int nth_set_bit(uint32_t m, int q)
{
    int pos = 0;
#pragma unroll
    for (int w = 16; w > 0; w >>= 1) {
        const uint32_t low = m & ((1u << w) - 1u);
        const int c = __popc(low);
        if (q >= c) {
            q -= c;
            m >>= w;
            pos += w;
        } else {
            m = low;
        }
    }
    return pos;
}

// root of x in the shared parent array, halving the path on the way (a
// halving store only ever replaces a non-root's parent by an ancestor)
__device__ __forceinline__ uint32_t sfind(volatile uint32_t* par, uint32_t x)
{
    uint32_t p = par[x];
    while (p != x) {
        const uint32_t g = par[p];
        if (g == p) return p;
        par[x] = g;
        x = g;
        p = par[x];
    }
    return x;
}

__device__ __forceinline__ bool bond_active(const SwArgs& a, uint8_t s0, uint8_t s1, uint32_t u)
{
    return (int)(s0 ^ s1) == a.anti && !a.never && u <= a.thr;
}

template <int D>
__global__ void __launch_bounds__(kSwThreads, 3) sw_local(const SwArgs a)
{
    constexpr int TX = SwTile<D>::TX, TY = SwTile<D>::TY, TZ = SwTile<D>::TZ;
    static_assert(TX == 64, "one warp lane per site pair of a 64-site row");
    constexpr int NS = TX * TY * TZ;
    constexpr int HX = TX + 2, HY = TY + 1, HZ = D == 3 ? TZ + 1 : 1;  // halo-padded spin tile
    constexpr int WORDS = SwFace<D>::WORDS;
    constexpr int NW = kSwThreads / 32;
    constexpr int ROWS = TY * TZ;
    constexpr int RPW = ROWS / NW;  // rows per warp
    __shared__ uint32_t par[NS];
    __shared__ uint8_t sp[HZ * HY * HX];
    __shared__ uint32_t fm[WORDS];
    // per row, per lane bit: active in-tile bonds of the lane's even (0) and
    // odd (1) site along +x, +y and +z
    __shared__ uint32_t bx[2][ROWS], by[2][ROWS], bz[2][D == 3 ? ROWS : 1];

    const long long b = blockIdx.x;
    int X0, Y0, Z0, nx, ny, nz;
    tile_origin<D>(a, b, X0, Y0, Z0, nx, ny, nz);
    const uint32_t L = (uint32_t)a.L;
    const uint32_t t = (uint32_t)a.ctrl->t;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int lx0 = 2 * lane;
    const bool ex = lx0 < nx;  // the lane's site pair lies in the tile

    for (int w = threadIdx.x; w < WORDS; w += blockDim.x) fm[w] = 0u;
    // the tile's rows plus the +y row and +z plane (one warp per row), and
    // the +x column
    for (int r = warp; r < HY * HZ; r += NW) {
        const int ly = r % HY, lz = r / HY;
        if (ly > ny || (D == 3 && lz > nz)) continue;
        const bool hy = ly == ny, hz = D == 3 && lz == nz;
        if (hy && hz) continue;
        const uint32_t y = (uint32_t)(Y0 + ly) == L ? 0u : (uint32_t)(Y0 + ly);
        const uint32_t z = D == 3 ? ((uint32_t)(Z0 + lz) == L ? 0u : (uint32_t)(Z0 + lz)) : 0u;
        const uint32_t rowbase = L * (y + L * z);
        const int ce = (int)((y + z) & 1u);  // colour of the even-x sites
        uint8_t* dst = sp + (lz * HY + ly) * HX;
        if (ex) {
            const uint32_t j = (rowbase + (uint32_t)(X0 + lx0)) >> 1;
            dst[lx0] = (uint8_t)a.s[ce][j];
            dst[lx0 + 1] = (uint8_t)a.s[ce ^ 1][j];
        }
        if (lane == 0 && !hy && !hz) {
            const uint32_t x = (uint32_t)(X0 + nx) == L ? 0u : (uint32_t)(X0 + nx);
            dst[nx] = (uint8_t)a.s[(x + y + z) & 1u][(rowbase + x) >> 1];
        }
    }
    // 2D: the bond uniforms of both of the warp's rows are drawn here, with
    // no branch between them, while the spin loads are in flight (rows
    // outside a ragged tile draw values nobody reads)
    uint4 pre[D == 2 ? RPW : 1];
    if (D == 2) {
#pragma unroll
        for (int k = 0; k < RPW; ++k) {
            const int ly = (warp + NW * k) % TY;
            const uint32_t i0 = (uint32_t)(X0 + lx0) + L * (uint32_t)(Y0 + ly);
            pre[k] = philox4x32_10(make_uint4(i0 >> 1, t, a.replica, kSwBond << 1), a.rk);
        }
    }
    __syncthreads();

    // Bond activation, one warp per row.  A row splits into x-runs of sites
    // joined by active bonds; every site's parent becomes the first site of
    // its run, found from the warp's ballots.  Bonds leaving the tile set
    // their face bit.
#pragma unroll
    for (int k = 0; k < RPW; ++k) {
        const int row = warp + NW * k;
        const int ly = row % TY, lz = row / TY;
        if (ly >= ny || lz >= nz) continue;  // uniform across the warp
        const int so = (lz * HY + ly) * HX + lx0;
        bool xb0 = false, xb1 = false, yb[2] = {false, false}, zb[2] = {false, false};
        if (ex) {
            const uint32_t i0 = (uint32_t)(X0 + lx0) + L * ((uint32_t)(Y0 + ly) + L * (uint32_t)(Z0 + lz));
            // uniforms of the x / y / z bonds of the even (e = 0) and odd site
            uint4 r0, r1;
            if (D == 2) {
                r0 = pre[D == 2 ? k : 0];
                r1 = make_uint4(r0.z, r0.w, 0u, 0u);
            } else {
                r0 = philox4x32_10(make_uint4(i0, t, a.replica, kSwBond << 1), a.rk);
                r1 = philox4x32_10(make_uint4(i0 + 1, t, a.replica, kSwBond << 1), a.rk);
            }
            const uint8_t s0 = sp[so], s1 = sp[so + 1], s2 = sp[so + 2];
            xb0 = bond_active(a, s0, s1, r0.x);
            xb1 = bond_active(a, s1, s2, r1.x);
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const uint8_t own = e ? s1 : s0;
                const int lx = lx0 + e;
                const uint4 re = e ? r1 : r0;
                if (bond_active(a, own, sp[so + e + HX], re.y)) {
                    if (ly + 1 == ny) {
                        const int bit = TY * TZ + lx + TX * lz;
                        atomicOr(&fm[bit >> 5], 1u << (bit & 31));
                    } else {
                        yb[e] = true;
                    }
                }
                if (D == 3 && bond_active(a, own, sp[so + e + HX * HY], re.z)) {
                    if (lz + 1 == nz) {
                        const int bit = TY * TZ + TX * TZ + lx + TX * ly;
                        atomicOr(&fm[bit >> 5], 1u << (bit & 31));
                    } else {
                        zb[e] = true;
                    }
                }
            }
        }
        const bool xcross = xb1 && lx0 + 2 == nx;
        if (xcross) {
            const int bit = ly + TY * lz;
            atomicOr(&fm[bit >> 5], 1u << (bit & 31));
        }
        const uint32_t B0 = __ballot_sync(0xFFFFFFFFu, xb0);
        const uint32_t B1 = __ballot_sync(0xFFFFFFFFu, xb1 && !xcross);
        const uint32_t Y0b = __ballot_sync(0xFFFFFFFFu, yb[0]);
        const uint32_t Y1b = __ballot_sync(0xFFFFFFFFu, yb[1]);
        uint32_t Z0b = 0u, Z1b = 0u;
        if (D == 3) {
            Z0b = __ballot_sync(0xFFFFFFFFu, zb[0]);
            Z1b = __ballot_sync(0xFFFFFFFFu, zb[1]);
        }
        if (lane == 0) {
            bx[0][row] = B0;
            bx[1][row] = B1;
            by[0][row] = Y0b;
            by[1][row] = Y1b;
            if (D == 3) {
                bz[0][D == 3 ? row : 0] = Z0b;
                bz[1][D == 3 ? row : 0] = Z1b;
            }
        }
        if (ex) {
            // run starts: the even site starts a run unless the bond from the
            // previous lane's odd site is active, the odd site unless xb0 is
            const uint32_t R0 = ~(B1 << 1);
            const uint32_t R1 = ~B0;
            int rs0 = 2 * (31 - __clz(R0 & ((2u << lane) - 1u)));
            const uint32_t m1 = R1 & ((1u << lane) - 1u);
            if (m1) rs0 = max(rs0, 2 * (31 - __clz(m1)) + 1);
            const int rs1 = xb0 ? rs0 : lx0 + 1;
            const int base = TX * (ly + TY * lz);
            par[base + lx0] = (uint32_t)(base + rs0);
            par[base + lx0 + 1] = (uint32_t)(base + rs1);
        }
    }
    __syncthreads();

    // The runs are joined along y and z by the active bonds between rows.  A
    // bond is left out when the bond at x - 1 is active and x - 1, x are
    // joined in both rows (the same two runs).
    uint32_t pend = 0;  // bit (k, e, mu): y/z bond of row k, site e, direction mu
    if (ex) {
#pragma unroll
        for (int k = 0; k < RPW; ++k) {
            const int row = warp + NW * k;
            const int ly = row % TY, lz = row / TY;
            if (ly >= ny || lz >= nz) continue;
#pragma unroll
            for (int mu = 1; mu < D; ++mu) {
                const int nrow = mu == 1 ? row + 1 : row + TY;
                const uint32_t c0 = mu == 1 ? by[0][row] : bz[0][D == 3 ? row : 0];
                const uint32_t c1 = mu == 1 ? by[1][row] : bz[1][D == 3 ? row : 0];
                // even site 2k: its left neighbour is lane k-1's odd site
                bool p0 = (c0 >> lane) & 1u;
                if (p0 && lane > 0 && ((c1 >> (lane - 1)) & 1u) &&
                    ((bx[1][row] >> (lane - 1)) & 1u) && ((bx[1][nrow] >> (lane - 1)) & 1u))
                    p0 = false;
                // odd site 2k+1: its left neighbour is lane k's even site
                bool p1 = (c1 >> lane) & 1u;
                if (p1 && ((c0 >> lane) & 1u) && ((bx[0][row] >> lane) & 1u) &&
                    ((bx[0][nrow] >> lane) & 1u))
                    p1 = false;
                const int base = k * 2 * (D - 1) + (mu - 1);
                if (p0) pend |= 1u << base;
                if (p1) pend |= 1u << (base + (D - 1));
            }
        }
    }
    // Every parent is a run head (the first site of an x-run), so after the
    // heads have jumped to their roots a label is read through the head (two
    // steps).  The warp lists the heads of its rows in shared memory (each
    // lane places its own by a population count of the ballot below it) and
    // deals the list out over its lanes for the jump; the heads are decided
    // by the x-bond ballots.
    // (3D, whose tile already fills most of the shared memory, keeps the
    // heads in registers instead: lane l takes the l-th and (l + 32)-th
    // head of each of its rows)
    __shared__ uint16_t hlist[NW][D == 2 ? RPW * TX : 1];
    unsigned nh = 0;                   // 2D: heads listed by the warp (warp-uniform)
    uint32_t heads[D == 2 ? 1 : RPW];  // 3D: per row two 16-bit sites, 0xFFFF = none
    {
        const uint32_t valid = nx >= 64 ? 0xFFFFFFFFu : ((1u << (nx >> 1)) - 1u);
        const uint32_t below = (1u << lane) - 1u;
#pragma unroll
        for (int k = 0; k < RPW; ++k) {
            if (D == 3) heads[D == 2 ? 0 : k] = 0xFFFFFFFFu;
            const int row = warp + NW * k;
            const int ly = row % TY, lz = row / TY;
            if (ly >= ny || lz >= nz) continue;
            const uint32_t h0 = ~(bx[1][row] << 1) & valid;  // even sites starting a run
            const uint32_t h1 = ~bx[0][row] & valid;         // odd sites starting a run
            const unsigned n0 = __popc(h0);
            if (D == 2) {
                if ((h0 >> lane) & 1u)
                    hlist[warp][nh + __popc(h0 & below)] = (uint16_t)(TX * row + lx0);
                if ((h1 >> lane) & 1u)
                    hlist[warp][nh + n0 + __popc(h1 & below)] = (uint16_t)(TX * row + lx0 + 1);
                nh += n0 + __popc(h1);
            } else {
                const int n = (int)n0 + __popc(h1);
                uint32_t w = 0;
#pragma unroll
                for (int slot = 0; slot < 2; ++slot) {
                    const int q = lane + 32 * slot;
                    uint32_t site = 0xFFFFu;
                    if (q < n)
                        site = (uint32_t)(TX * row) +
                               (q < (int)n0 ? 2u * (uint32_t)nth_set_bit(h0, q)
                                            : 2u * (uint32_t)nth_set_bit(h1, q - (int)n0) + 1u);
                    w |= site << (16 * slot);
                }
                heads[D == 2 ? 0 : k] = w;
            }
        }
        __syncwarp();
    }
    // One union per remaining y/z bond, lock-free: find both roots (path
    // halving), link the larger root below the smaller by compare-and-swap,
    // retry from the new roots if another link got there first.  Parents only
    // ever point to smaller indices and a root links only below a smaller
    // root, so the root of every tile cluster ends as its smallest site
    // whatever order the unions run in.  Then every head jumps to its root.
    volatile uint32_t* vp = par;
    auto unite = [&](uint32_t u, uint32_t v) {
        uint32_t ra = sfind(vp, u), rb = sfind(vp, v);
        while (ra != rb) {
            const uint32_t hi = max(ra, rb), lo = min(ra, rb);
            const uint32_t old = atomicCAS(par + hi, hi, lo);
            if (old == hi) break;
            ra = sfind(vp, old);
            rb = sfind(vp, lo);
        }
    };
    if (D == 2) {
        // the warp's bonds are packed into a shared list (a scan of the lanes'
        // counts places them) and dealt out evenly, so the warp runs as many
        // union rounds as its mean load needs rather than its busiest lane's
        __shared__ uint16_t plist[NW][D == 2 ? 2 * RPW * 32 : 1];
        const unsigned cnt = __popc(pend);
        unsigned incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned x = __shfl_up_sync(0xFFFFFFFFu, incl, o);
            if (lane >= o) incl += x;
        }
        const unsigned total = __shfl_sync(0xFFFFFFFFu, incl, 31);
        unsigned pos = incl - cnt;
        for (uint32_t bits = pend; bits; bits &= bits - 1) {
            const int bit = __ffs(bits) - 1;  // bit 2k + e: row k, site e
            plist[warp][pos++] = (uint16_t)(lx0 + (bit & 1) + TX * (warp + NW * (bit >> 1)));
        }
        __syncwarp();
        for (unsigned q = lane; q < total; q += 32) {
            const uint32_t u = plist[warp][q];
            unite(u, u + (uint32_t)TX);
        }
    } else {
        for (uint32_t bits = pend; bits; bits &= bits - 1) {
            const int bit = __ffs(bits) - 1;
            const int k = bit / (2 * (D - 1));
            const int e = (bit / (D - 1)) & 1;
            const int mu = 1 + bit % (D - 1);
            const uint32_t u = (uint32_t)(lx0 + e + TX * (warp + NW * k));
            unite(u, u + (mu == 1 ? (uint32_t)TX : (uint32_t)(TX * TY)));
        }
    }
    __syncthreads();
    auto jump = [&](uint32_t l) {
        uint32_t p = vp[l];
        while (true) {
            const uint32_t g = vp[p];
            if (g == p) break;
            p = g;
        }
        vp[l] = p;
    };
    if (D == 2) {
        for (unsigned q = lane; q < nh; q += 32) jump(hlist[warp][q]);
    } else {
#pragma unroll
        for (int k = 0; k < RPW; ++k)
#pragma unroll
            for (int slot = 0; slot < 2; ++slot) {
                const uint32_t l = (heads[D == 2 ? 0 : k] >> (16 * slot)) & 0xFFFFu;
                if (l != 0xFFFFu) jump(l);
            }
    }
    __syncthreads();

    // labels: the natural index of each site's tile root; tile roots marked
    // and counted (bit 2k + e of `mine`)
    uint32_t mine = 0;
    if (ex) {
#pragma unroll
        for (int k = 0; k < RPW; ++k) {
            const int row = warp + NW * k;
            const int ly = row % TY, lz = row / TY;
            if (ly >= ny || lz >= nz) continue;
            const uint32_t l0 = (uint32_t)(lx0 + TX * row);
            uint32_t w[2];
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const uint32_t m = vp[vp[l0 + e]];  // smallest site of the tile cluster
                const uint32_t rx = m % TX, rrow = m / TX;
                const uint32_t ry = rrow % TY, rz = rrow / TY;
                w[e] = ((uint32_t)X0 + rx) + L * (((uint32_t)Y0 + ry) + L * ((uint32_t)Z0 + rz));
                if (m == l0 + e) {
                    w[e] |= kTileRoot;
                    mine |= 1u << (2 * k + e);
                }
            }
            const uint32_t i0 = (uint32_t)(X0 + lx0) + L * ((uint32_t)(Y0 + ly) + L * (uint32_t)(Z0 + lz));
            *reinterpret_cast<uint2*>(a.lab + i0) = make_uint2(w[0], w[1]);
        }
    }
    for (int w = threadIdx.x; w < WORDS; w += blockDim.x) a.face[b * WORDS + w] = fm[w];
    // append the tile roots to the update's list: a warp scan of the counts,
    // one shared atomic per warp, one global atomic per block
    __shared__ unsigned blk_count, blk_base;
    if (threadIdx.x == 0) blk_count = 0;
    __syncthreads();
    const unsigned cnt = __popc(mine);
    unsigned incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned v = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += v;
    }
    unsigned wbase = 0;
    if (lane == 31) wbase = atomicAdd(&blk_count, incl);
    wbase = __shfl_sync(0xFFFFFFFFu, wbase, 31);
    __syncthreads();
    if (threadIdx.x == 0) blk_base = atomicAdd(a.nroots, blk_count);
    __syncthreads();
    unsigned pos = blk_base + wbase + incl - cnt;
    for (uint32_t bits = mine; bits; bits &= bits - 1) {
        const int bit = __ffs(bits) - 1;
        const int k = bit >> 1, e = bit & 1;
        const int row = warp + NW * k;
        const int ly = row % TY, lz = row / TY;
        a.roots[pos++] = (uint32_t)(X0 + lx0 + e) +
                         L * ((uint32_t)(Y0 + ly) + L * (uint32_t)(Z0 + lz));
    }
}

template <int D>
__global__ void __launch_bounds__(256) sw_merge(const SwArgs a)
{
    constexpr int TX = SwTile<D>::TX, TY = SwTile<D>::TY, TZ = SwTile<D>::TZ;
    constexpr int WORDS = SwFace<D>::WORDS;
    const long long total = a.ntiles * WORDS * 32;
    const int L = a.L;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total;
         q += (long long)gridDim.x * blockDim.x) {
        const long long b = q / (WORDS * 32);
        const int bit = (int)(q % (WORDS * 32));
        const uint32_t word = __ldg(a.face + b * WORDS + (bit >> 5));
        if (!((word >> (bit & 31)) & 1u)) continue;
        int X0, Y0, Z0, nx, ny, nz;
        tile_origin<D>(a, b, X0, Y0, Z0, nx, ny, nz);
        int lx, ly, lz, mu;
        if (bit < TY * TZ) {
            mu = 0;
            lx = nx - 1;
            ly = bit % TY;
            lz = bit / TY;
        } else if (bit < TY * TZ + TX * TZ) {
            mu = 1;
            const int k = bit - TY * TZ;
            lx = k % TX;
            ly = ny - 1;
            lz = k / TX;
        } else {
            mu = 2;
            const int k = bit - TY * TZ - TX * TZ;
            lx = k % TX;
            ly = k / TX;
            lz = nz - 1;
        }
        const int x = X0 + lx, y = Y0 + ly, z = Z0 + lz;
        int xn = x, yn = y, zn = z;
        if (mu == 0) xn = x + 1 == L ? 0 : x + 1;
        if (mu == 1) yn = y + 1 == L ? 0 : y + 1;
        if (mu == 2) zn = z + 1 == L ? 0 : z + 1;
        const uint32_t i = (uint32_t)x + (uint32_t)L * ((uint32_t)y + (uint32_t)L * (uint32_t)z);
        const uint32_t j = (uint32_t)xn + (uint32_t)L * ((uint32_t)yn + (uint32_t)L * (uint32_t)zn);
        gunion(a.lab, i, j);
    }
}

// One thread per listed tile root: follow the parents to the cluster root g
// (the smallest site of the cluster) and rewrite the tile root's word as g
// with g's flip bit, the top bit of output 0 of Philox(g, t, replica, 6 << 1).
// Tile roots are each other's parents, so a chase may read a word another
// thread has just rewritten; the new word points at g itself, so the chase
// still ends at g.
__global__ void __launch_bounds__(256) sw_resolve(const SwArgs a)
{
    const uint32_t t = (uint32_t)a.ctrl->t;
    const unsigned n = *a.nroots;
    const unsigned stride = gridDim.x * blockDim.x;
    // two roots per pass with their chases interleaved, so each thread keeps
    // two dependent load chains in flight (a missing second root repeats the
    // first and stores nothing)
    for (unsigned q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += 2 * stride) {
        const bool two = q + stride < n;
        const uint32_t r0 = __ldcg(a.roots + q);
        const uint32_t r1 = two ? __ldcg(a.roots + q + stride) : r0;
        uint32_t p0 = gload(a.lab + r0) & kMask, p1 = gload(a.lab + r1) & kMask;
        while (true) {
            const uint32_t g0 = gload(a.lab + p0) & kMask;
            const uint32_t g1 = gload(a.lab + p1) & kMask;
            if (g0 == p0 && g1 == p1) break;
            p0 = g0;
            p1 = g1;
        }
        const uint4 rnd0 = philox4x32_10(make_uint4(p0, t, a.replica, kSwFlip << 1), a.rk);
        const uint4 rnd1 = philox4x32_10(make_uint4(p1, t, a.replica, kSwFlip << 1), a.rk);
        gstore(a.lab + r0, p0 | kTileRoot | ((rnd0.x >> 31) ? kFlipBit : 0u));
        if (two) gstore(a.lab + r1, p1 | kTileRoot | ((rnd1.x >> 31) ? kFlipBit : 0u));
    }
}

// flip bit of site i's cluster from its label word l: a tile root carries it,
// any other site's parent is its tile root
__device__ __forceinline__ uint32_t root_bit(const SwArgs& a, uint32_t i, uint32_t l)
{
    const uint32_t word = (l & kTileRoot) ? l : __ldg(a.lab + (l & kMask));
    return (word & kFlipBit) ? 1u : 0u;
}

// Every site flips iff its cluster's root drew the flip bit.  A thread takes
// four site pairs (x even, x + 1): eight labels and one 32-bit word of each
// colour array.
// Threads of a block share rows: tq threads per row (the whole block on a
// long row), so the row's coordinates and colour come from one division per
// row rather than per word.
struct RowSplit {
    int tq, rpb, rsub, q0;
    __device__ RowSplit(int Q)
    {
        tq = Q >= (int)blockDim.x ? (int)blockDim.x : Q;
        rpb = (int)blockDim.x / tq;
        rsub = (int)threadIdx.x / tq;
        q0 = (int)threadIdx.x - rsub * tq;
    }
};

__global__ void __launch_bounds__(256) sw_flip(const SwArgs a)
{
    const long long H = a.N >> 1;
    const int L = a.L, W = L >> 1;
    if ((W & 3) == 0) {
        // rows of W colour entries, 4 per word of each colour array; the
        // labels of the 8 sites of word q are the uint4 pair 2q, 2q + 1
        const int Q = W >> 2;
        const long long rows = H / W;
        const RowSplit rs(Q);
        if (rs.rsub >= rs.rpb) return;
        for (long long row = (long long)blockIdx.x * rs.rpb + rs.rsub; row < rows;
             row += (long long)gridDim.x * rs.rpb) {
            const bool c0 = ((row % L + row / L) & 1) != 0;  // colour of the even sites
            for (int qi = rs.q0; qi < Q; qi += rs.tq) {
                const long long q = row * Q + qi;
                const uint4 la = __ldg(reinterpret_cast<const uint4*>(a.lab) + 2 * q);
                const uint4 lb = __ldg(reinterpret_cast<const uint4*>(a.lab) + 2 * q + 1);
                const uint32_t lw[8] = {la.x, la.y, la.z, la.w, lb.x, lb.y, lb.z, lb.w};
                const uint32_t i0 = (uint32_t)(8 * q);
                uint32_t fl0 = 0u, fl1 = 0u;  // flips of colour 0 / colour 1 bytes
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const uint32_t fe = root_bit(a, i0 + 2 * e, lw[2 * e]) << (8 * e);
                    const uint32_t fo = root_bit(a, i0 + 2 * e + 1, lw[2 * e + 1]) << (8 * e);
                    fl0 |= c0 ? fo : fe;
                    fl1 |= c0 ? fe : fo;
                }
                if (fl0) reinterpret_cast<uint32_t*>(a.s[0])[q] ^= fl0;
                if (fl1) reinterpret_cast<uint32_t*>(a.s[1])[q] ^= fl1;
            }
        }
        return;
    }
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < H;
         j += (long long)gridDim.x * blockDim.x) {
        const long long i0 = 2 * j;
        const long long row = i0 / L;
        const int c0 = (int)((row % L + row / L) & 1);
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const uint32_t i = (uint32_t)(i0 + e);
            const int8_t f = (int8_t)root_bit(a, i, __ldg(a.lab + i));
            int8_t* sp = a.s[c0 ^ e] + j;
            *sp = (int8_t)(*sp ^ f);
        }
    }
}

// E and M after an update, streaming 32-bit words (four colour-1 sites) of
// every colour-1 row against the colour-0 rows around it; closes the sweep
// like every other measured pass (series entry, sweep counter + 1).  Needs
// L % 8 == 0.  Every bond touches exactly one colour-1 site, so the bond sum
// is sum over colour-1 sites of 2d - 2 (unlike neighbours).
template <int D>
__global__ void __launch_bounds__(256) sw_measure(const SwArgs a, Partial* partials, double J)
{
    __shared__ long long red[32];
    const int L = a.L, W = L / 2, Q = W / 4;
    const long long rows = (long long)L * (D == 3 ? L : 1);
    const uint32_t* own = reinterpret_cast<const uint32_t*>(a.s[1]);
    const uint32_t* oth = reinterpret_cast<const uint32_t*>(a.s[0]);
    const uint32_t ones = 0x01010101u;
    long long bond = 0, down = 0;
    // one site word: A own, cur the other colour's word at the same place,
    // S its x-shifted neighbour word, nv the y (and z) neighbour words
    auto word = [&](uint32_t A, uint32_t cur, uint32_t S, uint32_t nv) {
        const uint32_t nd = cur + S + nv;
        const uint32_t na = (nd ^ (A * 7u)) - A * (uint32_t)(7 - 2 * D);
        bond += 8 * D - 2 * (long long)__dp4a(na, ones, 0u);
        down += (long long)__dp4a(A, ones, __dp4a(cur, ones, 0u));
    };
    if ((Q & 3) == 0) {
        // 16-byte chunks of four words: 128-bit loads, the x shift inside the
        // chunk, one edge word from the chunk beside it
        const int Q4 = Q >> 2;
        const uint4* own4 = reinterpret_cast<const uint4*>(own);
        const uint4* oth4 = reinterpret_cast<const uint4*>(oth);
        const RowSplit rs(Q4);
        for (long long row = (long long)blockIdx.x * rs.rpb + rs.rsub;
             rs.rsub < rs.rpb && row < rows; row += (long long)gridDim.x * rs.rpb) {
            const int y = (int)(row % L), z = D == 3 ? (int)(row / L) : 0;
            const int p = (y + z + 1) & 1;
            const long long ym = row - y + (y == 0 ? L - 1 : y - 1);
            const long long yp = row - y + (y == L - 1 ? 0 : y + 1);
            const long long zm = D == 3 ? ((z == 0 ? L - 1 : z - 1) * (long long)L + y) : 0;
            const long long zp = D == 3 ? ((z == L - 1 ? 0 : z + 1) * (long long)L + y) : 0;
            for (int c = rs.q0; c < Q4; c += rs.tq) {
                const uint4 A = __ldcs(own4 + row * Q4 + c);
                const uint4 cur = __ldg(oth4 + row * Q4 + c);
                const uint32_t edge =
                    __ldg(oth + row * Q + (p ? (c + 1 == Q4 ? 0 : 4 * c + 4) : (c == 0 ? Q - 1 : 4 * c - 1)));
                uint4 nv = __ldg(oth4 + ym * Q4 + c);
                const uint4 v2 = __ldg(oth4 + yp * Q4 + c);
                nv.x += v2.x;
                nv.y += v2.y;
                nv.z += v2.z;
                nv.w += v2.w;
                if (D == 3) {
                    const uint4 v3 = __ldg(oth4 + zm * Q4 + c);
                    const uint4 v4 = __ldg(oth4 + zp * Q4 + c);
                    nv.x += v3.x + v4.x;
                    nv.y += v3.y + v4.y;
                    nv.z += v3.z + v4.z;
                    nv.w += v3.w + v4.w;
                }
                if (p) {
                    word(A.x, cur.x, __funnelshift_r(cur.x, cur.y, 8), nv.x);
                    word(A.y, cur.y, __funnelshift_r(cur.y, cur.z, 8), nv.y);
                    word(A.z, cur.z, __funnelshift_r(cur.z, cur.w, 8), nv.z);
                    word(A.w, cur.w, __funnelshift_r(cur.w, edge, 8), nv.w);
                } else {
                    word(A.x, cur.x, __funnelshift_l(edge, cur.x, 8), nv.x);
                    word(A.y, cur.y, __funnelshift_l(cur.x, cur.y, 8), nv.y);
                    word(A.z, cur.z, __funnelshift_l(cur.y, cur.z, 8), nv.z);
                    word(A.w, cur.w, __funnelshift_l(cur.z, cur.w, 8), nv.w);
                }
            }
        }
    }
    const RowSplit rs(Q);
    for (long long row = (long long)blockIdx.x * rs.rpb + rs.rsub;
         (Q & 3) != 0 && rs.rsub < rs.rpb && row < rows; row += (long long)gridDim.x * rs.rpb) {
        const int y = (int)(row % L), z = D == 3 ? (int)(row / L) : 0;
        const int p = (y + z + 1) & 1;
        const long long base = row * Q;
        for (int q = rs.q0; q < Q; q += rs.tq) {
            const uint32_t A = __ldcs(own + base + q);
            const uint32_t cur = __ldg(oth + base + q);
            const uint32_t S =
                p ? __funnelshift_r(cur, __ldg(oth + base + (q + 1 == Q ? 0 : q + 1)), 8)
                  : __funnelshift_l(__ldg(oth + base + (q == 0 ? Q - 1 : q - 1)), cur, 8);
            const long long ym = row - y + (y == 0 ? L - 1 : y - 1);
            const long long yp = row - y + (y == L - 1 ? 0 : y + 1);
            uint32_t nv = __ldg(oth + ym * Q + q) + __ldg(oth + yp * Q + q);
            if (D == 3) {
                const long long zm = (z == 0 ? L - 1 : z - 1), zp = (z == L - 1 ? 0 : z + 1);
                nv += __ldg(oth + (zm * L + y) * Q + q) + __ldg(oth + (zp * L + y) * Q + q);
            }
            word(A, cur, S, nv);
        }
    }
    Partial mine;
    mine.i0 = block_sum(bond, red);
    mine.i1 = block_sum(down, red);
    mine.f[0] = mine.f[1] = mine.f[2] = mine.f[3] = 0.0;
    finish_pass(a.ctrl, partials, mine, [&](const Partial& tot) {
        Ctrl* C = a.ctrl;
        const double E = -J * (double)tot.i0;
        const double M = (double)(a.N - 2 * tot.i1);
        C->obs[0] = E;
        C->obs[1] = M;
        C->obs[2] = 0.0;
        C->obs[3] = 0.0;
        const long long k = (long long)C->t - C->series_base;
        if (C->series_E) C->series_E[k] = E;
        if (C->series_absm) C->series_absm[k] = fabs(M) / (double)a.N;
        C->t = C->t + 1;
    });
}

template <int D>
long long tiles_of(int L, int& ntx, int& nty, int& ntz)
{
    ntx = (L + SwTile<D>::TX - 1) / SwTile<D>::TX;
    nty = (L + SwTile<D>::TY - 1) / SwTile<D>::TY;
    ntz = D == 3 ? (L + SwTile<D>::TZ - 1) / SwTile<D>::TZ : 1;
    return (long long)ntx * nty * ntz;
}

template <int D>
cudaError_t sw_update(const SwArgs& a0, cudaStream_t s)
{
    SwArgs a = a0;
    const long long mergers = a.ntiles * SwFace<D>::WORDS * 32;
    cudaError_t e = cudaMemsetAsync(a.nroots, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    sw_local<D><<<(unsigned)a.ntiles, kSwThreads, 0, s>>>(a);
    sw_merge<D><<<grid_for(mergers, 256), 256, 0, s>>>(a);
    sw_resolve<<<grid_for(a.N, 256), 256, 0, s>>>(a);
    sw_flip<<<grid_for((a.N / 2 + 3) / 4, 256), 256, 0, s>>>(a);  // at most one block per row used
    return cudaGetLastError();
}

}  // namespace

size_t sw_workspace_bytes(int d, int L)
{
    int ntx, nty, ntz;
    const size_t N = (size_t)L * L * (d == 3 ? L : 1);
    const long long nt = d == 2 ? tiles_of<2>(L, ntx, nty, ntz) : tiles_of<3>(L, ntx, nty, ntz);
    const size_t words = d == 2 ? SwFace<2>::WORDS : SwFace<3>::WORDS;
    // labels, tile-face bits, the tile-root list and its count
    return align_up(N * 4) + align_up((size_t)nt * words * 4) + align_up(N * 4) + align_up(4);
}

cudaError_t ising_sw_sweeps(const sl_lattice* h, const SweepParams& p, int64_t count,
                            cudaStream_t s)
{
    SwArgs a;
    a.s[0] = (int8_t*)h->spins[0];
    a.s[1] = (int8_t*)h->spins[1];
    a.lab = (uint32_t*)h->ws;
    a.face = (uint32_t*)((char*)h->ws + align_up((size_t)h->N * 4));
    {
        int ntx, nty, ntz;
        const long long nt = h->d == 2 ? tiles_of<2>(h->L, ntx, nty, ntz)
                                       : tiles_of<3>(h->L, ntx, nty, ntz);
        const size_t words = h->d == 2 ? SwFace<2>::WORDS : SwFace<3>::WORDS;
        char* after_face = (char*)a.face + align_up((size_t)nt * words * 4);
        a.roots = (uint32_t*)after_face;
        a.nroots = (unsigned*)(after_face + align_up((size_t)h->N * 4));
    }
    a.L = h->L;
    a.N = h->N;
    a.ntiles = h->d == 2 ? tiles_of<2>(h->L, a.ntx, a.nty, a.ntz)
                         : tiles_of<3>(h->L, a.ntx, a.nty, a.ntz);
    a.thr = p.tab.sw_thr;
    a.never = p.tab.sw_never;
    a.anti = h->J < 0.0;
    a.replica = h->replica;
    a.rk = p.rk;
    a.ctrl = h->ctrl;
    for (int64_t k = 0; k < count; ++k) {
        cudaError_t e = h->d == 2 ? sw_update<2>(a, s) : sw_update<3>(a, s);
        if (e == cudaSuccess) {
            if (h->L % 8 == 0) {
                const long long items = (long long)h->L * (h->d == 3 ? h->L : 1) * (h->L / 8);
                if (h->d == 2) sw_measure<2><<<grid_for(items, 256), 256, 0, s>>>(a, h->partials, h->J);
                else sw_measure<3><<<grid_for(items, 256), 256, 0, s>>>(a, h->partials, h->J);
                e = cudaGetLastError();
            } else {
                e = ising_i8_measure_advance(h, s);
            }
        }
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace spinmc
