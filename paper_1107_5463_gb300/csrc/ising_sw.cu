// Swendsen-Wang cluster updates of the Ising model on byte storage
// (Weigel & Yavors'kii 2011, Section 3: activate bonds between like spins with
// p = 1 - exp(-2 beta J), build the clusters joined by active bonds, flip each
// cluster with probability 1/2; cluster identification in tiles first, then
// amalgamation of the tiles through a union-and-find structure).
//
// One update is four kernels plus the measurement that closes every sweep:
//   sw_local    one CTA per tile (64 x 32 sites in 2D, 32 x 16 x 16 in 3D):
//               loads the tile's spins and a one-site halo on its +x/+y/+z
//               faces into shared memory, draws the bond uniforms, unites the
//               sites joined by active bonds inside the tile with a
//               shared-memory union-find (roots hooked smaller-index-wins by
//               atomicCAS), writes every site's label (the natural index of
//               its tile-local root, the smallest site of its tile cluster)
//               and one bit per active bond that leaves the tile;
//   sw_merge    one thread per tile-face bond: unites the two labels of each
//               active face bond in global memory (same hooking rule, finds
//               with pointer jumping); afterwards the root of every cluster
//               is its smallest site;
//   sw_resolve  every site finds its root; roots draw their flip bit and keep
//               it in bit 31 of their own label;
//   sw_flip     every site reads its root's bit and flips.
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
constexpr uint32_t kMask = 0x7FFFFFFFu;
constexpr int kSwThreads = 512;

template <int D>
struct SwTile;
template <>
struct SwTile<2> {
    static constexpr int TX = 64, TY = 32, TZ = 1;
};
template <>
struct SwTile<3> {
    static constexpr int TX = 32, TY = 16, TZ = 16;
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
using bref = cuda::atomic_ref<uint32_t, cuda::thread_scope_block>;

__device__ __forceinline__ uint32_t gload(uint32_t* p)
{
    return gref(*p).load(cuda::memory_order_relaxed);
}

__device__ __forceinline__ void gstore(uint32_t* p, uint32_t v)
{
    gref(*p).store(v, cuda::memory_order_relaxed);
}

// shared-memory union-find over tile-local indices; parents only ever point
// to smaller indices
__device__ __forceinline__ uint32_t sfind(uint32_t* par, uint32_t x)
{
    while (true) {
        const uint32_t p = bref(par[x]).load(cuda::memory_order_relaxed);
        if (p == x) return x;
        x = p;
    }
}

__device__ __forceinline__ void sunion(uint32_t* par, uint32_t a, uint32_t b)
{
    a = sfind(par, a);
    b = sfind(par, b);
    while (a != b) {
        if (a < b) {
            const uint32_t t = a;
            a = b;
            b = t;
        }
        uint32_t expect = a;
        if (bref(par[a]).compare_exchange_strong(expect, b, cuda::memory_order_relaxed)) return;
        a = sfind(par, expect);
        b = sfind(par, b);
    }
}

// global find with pointer jumping: every store writes an ancestor into a
// non-root entry, so concurrent finds and hooks stay consistent
__device__ __forceinline__ uint32_t gfind(uint32_t* lab, uint32_t x)
{
    uint32_t p = gload(lab + x);
    if (p == x) return x;
    uint32_t prev = x;
    while (true) {
        const uint32_t g = gload(lab + p);
        if (g == p) return p;
        gstore(lab + prev, g);
        prev = p;
        p = g;
    }
}

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
        uint32_t expect = a;
        if (gref(lab[a]).compare_exchange_strong(expect, b, cuda::memory_order_relaxed)) return;
        a = gfind(lab, expect);
        b = gfind(lab, b);
    }
}

__device__ __forceinline__ int8_t spin_at(const SwArgs& a, int x, int y, int z)
{
    const long long i = x + (long long)a.L * (y + (long long)a.L * z);
    return a.s[(x + y + z) & 1][i >> 1];
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

template <int D>
__global__ void __launch_bounds__(kSwThreads) sw_local(const SwArgs a)
{
    constexpr int TX = SwTile<D>::TX, TY = SwTile<D>::TY, TZ = SwTile<D>::TZ;
    constexpr int NS = TX * TY * TZ;
    constexpr int HX = TX + 2, HY = TY + 1, HZ = D == 3 ? TZ + 1 : 1;  // halo-padded spin tile
    constexpr int WORDS = SwFace<D>::WORDS;
    __shared__ uint32_t par[NS];
    __shared__ uint8_t sp[HZ * HY * HX];
    __shared__ uint32_t fm[WORDS];

    const long long b = blockIdx.x;
    int X0, Y0, Z0, nx, ny, nz;
    tile_origin<D>(a, b, X0, Y0, Z0, nx, ny, nz);
    const int L = a.L;
    const uint32_t t = (uint32_t)a.ctrl->t;

    for (int l = threadIdx.x; l < NS; l += blockDim.x) par[l] = (uint32_t)l;
    for (int w = threadIdx.x; w < WORDS; w += blockDim.x) fm[w] = 0u;
    // the tile's spins plus the +x column, +y row and +z plane (no edges)
    for (int q = threadIdx.x; q < HZ * HY * (TX / 2 + 1); q += blockDim.x) {
        const int kx = q % (TX / 2 + 1);
        const int ly = (q / (TX / 2 + 1)) % HY;
        const int lz = q / ((TX / 2 + 1) * HY);
        if (ly > ny || lz > (D == 3 ? nz : 0)) continue;
        const int hy = ly == ny, hz = D == 3 && lz == nz;
        const int y = Y0 + ly == L ? 0 : Y0 + ly;
        const int z = D == 3 ? (Z0 + lz == L ? 0 : Z0 + lz) : 0;
        if (kx < nx / 2) {
            if (hy + hz > 1) continue;
            const int x = X0 + 2 * kx;
            sp[(lz * HY + ly) * HX + 2 * kx] = (uint8_t)spin_at(a, x, y, z);
            sp[(lz * HY + ly) * HX + 2 * kx + 1] = (uint8_t)spin_at(a, x + 1, y, z);
        } else if (kx == TX / 2) {
            if (hy || hz) continue;
            const int x = X0 + nx == L ? 0 : X0 + nx;
            sp[(lz * HY + ly) * HX + nx] = (uint8_t)spin_at(a, x, y, z);
        }
    }
    __syncthreads();

    // bond activation; unite inside the tile, record bonds leaving it
    for (int p = threadIdx.x; p < NS / 2; p += blockDim.x) {
        const int lx0 = 2 * (p % (TX / 2));
        const int ly = (p / (TX / 2)) % TY;
        const int lz = p / ((TX / 2) * TY);
        if (lx0 >= nx || ly >= ny || lz >= nz) continue;
        const long long i0 = (X0 + lx0) + (long long)L * ((Y0 + ly) + (long long)L * (Z0 + lz));
        uint32_t u[2][3];
        if (D == 2) {
            const uint4 r = philox4x32_10(
                make_uint4((uint32_t)(i0 >> 1), t, a.replica, kSwBond << 1), a.rk);
            u[0][0] = r.x;
            u[0][1] = r.y;
            u[1][0] = r.z;
            u[1][1] = r.w;
            u[0][2] = u[1][2] = 0u;
        } else {
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const uint4 r = philox4x32_10(
                    make_uint4((uint32_t)(i0 + e), t, a.replica, kSwBond << 1), a.rk);
                u[e][0] = r.x;
                u[e][1] = r.y;
                u[e][2] = r.z;
            }
        }
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int lx = lx0 + e;
            const int so = (lz * HY + ly) * HX + lx;
            const uint8_t own = sp[so];
            const uint32_t l = (uint32_t)(lx + TX * (ly + TY * lz));
#pragma unroll
            for (int mu = 0; mu < D; ++mu) {
                const int nb_off = mu == 0 ? 1 : (mu == 1 ? HX : HX * HY);
                const uint8_t nb = sp[so + nb_off];
                const int sat = (int)(own ^ nb) == a.anti;
                if (!sat || a.never || u[e][mu] > a.thr) continue;
                const int crosses = mu == 0 ? lx + 1 == nx : (mu == 1 ? ly + 1 == ny : lz + 1 == nz);
                if (crosses) {
                    const int bit = mu == 0 ? ly + TY * lz
                                            : (mu == 1 ? TY * TZ + lx + TX * lz
                                                       : TY * TZ + TX * TZ + lx + TX * ly);
                    atomicOr(&fm[bit >> 5], 1u << (bit & 31));
                } else {
                    const uint32_t stride = mu == 0 ? 1u : (mu == 1 ? (uint32_t)TX : (uint32_t)(TX * TY));
                    sunion(par, l, l + stride);
                }
            }
        }
    }
    __syncthreads();
    for (int l = threadIdx.x; l < NS; l += blockDim.x) par[l] = sfind(par, (uint32_t)l);
    __syncthreads();

    // labels: the natural index of each site's tile root
    for (int l = threadIdx.x; l < NS; l += blockDim.x) {
        const int lx = l % TX, ly = (l / TX) % TY, lz = l / (TX * TY);
        if (lx >= nx || ly >= ny || lz >= nz) continue;
        const uint32_t r = par[l];
        const int rx = (int)(r % TX), ry = (int)((r / TX) % TY), rz = (int)(r / (TX * TY));
        const long long i = (X0 + lx) + (long long)L * ((Y0 + ly) + (long long)L * (Z0 + lz));
        const long long ri = (X0 + rx) + (long long)L * ((Y0 + ry) + (long long)L * (Z0 + rz));
        a.lab[i] = (uint32_t)ri;
    }
    for (int w = threadIdx.x; w < WORDS; w += blockDim.x) a.face[b * WORDS + w] = fm[w];
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
        const uint32_t i = (uint32_t)(x + (long long)L * (y + (long long)L * z));
        const uint32_t j = (uint32_t)(xn + (long long)L * (yn + (long long)L * zn));
        gunion(a.lab, i, j);
    }
}

__global__ void __launch_bounds__(256) sw_resolve(const SwArgs a)
{
    const uint32_t t = (uint32_t)a.ctrl->t;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < a.N;
         q += (long long)gridDim.x * blockDim.x) {
        const uint32_t i = (uint32_t)q;
        const uint32_t p0 = gload(a.lab + i) & kMask;
        if (p0 == i) {
            const uint4 r = philox4x32_10(make_uint4(i, t, a.replica, kSwFlip << 1), a.rk);
            gstore(a.lab + i, i | (r.x & 0x80000000u));
            continue;
        }
        uint32_t p = p0;
        while (true) {
            const uint32_t g = gload(a.lab + p) & kMask;
            if (g == p) break;
            p = g;
        }
        if (p != p0) gstore(a.lab + i, p);
    }
}

__global__ void __launch_bounds__(256) sw_flip(const SwArgs a)
{
    const long long H = a.N >> 1;
    const int L = a.L;
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < H;
         j += (long long)gridDim.x * blockDim.x) {
        const long long i0 = 2 * j;
        const long long row = i0 / L;  // y + L z
        const int c0 = (int)((row % L + row / L) & 1);
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const uint32_t i = (uint32_t)(i0 + e);
            const uint32_t l = gload(a.lab + i);
            uint32_t r = l & kMask, root_word = l;
            if (r != i) {
                while (true) {
                    root_word = gload(a.lab + r);
                    const uint32_t g = root_word & kMask;
                    if (g == r) break;
                    r = g;
                }
            }
            const int8_t f = (int8_t)(root_word >> 31);
            int8_t* sp = a.s[c0 ^ e] + j;
            *sp = (int8_t)(*sp ^ f);
        }
    }
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
    sw_local<D><<<(unsigned)a.ntiles, kSwThreads, 0, s>>>(a);
    sw_merge<D><<<grid_for(mergers, 256), 256, 0, s>>>(a);
    sw_resolve<<<grid_for(a.N, 256), 256, 0, s>>>(a);
    sw_flip<<<grid_for(a.N / 2, 256), 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

size_t sw_workspace_bytes(int d, int L)
{
    int ntx, nty, ntz;
    const size_t N = (size_t)L * L * (d == 3 ? L : 1);
    const long long nt = d == 2 ? tiles_of<2>(L, ntx, nty, ntz) : tiles_of<3>(L, ntx, nty, ntz);
    const size_t words = d == 2 ? SwFace<2>::WORDS : SwFace<3>::WORDS;
    return align_up(N * 4) + align_up((size_t)nt * words * 4);
}

cudaError_t ising_sw_sweeps(const sl_lattice* h, const SweepParams& p, int64_t count,
                            cudaStream_t s)
{
    SwArgs a;
    a.s[0] = (int8_t*)h->spins[0];
    a.s[1] = (int8_t*)h->spins[1];
    a.lab = (uint32_t*)h->ws;
    a.face = (uint32_t*)((char*)h->ws + align_up((size_t)h->N * 4));
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
        if (e == cudaSuccess) e = ising_i8_measure_advance(h, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace spinmc
