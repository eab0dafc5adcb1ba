// Ising model (n = 1) with one byte per site, checkerboard
// Metropolis (Weigel & Yavors'kii 2011, Section 2, Eq. 1 and Eq. 2).
//
// Storage: two colour arrays S[c][j], j = i >> 1, each N/2 bytes holding 0
// for spin +1 and 1 for spin -1 (so neighbour counts are plain byte sums and
// flips a byte XOR); sl_get_spins / sl_set_spins convert to +-1.  Couplings
// are stored per colour and direction as 0 (+1), 1 (-1) or 2 (0).  A row of
// the lattice (fixed y, z) holds W = L/2 sites of each colour, contiguous in
// S[c]; the colour-c site at colour column k of row (y, z) sits at
// x = 2k + p with p = (y + z + c) & 1, so its -x / +x neighbours are the
// other colour's columns k-1 / k (p = 0) or k / k+1 (p = 1).
//
// Acceptance: class g of a site (number of unsatisfied bonds for +-1
// couplings, 2d - s_i h_i sign(J) when couplings may be zero) and the count
// q(u) of classes whose threshold lies below the site's 32-bit uniform u;
// the move is accepted iff g >= q(u), which equals u <= T[g] for g < ncmp and
// "always" for the classes with dE <= 0 (thresholds are non-decreasing in g).
//
// Two kernels compute the same decisions bit for bit:
//   i8_generic  one thread per Philox group of 4 sites, scalar, any even L and
//               any couplings; also the standalone measurement;
//   i8_stream   one thread per 16-byte column chunk marching through R rows
//               with a rolling window of the other colour's rows in registers,
//               128-bit loads and stores, SIMD-within-a-word neighbour
//               counts; needs W % 16 == 0 and +-1 couplings.
//
// Slabs (a lattice split along its slowest axis, y in 2D or z in 3D): the
// kernels see Lz local planes with a halo plane before the first and after
// the last in each colour array (no wrap along that axis), add the slab's
// global plane offset to every Philox group (gofs colour entries) and its
// parity to every colour, so each site makes the decisions it makes in the
// whole lattice.
#include "internal.h"

namespace spinmc {
namespace {

struct I8Args {
    int8_t* own;
    const int8_t* oth;
    const int8_t* Jown[3];
    const int8_t* Joth[3];
    int d, L, W, c, R;
    long long H, N;
    uint32_t replica;
    IsingTable tab;
    RoundKeys rk;
    Ctrl* ctrl;
    Partial* partials;
    double J;
    int measure;  // accumulate E and M and finish the pass
    int update;   // 0: standalone measurement (no moves, no sweep advance)
    int advance;  // a measurement that closes a sweep: write the series, t + 1
    int defer;    // i8_stream: add the block totals into the accumulator for i8_finish_kernel
    int Lz;       // planes along the slowest axis (L, or the slab's planes)
    int wrap;     // 1: periodic along the slowest axis; 0: halo planes at -1 and Lz
    int par;      // parity of the first plane's global index
    long long gofs;  // global colour index of local colour entry 0
};

__device__ __forceinline__ void i8_finish(const I8Args& a, const Partial& tot)
{
    Ctrl* C = a.ctrl;
    const double E = -a.J * (double)tot.i0;
    const double M = (double)(a.N - 2 * tot.i1);
    C->obs[0] = E;
    C->obs[1] = M;
    C->obs[2] = 0.0;
    C->obs[3] = 0.0;
    if (a.update || a.advance) {
        const long long k = (long long)C->t - C->series_base;
        if (C->series_E) C->series_E[k] = E;
        // a slab records its own M (summed over slabs, |M| / N is |m|)
        if (C->series_absm) C->series_absm[k] = a.wrap ? fabs(M) / (double)a.N : M;
        C->t = C->t + 1;
    }
}

__device__ __forceinline__ int spin_value(int8_t b) { return 1 - 2 * (int)b; }
__device__ __forceinline__ int bond_value(int8_t b) { return b == 2 ? 0 : 1 - 2 * (int)b; }

__device__ __forceinline__ int q_of(uint32_t u, const IsingTable& tab)
{
    int q = 0;
#pragma unroll
    for (int k = 0; k < 6; ++k)
        if (k < tab.ncmp) q += (u > tab.thr[k]) ? 1 : 0;
    return q;
}

// ----------------------------------------------------------- generic ----

template <int D>
__global__ void __launch_bounds__(256) i8_generic(const I8Args a)
{
    __shared__ long long red[32];
    const uint32_t t = (uint32_t)a.ctrl->t;
    const long long ngroups = (a.H + 3) >> 2;
    const int L = a.L;
    long long bond = 0, down = 0;
    for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < ngroups;
         g += (long long)gridDim.x * blockDim.x) {
        uint32_t rr[4] = {0u, 0u, 0u, 0u};
        if (a.update) {
            const uint4 r = philox4x32_10(
                make_uint4((uint32_t)(g + (a.gofs >> 2)), t, a.replica,
                           (kSweep << 1) | (uint32_t)a.c), a.rk);
            rr[0] = r.x; rr[1] = r.y; rr[2] = r.z; rr[3] = r.w;
        }
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const long long j = 4 * g + b;
            if (j >= a.H) break;
            const long long i0 = 2 * j;
            int x = (int)(i0 % L);
            const long long rrow = i0 / L;
            const int y = (int)(rrow % L);
            const int z = (int)(rrow / L);
            x += (a.c + y + z + a.par) & 1;
            int hs = 0;
#pragma unroll
            for (int mu = 0; mu < D; ++mu) {
                int cm[3] = {x, y, z}, cp[3] = {x, y, z};
                // the slowest axis of a slab ends in halo planes -1 and Lz
                const bool wr = mu != D - 1 || a.wrap;
                const int ext = mu == D - 1 ? a.Lz : L;
                cm[mu] = cm[mu] == 0 ? (wr ? ext - 1 : -1) : cm[mu] - 1;
                cp[mu] = cp[mu] == ext - 1 ? (wr ? 0 : ext) : cp[mu] + 1;
                const long long nm =
                    (cm[0] + (long long)L * (cm[1] + (long long)L * cm[2])) >> 1;
                const long long np =
                    (cp[0] + (long long)L * (cp[1] + (long long)L * cp[2])) >> 1;
                const int jm = a.Jown[0] ? bond_value(a.Joth[mu][nm]) : 1;
                const int jp = a.Jown[0] ? bond_value(a.Jown[mu][j]) : 1;
                hs += jm * spin_value(a.oth[nm]) + jp * spin_value(a.oth[np]);
            }
            int s = spin_value(a.own[j]);
            int sh = s * hs;
            if (a.update && a.tab.heatbath) {
                // heat-bath: the new spin from its conditional law alone
                const int snew = rr[b] <= a.tab.hb[hs + 2 * D] ? 1 : -1;
                if (snew != s) a.own[j] = (int8_t)(snew < 0);
                s = snew;
                sh = s * hs;
            } else if (a.update) {
                const int e = a.tab.sigma_neg ? -sh : sh;
                const int gcls = a.tab.scheme ? (2 * D - e) : ((2 * D - e) >> 1);
                if (gcls >= q_of(rr[b], a.tab)) {
                    s = -s;
                    sh = -sh;
                    a.own[j] = (int8_t)(s < 0);
                }
            }
            if (a.measure) {
                bond += sh;
                down += (s < 0) + (a.oth[j] != 0);
            }
        }
    }
    if (!a.measure) return;
    Partial mine;
    mine.i0 = block_sum(bond, red);
    mine.i1 = block_sum(down, red);
    mine.f[0] = mine.f[1] = mine.f[2] = mine.f[3] = 0.0;
    finish_pass(a.ctrl, a.partials, mine, [&](const Partial& tot) { i8_finish(a, tot); });
}

// ---------------------------------------------------------- streaming ----

__device__ __forceinline__ uint4 ld_rows(const int8_t* p)
{
    return __ldg(reinterpret_cast<const uint4*>(p));
}

// The other colour's row shifted by one column so that byte b holds the
// -x (p = 0) or +x (p = 1) neighbour of own byte b; `edge` is the byte that
// enters from the adjacent chunk.
__device__ __forceinline__ uint4 shift_row(uint4 v, uint32_t edge, int p)
{
    uint4 s;
    if (p == 0) {
        s.x = __funnelshift_l(edge << 24, v.x, 8);
        s.y = __funnelshift_l(v.x, v.y, 8);
        s.z = __funnelshift_l(v.y, v.z, 8);
        s.w = __funnelshift_l(v.z, v.w, 8);
    } else {
        s.x = __funnelshift_r(v.x, v.y, 8);
        s.y = __funnelshift_r(v.y, v.z, 8);
        s.z = __funnelshift_r(v.z, v.w, 8);
        s.w = __funnelshift_r(v.w, edge, 8);
    }
    return s;
}

__device__ __forceinline__ uint32_t w_of(const uint4& v, int k)
{
    return k == 0 ? v.x : k == 1 ? v.y : k == 2 ? v.z : v.w;
}

// Per byte: 0x80 minus the number of thresholds below u, i.e. 0x80 - q(u)
// for the four sites of one Philox block (byte b <- output b).
template <int NCMP>
__device__ __forceinline__ uint32_t q_bias(const uint4& r, const IsingTable& tab)
{
    uint32_t acc = 0x80808080u;
    const uint32_t u[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
        for (int k = 0; k < NCMP; ++k) acc -= (u[b] > tab.thr[k]) ? (1u << (8 * b)) : 0u;
    return acc;
}

// MEAS: the measuring (colour-1) pass; the other pass is compiled without the
// counters, which keeps its register count, and so its occupancy, lower.
// SLAB: a slab of a split lattice (halo planes, global offsets); a whole
// lattice compiles without them.
template <int D, int BONDS, int JNEG, int HB, bool MEAS, bool SLAB = false>
__global__ void __launch_bounds__(128) i8_stream(const I8Args a)
{
    __shared__ long long red[32];
    __shared__ uint32_t s_hb[16];  // heat-bath thresholds by h + 2d
    if (HB) {
        if (threadIdx.x < 13) s_hb[threadIdx.x] = a.tab.hb[threadIdx.x];
        __syncthreads();
    }
    const uint32_t t = (uint32_t)a.ctrl->t;
    const int W = a.W, L = a.L, R = a.R, Lz = SLAB ? a.Lz : a.L;
    const int W16 = W >> 4;
    const long long nseg = Lz / R;
    const int par = SLAB ? a.par : 0;
    const long long gofs = SLAB ? a.gofs : 0;
    // neighbouring plane along the slowest axis: periodic, or a halo plane
    auto zprev = [&](int m) { return m == 0 ? (SLAB ? -1 : Lz - 1) : m - 1; };
    auto znext = [&](int m) { return m == Lz - 1 ? (SLAB ? Lz : 0) : m + 1; };
    const long long nitems = (long long)W16 * (D == 3 ? L : 1) * nseg;
    const uint32_t ctr_w = (kSweep << 1) | (uint32_t)a.c;
    const uint32_t two_d = 0x01010101u * (uint32_t)(2 * D);
    const uint32_t ones = 0x01010101u;
    // Counts of the measuring pass.  2D: 32-bit per-thread counters across
    // all of a thread's items (at most a few hundred items of 16 R sites
    // reach one thread at the grid cap) and an item count; 3D: 32-bit
    // counters per item added into 64-bit totals, and a site count.  Each
    // form measured 1.5-2% faster than the other in its dimension.
    uint32_t t_na = 0, t_flip = 0, t_flipna = 0, t_down = 0, nitem = 0;
    unsigned long long w_na = 0, w_flip = 0, w_flipna = 0, w_down = 0, w_site = 0;

    for (long long it = (long long)blockIdx.x * blockDim.x + threadIdx.x; it < nitems;
         it += (long long)gridDim.x * blockDim.x) {
        const int cx = (int)(it % W16);
        const long long rest = it / W16;
        const int y3 = D == 3 ? (int)(rest % L) : 0;
        const int seg = D == 3 ? (int)(rest / L) : (int)rest;
        const int k0 = cx << 4;
        const int m0 = seg * R;
        auto off = [&](int yy, int zz) -> long long { return ((long long)zz * L + yy) * W; };
        auto moff = [&](int m) -> long long { return D == 3 ? off(y3, m) : off(m, 0); };
        const int mprev = zprev(m0);
        uint4 prev = ld_rows(a.oth + moff(mprev) + k0);
        uint4 cur = ld_rows(a.oth + moff(m0) + k0);
        uint4 jprev = make_uint4(0, 0, 0, 0);
        if (BONDS) jprev = ld_rows(a.Joth[D == 3 ? 2 : 1] + moff(mprev) + k0);
        uint32_t l_na = 0, l_flip = 0, l_flipna = 0, l_down = 0;
        uint32_t& i_na = D == 2 ? t_na : l_na;
        uint32_t& i_flip = D == 2 ? t_flip : l_flip;
        uint32_t& i_flipna = D == 2 ? t_flipna : l_flipna;
        uint32_t& i_down = D == 2 ? t_down : l_down;
        // Metropolis measurement: per-byte counts packed in words (integer
        // adds, no multiplier), folded into the totals every 8 rows, where a
        // byte holds at most 8 x 4 x 2d <= 192
        uint32_t p_na = 0, p_flip = 0, p_down = 0;
        // software pipeline: row m's own chunk, its edge byte and row m+1 of
        // the other colour are loaded one iteration ahead
        auto row_of = [&](int m, int& yy, int& zz) {
            yy = D == 3 ? y3 : m;
            zz = D == 3 ? m : 0;
        };
        auto edge_idx = [&](int p) {
            return p ? (k0 + 16 == W ? 0 : k0 + 16) : (k0 == 0 ? W - 1 : k0 - 1);
        };
        int yy0, zz0;
        row_of(m0, yy0, zz0);
        uint4 next = ld_rows(a.oth + moff(znext(m0)) + k0);
        uint4 A_nx = *reinterpret_cast<const uint4*>(a.own + off(yy0, zz0) + k0);
        uint32_t edge_nx =
            (uint8_t)a.oth[off(yy0, zz0) + edge_idx((yy0 + zz0 + a.c + par) & 1)];
        // 3D: rows y -/+ 1 of the current plane, also one iteration ahead
        const int y_m = y3 == 0 ? L - 1 : y3 - 1, y_p = y3 == L - 1 ? 0 : y3 + 1;
        uint4 ym_nx = make_uint4(0, 0, 0, 0), yp_nx = ym_nx;
        if (D == 3) {
            ym_nx = ld_rows(a.oth + off(y_m, zz0) + k0);
            yp_nx = ld_rows(a.oth + off(y_p, zz0) + k0);
        }
        // two rows per loop pass, so their Philox blocks interleave (not for
        // the 3D measuring pass, whose extra registers cost more than the
        // overlap gains)
#pragma unroll ((D == 2 || !MEAS) ? 2 : 1)
        for (int r = 0; r < R; ++r) {
            const int m = m0 + r;
            int yy, zz;
            row_of(m, yy, zz);
            const int p = (yy + zz + a.c + par) & 1;
            const long long ro = off(yy, zz);
            const int eidx = edge_idx(p);
            const uint4 A = A_nx;
            const uint32_t edge = edge_nx;
            const uint4 nxt = next;
            const uint4 ym = ym_nx, yp = yp_nx;
            if (r + 1 < R) {
                const int m1 = m + 1;
                const int m2 = znext(m1);
                int y1, z1;
                row_of(m1, y1, z1);
                next = ld_rows(a.oth + moff(m2) + k0);
                A_nx = *reinterpret_cast<const uint4*>(a.own + off(y1, z1) + k0);
                edge_nx = (uint8_t)a.oth[off(y1, z1) + edge_idx((y1 + z1 + a.c + par) & 1)];
                if (D == 3) {
                    ym_nx = ld_rows(a.oth + off(y_m, z1) + k0);
                    yp_nx = ld_rows(a.oth + off(y_p, z1) + k0);
                }
            }
            const uint4 S = shift_row(cur, edge, p);
            // couplings (0 = +1, 1 = -1): +x/+y/+z from own forward bonds; -x
            // from the other colour's x bonds (shifted when the -x neighbour is
            // column k-1); -y / -z from the other colour's rows behind.
            uint4 jx_own, jx_oth, jy_own, jy_oth, jz_own, jz_oth, jnext;
            if (BONDS) {
                jx_own = ld_rows(a.Jown[0] + ro + k0);
                const uint4 jo = ld_rows(a.Joth[0] + ro + k0);
                jx_oth = p == 0 ? shift_row(jo, (uint8_t)a.Joth[0][ro + eidx], 0) : jo;
                jy_own = ld_rows(a.Jown[1] + ro + k0);
                if (D == 2) {
                    jy_oth = jprev;
                    jnext = ld_rows(a.Joth[1] + ro + k0);
                } else {
                    const int ym_ = yy == 0 ? L - 1 : yy - 1;
                    jy_oth = ld_rows(a.Joth[1] + off(ym_, zz) + k0);
                    jz_own = ld_rows(a.Jown[2] + ro + k0);
                    jz_oth = jprev;
                    jnext = ld_rows(a.Joth[2] + ro + k0);
                }
            }
            const uint32_t g0 = (uint32_t)((ro + gofs + k0) >> 2);
            uint4 Anew;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const uint32_t av = w_of(A, k);
                const uint32_t nxm = p ? w_of(cur, k) : w_of(S, k);
                const uint32_t nxp = p ? w_of(S, k) : w_of(cur, k);
                uint32_t na;  // unsatisfied bonds per byte (ferromagnetic sense)
                if (HB) {
                    // heat-bath: na = neighbours with Jb_k s_k = -1, so h = 2d - 2 na;
                    // the new spin is down iff u > hb[h + 2d]
                    if (!BONDS) {
                        na = nxm + nxp + w_of(prev, k) + w_of(nxt, k);
                        if (D == 3) na += w_of(ym, k) + w_of(yp, k);
                    } else {
                        na = (nxm ^ w_of(jx_oth, k)) + (nxp ^ w_of(jx_own, k));
                        if (D == 2) {
                            na += (w_of(prev, k) ^ w_of(jy_oth, k)) + (w_of(nxt, k) ^ w_of(jy_own, k));
                        } else {
                            na += (w_of(ym, k) ^ w_of(jy_oth, k)) + (w_of(yp, k) ^ w_of(jy_own, k)) +
                                  (w_of(prev, k) ^ w_of(jz_oth, k)) + (w_of(nxt, k) ^ w_of(jz_own, k));
                        }
                    }
                    const uint4 rnd = philox4x32_10(make_uint4(g0 + k, t, a.replica, ctr_w), a.rk);
                    const uint32_t u[4] = {rnd.x, rnd.y, rnd.z, rnd.w};
                    uint32_t down_new = 0;
#pragma unroll
                    for (int b = 0; b < 4; ++b) {
                        const uint32_t nb = (na >> (8 * b)) & 0xFFu;
                        if (u[b] > s_hb[4 * D - 2 * nb]) down_new |= 1u << (8 * b);
                    }
                    // after the update na' = na + new_down (2d - 2 na), as for a flip
                    if (k == 0) Anew.x = down_new;
                    else if (k == 1) Anew.y = down_new;
                    else if (k == 2) Anew.z = down_new;
                    else Anew.w = down_new;
                    if (MEAS) {
                        i_na = __dp4a(na, ones, i_na);
                        i_flip = __dp4a(down_new, ones, i_flip);
                        i_flipna = __dp4a(down_new, na, i_flipna);
                        i_down = __dp4a(down_new, ones, __dp4a(w_of(cur, k), ones, i_down));
                    }
                    continue;
                }
                if (!BONDS) {
                    uint32_t nd = nxm + nxp + w_of(prev, k) + w_of(nxt, k);
                    if (D == 3) nd += w_of(ym, k) + w_of(yp, k);
                    // own spin down: na = 2d - nd = (nd ^ 7) - (7 - 2d)
                    na = (nd ^ (av * 7u)) - av * (uint32_t)(7 - 2 * D);
                } else {
                    na = (av ^ nxm ^ w_of(jx_oth, k)) + (av ^ nxp ^ w_of(jx_own, k));
                    if (D == 2) {
                        na += (av ^ w_of(prev, k) ^ w_of(jy_oth, k)) +
                              (av ^ w_of(nxt, k) ^ w_of(jy_own, k));
                    } else {
                        na += (av ^ w_of(ym, k) ^ w_of(jy_oth, k)) +
                              (av ^ w_of(yp, k) ^ w_of(jy_own, k)) +
                              (av ^ w_of(prev, k) ^ w_of(jz_oth, k)) +
                              (av ^ w_of(nxt, k) ^ w_of(jz_own, k));
                    }
                }
                if (JNEG) na = two_d - na;
                const uint4 rnd = philox4x32_10(make_uint4(g0 + k, t, a.replica, ctr_w), a.rk);
                // byte bit 7 set iff na >= q(u): accept
                const uint32_t flip = ((na + q_bias<D>(rnd, a.tab)) & 0x80808080u) >> 7;
                const uint32_t an = av ^ flip;
                if (k == 0) Anew.x = an;
                else if (k == 1) Anew.y = an;
                else if (k == 2) Anew.z = an;
                else Anew.w = an;
                if (MEAS) {
                    p_na += na;
                    p_flip += flip;
                    p_down += an + w_of(cur, k);
                    i_flipna = __dp4a(flip, na, i_flipna);
                }
            }
            if (!HB && MEAS && ((r & 7) == 7 || r + 1 == R)) {
                i_na = __dp4a(p_na, ones, i_na);
                i_flip = __dp4a(p_flip, ones, i_flip);
                i_down = __dp4a(p_down, ones, i_down);
                p_na = p_flip = p_down = 0;
            }
            *reinterpret_cast<uint4*>(a.own + ro + k0) = Anew;
            prev = cur;
            cur = nxt;
            if (BONDS) jprev = jnext;
        }
        if (MEAS) {
            if (D == 3) {
                w_na += l_na;
                w_flip += l_flip;
                w_flipna += l_flipna;
                w_down += l_down;
                w_site += 16 * R;
            } else {
                ++nitem;
            }
        }
    }
    if (!MEAS) return;
    const long long nsite = D == 2 ? 16LL * R * nitem : (long long)w_site;
    const long long s_na = D == 2 ? (long long)t_na : (long long)w_na;
    const long long s_flip = D == 2 ? (long long)t_flip : (long long)w_flip;
    const long long s_flipna = D == 2 ? (long long)t_flipna : (long long)w_flipna;
    const unsigned long long down = D == 2 ? (unsigned long long)t_down : w_down;
    // sum over colour-1 sites of the unsatisfied bonds after the move:
    // na' = na + flip (2d - 2 na)
    const long long na_after = s_na + 2 * D * s_flip - 2 * s_flipna;
    long long bond = (long long)(2 * D) * (long long)nsite - 2 * na_after;
    if (JNEG && !HB) bond = -bond;
    Partial mine;
    mine.i0 = block_sum(bond, red);
    mine.i1 = block_sum((long long)down, red);
    mine.f[0] = mine.f[1] = mine.f[2] = mine.f[3] = 0.0;
    if (a.defer) {
        // integer totals: the order of the additions does not matter, so
        // every block adds its own into the pass's accumulator
        if (threadIdx.x == 0) {
            Partial* acc = a.partials + kMaxBlocks;
            atomicAdd(reinterpret_cast<unsigned long long*>(&acc->i0), (unsigned long long)mine.i0);
            atomicAdd(reinterpret_cast<unsigned long long*>(&acc->i1), (unsigned long long)mine.i1);
        }
        return;
    }
    finish_pass(a.ctrl, a.partials, mine, [&](const Partial& tot) { i8_finish(a, tot); });
}

// Closes an i8_stream measuring pass from the totals its blocks added into
// the accumulator after the block partials, and clears the accumulator for
// the next pass (one thread; the kernel boundary orders it after the pass).
__global__ void i8_finish_kernel(const I8Args a)
{
    Partial* acc = a.partials + kMaxBlocks;
    Partial tot = *acc;
    acc->i0 = 0;
    acc->i1 = 0;
    i8_finish(a, tot);
}

// ------------------------------------------------------ init / layout ----

// gofs: global colour index of local entry 0 (a multiple of 4; 0 for a whole lattice)
__global__ void i8_init_kernel(int8_t* s0, int8_t* s1, long long H, uint32_t replica, RoundKeys rk,
                               long long gofs)
{
    const long long ng = (H + 3) >> 2;
    for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < 2 * ng;
         g += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(g / ng);
        const long long gg = g % ng;
        const uint4 r = philox4x32_10(
            make_uint4((uint32_t)(gg + (gofs >> 2)), 0u, replica, (kInit << 1) | (uint32_t)c), rk);
        const uint32_t rr[4] = {r.x, r.y, r.z, r.w};
        int8_t* s = c ? s1 : s0;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const long long j = 4 * gg + b;
            if (j < H) s[j] = (rr[b] >> 31) ? (int8_t)0 : (int8_t)1;
        }
    }
}

// colour of local natural site i; par = parity of the first plane's global index
__device__ __forceinline__ int colour_of(long long i, int L, int par)
{
    const int x = (int)(i % L);
    const long long r = i / L;
    return (x + (int)(r % L) + (int)(r / L) + par) & 1;
}

__global__ void i8_scatter_kernel(int8_t* s0, int8_t* s1, const int8_t* nat, long long N, int L,
                                  int par)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (long long)gridDim.x * blockDim.x)
        (colour_of(i, L, par) ? s1 : s0)[i >> 1] = (int8_t)(nat[i] < 0);
}

__global__ void i8_gather_kernel(const int8_t* s0, const int8_t* s1, int8_t* nat, long long N,
                                 int L, int par)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (long long)gridDim.x * blockDim.x)
        nat[i] = (colour_of(i, L, par) ? s1 : s0)[i >> 1] ? (int8_t)-1 : (int8_t)1;
}

struct BondPtrs {
    int8_t* p[2][3];
};

__global__ void bonds_scatter_kernel(BondPtrs bp, const int8_t* nat, long long N, int L, int d,
                                     unsigned* flags)
{
    unsigned f = 0;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < d * N;
         k += (long long)gridDim.x * blockDim.x) {
        const int mu = (int)(k / N);
        const long long i = k % N;
        const int8_t v = nat[k];
        if (v == 0) f |= 1u;
        if (v < -1 || v > 1) f |= 2u;
        bp.p[colour_of(i, L, 0)][mu][i >> 1] = (int8_t)(v == 0 ? 2 : (v < 0 ? 1 : 0));
    }
    if (f) atomicOr(flags, f);
}

int grid_for(long long work, int block)
{
    long long g = (work + block - 1) / block;
    if (g < 1) g = 1;
    if (g > kMaxBlocks) g = kMaxBlocks;
    return (int)g;
}

I8Args make_args(const sl_lattice* h, int c)
{
    I8Args a;
    a.own = (int8_t*)h->spins[c];
    a.oth = (const int8_t*)h->spins[1 - c];
    for (int mu = 0; mu < 3; ++mu) {
        a.Jown[mu] = (const int8_t*)h->bonds[c][mu];
        a.Joth[mu] = (const int8_t*)h->bonds[1 - c][mu];
    }
    a.d = h->d;
    a.L = h->L;
    a.W = h->W;
    a.c = c;
    a.R = 1;
    a.H = h->H;
    a.N = h->N;
    a.replica = h->replica;
    a.ctrl = h->ctrl;
    a.partials = h->partials;
    a.J = h->J;
    a.measure = c == 1;
    a.update = 1;
    a.advance = 0;
    a.defer = 0;
    a.Lz = h->Lz;
    a.wrap = !h->slab;
    a.par = h->z0 & 1;
    a.gofs = (long long)h->z0 * h->P;
    return a;
}

bool stream_ok(const sl_lattice* h)
{
    return h->W % 16 == 0 && !h->bonds_have_zero;
}

int pick_rows(const sl_lattice* h)
{
    if (h->rows > 0) return h->rows;
    // measured on GB300: 16 rows per thread for 2D (1040 flips/ns at L =
    // 16384, against 1027 for 8 and 999 for 32), 8 for 3D (807 at L = 512,
    // against 803 for 16 and 795 for 32: more, shorter items balance the SMs
    // better); fewer rows only when the grid would not fill the GPU
    const long long W16 = h->W / 16;
    const long long cross = h->d == 3 ? h->L : 1;
    int R = h->d == 3 ? 8 : 16;
    while (R > 1 && (h->Lz % R != 0 || W16 * cross * (h->Lz / R) < (long long)h->sms * 512))
        R >>= 1;
    return R;
}

cudaError_t launch_pass(const sl_lattice* h, I8Args a, cudaStream_t s, bool stream)
{
    if (stream) {
        a.R = pick_rows(h);
        const long long items = (long long)(h->W / 16) * (h->d == 3 ? h->L : 1) * (h->Lz / a.R);
        int grid = grid_for(items, 128);
        if (h->blocks_per_sm > 0 && grid > h->sms * h->blocks_per_sm)
            grid = h->sms * h->blocks_per_sm;
        const bool bonds = a.Jown[0] != nullptr;
        const bool jneg = a.tab.sigma_neg != 0;
        a.defer = a.measure;
        // slabs have uniform couplings: their instantiations have BONDS = 0
#define SPINMC_LAUNCH(D, B, N, HB)                                                        \
    do {                                                                                  \
        if (h->slab && !(B)) {                                                            \
            if (a.measure) i8_stream<D, 0, N, HB, true, true><<<grid, 128, 0, s>>>(a);    \
            else i8_stream<D, 0, N, HB, false, true><<<grid, 128, 0, s>>>(a);             \
        } else {                                                                          \
            if (a.measure) i8_stream<D, B, N, HB, true><<<grid, 128, 0, s>>>(a);          \
            else i8_stream<D, B, N, HB, false><<<grid, 128, 0, s>>>(a);                   \
        }                                                                                 \
    } while (0)
        if (a.tab.heatbath && a.update) {
            if (h->d == 2) {
                if (bonds) SPINMC_LAUNCH(2, 1, 0, 1); else SPINMC_LAUNCH(2, 0, 0, 1);
            } else {
                if (bonds) SPINMC_LAUNCH(3, 1, 0, 1); else SPINMC_LAUNCH(3, 0, 0, 1);
            }
        } else if (h->d == 2) {
            if (bonds) { if (jneg) SPINMC_LAUNCH(2, 1, 1, 0); else SPINMC_LAUNCH(2, 1, 0, 0); }
            else { if (jneg) SPINMC_LAUNCH(2, 0, 1, 0); else SPINMC_LAUNCH(2, 0, 0, 0); }
        } else {
            if (bonds) { if (jneg) SPINMC_LAUNCH(3, 1, 1, 0); else SPINMC_LAUNCH(3, 1, 0, 0); }
            else { if (jneg) SPINMC_LAUNCH(3, 0, 1, 0); else SPINMC_LAUNCH(3, 0, 0, 0); }
        }
#undef SPINMC_LAUNCH
        if (a.defer) {
            const cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) return e;
            i8_finish_kernel<<<1, 1, 0, s>>>(a);
        }
    } else {
        const int grid = grid_for((h->H + 3) >> 2, 256);
        if (h->d == 2) i8_generic<2><<<grid, 256, 0, s>>>(a);
        else i8_generic<3><<<grid, 256, 0, s>>>(a);
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t ising_i8_init(const sl_lattice* h, cudaStream_t s)
{
    i8_init_kernel<<<grid_for(2 * ((h->H + 3) >> 2), 256), 256, 0, s>>>(
        (int8_t*)h->spins[0], (int8_t*)h->spins[1], h->H, h->replica,
        make_round_keys(h->init_seed), (long long)h->z0 * h->P);
    return cudaGetLastError();
}

cudaError_t ising_i8_scatter(const sl_lattice* h, const int8_t* nat, cudaStream_t s)
{
    i8_scatter_kernel<<<grid_for(h->N, 256), 256, 0, s>>>(
        (int8_t*)h->spins[0], (int8_t*)h->spins[1], nat, h->N, h->L, h->z0 & 1);
    return cudaGetLastError();
}

cudaError_t ising_i8_gather(const sl_lattice* h, int8_t* nat, cudaStream_t s)
{
    i8_gather_kernel<<<grid_for(h->N, 256), 256, 0, s>>>(
        (const int8_t*)h->spins[0], (const int8_t*)h->spins[1], nat, h->N, h->L, h->z0 & 1);
    return cudaGetLastError();
}

cudaError_t ising_bonds_scatter(const sl_lattice* h, const int8_t* nat, unsigned* flags,
                                cudaStream_t s)
{
    BondPtrs bp;
    for (int c = 0; c < 2; ++c)
        for (int mu = 0; mu < 3; ++mu) bp.p[c][mu] = (int8_t*)h->bonds[c][mu];
    bonds_scatter_kernel<<<grid_for(h->d * h->N, 256), 256, 0, s>>>(bp, nat, h->N, h->L, h->d,
                                                                    flags);
    return cudaGetLastError();
}

cudaError_t ising_i8_sweeps(const sl_lattice* h, const SweepParams& p, int64_t count,
                            cudaStream_t s)
{
    if (h->update == SL_UPDATE_SW) return ising_sw_sweeps(h, p, count, s);
    if (h->multihit > 0) {
        for (int64_t k = 0; k < count; ++k) {
            cudaError_t e = ising_tile_sweep(h, p, s);
            if (e == cudaSuccess) e = ising_i8_measure_advance(h, s);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
    const bool stream = h->kernel == 2 || (h->kernel == 0 && stream_ok(h));
    for (int64_t k = 0; k < count; ++k) {
        for (int c = 0; c < 2; ++c) {
            I8Args a = make_args(h, c);
            a.tab = p.tab;
            a.rk = p.rk;
            const cudaError_t e = launch_pass(h, a, s, stream);
            if (e != cudaSuccess) return e;
        }
    }
    return cudaSuccess;
}

bool i8_streams(const sl_lattice* h)
{
    return h->multihit == 0 && h->update != SL_UPDATE_SW &&
           (h->kernel == 2 || (h->kernel == 0 && stream_ok(h)));
}

cudaError_t ising_i8_pass(const sl_lattice* h, const SweepParams& p, int c, cudaStream_t s)
{
    const bool stream = h->kernel == 2 || (h->kernel == 0 && stream_ok(h));
    I8Args a = make_args(h, c);
    a.tab = p.tab;
    a.rk = p.rk;
    return launch_pass(h, a, s, stream);
}

cudaError_t ising_i8_measure_advance(const sl_lattice* h, cudaStream_t s)
{
    I8Args a = make_args(h, 1);
    a.update = 0;
    a.measure = 1;
    a.advance = 1;
    memset(&a.tab, 0, sizeof(a.tab));
    memset(&a.rk, 0, sizeof(a.rk));
    return launch_pass(h, a, s, false);
}

cudaError_t ising_i8_measure(const sl_lattice* h, cudaStream_t s)
{
    I8Args a = make_args(h, 1);
    a.update = 0;
    a.measure = 1;
    memset(&a.tab, 0, sizeof(a.tab));
    memset(&a.rk, 0, sizeof(a.rk));
    return launch_pass(h, a, s, false);
}

}  // namespace spinmc
