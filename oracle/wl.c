/*
 * Windowed multicanonical (MUCA) and Wang-Landau (WL) walkers of the 2D
 * Ising model (Section 4 of the paper: one copy of the system per walker in
 * a fixed energy window, windows overlapping by one energy value, start
 * configurations from a nearest ground state raised into the window, flat
 * histograms over each window, estimates glued into S(E)).
 *
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Energies are counted in levels k = (E + 2N) / 4, 0 <= k <= N (J = 1,
 * periodic L x L, E = -sum over bonds of s_i s_j).  A window is the level
 * range [klo, khi]; a walker's arrays are indexed by k - klo.
 *
 * Readings where the paper is silent:
 *   - L is a power of two; every sweep visits each site once, all walkers in
 *     the same order (so that a warp's walkers touch one site at a time):
 *     step q of sweep t visits site (a q + b) mod N with
 *     (x, y) = outputs 0, 1 of Philox(ctr = (0, t, 0, 11 << 1)),
 *     a = (x mod N) | 1 and b = y mod N, a fresh permutation every sweep (a
 *     fixed order lets a walker whose decisions have all become certain
 *     repeat one cycle of states for ever);
 *   - step q of sweep t draws output q & 3 of
 *     Philox(ctr = (q >> 2, t, walker, purpose << 1)), purpose 9 for WL and
 *     10 for MUCA; a move leaving the window is rejected;
 *   - MUCA with weights S (ln W, FP64): accept iff S(k) >= S(k') or
 *     u < exp(S(k) - S(k')) * 2^32; H(k) counts the level after every
 *     attempt;
 *   - WL: ln g is kept in fixed point, units of 2^-32 (ln f = 2^-stage, so
 *     every update is exact): accept iff D >= 0 or u < exp(D 2^-32) * 2^32,
 *     D = S(k) - S(k'); after every attempt S(k) += 2^(32 - stage), H(k) += 1
 *     and level k is marked visited.  After every sweep of a walker whose
 *     stage is <= final_stage: if every visited level has
 *     H(k) * nvisited * 100 >= flat_percent * sum(H), the stage is flat:
 *     stage += 1, H = 0, and S of the visited levels is lowered by its
 *     minimum over them.  A walker past final_stage makes no more moves;
 *   - start state: the two ferromagnetic ground states (E = -2N) serve a
 *     window whose middle level is <= N/2, the two Neel states (E = +2N) the
 *     others; the top bit of output 0 of Philox(ctr = (0, 1, walker, 8 << 1))
 *     picks the one with spin 0 down.  Attempt a draws output 0 of
 *     Philox(ctr = (a, 0, walker, 8 << 1)) and takes site (u * N) >> 32; the
 *     spin flips iff that moves the energy towards the window without
 *     passing its far edge.  The walk stops inside the window or fails after
 *     1000 N attempts.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "oracle.h"
#include "lattice.h"

enum { ORC_WALK_INIT = 8, ORC_WL = 9, ORC_MUCA = 10, ORC_ORDER = 11 };

/* the site visit order of sweep t: site (a q + b) mod N at step q */
static void wl_order(int64_t N, uint32_t t, const uint32_t key[2], uint64_t* a, uint64_t* b)
{
    uint32_t c[4] = {0u, t, 0u, (uint32_t)(ORC_ORDER << 1)};
    uint32_t out[4];
    orc_philox4x32_10(c, key, out);
    *a = ((uint64_t)out[0] % (uint64_t)N) | 1u;
    *b = (uint64_t)out[1] % (uint64_t)N;
}

/* 4 - 2 (unlike neighbours) = s_i h_i for site i of an L x L torus */
static int wl_sh(const int8_t* s, int L, int64_t i)
{
    const int x = (int)(i % L), y = (int)(i / L);
    const int xm = x == 0 ? L - 1 : x - 1, xp = x == L - 1 ? 0 : x + 1;
    const int ym = y == 0 ? L - 1 : y - 1, yp = y == L - 1 ? 0 : y + 1;
    const int h = s[y * L + xm] + s[y * L + xp] + s[ym * L + x] + s[yp * L + x];
    return s[i] * h;
}

int orc_walker_init(int L, int klo, int khi, uint64_t seed, uint32_t walker, int8_t* s, int* level)
{
    const int64_t N = (int64_t)L * L;
    const uint32_t key[2] = {orc_key_lo(seed), orc_key_hi(seed)};
    uint32_t out[4];
    uint32_t c0[4] = {0u, 1u, walker, (uint32_t)(ORC_WALK_INIT << 1)};
    orc_philox4x32_10(c0, key, out);
    const int down0 = (int)(out[0] >> 31);
    const int ferro = 2 * ((klo + khi) / 2) <= N;   /* middle level <= N / 2 */
    for (int64_t i = 0; i < N; ++i) {
        const int x = (int)(i % L), y = (int)(i / L);
        int up = ferro ? 1 : ((x + y) % 2 == 0);
        if (down0) up = !up;
        s[i] = up ? 1 : -1;
    }
    int k = ferro ? 0 : (int)N;
    const int64_t cap = 1000 * N;
    for (int64_t a = 0; a < cap && (k < klo || k > khi); ++a) {
        uint32_t ca[4] = {(uint32_t)a, 0u, walker, (uint32_t)(ORC_WALK_INIT << 1)};
        orc_philox4x32_10(ca, key, out);
        const int64_t i = (int64_t)(((uint64_t)out[0] * (uint64_t)N) >> 32);
        const int dk = 2 * wl_sh(s, L, i) / 4;   /* dE = 2 s h, in levels */
        const int k2 = k + dk;
        if ((k < klo && dk > 0 && k2 <= khi) || (k > khi && dk < 0 && k2 >= klo)) {
            s[i] = (int8_t)-s[i];
            k = k2;
        }
    }
    *level = k;
    return (k >= klo && k <= khi) ? 0 : -1;
}

static int muca_accept(const void* ctx, int k, int k2, uint32_t u)
{
    const double* S = (const double*)ctx;
    const double d = S[k] - S[k2];
    if (d >= 0.0) return 1;
    return (double)u < exp(d) * 4294967296.0;
}

typedef struct {
    const int64_t* S;
    double tie_tol;
    int64_t ties;
} wl_ctx;

static int wl_accept(const void* ctx, int k, int k2, uint32_t u)
{
    wl_ctx* c = (wl_ctx*)ctx;
    const int64_t D = c->S[k] - c->S[k2];
    if (D >= 0) return 1;
    const double p = exp((double)D * (1.0 / 4294967296.0));
    const double uu = (double)u * (1.0 / 4294967296.0);
    if (fabs(uu - p) < c->tie_tol) c->ties++;
    return uu < p;
}

int64_t orc_wl_sweeps(int L, int klo, int khi, uint64_t seed, uint32_t walker, int64_t t0,
                      int64_t nsweeps, int final_stage, int flat_percent, int8_t* s, int* level,
                      int64_t* S, uint32_t* H, uint64_t* visited, int* stage, double tie_tol)
{
    const int64_t N = (int64_t)L * L;
    const int K = khi - klo + 1;
    const uint32_t key[2] = {orc_key_lo(seed), orc_key_hi(seed)};
    wl_ctx ctx = {S, tie_tol, 0};
    int k = *level - klo;
    for (int64_t step = 0; step < nsweeps; ++step) {
        if (*stage > final_stage) break;
        const uint32_t t = (uint32_t)(t0 + step);
        const int64_t inc = (int64_t)1 << (32 - *stage);
        uint64_t oa, ob;
        wl_order(N, t, key, &oa, &ob);
        uint32_t out[4] = {0, 0, 0, 0};
        for (int64_t q = 0; q < N; ++q) {
            if ((q & 3) == 0) {
                uint32_t c[4] = {(uint32_t)(q >> 2), t, walker, (uint32_t)(ORC_WL << 1)};
                orc_philox4x32_10(c, key, out);
            }
            const int64_t i = (int64_t)((oa * (uint64_t)q + ob) % (uint64_t)N);
            const int k2 = k + 2 * wl_sh(s, L, i) / 4;
            if (k2 >= 0 && k2 < K && wl_accept(&ctx, k, k2, out[q & 3])) {
                s[i] = (int8_t)-s[i];
                k = k2;
            }
            S[k] += inc;
            H[k] += 1u;
            *visited |= (uint64_t)1 << k;
        }
        /* flatness of the visited levels */
        int nv = 0;
        uint64_t sum = 0;
        for (int q = 0; q < K; ++q)
            if ((*visited >> q) & 1u) {
                nv++;
                sum += H[q];
            }
        int flat = nv > 0;
        for (int q = 0; q < K && flat; ++q)
            if (((*visited >> q) & 1u) && (uint64_t)H[q] * (uint64_t)nv * 100u <
                                              (uint64_t)flat_percent * sum)
                flat = 0;
        if (flat) {
            int64_t mn = INT64_MAX;
            for (int q = 0; q < K; ++q)
                if (((*visited >> q) & 1u) && S[q] < mn) mn = S[q];
            for (int q = 0; q < K; ++q) {
                if ((*visited >> q) & 1u) S[q] -= mn;
                H[q] = 0u;
            }
            *stage += 1;
        }
    }
    *level = k + klo;
    return ctx.ties;
}

void orc_muca_sweeps(int L, int klo, int khi, const double* Sw, uint64_t seed, uint32_t walker,
                     int64_t t0, int64_t nsweeps, int8_t* s, int* level, uint64_t* H)
{
    const int64_t N = (int64_t)L * L;
    const int K = khi - klo + 1;
    const uint32_t key[2] = {orc_key_lo(seed), orc_key_hi(seed)};
    int k = *level - klo;
    for (int64_t step = 0; step < nsweeps; ++step) {
        const uint32_t t = (uint32_t)(t0 + step);
        uint64_t oa, ob;
        wl_order(N, t, key, &oa, &ob);
        uint32_t out[4] = {0, 0, 0, 0};
        for (int64_t q = 0; q < N; ++q) {
            if ((q & 3) == 0) {
                uint32_t c[4] = {(uint32_t)(q >> 2), t, walker, (uint32_t)(ORC_MUCA << 1)};
                orc_philox4x32_10(c, key, out);
            }
            const int64_t i = (int64_t)((oa * (uint64_t)q + ob) % (uint64_t)N);
            const int k2 = k + 2 * wl_sh(s, L, i) / 4;
            if (k2 >= 0 && k2 < K && muca_accept(Sw, k, k2, out[q & 3])) {
                s[i] = (int8_t)-s[i];
                k = k2;
            }
            H[k] += 1u;
        }
    }
    *level = k + klo;
}

/* Glue per-window estimates S_w (levels klo[w] .. khi[w], the entries of
 * levels a window never visited marked by visited[w]) into one S over
 * 0..N: window 0 is taken as it is; window w + 1 is shifted so that its
 * value at the level it shares with window w (its first level, which must be
 * window w's last) equals window w's there.  Levels no window visited are
 * NAN.  Returns 0, or -1 if consecutive windows do not share their edge
 * level or the shared level was not visited in both. */
int orc_dos_glue(int N, int nwin, const int* klo, const int* khi, const double* S, int stride,
                 const uint64_t* visited, double* out)
{
    for (int k = 0; k <= N; ++k) out[k] = NAN;
    double shift = 0.0;
    for (int w = 0; w < nwin; ++w) {
        const double* Sw = S + (int64_t)w * stride;
        if (w > 0) {
            if (klo[w] != khi[w - 1]) return -1;
            const double* Sp = S + (int64_t)(w - 1) * stride;
            const int qp = khi[w - 1] - klo[w - 1];
            if (!((visited[w - 1] >> qp) & 1u) || !(visited[w] & 1u)) return -1;
            shift += Sp[qp] - Sw[0];
        }
        for (int k = klo[w]; k <= khi[w]; ++k)
            if ((visited[w] >> (k - klo[w])) & 1u) out[k] = Sw[k - klo[w]] + shift;
    }
    return 0;
}
