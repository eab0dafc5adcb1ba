/*
 * Ising model (n = 1) under checkerboard single-spin-flip Metropolis.
 *
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Follows Section 2 of the paper: Hamiltonian Eq. (1) with s_i = +-1 and
 * nearest-neighbour couplings J_ij = J * Jb_ij, acceptance Eq. (2)
 * p = min[1, exp(-beta dE)], and the checkerboard order (all sites of one
 * colour, then all sites of the other).  Readings where the paper is silent:
 *   - dE = 2 J s_i sum_k Jb_k s_k, evaluated as 2.0 * J * (integer s_i h);
 *   - a move with dE <= 0 is always accepted; otherwise it is accepted iff
 *     u < exp(-beta dE) * 2^32 with u the site's raw 32-bit Philox output,
 *     i.e. with probability exp(-beta dE) resolved to 2^-32;
 *   - Jb = NULL means every coupling is +1.
 */
#include <math.h>
#include <stddef.h>
#include "oracle.h"
#include "lattice.h"

void orc_ising_init(int d, int L, uint64_t seed, uint32_t replica, int8_t* s)
{
    orc_geom g = orc_make_geom(d, L);
    const uint32_t key[2] = {orc_key_lo(seed), orc_key_hi(seed)};
    for (int64_t i = 0; i < g.N; ++i) {
        int c = orc_colour(&g, i);
        int64_t j = i >> 1;
        uint32_t ctr[4] = {(uint32_t)(j >> 2), 0u, replica, (uint32_t)(ORC_INIT << 1 | c)};
        uint32_t out[4];
        orc_philox4x32_10(ctr, key, out);
        s[i] = (out[j & 3] >> 31) ? 1 : -1;
    }
}

void orc_ea_couplings(int d, int L, uint64_t seed, uint32_t sample, int8_t* Jb)
{
    orc_geom g = orc_make_geom(d, L);
    const uint32_t key[2] = {orc_key_lo(seed), orc_key_hi(seed)};
    for (int mu = 0; mu < d; ++mu)
        for (int64_t i = 0; i < g.N; ++i) {
            uint32_t ctr[4] = {(uint32_t)i, (uint32_t)mu, sample, (uint32_t)(ORC_COUPLING << 1)};
            uint32_t out[4];
            orc_philox4x32_10(ctr, key, out);
            Jb[(int64_t)mu * g.N + i] = (out[0] >> 31) ? 1 : -1;
        }
}

void orc_ising_measure(int d, int L, double J, const int8_t* Jb, const int8_t* s,
                       double* E, double* M)
{
    orc_geom g = orc_make_geom(d, L);
    int64_t bond_sum = 0, m = 0;
    for (int64_t i = 0; i < g.N; ++i) {
        int x[3];
        orc_coords(&g, i, x);
        m += s[i];
        for (int mu = 0; mu < d; ++mu) {
            int64_t nb = orc_neighbour_at(&g, x, 2 * mu + 1);
            int jb = Jb ? Jb[(int64_t)mu * g.N + i] : 1;
            bond_sum += (int64_t)jb * s[i] * s[nb];
        }
    }
    *E = -J * (double)bond_sum;
    *M = (double)m;
}

/* one Metropolis decision for site i of colour c, given its uniform u */
static int ising_accept(const orc_geom* g, double J, const int8_t* Jb, double beta,
                        const int8_t* s, const int x[3], int64_t i, uint32_t u)
{
    int hsum = 0;
    for (int k = 0; k < 2 * g->d; ++k) {
        int64_t nb = orc_neighbour_at(g, x, k);
        int jb = Jb ? Jb[(int64_t)(k >> 1) * g->N + orc_bond_owner_at(g, x, i, k)] : 1;
        hsum += jb * s[nb];
    }
    int sh = s[i] * hsum;
    double dE = 2.0 * J * (double)sh;
    if (dE <= 0.0) return 1;
    return (double)u < exp(-beta * dE) * 4294967296.0;
}

/* sum_k Jb_k s_k over the 2d neighbours of the site at coordinates x */
static int ising_field(const orc_geom* g, const int8_t* Jb, const int8_t* s, const int x[3],
                       int64_t i)
{
    int hsum = 0;
    for (int k = 0; k < 2 * g->d; ++k) {
        int64_t nb = orc_neighbour_at(g, x, k);
        int jb = Jb ? Jb[(int64_t)(k >> 1) * g->N + orc_bond_owner_at(g, x, i, k)] : 1;
        hsum += jb * s[nb];
    }
    return hsum;
}

static void ising_sweeps_rule(int d, int L, double J, const int8_t* Jb, double beta,
                              uint64_t seed, uint32_t replica, int64_t t0, int64_t nsweeps,
                              int8_t* s, double* E_out, double* absm_out, int heatbath);

void orc_ising_sweeps(int d, int L, double J, const int8_t* Jb, double beta,
                      uint64_t seed, uint32_t replica, int64_t t0, int64_t nsweeps,
                      int8_t* s, double* E_out, double* absm_out)
{
    ising_sweeps_rule(d, L, J, Jb, beta, seed, replica, t0, nsweeps, s, E_out, absm_out, 0);
}

void orc_ising_heatbath_sweeps(int d, int L, double J, const int8_t* Jb, double beta,
                               uint64_t seed, uint32_t replica, int64_t t0, int64_t nsweeps,
                               int8_t* s, double* E_out, double* absm_out)
{
    ising_sweeps_rule(d, L, J, Jb, beta, seed, replica, t0, nsweeps, s, E_out, absm_out, 1);
}

static void ising_sweeps_rule(int d, int L, double J, const int8_t* Jb, double beta,
                              uint64_t seed, uint32_t replica, int64_t t0, int64_t nsweeps,
                              int8_t* s, double* E_out, double* absm_out, int heatbath)
{
    orc_geom g = orc_make_geom(d, L);
    const uint32_t key[2] = {orc_key_lo(seed), orc_key_hi(seed)};
    const int Lz = d == 3 ? L : 1;
    for (int64_t step = 0; step < nsweeps; ++step) {
        uint32_t t = (uint32_t)(t0 + step);
        for (int c = 0; c < 2; ++c) {
            int64_t cached_group = -1;
            uint32_t out[4] = {0, 0, 0, 0};
            for (int z = 0; z < Lz; ++z)
                for (int y = 0; y < L; ++y)
                    for (int x = (c + y + z) & 1; x < L; x += 2) {
                        int xyz[3] = {x, y, z};
                        int64_t i = orc_index(&g, xyz);
                        int64_t j = i >> 1;
                        if ((j >> 2) != cached_group) {
                            cached_group = j >> 2;
                            uint32_t ctr[4] = {(uint32_t)(j >> 2), t, replica,
                                               (uint32_t)(ORC_SWEEP << 1 | c)};
                            orc_philox4x32_10(ctr, key, out);
                        }
                        if (heatbath) {
                            /* P(s_i = +1) = 1 / (1 + exp(-2 beta J h)) */
                            double a = 2.0 * J * (double)ising_field(&g, Jb, s, xyz, i);
                            double thr = 4294967296.0 / (1.0 + exp(-beta * a));
                            s[i] = (double)out[j & 3] < thr ? 1 : -1;
                        } else if (ising_accept(&g, J, Jb, beta, s, xyz, i, out[j & 3])) {
                            s[i] = (int8_t)-s[i];
                        }
                    }
        }
        if (E_out || absm_out) {
            double E, M;
            orc_ising_measure(d, L, J, Jb, s, &E, &M);
            if (E_out) E_out[step] = E;
            if (absm_out) absm_out[step] = fabs(M) / (double)g.N;
        }
    }
}

int orc_ising_site_update(int d, int L, double J, const int8_t* Jb, double beta, uint64_t seed,
                          uint32_t replica, int64_t t, int heatbath, const int8_t* s, int64_t i)
{
    orc_geom g = orc_make_geom(d, L);
    const uint32_t key[2] = {orc_key_lo(seed), orc_key_hi(seed)};
    int xyz[3];
    orc_coords(&g, i, xyz);
    const int c = orc_colour(&g, i);
    const int64_t j = i >> 1;
    uint32_t ctr[4] = {(uint32_t)(j >> 2), (uint32_t)t, replica, (uint32_t)(ORC_SWEEP << 1 | c)};
    uint32_t out[4];
    orc_philox4x32_10(ctr, key, out);
    if (heatbath) {
        double a = 2.0 * J * (double)ising_field(&g, Jb, s, xyz, i);
        return (double)out[j & 3] < 4294967296.0 / (1.0 + exp(-beta * a)) ? 1 : -1;
    }
    return ising_accept(&g, J, Jb, beta, s, xyz, i, out[j & 3]) ? -s[i] : s[i];
}

void orc_ising_multihit_sweeps(int d, int L, int T, int k, double J, const int8_t* Jb,
                               double beta, uint64_t seed, uint32_t replica, int64_t t0,
                               int64_t nsweeps, int8_t* s, double* E_out, double* absm_out)
{
    orc_geom g = orc_make_geom(d, L);
    const uint32_t key[2] = {orc_key_lo(seed), orc_key_hi(seed)};
    const int Lz = d == 3 ? L : 1;
    for (int64_t step = 0; step < nsweeps; ++step) {
        const int64_t t = t0 + step;
        for (int tc = 0; tc < 2; ++tc)          /* tile colour */
            for (int h = 0; h < k; ++h)           /* hit */
                for (int c = 0; c < 2; ++c)       /* site colour */
                    for (int z = 0; z < Lz; ++z)
                        for (int y = 0; y < L; ++y)
                            for (int x = (c + y + z) & 1; x < L; x += 2) {
                                int tile_colour = (x / T + y / T + (d == 3 ? z / T : 0)) & 1;
                                if (tile_colour != tc) continue;
                                int xyz[3] = {x, y, z};
                                int64_t i = orc_index(&g, xyz);
                                int64_t j = i >> 1;
                                uint32_t ctr[4] = {(uint32_t)(j >> 2), (uint32_t)(t * k + h),
                                                   replica, (uint32_t)(ORC_MULTIHIT << 1 | c)};
                                uint32_t out[4];
                                orc_philox4x32_10(ctr, key, out);
                                if (ising_accept(&g, J, Jb, beta, s, xyz, i, out[j & 3]))
                                    s[i] = (int8_t)-s[i];
                            }
        if (E_out || absm_out) {
            double E, M;
            orc_ising_measure(d, L, J, Jb, s, &E, &M);
            if (E_out) E_out[step] = E;
            if (absm_out) absm_out[step] = fabs(M) / (double)g.N;
        }
    }
}
