/*
 * Lattice geometry for the oracle: natural index <-> coordinates, colour,
 * periodic nearest neighbours (Eq. 1: square d = 2 or simple-cubic d = 3
 * lattices, nearest-neighbour bonds).
 *
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 */
#ifndef SPINMC_ORACLE_LATTICE_H
#define SPINMC_ORACLE_LATTICE_H
#include <stdint.h>

typedef struct {
    int d, L;
    int64_t N;
} orc_geom;

static inline orc_geom orc_make_geom(int d, int L)
{
    orc_geom g;
    g.d = d;
    g.L = L;
    g.N = (int64_t)L * L * (d == 3 ? L : 1);
    return g;
}

/* coordinates x[0..d-1] of natural index i */
static inline void orc_coords(const orc_geom* g, int64_t i, int x[3])
{
    x[0] = (int)(i % g->L);
    x[1] = (int)((i / g->L) % g->L);
    x[2] = g->d == 3 ? (int)(i / ((int64_t)g->L * g->L)) : 0;
}

static inline int64_t orc_index(const orc_geom* g, const int x[3])
{
    int64_t i = x[0] + (int64_t)g->L * x[1];
    if (g->d == 3) i += (int64_t)g->L * g->L * x[2];
    return i;
}

static inline int orc_colour(const orc_geom* g, int64_t i)
{
    int x[3];
    orc_coords(g, i, x);
    return (x[0] + x[1] + (g->d == 3 ? x[2] : 0)) & 1;
}

/* neighbour k of site i, k = 2*mu + (0 for -e_mu, 1 for +e_mu) */
static inline int64_t orc_neighbour(const orc_geom* g, int64_t i, int k)
{
    int x[3];
    orc_coords(g, i, x);
    int mu = k >> 1;
    int step = (k & 1) ? 1 : -1;
    x[mu] = (x[mu] + step + g->L) % g->L;
    return orc_index(g, x);
}

/* neighbour k of the site at coordinates x (no division needed) */
static inline int64_t orc_neighbour_at(const orc_geom* g, const int x[3], int k)
{
    int y[3] = {x[0], x[1], x[2]};
    int mu = k >> 1;
    y[mu] = (k & 1) ? (y[mu] + 1 == g->L ? 0 : y[mu] + 1) : (y[mu] == 0 ? g->L - 1 : y[mu] - 1);
    return orc_index(g, y);
}

/* the forward-bond coupling (in units of J) of the bond from i to its
 * neighbour k: Jb[mu][i] for +e_mu, Jb[mu][i - e_mu] for -e_mu */
static inline int64_t orc_bond_owner(const orc_geom* g, int64_t i, int k)
{
    return (k & 1) ? i : orc_neighbour(g, i, k);
}

static inline int64_t orc_bond_owner_at(const orc_geom* g, const int x[3], int64_t i, int k)
{
    return (k & 1) ? i : orc_neighbour_at(g, x, k);
}

static inline uint32_t orc_key_lo(uint64_t seed) { return (uint32_t)(seed & 0xffffffffu); }
static inline uint32_t orc_key_hi(uint64_t seed) { return (uint32_t)(seed >> 32); }

/* u24 in [0,1): the top 24 bits of a 32-bit output, scaled by 2^-24 (exact
 * in FP32 and FP64). */
static inline double orc_u24(uint32_t x) { return (double)(x >> 8) * (1.0 / 16777216.0); }

enum { ORC_SWEEP = 0, ORC_INIT = 1, ORC_COUPLING = 2, ORC_EXCHANGE = 3, ORC_MULTIHIT = 4,
       ORC_SW_BOND = 5, ORC_SW_FLIP = 6 };

#endif
