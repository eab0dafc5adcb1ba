/*
 * Swendsen-Wang cluster update of the Ising model (Section 3 of the paper,
 * its three steps: activate bonds between like spins with probability
 * p = 1 - exp(-2 beta J), build the clusters connected by active bonds, flip
 * every cluster independently with probability 1/2).
 *
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Readings where the paper is silent:
 *   - "like spins" is read for either sign of J as a satisfied bond,
 *     J s_i s_j > 0, and p = 1 - exp(-2 beta |J|); a bond is active iff it is
 *     satisfied and u < p * 2^32 for its raw 32-bit uniform u;
 *   - bond uniforms: the forward bond (i, i + e_mu) draws output
 *     2 (i & 1) + mu of Philox(ctr = (i >> 1, t, replica, 5 << 1)) in 2D, and
 *     output mu of Philox(ctr = (i, t, replica, 5 << 1)) in 3D;
 *   - a cluster is named by its smallest natural site index r and flips iff
 *     the top bit of output 0 of Philox(ctr = (r, t, replica, 6 << 1)) is set;
 *   - one update consumes one sweep index t, like a Metropolis sweep.
 * Clusters are found by a breadth-first search started from every site not
 * yet reached, in increasing site order, so the site that starts a search is
 * the smallest of its cluster.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "oracle.h"
#include "lattice.h"

/* the raw uniforms of the forward bonds of site i: u[mu], mu < d */
static void sw_bond_uniforms(const orc_geom* g, int64_t i, uint32_t t, uint32_t replica,
                             const uint32_t key[2], uint32_t u[3])
{
    uint32_t out[4];
    if (g->d == 2) {
        uint32_t ctr[4] = {(uint32_t)(i >> 1), t, replica, (uint32_t)(ORC_SW_BOND << 1)};
        orc_philox4x32_10(ctr, key, out);
        u[0] = out[2 * (i & 1)];
        u[1] = out[2 * (i & 1) + 1];
        u[2] = 0;
    } else {
        uint32_t ctr[4] = {(uint32_t)i, t, replica, (uint32_t)(ORC_SW_BOND << 1)};
        orc_philox4x32_10(ctr, key, out);
        u[0] = out[0];
        u[1] = out[1];
        u[2] = out[2];
    }
}

int orc_ising_sw_sweeps(int d, int L, double J, double beta, uint64_t seed, uint32_t replica,
                        int64_t t0, int64_t nsweeps, int8_t* s, double* E_out,
                        double* absm_out, uint8_t* active_out, int64_t* label_out)
{
    orc_geom g = orc_make_geom(d, L);
    const uint32_t key[2] = {orc_key_lo(seed), orc_key_hi(seed)};
    const double pact = (1.0 - exp(-2.0 * beta * fabs(J))) * 4294967296.0;
    uint8_t* active = malloc((size_t)g.N * 3);
    int64_t* label = malloc((size_t)g.N * sizeof(int64_t));
    int64_t* queue = malloc((size_t)g.N * sizeof(int64_t));
    if (!active || !label || !queue) {
        free(active);
        free(label);
        free(queue);
        return -1;
    }
    for (int64_t step = 0; step < nsweeps; ++step) {
        const uint32_t t = (uint32_t)(t0 + step);
        /* 1. bond activation */
        for (int64_t i = 0; i < g.N; ++i) {
            uint32_t u[3];
            sw_bond_uniforms(&g, i, t, replica, key, u);
            for (int mu = 0; mu < 3; ++mu) {
                int on = 0;
                if (mu < d) {
                    const int64_t nb = orc_neighbour(&g, i, 2 * mu + 1);
                    const int satisfied = J * (double)(s[i] * s[nb]) > 0.0;
                    on = satisfied && (double)u[mu] < pact;
                }
                active[3 * i + mu] = (uint8_t)on;
            }
        }
        /* 2. clusters: breadth-first search over active bonds, both ends */
        for (int64_t i = 0; i < g.N; ++i) label[i] = -1;
        for (int64_t r = 0; r < g.N; ++r) {
            if (label[r] >= 0) continue;
            int64_t head = 0, tail = 0;
            queue[tail++] = r;
            label[r] = r;
            while (head < tail) {
                const int64_t a = queue[head++];
                for (int k = 0; k < 2 * d; ++k) {
                    const int mu = k >> 1;
                    const int64_t b = orc_neighbour(&g, a, k);
                    /* bond (a, a + e_mu) belongs to a; (a - e_mu, a) to b */
                    const int on = (k & 1) ? active[3 * a + mu] : active[3 * b + mu];
                    if (on && label[b] < 0) {
                        label[b] = r;
                        queue[tail++] = b;
                    }
                }
            }
        }
        /* 3. flip each cluster with probability 1/2 */
        for (int64_t i = 0; i < g.N; ++i) {
            const int64_t r = label[i];
            uint32_t ctr[4] = {(uint32_t)r, t, replica, (uint32_t)(ORC_SW_FLIP << 1)};
            uint32_t out[4];
            orc_philox4x32_10(ctr, key, out);
            if (out[0] >> 31) s[i] = (int8_t)-s[i];
        }
        if (E_out || absm_out) {
            double E, M;
            orc_ising_measure(d, L, J, NULL, s, &E, &M);
            if (E_out) E_out[step] = E;
            if (absm_out) absm_out[step] = fabs(M) / (double)g.N;
        }
    }
    if (nsweeps > 0 && active_out)
        for (int64_t i = 0; i < g.N; ++i)
            for (int mu = 0; mu < d; ++mu) active_out[(int64_t)mu * g.N + i] = active[3 * i + mu];
    if (nsweeps > 0 && label_out) memcpy(label_out, label, (size_t)g.N * sizeof(int64_t));
    free(active);
    free(label);
    free(queue);
    return 0;
}
