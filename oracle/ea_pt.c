/*
 * Edwards-Anderson +-J Ising spin glass (Section 2: couplings drawn from the
 * bimodal distribution, trivially parallel over disorder samples) with
 * replica exchange between temperatures.
 *
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * The paper has no replica exchange; the reading implemented here is the
 * standard Metropolis swap between neighbouring temperatures: after sweep t
 * the pairs (k, k+1) with k = t mod 2, t mod 2 + 2, ... are visited in order,
 * Delta = (b_k - b_{k+1}) (E_{r(k)} - E_{r(k+1)}), and the swap of the
 * temperature labels is accepted iff Delta >= 0 or U < exp(Delta) * 2^32.
 * Configurations stay in their slots; a slot's random stream is keyed by the
 * slot, never by its current temperature.
 */
#include <math.h>
#include <stdlib.h>
#include "oracle.h"
#include "lattice.h"

void orc_ea_pt_sweeps(int d, int L, const int8_t* Jb, int ntemps, const double* betas,
                      uint64_t seed, uint32_t sample, int64_t t0, int64_t nsweeps,
                      int8_t* spins, int32_t* slot_of_temp, double* E_out)
{
    orc_geom g = orc_make_geom(d, L);
    const uint32_t key[2] = {orc_key_lo(seed), orc_key_hi(seed)};
    int* temp_of_slot = (int*)malloc(sizeof(int) * (size_t)ntemps);
    double* E_slot = (double*)malloc(sizeof(double) * (size_t)ntemps);
    for (int64_t step = 0; step < nsweeps; ++step) {
        int64_t t = t0 + step;
        for (int k = 0; k < ntemps; ++k) temp_of_slot[slot_of_temp[k]] = k;
        for (int r = 0; r < ntemps; ++r) {
            int8_t* s = spins + (int64_t)r * g.N;
            uint32_t replica = sample * (uint32_t)ntemps + (uint32_t)r;
            orc_ising_sweeps(d, L, 1.0, Jb, betas[temp_of_slot[r]], seed, replica, t, 1,
                             s, NULL, NULL);
            double M;
            orc_ising_measure(d, L, 1.0, Jb, s, &E_slot[r], &M);
        }
        for (int k = 0; k < ntemps; ++k)
            E_out[step * ntemps + k] = E_slot[slot_of_temp[k]];
        for (int k = (int)(t & 1); k + 1 < ntemps; k += 2) {
            int ra = slot_of_temp[k], rb = slot_of_temp[k + 1];
            double delta = (betas[k] - betas[k + 1]) * (E_slot[ra] - E_slot[rb]);
            int accept = delta >= 0.0;
            if (!accept) {
                uint32_t ctr[4] = {(uint32_t)k, (uint32_t)t, sample,
                                   (uint32_t)(ORC_EXCHANGE << 1)};
                uint32_t out[4];
                orc_philox4x32_10(ctr, key, out);
                accept = (double)out[0] < exp(delta) * 4294967296.0;
            }
            if (accept) {
                slot_of_temp[k] = rb;
                slot_of_temp[k + 1] = ra;
            }
        }
    }
    free(temp_of_slot);
    free(E_slot);
}
