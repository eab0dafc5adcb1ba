/*
 * Philox4x32-10 counter-based generator, written from its published
 * definition (Salmon, Moraes, Dror & Shaw, "Parallel random numbers: as easy
 * as 1, 2, 3", SC'11, Section 3 and its Philox-4x32 parameters).
 *
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * The paper under study uses one 32-bit LCG per thread (Section 2) and points
 * to "more generally appropriate generators"; the method here keys a
 * counter-based generator by (seed, sweep, site) instead.
 *
 * One round maps (c0, c1, c2, c3) under key (k0, k1) to
 *   (hi(M1*c2) ^ c1 ^ k0,  lo(M1*c2),  hi(M0*c0) ^ c3 ^ k1,  lo(M0*c0))
 * with M0 = 0xD2511F53, M1 = 0xCD9E8D57; between rounds the key is bumped by
 * the Weyl constants (0x9E3779B9, 0xBB67AE85).  Ten rounds.
 */
#include "oracle.h"

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}
