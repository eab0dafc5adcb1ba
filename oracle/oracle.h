/*
 * CPU oracle for the checkerboard single-spin-flip Metropolis method of
 * Weigel & Yavors'kii, "GPU accelerated Monte Carlo simulations of lattice
 * spin models" (Physics Procedia 15, 2011), Section 2.
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the slow, plain, obviously
 * correct restatement of the method that the CUDA library is checked against.
 * Only the test suite, the smoke check and the CPU-baseline leg of the bench
 * may load it.  It shares no code, header, table or constant generator with
 * the CUDA library, and the CUDA library never calls it.
 *
 * Conventions (the paper is silent on all of them; they are the readings the
 * CUDA library implements too, written here independently):
 *   - d in {2,3}, L even (the checkerboard needs an even period), N = L^d.
 *   - natural index i = x + L*y (+ L*L*z); colour c(i) = (x+y(+z)) & 1;
 *     colour index j = i >> 1 (the rank of i among the sites of its colour).
 *   - a sweep updates every colour-0 site, then every colour-1 site
 *     (Section 2: one sub-lattice, a barrier, then the other).
 *   - neighbours are taken in the order -x,+x,-y,+y(,-z,+z) with periodic
 *     wrap; for L = 2 a neighbour appears twice (a multigraph), so every site
 *     always has 2d bonds and E counts d*N bonds.
 *   - forward-bond couplings Jb[mu][i] give the bond (i, i + e_mu); the bond
 *     to i - e_mu is Jb[mu][i - e_mu].  J_ij = J * Jb (Eq. 1 with the scalar
 *     J factored out).
 *   - random numbers: Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11),
 *     key = (seed & 0xffffffff, seed >> 32), counter
 *       ctr = (group, t, replica, purpose << 1 | colour)
 *     with purpose 0 = sweep, 1 = initial state, 2 = couplings, 3 = replica
 *     exchange, 4 = multi-hit sweep, 5 = Swendsen-Wang bond, 6 = Swendsen-Wang
 *     cluster flip.  The group is j >> 2 for Ising (site j uses output j & 3),
 *     j >> 1 for XY (site j uses outputs 2(j&1), 2(j&1)+1), and j for
 *     Heisenberg (outputs 0, 1, 2).
 */
#ifndef SPINMC_ORACLE_H
#define SPINMC_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- Philox4x32-10 (published definition, SC'11) ---------------------- */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* ---- Ising model, n = 1 (Eq. 1 with s_i = +-1; Eq. 2) ------------------ */

/* Start configuration: s = +1 if the top bit of the site's Philox output
 * (purpose 1, t = 0) is set, else -1.  s is in natural order, N entries. */
void orc_ising_init(int d, int L, uint64_t seed, uint32_t replica, int8_t* s);

/* Edwards-Anderson couplings: Jb[mu][i] = +1 if the top bit of output 0 of
 * Philox(ctr = (i, mu, sample, 2 << 1)) is set, else -1. */
void orc_ea_couplings(int d, int L, uint64_t seed, uint32_t sample, int8_t* Jb);

/* Energy (Eq. 1) and total magnetisation of an Ising configuration. */
void orc_ising_measure(int d, int L, double J, const int8_t* Jb, const int8_t* s,
                       double* E, double* M);

/* nsweeps Metropolis sweeps with sweep indices t0 .. t0+nsweeps-1.  After
 * sweep k the energy and |m| = |M|/N are written to E_out[k], absm_out[k]
 * (either may be NULL).  Jb may be NULL (all bonds +1). */
void orc_ising_sweeps(int d, int L, double J, const int8_t* Jb, double beta,
                      uint64_t seed, uint32_t replica, int64_t t0, int64_t nsweeps,
                      int8_t* s, double* E_out, double* absm_out);

/* Heat-bath sweeps (Section 2: the heat-bath prescription as the alternative
 * local update).  Same arguments, random stream and measurement as
 * orc_ising_sweeps; each visited spin is drawn afresh from its conditional
 * law: s_i = +1 iff u < 2^32 / (1 + exp(-beta a)), a = 2 J sum_k Jb_k s_k. */
void orc_ising_heatbath_sweeps(int d, int L, double J, const int8_t* Jb, double beta,
                               uint64_t seed, uint32_t replica, int64_t t0, int64_t nsweeps,
                               int8_t* s, double* E_out, double* absm_out);

/* The update of the single site i in sweep t (Metropolis, or heat-bath if
 * heatbath): its new spin from the configuration s, which holds the values the
 * site's neighbours have when its colour is updated (the other colour before
 * the sweep for colour 0, after the colour-0 pass for colour 1; sites of one
 * colour do not interact).  Checks sampled sites of lattices too large to
 * sweep on the CPU. */
int orc_ising_site_update(int d, int L, double J, const int8_t* Jb, double beta, uint64_t seed,
                          uint32_t replica, int64_t t, int heatbath, const int8_t* s, int64_t i);

/* k-fold multi-hit sweeps in big tiles (Section 2: the lattice is cut into
 * big tiles of side T forming a checkerboard; for tile colour 0 and then 1,
 * every tile of that colour receives k updates of all its spins, each an
 * inner checkerboard pass over site colour 0 and then 1, while the
 * neighbouring tiles stay fixed).  T must be even and L % (2T) == 0 so the
 * tile checkerboard closes under the periodic wrap.  Hit h of sweep t
 * draws output j & 3 of Philox(ctr = (j >> 2, t*k + h, replica,
 * 4 << 1 | colour)); acceptance as in orc_ising_sweeps.  E_out / absm_out
 * receive the energy and |m| after each full sweep. */
void orc_ising_multihit_sweeps(int d, int L, int T, int k, double J, const int8_t* Jb,
                               double beta, uint64_t seed, uint32_t replica, int64_t t0,
                               int64_t nsweeps, int8_t* s, double* E_out, double* absm_out);

/* Swendsen-Wang updates (Section 3: activate satisfied bonds with
 * p = 1 - exp(-2 beta |J|), form the clusters joined by active bonds, flip each
 * with probability 1/2), uniform coupling J.  Update t: the forward bond
 * (i, i + e_mu) is active iff J s_i s_j > 0 and u < p 2^32, u = output
 * 2 (i & 1) + mu of Philox(ctr = (i >> 1, t, replica, 5 << 1)) in 2D or output
 * mu of Philox(ctr = (i, t, replica, 5 << 1)) in 3D; the cluster whose
 * smallest site is r flips iff the top bit of output 0 of
 * Philox(ctr = (r, t, replica, 6 << 1)) is set.  E_out / absm_out as for
 * orc_ising_sweeps.  If non-NULL, active_out ([d][N] bytes) and label_out
 * (N entries, the smallest site of each site's cluster) receive the bonds and
 * clusters of the last update.  Returns 0, or -1 if memory ran out. */
int orc_ising_sw_sweeps(int d, int L, double J, double beta, uint64_t seed, uint32_t replica,
                        int64_t t0, int64_t nsweeps, int8_t* s, double* E_out,
                        double* absm_out, uint8_t* active_out, int64_t* label_out);

/* ---- Windowed multicanonical and Wang-Landau walkers (Section 4), 2D
 * Ising, J = 1, L x L torus with L a power of two; energies in levels
 * k = (E + 2N) / 4; a walker
 * lives in the window [klo, khi] and its arrays are indexed by k - klo (see
 * wl.c for every rule and counter).  s is natural order, +-1. */

/* Start state in the window: a nearest ground state raised (or lowered) by
 * flips of randomly drawn spins.  Returns 0, or -1 if 1000 N attempts did
 * not reach the window. */
int orc_walker_init(int L, int klo, int khi, uint64_t seed, uint32_t walker, int8_t* s, int* level);

/* Wang-Landau sweeps t0 .. t0+nsweeps-1 with ln g in fixed point (units of
 * 2^-32) in S, histogram H, visited-level mask and stage (ln f = 2^-stage);
 * returns the number of decisions within tie_tol of the threshold. */
int64_t orc_wl_sweeps(int L, int klo, int khi, uint64_t seed, uint32_t walker, int64_t t0,
                      int64_t nsweeps, int final_stage, int flat_percent, int8_t* s, int* level,
                      int64_t* S, uint32_t* H, uint64_t* visited, int* stage, double tie_tol);

/* Multicanonical sweeps with fixed weights Sw (ln W per window level);
 * H[k - klo] counts the level after every attempt. */
void orc_muca_sweeps(int L, int klo, int khi, const double* Sw, uint64_t seed, uint32_t walker,
                     int64_t t0, int64_t nsweeps, int8_t* s, int* level, uint64_t* H);

/* Glue window estimates (row w of S, stride entries apart) into S over the
 * levels 0..N by matching consecutive windows at their shared edge level. */
int orc_dos_glue(int N, int nwin, const int* klo, const int* khi, const double* S, int stride,
                 const uint64_t* visited, double* out);

/* ---- O(n) models with continuous spins, n = 2 (XY), n = 3 (Heisenberg) ---
 * XY spins are angles theta (s = (cos theta, sin theta)); Heisenberg spins
 * are unit vectors stored as s[3*i + a].  All arithmetic is FP64. */

void orc_xy_init(int d, int L, uint64_t seed, uint32_t replica, double* theta);
void orc_heis_init(int d, int L, uint64_t seed, uint32_t replica, double* s);

/* Energy and magnetisation vector M[0..n-1] (Eq. 1). Jb (float per forward
 * bond, [d][N]) may be NULL. */
void orc_xy_measure(int d, int L, double J, const float* Jb, const double* theta,
                    double* E, double* M);
void orc_heis_measure(int d, int L, double J, const float* Jb, const double* s,
                      double* E, double* M);

/* Decisions whose margin |u - exp(-beta dE)| is below tie_tol are recorded as
 * (t, site) pairs in ties[2*k], ties[2*k+1] for k < ties_cap, and, if tie_info
 * is not NULL, as (margin, K) in tie_info[2*k], tie_info[2*k+1] with the
 * condition factor K = p (beta (A + |dE|) + 1), A = 2 sum_a |h_a| +
 * sum_a |s'_a - s_a| sum_k |J_ik| (an evaluation whose spin components and
 * operations err by at most eps moves p by at most eps K); the return value
 * is the total number of such near-ties.  E_out / absm_out as for Ising.
 * renorm_every > 0 renormalises each spin of the colour being updated right
 * after its decision in every sweep t with (t+1) % renorm_every == 0. */
int64_t orc_xy_sweeps(int d, int L, double J, const float* Jb, double beta,
                      uint64_t seed, uint32_t replica, int64_t t0, int64_t nsweeps,
                      double* theta, double* E_out, double* absm_out,
                      double tie_tol, int64_t* ties, double* tie_info, int64_t ties_cap);
int64_t orc_heis_sweeps(int d, int L, double J, const float* Jb, double beta,
                        uint64_t seed, uint32_t replica, int64_t t0, int64_t nsweeps,
                        int renorm_every, double* s, double* E_out, double* absm_out,
                        double tie_tol, int64_t* ties, double* tie_info, int64_t ties_cap);

/* Heat-bath sweeps (Section 2: each spin drawn from its conditional law given
 * its neighbours), same arguments plus `colours`: bit c set runs the pass of
 * colour c (3 = whole sweeps; a single pass repeats one colour update from
 * given inputs).  Near-ties are XY rejection-test margins below tie_tol and
 * Heisenberg sites whose field has |h_z| / |h| < tie_tol (where the sampling
 * basis changes sign). */
int64_t orc_xy_heatbath_sweeps(int d, int L, double J, const float* Jb, double beta,
                               uint64_t seed, uint32_t replica, int64_t t0, int64_t nsweeps,
                               int colours, double* theta, double* E_out, double* absm_out,
                               double tie_tol, int64_t* ties, int64_t ties_cap);
int64_t orc_heis_heatbath_sweeps(int d, int L, double J, const float* Jb, double beta,
                                 uint64_t seed, uint32_t replica, int64_t t0, int64_t nsweeps,
                                 int colours, int renorm_every, double* s, double* E_out,
                                 double* absm_out, double tie_tol, int64_t* ties,
                                 int64_t ties_cap);

/* ---- Edwards-Anderson +-J spin glass with replica exchange --------------
 * One disorder sample of side L with ntemps replicas (slots).  spins holds
 * ntemps configurations [slot][N]; slot_of_temp[k] is the slot currently at
 * inverse temperature betas[k].  Each sweep t: every slot r performs one
 * Metropolis sweep at betas[temp of r] with replica id sample*ntemps + r;
 * the energy of every slot is measured and E_out[(step)*ntemps + k] receives
 * the energy at temperature k; then pairs (k, k+1) with k = t mod 2, t mod 2
 * + 2, ... attempt a swap accepted iff Delta >= 0 or U < exp(Delta) * 2^32,
 * Delta = (b_k - b_{k+1}) (E_{r(k)} - E_{r(k+1)}), U = output 0 of
 * Philox(ctr = (k, t, sample, 3 << 1)). */
void orc_ea_pt_sweeps(int d, int L, const int8_t* Jb, int ntemps, const double* betas,
                      uint64_t seed, uint32_t sample, int64_t t0, int64_t nsweeps,
                      int8_t* spins, int32_t* slot_of_temp, double* E_out);

#ifdef __cplusplus
}
#endif
#endif
