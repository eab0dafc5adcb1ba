/*
 * Continuous-spin O(n) models, n = 2 (XY) and n = 3 (Heisenberg), under
 * checkerboard single-spin-flip Metropolis, in FP64.
 *
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Section 2 of the paper: Hamiltonian Eq. (1), acceptance Eq. (2), and the
 * remark that continuous spins make floating-point precision matter (the
 * "Metro. double" row of Table 1 is this FP64 computation).  Readings where
 * the paper is silent:
 *   - proposal: a fresh uniform angle (XY) or a fresh uniform direction on
 *     the sphere (Heisenberg), independent of the current spin;
 *   - u24(x) = (x >> 8) * 2^-24; XY angle theta' = 2 pi u24; Heisenberg
 *     z = 2 u24 - 1, phi = 2 pi u24', s' = (sqrt(1-z^2) cos phi,
 *     sqrt(1-z^2) sin phi, z);
 *   - dE = -(s' - s) . h with h = sum_k J Jb_k s_k; accepted iff dE <= 0
 *     or u24 < exp(-beta dE);
 *   - renormalisation s <- s/|s| of each updated spin, right after its
 *     decision, in every sweep t with (t+1) % renorm_every == 0.
 */
#include <math.h>
#include <stddef.h>
#include "oracle.h"
#include "lattice.h"

static const double TWO_PI = 6.283185307179586476925286766559;

static double bond_j(const orc_geom* g, double J, const float* Jb, const int x[3],
                     int64_t i, int k)
{
    if (!Jb) return J;
    return J * (double)Jb[(int64_t)(k >> 1) * g->N + orc_bond_owner_at(g, x, i, k)];
}

static void log_tie(int64_t* count, int64_t* ties, int64_t cap, int64_t t, int64_t i)
{
    if (ties && *count < cap) {
        ties[2 * *count] = t;
        ties[2 * *count + 1] = i;
    }
    ++*count;
}

/* ---------------------------------------------------------------- XY ---- */

void orc_xy_init(int d, int L, uint64_t seed, uint32_t replica, double* theta)
{
    orc_geom g = orc_make_geom(d, L);
    const uint32_t key[2] = {orc_key_lo(seed), orc_key_hi(seed)};
    for (int64_t i = 0; i < g.N; ++i) {
        int c = orc_colour(&g, i);
        int64_t j = i >> 1;
        uint32_t ctr[4] = {(uint32_t)(j >> 1), 0u, replica, (uint32_t)(ORC_INIT << 1 | c)};
        uint32_t out[4];
        orc_philox4x32_10(ctr, key, out);
        theta[i] = TWO_PI * orc_u24(out[2 * (j & 1) + 1]);
    }
}

void orc_xy_measure(int d, int L, double J, const float* Jb, const double* theta,
                    double* E, double* M)
{
    orc_geom g = orc_make_geom(d, L);
    double e = 0.0, mx = 0.0, my = 0.0;
    for (int64_t i = 0; i < g.N; ++i) {
        int x[3];
        orc_coords(&g, i, x);
        mx += cos(theta[i]);
        my += sin(theta[i]);
        for (int mu = 0; mu < d; ++mu) {
            int64_t nb = orc_neighbour_at(&g, x, 2 * mu + 1);
            double jij = bond_j(&g, J, Jb, x, i, 2 * mu + 1);
            e -= jij * (cos(theta[i]) * cos(theta[nb]) + sin(theta[i]) * sin(theta[nb]));
        }
    }
    *E = e;
    M[0] = mx;
    M[1] = my;
}

int64_t orc_xy_sweeps(int d, int L, double J, const float* Jb, double beta,
                      uint64_t seed, uint32_t replica, int64_t t0, int64_t nsweeps,
                      double* theta, double* E_out, double* absm_out,
                      double tie_tol, int64_t* ties, int64_t ties_cap)
{
    orc_geom g = orc_make_geom(d, L);
    const uint32_t key[2] = {orc_key_lo(seed), orc_key_hi(seed)};
    const int Lz = d == 3 ? L : 1;
    int64_t nties = 0;
    for (int64_t step = 0; step < nsweeps; ++step) {
        int64_t t = t0 + step;
        for (int c = 0; c < 2; ++c)
            for (int z = 0; z < Lz; ++z)
                for (int y = 0; y < L; ++y)
                    for (int x0 = (c + y + z) & 1; x0 < L; x0 += 2) {
                        int x[3] = {x0, y, z};
                        int64_t i = orc_index(&g, x);
                        int64_t j = i >> 1;
                        uint32_t ctr[4] = {(uint32_t)(j >> 1), (uint32_t)t, replica,
                                           (uint32_t)(ORC_SWEEP << 1 | c)};
                        uint32_t out[4];
                        orc_philox4x32_10(ctr, key, out);
                        double u = orc_u24(out[2 * (j & 1)]);
                        double th_new = TWO_PI * orc_u24(out[2 * (j & 1) + 1]);
                        double hx = 0.0, hy = 0.0;
                        for (int k = 0; k < 2 * d; ++k) {
                            int64_t nb = orc_neighbour_at(&g, x, k);
                            double jij = bond_j(&g, J, Jb, x, i, k);
                            hx += jij * cos(theta[nb]);
                            hy += jij * sin(theta[nb]);
                        }
                        double dE = -((cos(th_new) - cos(theta[i])) * hx +
                                      (sin(th_new) - sin(theta[i])) * hy);
                        int accept = 1;
                        if (dE > 0.0) {
                            double p = exp(-beta * dE);
                            accept = u < p;
                            if (fabs(u - p) < tie_tol) log_tie(&nties, ties, ties_cap, t, i);
                        }
                        if (accept) theta[i] = th_new;
                    }
        if (E_out || absm_out) {
            double E, M[2];
            orc_xy_measure(d, L, J, Jb, theta, &E, M);
            if (E_out) E_out[step] = E;
            if (absm_out) absm_out[step] = sqrt(M[0] * M[0] + M[1] * M[1]) / (double)g.N;
        }
    }
    return nties;
}

/* -------------------------------------------------------- Heisenberg ---- */

static void sphere_point(uint32_t uz, uint32_t uphi, double v[3])
{
    double z = 2.0 * orc_u24(uz) - 1.0;
    double phi = TWO_PI * orc_u24(uphi);
    double r = sqrt(1.0 - z * z);
    v[0] = r * cos(phi);
    v[1] = r * sin(phi);
    v[2] = z;
}

void orc_heis_init(int d, int L, uint64_t seed, uint32_t replica, double* s)
{
    orc_geom g = orc_make_geom(d, L);
    const uint32_t key[2] = {orc_key_lo(seed), orc_key_hi(seed)};
    for (int64_t i = 0; i < g.N; ++i) {
        int c = orc_colour(&g, i);
        int64_t j = i >> 1;
        uint32_t ctr[4] = {(uint32_t)j, 0u, replica, (uint32_t)(ORC_INIT << 1 | c)};
        uint32_t out[4];
        orc_philox4x32_10(ctr, key, out);
        sphere_point(out[1], out[2], s + 3 * i);
    }
}

void orc_heis_measure(int d, int L, double J, const float* Jb, const double* s,
                      double* E, double* M)
{
    orc_geom g = orc_make_geom(d, L);
    double e = 0.0;
    M[0] = M[1] = M[2] = 0.0;
    for (int64_t i = 0; i < g.N; ++i) {
        int x[3];
        orc_coords(&g, i, x);
        for (int a = 0; a < 3; ++a) M[a] += s[3 * i + a];
        for (int mu = 0; mu < d; ++mu) {
            int64_t nb = orc_neighbour_at(&g, x, 2 * mu + 1);
            double jij = bond_j(&g, J, Jb, x, i, 2 * mu + 1);
            double dot = s[3 * i] * s[3 * nb] + s[3 * i + 1] * s[3 * nb + 1] +
                         s[3 * i + 2] * s[3 * nb + 2];
            e -= jij * dot;
        }
    }
    *E = e;
}

int64_t orc_heis_sweeps(int d, int L, double J, const float* Jb, double beta,
                        uint64_t seed, uint32_t replica, int64_t t0, int64_t nsweeps,
                        int renorm_every, double* s, double* E_out, double* absm_out,
                        double tie_tol, int64_t* ties, int64_t ties_cap)
{
    orc_geom g = orc_make_geom(d, L);
    const uint32_t key[2] = {orc_key_lo(seed), orc_key_hi(seed)};
    const int Lz = d == 3 ? L : 1;
    int64_t nties = 0;
    for (int64_t step = 0; step < nsweeps; ++step) {
        int64_t t = t0 + step;
        int renorm = renorm_every > 0 && (t + 1) % renorm_every == 0;
        for (int c = 0; c < 2; ++c)
            for (int z = 0; z < Lz; ++z)
                for (int y = 0; y < L; ++y)
                    for (int x0 = (c + y + z) & 1; x0 < L; x0 += 2) {
                        int x[3] = {x0, y, z};
                        int64_t i = orc_index(&g, x);
                        int64_t j = i >> 1;
                        uint32_t ctr[4] = {(uint32_t)j, (uint32_t)t, replica,
                                           (uint32_t)(ORC_SWEEP << 1 | c)};
                        uint32_t out[4];
                        orc_philox4x32_10(ctr, key, out);
                        double u = orc_u24(out[0]);
                        double sn[3];
                        sphere_point(out[1], out[2], sn);
                        double h[3] = {0.0, 0.0, 0.0};
                        for (int k = 0; k < 2 * d; ++k) {
                            int64_t nb = orc_neighbour_at(&g, x, k);
                            double jij = bond_j(&g, J, Jb, x, i, k);
                            for (int a = 0; a < 3; ++a) h[a] += jij * s[3 * nb + a];
                        }
                        double dE = 0.0;
                        for (int a = 0; a < 3; ++a) dE -= (sn[a] - s[3 * i + a]) * h[a];
                        int accept = 1;
                        if (dE > 0.0) {
                            double p = exp(-beta * dE);
                            accept = u < p;
                            if (fabs(u - p) < tie_tol) log_tie(&nties, ties, ties_cap, t, i);
                        }
                        if (accept)
                            for (int a = 0; a < 3; ++a) s[3 * i + a] = sn[a];
                        if (renorm) {
                            double nrm = sqrt(s[3 * i] * s[3 * i] + s[3 * i + 1] * s[3 * i + 1] +
                                              s[3 * i + 2] * s[3 * i + 2]);
                            for (int a = 0; a < 3; ++a) s[3 * i + a] /= nrm;
                        }
                    }
        if (E_out || absm_out) {
            double E, M[3];
            orc_heis_measure(d, L, J, Jb, s, &E, M);
            if (E_out) E_out[step] = E;
            if (absm_out)
                absm_out[step] = sqrt(M[0] * M[0] + M[1] * M[1] + M[2] * M[2]) / (double)g.N;
        }
    }
    return nties;
}
