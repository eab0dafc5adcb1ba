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
 *
 * Heat-bath rule (Section 2 names it as the other local update, a small local
 * change of the Metropolis code): the new spin is drawn from its conditional
 * law, density proportional to exp(beta s' . h) with h = sum_k J Jb_k s_k,
 * independent of the old spin.  Readings where the paper is silent:
 *   - Heisenberg: with kappa = beta |h| and c = s' . h / |h|, c has density
 *     proportional to exp(kappa c) on [-1, 1]; inverting its distribution
 *     function at u = u24(output 0) gives
 *       1 - c = -log1p((1 - u) expm1(-2 kappa)) / kappa,
 *       1 + c =  log1p(u expm1(2 kappa)) / kappa
 *     (the first is used when it is <= 1, else the second; both are exact
 *     forms of the same inverse); the azimuth about h is phi = 2 pi
 *     u24(output 1), measured in the orthonormal basis (e1, e2, h/|h|) of
 *     Duff et al., "Building an Orthonormal Basis, Revisited" (JCGT 6(1),
 *     2017); kappa = 0 draws c = 2u - 1 (about the z axis if h = 0).  The
 *     basis changes sign with the z component of h/|h|, so a site with
 *     |h_z|/|h| below tie_tol is recorded as a near-tie;
 *   - XY: the angle offset delta from the angle of h has density
 *     proportional to exp(kappa cos delta), drawn by the rejection method of
 *     Best and Fisher (Appl. Statist. 28, 152 (1979)), wrapped-Cauchy
 *     envelope with parameter rho = 2 kappa / (tau + sqrt(2 tau)),
 *     tau = 1 + sqrt(1 + 4 kappa^2) (their rho, free of cancellation).
 *     Attempt a = 0, 1, ..., 31 of site i takes U1, U2 from outputs
 *     2 (j & 1) and 2 (j & 1) + 1 of Philox(ctr = (j >> 1, t, replica,
 *     a << 16 | colour)), j = i >> 1; with w = pi U1 / 2 the candidate is
 *     tan(delta / 2) = ((1 - rho) / (1 + rho)) tan w (their arccos f,
 *     f = (1 + r cos 2w) / (r + cos 2w), written without cancellation), and
 *     their test quantity is c = kappa (r - f) = (tau + sqrt(2 tau))
 *     (1 - rho^2)^2 / (4 ((1 - rho)^2 + 4 rho cos^2 w)); the candidate is
 *     accepted iff c (2 - c) > U2 or log(c / U2) + 1 - c >= 0, and delta is
 *     negated iff bit 0 of the U1 output is set.  A site with no acceptance
 *     in 32 attempts keeps its angle.  Test margins below tie_tol are
 *     recorded as near-ties.
 */
#include <math.h>
#include <stddef.h>
#include "oracle.h"
#include "lattice.h"

static const double TWO_PI = 6.283185307179586476925286766559;
static const double HALF_PI = 1.5707963267948966192313216916398;

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

/* A Metropolis near-tie with its margin |u - p| and the condition factor
 * K = p (beta (A + |dE|) + 1), A = 2 sum_a |h_a| + sum_a |s'_a - s_a| sum_k |J_ik|
 * (components a of the spin vectors; cos and sin of the angles for XY).  If
 * every spin component, the field's inputs and the evaluation carry relative
 * or absolute errors up to eps, then dE is off by at most eps (A + |dE|) and
 * p by at most eps K, so a decision can only differ where the margin is below
 * eps K: this is instrumentation for the caller's tolerance, not part of the
 * method. */
static void log_tie_info(int64_t* count, int64_t* ties, double* info, int64_t cap, int64_t t,
                         int64_t i, double margin, double K)
{
    if (info && *count < cap) {
        info[2 * *count] = margin;
        info[2 * *count + 1] = K;
    }
    log_tie(count, ties, cap, t, i);
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

/* Heat-bath draw of one XY angle (rejection method of Best and Fisher, as
 * read in the header); returns 1 if a candidate was accepted. */
static int xy_heatbath_draw(double hx, double hy, double beta, const uint32_t key[2],
                            uint32_t group, uint32_t t, uint32_t replica, int c, int lane,
                            double tie_tol, int* tie, double* theta)
{
    const double kappa = beta * sqrt(hx * hx + hy * hy);
    const double tau = 1.0 + sqrt(1.0 + 4.0 * kappa * kappa);
    const double s2 = sqrt(2.0 * tau);
    const double rho = 2.0 * kappa / (tau + s2);
    const double g = (1.0 - rho) / (1.0 + rho);
    const double cnum = (tau + s2) * (1.0 - rho * rho) * (1.0 - rho * rho) / 4.0;
    for (uint32_t a = 0; a < 32u; ++a) {
        uint32_t ctr[4] = {group, t, replica, (a << 16) | (uint32_t)(ORC_SWEEP << 1 | c)};
        uint32_t out[4];
        orc_philox4x32_10(ctr, key, out);
        const uint32_t o1 = out[2 * lane];
        const double U1 = orc_u24(o1), U2 = orc_u24(out[2 * lane + 1]);
        const double w = HALF_PI * U1;
        const double cw = cos(w), sw = sin(w);
        const double cc = cnum / ((1.0 - rho) * (1.0 - rho) + 4.0 * rho * cw * cw);
        const double m1 = cc * (2.0 - cc) - U2;
        int accept = m1 > 0.0;
        if (fabs(m1) < tie_tol) *tie = 1;
        if (!accept) {
            const double m2 = log(cc / U2) + 1.0 - cc;
            accept = m2 >= 0.0;
            if (fabs(m2) < tie_tol) *tie = 1;
        }
        if (accept) {
            double delta = 2.0 * atan2(g * sw, cw);
            if (o1 & 1u) delta = -delta;
            double th = atan2(hy, hx) + delta;
            if (th < 0.0) th += TWO_PI;
            if (th >= TWO_PI) th -= TWO_PI;
            *theta = th;
            return 1;
        }
    }
    return 0;
}

static int64_t xy_sweeps(int d, int L, double J, const float* Jb, double beta, uint64_t seed,
                         uint32_t replica, int64_t t0, int64_t nsweeps, int heatbath,
                         int colours, double* theta, double* E_out, double* absm_out,
                         double tie_tol, int64_t* ties, double* tie_info, int64_t ties_cap)
{
    orc_geom g = orc_make_geom(d, L);
    const uint32_t key[2] = {orc_key_lo(seed), orc_key_hi(seed)};
    const int Lz = d == 3 ? L : 1;
    int64_t nties = 0;
    for (int64_t step = 0; step < nsweeps; ++step) {
        int64_t t = t0 + step;
        for (int c = 0; c < 2; ++c)
            for (int z = 0; z < Lz && ((colours >> c) & 1); ++z)
                for (int y = 0; y < L; ++y)
                    for (int x0 = (c + y + z) & 1; x0 < L; x0 += 2) {
                        int x[3] = {x0, y, z};
                        int64_t i = orc_index(&g, x);
                        int64_t j = i >> 1;
                        double hx = 0.0, hy = 0.0, jsum = 0.0;
                        for (int k = 0; k < 2 * d; ++k) {
                            int64_t nb = orc_neighbour_at(&g, x, k);
                            double jij = bond_j(&g, J, Jb, x, i, k);
                            hx += jij * cos(theta[nb]);
                            hy += jij * sin(theta[nb]);
                            jsum += fabs(jij);
                        }
                        if (heatbath) {
                            int tie = 0;
                            xy_heatbath_draw(hx, hy, beta, key, (uint32_t)(j >> 1), (uint32_t)t,
                                             replica, c, (int)(j & 1), tie_tol, &tie, theta + i);
                            if (tie) log_tie(&nties, ties, ties_cap, t, i);
                            continue;
                        }
                        uint32_t ctr[4] = {(uint32_t)(j >> 1), (uint32_t)t, replica,
                                           (uint32_t)(ORC_SWEEP << 1 | c)};
                        uint32_t out[4];
                        orc_philox4x32_10(ctr, key, out);
                        double u = orc_u24(out[2 * (j & 1)]);
                        double th_new = TWO_PI * orc_u24(out[2 * (j & 1) + 1]);
                        double dE = -((cos(th_new) - cos(theta[i])) * hx +
                                      (sin(th_new) - sin(theta[i])) * hy);
                        int accept = 1;
                        if (dE > 0.0) {
                            double p = exp(-beta * dE);
                            accept = u < p;
                            if (fabs(u - p) < tie_tol) {
                                double A = 2.0 * (fabs(hx) + fabs(hy)) +
                                           (fabs(cos(th_new) - cos(theta[i])) +
                                            fabs(sin(th_new) - sin(theta[i]))) * jsum;
                                log_tie_info(&nties, ties, tie_info, ties_cap, t, i, fabs(u - p),
                                             p * (beta * (A + fabs(dE)) + 1.0));
                            }
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

int64_t orc_xy_sweeps(int d, int L, double J, const float* Jb, double beta,
                      uint64_t seed, uint32_t replica, int64_t t0, int64_t nsweeps,
                      double* theta, double* E_out, double* absm_out,
                      double tie_tol, int64_t* ties, double* tie_info, int64_t ties_cap)
{
    return xy_sweeps(d, L, J, Jb, beta, seed, replica, t0, nsweeps, 0, 3, theta, E_out,
                     absm_out, tie_tol, ties, tie_info, ties_cap);
}

int64_t orc_xy_heatbath_sweeps(int d, int L, double J, const float* Jb, double beta,
                               uint64_t seed, uint32_t replica, int64_t t0, int64_t nsweeps,
                               int colours, double* theta, double* E_out, double* absm_out,
                               double tie_tol, int64_t* ties, int64_t ties_cap)
{
    return xy_sweeps(d, L, J, Jb, beta, seed, replica, t0, nsweeps, 1, colours, theta, E_out,
                     absm_out, tie_tol, ties, NULL, ties_cap);
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

/* Heat-bath draw of one Heisenberg spin in the field h from the uniforms u
 * (for c = s'.h/|h|) and v (azimuth); returns |h_z| / |h| (1 for h = 0,
 * whose basis is fixed). */
static double heis_heatbath_draw(const double h[3], double beta, double u, double v,
                                 double sn[3])
{
    const double H = sqrt(h[0] * h[0] + h[1] * h[1] + h[2] * h[2]);
    double n[3] = {0.0, 0.0, 1.0};
    double omc, opc;  /* 1 - c, 1 + c */
    const double kappa = beta * H;
    if (H > 0.0)
        for (int a = 0; a < 3; ++a) n[a] = h[a] / H;
    if (kappa > 0.0) {
        omc = -log1p((1.0 - u) * expm1(-2.0 * kappa)) / kappa;
        if (omc <= 1.0) {
            opc = 2.0 - omc;
        } else {
            /* where expm1 overflows, log1p(u e^{2 kappa}) = log(u) + 2 kappa */
            opc = 2.0 * kappa < 700.0 ? log1p(u * expm1(2.0 * kappa)) / kappa
                                      : fmax(0.0, 2.0 + log(u) / kappa);
            omc = 2.0 - opc;
        }
    } else {
        omc = 2.0 * (1.0 - u);
        opc = 2.0 * u;
    }
    if (omc < 0.0) omc = 0.0;
    if (opc < 0.0) opc = 0.0;
    const double c = omc <= 1.0 ? 1.0 - omc : opc - 1.0;
    const double r = sqrt(omc * opc);
    /* orthonormal basis (e1, e2, n), Duff et al. 2017 */
    const double sg = copysign(1.0, n[2]);
    const double a = -1.0 / (sg + n[2]);
    const double b = n[0] * n[1] * a;
    const double e1[3] = {1.0 + sg * n[0] * n[0] * a, sg * b, -sg * n[0]};
    const double e2[3] = {b, sg + n[1] * n[1] * a, -n[1]};
    const double phi = TWO_PI * v;
    const double cp = cos(phi), sp = sin(phi);
    for (int k = 0; k < 3; ++k) sn[k] = c * n[k] + r * (cp * e1[k] + sp * e2[k]);
    return fabs(n[2]);
}

static int64_t heis_sweeps(int d, int L, double J, const float* Jb, double beta, uint64_t seed,
                           uint32_t replica, int64_t t0, int64_t nsweeps, int heatbath,
                           int colours, int renorm_every, double* s, double* E_out,
                           double* absm_out, double tie_tol, int64_t* ties, double* tie_info,
                           int64_t ties_cap)
{
    orc_geom g = orc_make_geom(d, L);
    const uint32_t key[2] = {orc_key_lo(seed), orc_key_hi(seed)};
    const int Lz = d == 3 ? L : 1;
    int64_t nties = 0;
    for (int64_t step = 0; step < nsweeps; ++step) {
        int64_t t = t0 + step;
        int renorm = renorm_every > 0 && (t + 1) % renorm_every == 0;
        for (int c = 0; c < 2; ++c)
            for (int z = 0; z < Lz && ((colours >> c) & 1); ++z)
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
                        double h[3] = {0.0, 0.0, 0.0};
                        double jsum = 0.0;
                        for (int k = 0; k < 2 * d; ++k) {
                            int64_t nb = orc_neighbour_at(&g, x, k);
                            double jij = bond_j(&g, J, Jb, x, i, k);
                            for (int a = 0; a < 3; ++a) h[a] += jij * s[3 * nb + a];
                            jsum += fabs(jij);
                        }
                        int accept = 1;
                        if (heatbath) {
                            if (heis_heatbath_draw(h, beta, u, orc_u24(out[1]), sn) < tie_tol)
                                log_tie(&nties, ties, ties_cap, t, i);
                        } else {
                            sphere_point(out[1], out[2], sn);
                        }
                        double dE = 0.0;
                        for (int a = 0; a < 3; ++a) dE -= (sn[a] - s[3 * i + a]) * h[a];
                        if (!heatbath && dE > 0.0) {
                            double p = exp(-beta * dE);
                            accept = u < p;
                            if (fabs(u - p) < tie_tol) {
                                double A = 0.0;
                                for (int a = 0; a < 3; ++a)
                                    A += 2.0 * fabs(h[a]) + fabs(sn[a] - s[3 * i + a]) * jsum;
                                log_tie_info(&nties, ties, tie_info, ties_cap, t, i, fabs(u - p),
                                             p * (beta * (A + fabs(dE)) + 1.0));
                            }
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

int64_t orc_heis_sweeps(int d, int L, double J, const float* Jb, double beta,
                        uint64_t seed, uint32_t replica, int64_t t0, int64_t nsweeps,
                        int renorm_every, double* s, double* E_out, double* absm_out,
                        double tie_tol, int64_t* ties, double* tie_info, int64_t ties_cap)
{
    return heis_sweeps(d, L, J, Jb, beta, seed, replica, t0, nsweeps, 0, 3, renorm_every, s,
                       E_out, absm_out, tie_tol, ties, tie_info, ties_cap);
}

int64_t orc_heis_heatbath_sweeps(int d, int L, double J, const float* Jb, double beta,
                                 uint64_t seed, uint32_t replica, int64_t t0, int64_t nsweeps,
                                 int colours, int renorm_every, double* s, double* E_out,
                                 double* absm_out, double tie_tol, int64_t* ties,
                                 int64_t ties_cap)
{
    return heis_sweeps(d, L, J, Jb, beta, seed, replica, t0, nsweeps, 1, colours, renorm_every, s,
                       E_out, absm_out, tie_tol, ties, NULL, ties_cap);
}
