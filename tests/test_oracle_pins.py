"""Pins of the CPU oracle to things other than itself (no GPU).

Each test ties one part of the oracle to a library routine, a closed form, an
exact enumeration or an invariant of the method (Weigel & Yavors'kii 2011,
Section 2: Eq. 1, Eq. 2, checkerboard order), chosen so that a dropped term,
a wrong sign or index, or a swapped colour order fails at least one of them.
Statistical checks run from fixed seeds, so they are deterministic.
"""
import ctypes
import ctypes.util
import math

import numpy as np
import pytest
from scipy import stats

import oracle
from paper_1107_5463_gb300 import inputs
from tests import exact

BETA_C = inputs.BETA_C_2D_ISING


# ------------------------------------------------------------- Philox ----

def _curand():
    for name in ("libcurand.so.10", "libcurand.so", ctypes.util.find_library("curand")):
        if not name:
            continue
        try:
            return ctypes.CDLL(name)
        except OSError:
            continue
    pytest.skip("cuRAND not available")


def _curand_host_philox(lib, seed, first_block, nblocks):
    """nblocks x 4 outputs of cuRAND's host Philox4_32_10 generator."""
    gen = ctypes.c_void_p()
    assert lib.curandCreateGeneratorHost(ctypes.byref(gen), 161) == 0  # PHILOX4_32_10
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        assert lib.curandSetGeneratorOffset(gen, ctypes.c_ulonglong(4 * first_block)) == 0
        buf = (ctypes.c_uint32 * (4 * nblocks))()
        assert lib.curandGenerate(gen, buf, 4 * nblocks) == 0
    finally:
        lib.curandDestroyGenerator(gen)
    return np.frombuffer(buf, np.uint32).reshape(nblocks, 4).copy()


@pytest.mark.parametrize("seed", [0, 1, 0xFFFFFFFF, 1 << 32, inputs.DEFAULT_SEED, 2**64 - 1])
def test_philox_matches_curand_host_generator(seed):
    """cuRAND's host Philox4_32_10 generator (a library routine) emits block B
    as Philox4x32-10 of counter (B >> 16, B >> 48, B & 0xffff, 0) under key
    (seed_lo, seed_hi); the oracle must reproduce it.  Blocks with non-zero
    words 0, 1 and 2 are covered, so each counter word and both key words
    reach the check."""
    lib = _curand()
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for first in (0, 65536 * 5 + 7, (3 << 48) + (11 << 16) + 65530):
        got = _curand_host_philox(lib, seed, first, 12)
        for b in range(12):
            B = first + b
            ctr = [(B >> 16) & 0xFFFFFFFF, B >> 48, B & 0xFFFF, 0]
            np.testing.assert_array_equal(oracle.philox4x32_10(ctr, key), got[b])


def test_philox_is_a_bijection_on_sampled_counters():
    """Distinct counters give distinct outputs (Philox is a bijection for a
    fixed key) and one flipped input bit changes about half the output bits."""
    key = [0x1234, 0x5678]
    rng = np.random.default_rng(7)
    ctrs = rng.integers(0, 2**32, size=(2000, 4), dtype=np.uint64).astype(np.uint32)
    outs = {tuple(oracle.philox4x32_10(c, key)) for c in ctrs}
    assert len(outs) == len({tuple(c) for c in ctrs})
    flips = []
    for c in ctrs[:200]:
        a = oracle.philox4x32_10(c, key)
        c2 = c.copy()
        c2[rng.integers(4)] ^= np.uint32(1 << int(rng.integers(32)))
        b = oracle.philox4x32_10(c2, key)
        flips.append(sum(bin(int(x) ^ int(y)).count("1") for x, y in zip(a, b)))
    assert abs(np.mean(flips) - 64) < 3


# ------------------------------------------------------------ energy ----

@pytest.mark.parametrize("d,L", [(2, 2), (2, 6), (3, 2), (3, 4)])
def test_ising_measure_matches_roll_energy(d, L):
    s = inputs.ising_spins(d, L, 11)
    jb = inputs.ising_bonds(d, L, 12, p_zero=0.2)
    for J, bonds in ((1.0, None), (-0.7, jb)):
        E, M = oracle.ising_measure(d, L, s, J=J, Jb=bonds)
        assert E == pytest.approx(exact.roll_energy(s, d, L, J, bonds), abs=1e-12)
        assert M == s.sum()


@pytest.mark.parametrize("d,L,rows", [(2, 10, 3), (2, 8, 512), (3, 6, 4), (3, 4, 1)])
def test_chunked_energy_matches_roll_energy(d, L, rows):
    """The slab-wise energy used at the largest sizes equals the whole-array
    roll energy."""
    s = inputs.ising_spins(d, L, 7)
    assert exact.chunked_energy(s, d, L, rows) == exact.roll_energy(s, d, L)


@pytest.mark.parametrize("d", [2, 3])
def test_ising_measure_special_states(d):
    L = 4
    N = L ** d
    up = np.ones(N, np.int8)
    assert oracle.ising_measure(d, L, up)[0] == -d * N
    neel = (1 - 2 * exact.colour_of_site(d, L)).astype(np.int8)
    assert oracle.ising_measure(d, L, neel)[0] == d * N
    one = up.copy()
    one[5] = -1
    assert oracle.ising_measure(d, L, one)[0] == -d * N + 4 * d


@pytest.mark.parametrize("d,L", [(2, 4), (3, 2)])
def test_continuous_measure_matches_roll_energy(d, L):
    th = inputs.angles(d, L, 3)
    jbf = inputs.float_bonds(d, L, 4)
    E, M = oracle.xy_measure(d, L, th, J=0.9, Jb=jbf)
    v = np.stack([np.cos(th), np.sin(th)], axis=1)
    assert E == pytest.approx(exact.roll_energy(v, d, L, 0.9, jbf.astype(np.float64)), abs=1e-12)
    np.testing.assert_allclose(M, v.sum(axis=0), atol=1e-12)
    s = inputs.unit_vectors(d, L, 5)
    E, M = oracle.heis_measure(d, L, s, J=1.3, Jb=jbf)
    assert E == pytest.approx(exact.roll_energy(s, d, L, 1.3, jbf.astype(np.float64)), abs=1e-12)
    np.testing.assert_allclose(M, s.sum(axis=0), atol=1e-12)


# ---------------------------------------------- exact small lattices ----

def test_ising_4x4_equilibrium_matches_enumeration():
    """<E>, <E^2>, <|m|> of the 4x4 torus at beta_c from all 2^16 states; the
    oracle's Metropolis chain must agree within 3 sigma (binning errors)."""
    ex = exact.enumerate_ising(2, 4, BETA_C)
    s = oracle.ising_init(2, 4, 99)
    E, m = oracle.ising_sweeps(2, 4, s, BETA_C, 99, 0, 200_000)
    E, m = E[1000:], m[1000:]
    for obs, ref in ((E, ex["E"]), (E * E, ex["E2"]), (m, ex["absm"])):
        mean, err = exact.binned_mean(obs, 40)
        assert abs(mean - ref) < 3 * err, (mean, ref, err)


def _chi2_rows(counts, T, rows):
    """Pooled chi-square p-value over the given rows; cells with an expected
    count below 5 are lumped into one cell per row."""
    chi2, dof = 0.0, 0
    for a in rows:
        n = counts[a].sum()
        expct = n * T[a]
        assert counts[a][expct == 0].sum() == 0, "transition with zero exact probability"
        big = expct >= 5
        obs = list(counts[a][big])
        exp_ = list(expct[big])
        if (~big).any() and expct[~big].sum() > 0:
            obs.append(counts[a][~big].sum())
            exp_.append(expct[~big].sum())
        obs, exp_ = np.array(obs), np.array(exp_)
        chi2 += ((obs - exp_) ** 2 / exp_).sum()
        dof += len(obs) - 1
    return stats.chi2.sf(chi2, dof)


@pytest.mark.parametrize("d,beta", [(2, 0.15), (3, 0.1)])
def test_one_sweep_transition_matrix_on_L2(d, beta):
    """Exact matrix of one sweep (colour 0 then colour 1, each site of a colour
    flipped independently with min[1, e^{-beta dE}], dE from the full Eq. 1)
    against the oracle's empirical transitions.  T0 and T1 each satisfy
    detailed balance and the Boltzmann weights are stationary under T0 T1."""
    L = 2
    T0, T1, S, E = exact.exact_sweep_matrix(d, L, beta)
    pi = np.exp(-beta * E)
    pi /= pi.sum()
    for T in (T0, T1):
        np.testing.assert_allclose(pi[:, None] * T, (pi[:, None] * T).T, atol=1e-14)
    T = T0 @ T1
    np.testing.assert_allclose(pi @ T, pi, atol=1e-14)
    if d == 2:
        assert np.abs(T0 @ T1 - T1 @ T0).max() > 1e-3  # the colour order is visible
    index = {tuple(s): k for k, s in enumerate(S)}
    nst = len(S)
    rows = range(nst) if d == 2 else range(0, nst, 37)
    reps = 3000
    counts = np.zeros((nst, nst))
    for a in rows:
        for r in range(reps):
            s = S[a].copy()
            oracle.ising_sweeps(d, L, s, beta, 1234, r, 1, series=False)
            counts[a, index[tuple(s)]] += 1
    assert _chi2_rows(counts, T, rows) > 1e-4


@pytest.mark.slow
def test_kaufman_energy_tends_to_onsager():
    """Kaufman's exact finite-torus energy per site at beta_c approaches
    Onsager's critical energy -sqrt(2) with a 1/L correction: (E + sqrt 2) L
    is the same for L = 64, 256 and 1024, and E(1024) is within 7e-4 of
    -sqrt(2).  With the L = 64 chain below this ties the oracle to Onsager's
    value."""
    prods = [(exact.kaufman_energy_per_site(BETA_C, L) + math.sqrt(2)) * L
             for L in (64, 256, 1024)]
    assert max(prods) - min(prods) < 1e-3, prods
    assert abs(exact.kaufman_energy_per_site(BETA_C, 1024) + math.sqrt(2)) < 7e-4


def test_ising_L64_energy_matches_kaufman():
    """The 2D Ising workload of side 64 at beta_c = ln(1+sqrt2)/2, 4 x 10^4
    sweeps from a random start: mean energy per site against Kaufman's exact
    finite-torus value (about -1.4239; Onsager's -sqrt(2) is the L -> infinity
    limit)."""
    L = 64
    ref = exact.kaufman_energy_per_site(BETA_C, L)
    assert -1.43 < ref < -1.42
    s = oracle.ising_init(2, L, inputs.DEFAULT_SEED)
    E, _ = oracle.ising_sweeps(2, L, s, BETA_C, inputs.DEFAULT_SEED, 0, 40_000)
    mean, err = exact.binned_mean(E[2000:] / L**2, 16)
    assert abs(mean - ref) < 3 * err, (mean, ref, err)
    assert err < 5e-3


# ---------------------------------------------------- two-spin laws ----

@pytest.mark.parametrize("n,beta", [(1, 0.8), (2, 1.3), (3, 1.7)])
def test_two_spin_bond_distribution(n, beta):
    """A 4x4 lattice whose only non-zero coupling joins sites 0 and 1: the bond
    variable x = s_0 . s_1 = -E must follow p(x) ~ e^{beta x}(1-x^2)^{(n-3)/2}
    (mean tanh, I1/I0, Langevin) and, for n = 2, 3, its full CDF (KS test)."""
    d, L = 2, 4
    jb = inputs.two_spin_bonds(d, L, 0, 0)
    nsw = 60_000
    if n == 1:
        s = oracle.ising_init(d, L, 5)
        E, _ = oracle.ising_sweeps(d, L, s, beta, 6, 0, nsw, Jb=jb)
    elif n == 2:
        th = oracle.xy_init(d, L, 5)
        E, _, _, _ = oracle.xy_sweeps(d, L, th, beta, 6, 0, nsw, Jb=jb.astype(np.float32))
    else:
        s = oracle.heis_init(d, L, 5)
        E, _, _, _ = oracle.heis_sweeps(d, L, s, beta, 6, 0, nsw, Jb=jb.astype(np.float32))
    x = -E[100:]
    mean, err = exact.binned_mean(x, 50)
    assert abs(mean - exact.two_spin_mean(n, beta)) < 3 * err, (mean, err)
    if n > 1:
        sample = x[::10][:2000]
        assert stats.kstest(sample, exact.two_spin_cdf(n, beta)).pvalue > 1e-3


# ------------------------------------------------------ limiting beta ----

@pytest.mark.parametrize("d", [2, 3])
def test_beta_zero_accepts_every_move(d):
    """At beta = 0 every proposal is accepted: every Ising spin flips and every
    continuous spin becomes its proposal, which is the Philox stream itself."""
    L, seed, t = 4, 77, 5
    N = L ** d
    s0 = inputs.ising_spins(d, L, 1)
    s = s0.copy()
    oracle.ising_sweeps(d, L, s, 0.0, seed, t, 1, series=False)
    np.testing.assert_array_equal(s, -s0)

    key = [seed & 0xFFFFFFFF, seed >> 32]
    colour = exact.colour_of_site(d, L)
    u24 = lambda x: (int(x) >> 8) * 2.0**-24
    th = inputs.angles(d, L, 2)
    oracle.xy_sweeps(d, L, th, 0.0, seed, t, 1, series=False)
    v = inputs.unit_vectors(d, L, 3)
    oracle.heis_sweeps(d, L, v, 0.0, seed, t, 1, renorm_every=0, series=False)
    for i in range(N):
        j, c = i >> 1, int(colour[i])
        out = oracle.philox4x32_10([j >> 1, t, 0, c], key)
        assert th[i] == 2 * math.pi * u24(out[2 * (j & 1) + 1])
        out = oracle.philox4x32_10([j, t, 0, c], key)
        z = 2 * u24(out[1]) - 1
        phi = 2 * math.pi * u24(out[2])
        r = math.sqrt(1 - z * z)
        np.testing.assert_allclose(v[i], [r * math.cos(phi), r * math.sin(phi), z], atol=1e-15)


@pytest.mark.parametrize("d", [2, 3])
def test_large_beta_never_raises_energy(d):
    """With beta large, no move with dE > 0 is accepted: the ordered Ising
    ground state survives and continuous-spin energies never increase."""
    L = 6
    up = np.ones(L ** d, np.int8)
    oracle.ising_sweeps(d, L, up, 40.0, 3, 0, 50, series=False)
    assert (up == 1).all()
    th = inputs.angles(d, L, 8)
    E, _, _, _ = oracle.xy_sweeps(d, L, th, 1e12, 3, 0, 30)
    assert (np.diff(E) <= 1e-8).all()
    assert E[-1] < E[0]
    v = inputs.unit_vectors(d, L, 9)
    E, _, _, _ = oracle.heis_sweeps(d, L, v, 1e12, 3, 0, 30)
    assert (np.diff(E) <= 1e-8).all()
    assert E[-1] < E[0]


# ------------------------------------------------------- bookkeeping ----

@pytest.mark.parametrize("d,L", [(2, 6), (2, 8), (3, 4)])
def test_series_matches_recomputed_state(d, L):
    """The series after the last sweep equals Eq. 1 recomputed by rolls; the
    2D energy is 2N mod 4 (unsatisfied bonds come in even numbers on a torus);
    sweeps a then b equal a + b sweeps (the stream is keyed by sweep index)."""
    s = oracle.ising_init(d, L, 4)
    s2 = s.copy()
    E, m = oracle.ising_sweeps(d, L, s, 0.3, 9, 0, 20)
    assert E[-1] == exact.roll_energy(s, d, L)
    assert m[-1] == abs(int(s.astype(np.int64).sum())) / L**d
    if d == 2:
        assert all(int(e) % 4 == (2 * L * L) % 4 for e in E)
    oracle.ising_sweeps(d, L, s2, 0.3, 9, 0, 7, series=False)
    oracle.ising_sweeps(d, L, s2, 0.3, 9, 7, 13, series=False)
    np.testing.assert_array_equal(s, s2)


def test_heisenberg_renormalisation_keeps_unit_length():
    d, L = 3, 4
    v = inputs.unit_vectors(d, L, 1) * 1.5
    oracle.heis_sweeps(d, L, v, 0.7, 2, 15, 1, renorm_every=16, series=False)
    np.testing.assert_allclose(np.linalg.norm(v, axis=1), 1.0, atol=1e-14)


# ---------------------------------------------------------- EA + PT ----

def test_ea_couplings_are_balanced_pm1():
    jb = oracle.ea_couplings(3, 16, 5, 0)
    assert set(np.unique(jb)) == {-1, 1}
    p = (jb == 1).mean()
    assert abs(p - 0.5) < 3 * math.sqrt(0.25 / jb.size)
    assert not np.array_equal(jb, oracle.ea_couplings(3, 16, 5, 1))


def test_exchange_with_equal_betas_always_swaps():
    """Delta = 0 when all temperatures are equal, so every attempted pair
    swaps: the labels follow the fixed even/odd transposition pattern."""
    d, L, nt = 3, 2, 5
    jb = oracle.ea_couplings(d, L, 1, 0)
    spins = np.stack([oracle.ising_init(d, L, 1, r) for r in range(nt)])
    perm = np.arange(nt, dtype=np.int32)
    expect = list(range(nt))
    for t in range(6):
        oracle.ea_pt_sweeps(d, L, jb, [0.4] * nt, 2, 0, t, 1, spins, perm)
        for k in range(t % 2, nt - 1, 2):
            expect[k], expect[k + 1] = expect[k + 1], expect[k]
        assert list(perm) == expect


def test_exchange_keeps_canonical_energies_on_L2_sample():
    """Replica exchange must leave each temperature canonical: the mean energy
    at every beta of a 3D L = 2 EA sample (256 states, enumerated exactly)
    agrees with the exact value within 3 sigma."""
    d, L = 3, 2
    jb = oracle.ea_couplings(d, L, 21, 3)
    betas = np.array([0.2, 0.45, 0.8, 1.4])
    spins = np.stack([oracle.ising_init(d, L, 21, 3 * 4 + r) for r in range(4)])
    perm = np.arange(4, dtype=np.int32)
    E = oracle.ea_pt_sweeps(d, L, jb, betas, 22, 3, 0, 200_000, spins, perm)
    assert sorted(perm) == [0, 1, 2, 3]
    for k, b in enumerate(betas):
        ex = exact.enumerate_ising(d, L, b, Jb=jb.astype(np.int64))
        mean, err = exact.binned_mean(E[1000:, k], 40)
        assert abs(mean - ex["E"]) < 3 * err, (k, mean, ex["E"], err)


# ------------------------------------------------------------ heat-bath --

@pytest.mark.parametrize("d,beta", [(2, 0.15), (2, 0.6)])
def test_heatbath_transition_matrix_on_L2(d, beta):
    """Exact one-sweep matrix of the heat-bath rule (each site of a colour set
    to its flipped value with probability e^{-beta E'}/(e^{-beta E}+e^{-beta
    E'}), energies from Eq. 1) against the oracle's empirical transitions;
    the Boltzmann law is stationary and each half-sweep is reversible."""
    L = 2
    T0, T1, S, E = exact.exact_sweep_matrix(d, L, beta, heatbath=True)
    pi = np.exp(-beta * E)
    pi /= pi.sum()
    for T in (T0, T1):
        np.testing.assert_allclose(pi[:, None] * T, (pi[:, None] * T).T, atol=1e-14)
    T = T0 @ T1
    np.testing.assert_allclose(pi @ T, pi, atol=1e-14)
    M0, M1, _, _ = exact.exact_sweep_matrix(d, L, beta)
    assert np.abs(T - M0 @ M1).max() > 1e-3  # a different chain from Metropolis
    index = {tuple(s): k for k, s in enumerate(S)}
    counts = np.zeros((len(S), len(S)))
    for a in range(len(S)):
        for r in range(3000):
            s = S[a].copy()
            oracle.ising_heatbath_sweeps(d, L, s, beta, 4321, r, 1, series=False)
            counts[a, index[tuple(s)]] += 1
    assert _chi2_rows(counts, T, range(len(S))) > 1e-4


def test_heatbath_4x4_equilibrium_matches_enumeration():
    ex = exact.enumerate_ising(2, 4, BETA_C)
    s = oracle.ising_init(2, 4, 7)
    E, m = oracle.ising_heatbath_sweeps(2, 4, s, BETA_C, 8, 0, 200_000)
    E, m = E[1000:], m[1000:]
    for obs, ref in ((E, ex["E"]), (E * E, ex["E2"]), (m, ex["absm"])):
        mean, err = exact.binned_mean(obs, 40)
        assert abs(mean - ref) < 3 * err, (mean, ref, err)


def test_heatbath_two_spin_bond_and_beta_zero():
    """One bond: <s0 s1> = tanh(beta J).  beta = 0: every spin is +1 exactly
    when its Philox output is below 2^31, independent of the old state."""
    d, L = 2, 4
    jb = inputs.two_spin_bonds(d, L, 0, 0)
    s = oracle.ising_init(d, L, 5)
    E, _ = oracle.ising_heatbath_sweeps(d, L, s, 0.9, 6, 0, 40_000, Jb=jb)
    mean, err = exact.binned_mean(-E[100:], 40)
    assert abs(mean - math.tanh(0.9)) < 3 * err
    seed, t = 31, 4
    s = inputs.ising_spins(d, L, 3)
    oracle.ising_heatbath_sweeps(d, L, s, 0.0, seed, t, 1, series=False)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    colour = exact.colour_of_site(d, L)
    for i in range(L ** d):
        j = i >> 1
        out = oracle.philox4x32_10([j >> 2, t, 0, int(colour[i])], key)
        assert s[i] == (1 if int(out[j & 3]) < 2**31 else -1)


# ------------------------------------------- continuous-spin heat-bath --

def _perp_basis(n):
    """Any orthonormal pair perpendicular to the unit vector n (numpy)."""
    a = np.array([1.0, 0.0, 0.0]) if abs(n[0]) < 0.9 else np.array([0.0, 1.0, 0.0])
    e1 = np.cross(n, a)
    e1 /= np.linalg.norm(e1)
    return e1, np.cross(n, e1)


@pytest.mark.parametrize("kappa", [0.3, 2.5, 15.0])
def test_xy_heatbath_draws_the_von_mises_conditional(kappa):
    """One heat-bath sweep from a fixed state, repeated over 3000 seeds: the
    new angle of a colour-0 site minus the angle of its (fixed) local field
    follows the von Mises law with concentration beta |h| (scipy's CDF)."""
    d, L = 2, 4
    th0 = inputs.angles(d, L, 8)
    N = L * L
    nb = [exact.neighbour(d, L, 0, k) for k in range(4)]
    hx, hy = sum(math.cos(th0[q]) for q in nb), sum(math.sin(th0[q]) for q in nb)
    beta = kappa / math.hypot(hx, hy)
    offs = np.empty(3000)
    for sd in range(offs.size):
        th = th0.copy()
        oracle.xy_sweeps(d, L, th, beta, 1000 + sd, 0, 1, heatbath=True, series=False)
        offs[sd] = (th[0] - math.atan2(hy, hx) + math.pi) % (2 * math.pi) - math.pi
        assert 0.0 <= th[N - 1] < 2 * math.pi
    assert stats.kstest(offs, stats.vonmises(kappa).cdf).pvalue > 1e-3
    assert abs(np.mean(np.cos(offs)) - exact.two_spin_mean(2, kappa)) < 4 / math.sqrt(offs.size)


@pytest.mark.parametrize("kappa", [0.3, 2.5, 15.0])
def test_heisenberg_heatbath_draws_the_exponential_conditional(kappa):
    """As above for a Heisenberg site: c = s'.h/|h| has the distribution
    function (e^{kappa (c+1)} - 1) / (e^{2 kappa} - 1), the azimuth about h
    is uniform, and the new spin has unit length."""
    d, L = 3, 4
    s0 = inputs.unit_vectors(d, L, 9)
    nb = [exact.neighbour(d, L, 0, k) for k in range(6)]
    h = s0[nb].sum(axis=0)
    H = np.linalg.norm(h)
    n = h / H
    e1, e2 = _perp_basis(n)
    beta = kappa / H
    cs, phis = np.empty(3000), np.empty(3000)
    for sd in range(cs.size):
        s = s0.copy()
        oracle.heis_sweeps(d, L, s, beta, 1000 + sd, 0, 1, renorm_every=0, heatbath=True,
                           series=False)
        v = s[0]
        assert abs(np.linalg.norm(v) - 1.0) < 1e-12
        cs[sd] = v @ n
        phis[sd] = math.atan2(v @ e2, v @ e1)
    cdf = lambda c: np.expm1(kappa * (np.asarray(c) + 1)) / math.expm1(2 * kappa)
    assert stats.kstest(cs, cdf).pvalue > 1e-3
    assert stats.kstest(phis, stats.uniform(-math.pi, 2 * math.pi).cdf).pvalue > 1e-3


@pytest.mark.parametrize("n", [2, 3])
def test_continuous_heatbath_two_spin_bond(n):
    """The single-bond lattice under heat-bath sweeps: the bond variable
    follows the exact two-spin law (mean and KS), as under Metropolis; every
    other site has h = 0 and is redrawn uniformly."""
    d, L, beta = 2, 4, 1.4
    jb = inputs.two_spin_bonds(d, L, 0, 0).astype(np.float32)
    nsw = 40_000
    if n == 2:
        th = oracle.xy_init(d, L, 5)
        E, _, _, _ = oracle.xy_sweeps(d, L, th, beta, 6, 0, nsw, Jb=jb, heatbath=True)
    else:
        s = oracle.heis_init(d, L, 5)
        E, _, _, _ = oracle.heis_sweeps(d, L, s, beta, 6, 0, nsw, Jb=jb, heatbath=True)
    x = -E[10:]
    mean, err = exact.binned_mean(x, 50)
    assert abs(mean - exact.two_spin_mean(n, beta)) < 3 * err, (mean, err)
    assert stats.kstest(x[::7][:3000], exact.two_spin_cdf(n, beta)).pvalue > 1e-3


def test_continuous_heatbath_at_beta_zero_is_uniform():
    """beta = 0: every new XY angle is uniform on the circle and every new
    Heisenberg spin uniform on the sphere (z uniform on [-1, 1], azimuth
    uniform), whatever the old state."""
    th = np.zeros(64 * 64)
    oracle.xy_sweeps(2, 64, th, 0.0, 3, 0, 1, heatbath=True, series=False)
    assert stats.kstest(th, stats.uniform(0, 2 * math.pi).cdf).pvalue > 1e-3
    s = np.tile([0.0, 0.0, 1.0], (16 ** 3, 1))
    oracle.heis_sweeps(3, 16, s, 0.0, 3, 0, 1, heatbath=True, series=False)
    assert stats.kstest(s[:, 2], stats.uniform(-1, 2).cdf).pvalue > 1e-3
    assert stats.kstest(np.arctan2(s[:, 1], s[:, 0]),
                        stats.uniform(-math.pi, 2 * math.pi).cdf).pvalue > 1e-3


@pytest.mark.parametrize("n", [2, 3])
def test_continuous_heatbath_colour_passes_compose_to_sweeps(n):
    """The pass of colour 0 followed by the pass of colour 1 (same sweep
    index) is exactly one whole sweep, and a pass touches only its colour."""
    d, L, beta = 3, 4, 0.9
    init = oracle.xy_init if n == 2 else oracle.heis_init
    run = oracle.xy_sweeps if n == 2 else oracle.heis_sweeps
    a, b = init(d, L, 3), init(d, L, 3)
    run(d, L, a, beta, 5, 7, 1, heatbath=True, series=False)
    start = b.copy()
    run(d, L, b, beta, 5, 7, 1, heatbath=True, series=False, colours=1)
    colour = exact.colour_of_site(d, L)
    np.testing.assert_array_equal(b[colour == 1], start[colour == 1])
    assert (b[colour == 0] != start[colour == 0]).any()
    run(d, L, b, beta, 5, 7, 1, heatbath=True, series=False, colours=2)
    np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("n,d,L,beta", [(2, 2, 8, 1.12), (3, 3, 4, 0.693)])
def test_continuous_heatbath_and_metropolis_agree_in_equilibrium(n, d, L, beta):
    """Both rules leave the Boltzmann law invariant: their mean energies on
    the same lattice agree within three combined standard errors."""
    nsw = 30_000
    res = []
    for hb in (False, True):
        if n == 2:
            st = oracle.xy_init(d, L, 11)
            E, _, _, _ = oracle.xy_sweeps(d, L, st, beta, 12, 0, nsw, heatbath=hb)
        else:
            st = oracle.heis_init(d, L, 11)
            E, _, _, _ = oracle.heis_sweeps(d, L, st, beta, 12, 0, nsw, heatbath=hb)
        res.append(exact.binned_mean(E[2000:] / L ** d, 40))
    (m0, e0), (m1, e1) = res
    assert abs(m0 - m1) < 3 * math.hypot(e0, e1), res
    assert max(e0, e1) < 1e-2


@pytest.mark.parametrize("d,L,heatbath,J", [(2, 6, False, 1.0), (3, 4, False, -0.7),
                                             (2, 8, True, 1.0), (3, 4, True, 1.3)])
def test_site_updates_reproduce_a_sweep(d, L, heatbath, J):
    """The single-site update, fed the configuration each colour's pass sees
    (colour 0: the state before the sweep; colour 1: after the colour-0
    pass), gives every site of one oracle sweep, on random +-1 couplings."""
    beta, seed, t = 0.4, 21, 5
    jb = inputs.ising_bonds(d, L, 3)
    before = inputs.ising_spins(d, L, 4)
    after = before.copy()
    sweep = oracle.ising_heatbath_sweeps if heatbath else oracle.ising_sweeps
    sweep(d, L, after, beta, seed, t, 1, J=J, Jb=jb, series=False)
    colour = exact.colour_of_site(d, L)
    mid = np.where(colour == 0, after, before).astype(np.int8)
    for c, state in ((0, before), (1, mid)):
        sites = np.flatnonzero(colour == c)
        got = oracle.ising_site_updates(d, L, np.ascontiguousarray(state), sites, beta, seed, t,
                                        J=J, Jb=jb, heatbath=heatbath)
        np.testing.assert_array_equal(got, after[sites])


# ------------------------------------------------------------ multi-hit --

@pytest.mark.parametrize("k,beta", [(1, 0.35), (2, 0.2)])
def test_multihit_one_sweep_distribution_on_4x4(k, beta):
    """The tile schedule of the k-fold multi-hit sweep (tiles of side 2 on the
    4x4 torus): the exact distribution of the state after one sweep from a
    fixed start (all 2^16 states propagated through the tile / hit / colour
    sub-steps) against the oracle's empirical outcomes (chi-square)."""
    d, L, T = 2, 4, 2
    start = inputs.ising_spins(d, L, 12)
    p = exact.multihit_sweep_distribution(d, L, T, k, beta, start)
    assert abs(p.sum() - 1) < 1e-12
    reps = 20000
    counts = np.zeros(p.size)
    weights = 1 << np.arange(L * L)
    for r in range(reps):
        s = start.copy()
        oracle.ising_multihit_sweeps(d, L, T, k, s, beta, 99, r, 1, series=False)
        counts[int(((s < 0) * weights).sum())] += 1
    big = reps * p >= 5
    assert counts[p == 0].sum() == 0, "an outcome with zero exact probability"
    obs = np.append(counts[big], counts[~big].sum())
    exp_ = np.append(reps * p[big], reps * p[~big].sum())
    keep = exp_ > 0
    chi2 = ((obs[keep] - exp_[keep]) ** 2 / exp_[keep]).sum()
    assert stats.chi2.sf(chi2, keep.sum() - 1) > 1e-4
    # a schedule with one tile (the plain checkerboard) is a different chain
    q = exact.multihit_sweep_distribution(d, L, 4, k, beta, start)
    assert np.abs(p - q).max() > 1e-3


def test_multihit_equilibrium_and_beta_zero():
    ex = exact.enumerate_ising(2, 4, BETA_C)
    s = oracle.ising_init(2, 4, 3)
    E, m = oracle.ising_multihit_sweeps(2, 4, 2, 3, s, BETA_C, 4, 0, 60_000)
    for obs, ref in ((E[500:], ex["E"]), (m[500:], ex["absm"])):
        mean, err = exact.binned_mean(obs, 40)
        assert abs(mean - ref) < 3 * err, (mean, ref, err)
    for k in (1, 2, 5):
        s0 = inputs.ising_spins(3, 8, k)
        s = s0.copy()
        oracle.ising_multihit_sweeps(3, 8, 4, k, s, 0.0, 1, 0, 1, series=False)
        np.testing.assert_array_equal(s, s0 * (-1) ** k)


# ------------------------------------------------------ Swendsen-Wang ----

@pytest.mark.parametrize("beta", [0.2, 0.45])
def test_sw_transition_matrix_on_L2(beta):
    """Exact matrix of one Swendsen-Wang update on the 2 x 2 torus (Section 3:
    satisfied bonds activated with 1 - e^{-2 beta J}, connected components by
    scipy, clusters flipped with probability 1/2, summed over all bond
    subsets) satisfies detailed balance for the Boltzmann weights of Eq. 1,
    and the oracle's empirical transitions from every start state follow it."""
    d, L = 2, 2
    T, S, E = exact.exact_sw_matrix(d, L, beta)
    pi = np.exp(-beta * E)
    pi /= pi.sum()
    np.testing.assert_allclose(pi[:, None] * T, (pi[:, None] * T).T, atol=1e-15)
    np.testing.assert_allclose(T.sum(axis=1), 1.0, atol=1e-13)
    codes = {tuple(s): k for k, s in enumerate(S)}
    reps = 4000
    counts = np.zeros((len(S), len(S)))
    for a in range(len(S)):
        for r in range(reps):
            s = S[a].copy()
            oracle.ising_sw_sweeps(d, L, s, beta, 4321, r, 1, series=False)
            counts[a, codes[tuple(s)]] += 1
    assert _chi2_rows(counts, T, range(len(S))) > 1e-4


@pytest.mark.parametrize("d,L,beta", [(2, 16, BETA_C), (3, 6, 0.2216546)])
def test_sw_clusters_are_connected_components(d, L, beta):
    """The last update's clusters are exactly the connected components of its
    active bonds (scipy), each named by its smallest site; active bonds join
    like spins only, a fraction 1 - e^{-2 beta J} of the satisfied bonds is
    active, every cluster flips as a whole, and about half of them flip."""
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import connected_components
    N = L ** d
    A, B = exact.forward_bonds(d, L)
    n_sat = n_act = n_cl = n_flip = 0
    for t in range(6):
        s0 = oracle.ising_init(d, L, 11 + t)
        s = s0.copy()
        _, _, act, lab = oracle.ising_sw_sweeps(d, L, s, beta, 77, t, 1, series=False,
                                                clusters=True)
        on = act.reshape(-1).astype(bool)
        sat = s0[A] == s0[B]
        assert not (on & ~sat).any()
        n_sat += sat.sum()
        n_act += on.sum()
        g = coo_matrix((np.ones(on.sum()), (A[on], B[on])), shape=(N, N))
        ncl, comp = connected_components(g, directed=False)
        cmin = np.full(ncl, N)
        np.minimum.at(cmin, comp, np.arange(N))
        np.testing.assert_array_equal(lab, cmin[comp])
        flipped = (s != s0)
        # a cluster flips as a whole
        per = np.zeros(ncl)
        np.add.at(per, comp, flipped)
        sizes = np.bincount(comp, minlength=ncl)
        assert np.all((per == 0) | (per == sizes))
        n_cl += ncl
        n_flip += (per > 0).sum()
    p = 1.0 - math.exp(-2.0 * beta)
    assert abs(n_act / n_sat - p) < 5 * math.sqrt(p * (1 - p) / n_sat)
    assert abs(n_flip / n_cl - 0.5) < 5 * math.sqrt(0.25 / n_cl)


@pytest.mark.parametrize("d", [2, 3])
def test_sw_beta_zero_and_large_beta(d):
    """beta = 0: no bond is active, every site is its own cluster and flips iff
    the top bit of output 0 of Philox(i, t, replica, 6 << 1) is set.  Large
    beta from the ground state: every bond is active, one cluster named 0
    flips as a whole and the energy stays -d N J."""
    L = 4
    N = L ** d
    s0 = oracle.ising_init(d, L, 5)
    s = s0.copy()
    seed, t, rep = 0x1234_5678_9ABC, 7, 3
    _, _, act, lab = oracle.ising_sw_sweeps(d, L, s, 0.0, seed, t, 1, replica=rep,
                                            series=False, clusters=True)
    assert act.sum() == 0
    np.testing.assert_array_equal(lab, np.arange(N))
    key = [seed & 0xFFFFFFFF, seed >> 32]
    bits = np.array([oracle.philox4x32_10([i, t, rep, 6 << 1], key)[0] >> 31 for i in range(N)])
    np.testing.assert_array_equal(s, np.where(bits == 1, -s0, s0))
    g = np.ones(N, np.int8)
    flips = 0
    for t in range(8):
        E, _, act, lab = oracle.ising_sw_sweeps(d, L, g, 50.0, seed, t, 1, clusters=True)
        assert act.all() and (lab == 0).all()
        assert E[0] == -d * N
        assert abs(int(g.sum())) == N
        flips += g[0] < 0
    assert 0 < flips < 8


def test_sw_equilibrium_matches_enumeration_and_kaufman():
    """Swendsen-Wang chains reach the Boltzmann law of Eq. 1: <E>, <E^2> and
    <|m|> on the 4 x 4 torus at beta_c against exact enumeration, <E> on the
    2 x 2 x 2 torus at beta = 0.3, and <E>/N on the 16 x 16 torus at beta_c
    against Kaufman's exact value (all within 3 binned standard errors)."""
    ex = exact.enumerate_ising(2, 4, BETA_C)
    s = oracle.ising_init(2, 4, 21)
    E, m = oracle.ising_sw_sweeps(2, 4, s, BETA_C, 21, 0, 100_000)
    for obs, ref in ((E, ex["E"]), (E * E, ex["E2"]), (m, ex["absm"])):
        mean, err = exact.binned_mean(obs[100:], 40)
        assert abs(mean - ref) < 3 * err, (mean, ref, err)
    ex3 = exact.enumerate_ising(3, 2, 0.3)
    s = oracle.ising_init(3, 2, 22)
    E, _ = oracle.ising_sw_sweeps(3, 2, s, 0.3, 22, 0, 100_000)
    mean, err = exact.binned_mean(E[100:], 40)
    assert abs(mean - ex3["E"]) < 3 * err, (mean, ex3["E"], err)
    L = 16
    ref = exact.kaufman_energy_per_site(BETA_C, L)
    s = oracle.ising_init(2, L, 23)
    E, _ = oracle.ising_sw_sweeps(2, L, s, BETA_C, 23, 0, 20_000)
    mean, err = exact.binned_mean(E[200:] / L**2, 20)
    assert abs(mean - ref) < 3 * err, (mean, ref, err)


# ------------------------------------------- multicanonical / Wang-Landau ----

def test_exact_dos_methods_agree():
    """The transfer-matrix density of states equals enumeration on 4x4 and
    sums to 2^36 on 6x6; g is symmetric (k <-> N - k by flipping a
    sublattice), g(0) = 2 and level 1 (one broken bond pair) is empty."""
    g4 = exact.ising_dos_enumerated(4)
    np.testing.assert_array_equal(exact.ising_dos_transfer(4), g4)
    g6 = exact.ising_dos_transfer(6)
    assert g6.sum() == 2.0 ** 36
    for g in (g4, g6):
        np.testing.assert_array_equal(g, g[::-1])
        assert g[0] == 2 and g[1] == 0


@pytest.mark.parametrize("klo,khi", [(0, 4), (10, 14), (30, 34), (50, 54), (60, 64)])
def test_walker_init_reaches_window(klo, khi):
    """Start states (8x8): every walker lands inside its window, its level is
    the Eq. 1 energy of its spins, and the bottom (top) window starts in a
    ferromagnetic (Neel) ground state."""
    L = 8
    N = L * L
    for w in range(8):
        wk = oracle.Walker(L, klo, khi, 77, w)
        assert klo <= wk.level <= khi
        E = exact.roll_energy(wk.s, 2, L)
        assert (E + 2 * N) // 4 == wk.level
        if klo == 0:
            assert abs(int(wk.s.sum())) == N
        if khi == N:
            x, y = np.meshgrid(np.arange(L), np.arange(L))
            neel = np.where((x + y) % 2 == 0, 1, -1).reshape(-1)
            assert abs(int((wk.s * neel).sum())) == N


def test_muca_with_exact_weights_is_flat():
    """Multicanonical sampling with W = the exact density of states (4x4,
    levels 2..8) visits every level equally often (within 5%)."""
    g = exact.ising_dos_enumerated(4)
    klo, khi = 2, 8
    Sw = np.log(g[klo:khi + 1])
    H = np.zeros(khi - klo + 1)
    for w in range(4):
        wk = oracle.Walker(4, klo, khi, 9, w)
        H += wk.muca(Sw, 20_000)
    frac = H / H.sum()
    assert np.abs(frac * len(frac) - 1).max() < 0.05, frac


def test_muca_canonical_weights_reproduce_boltzmann():
    """W(E) = exp(beta E) over all levels turns the multicanonical rule into
    Metropolis at beta: <E> on the 4x4 torus at beta = 0.3 matches
    enumeration within 3 standard errors over 8 walkers."""
    L, beta = 4, 0.3
    N = L * L
    ex = exact.enumerate_ising(2, L, beta)
    k = np.arange(N + 1)
    Sw = beta * (4 * k - 2 * N)
    means = []
    for w in range(8):
        wk = oracle.Walker(L, 0, N, 11, w)
        wk.muca(Sw, 500)
        H = wk.muca(Sw, 20_000)
        means.append(((4 * k - 2 * N) * H).sum() / H.sum())
    m, err = np.mean(means), np.std(means, ddof=1) / np.sqrt(len(means))
    assert abs(m - ex["E"]) < 3 * err + 1e-3, (m, ex["E"], err)


def test_wl_bookkeeping_is_exact():
    """Fixed-point Wang-Landau: with flatness never reached, every attempt
    adds exactly 2^32 (ln f = 1) to its level and one count to H; the level
    is the energy of the spins.  After a flat stage the minimum over the
    visited levels is 0 and H restarts."""
    L, klo, khi = 4, 2, 8
    wk = oracle.Walker(L, klo, khi, 12, 0)
    wk.wl(37, final_stage=5, flat_percent=101)
    assert int(wk.H.sum()) == 37 * 16
    assert int(wk.S.sum()) == 37 * 16 * 2 ** 32
    assert wk.stage == 0
    assert (exact.roll_energy(wk.s, 2, L) + 32) // 4 == wk.level
    vis = np.array([(wk.visited >> q) & 1 for q in range(wk.K)], bool)
    assert ((wk.H > 0) == vis).all()
    wk2 = oracle.Walker(L, klo, khi, 12, 1)
    wk2.wl(2000, final_stage=1, flat_percent=50)
    assert wk2.stage >= 1
    vis = np.array([(wk2.visited >> q) & 1 for q in range(wk2.K)], bool)
    assert wk2.S[vis].min() >= 0


def test_wl_converges_to_exact_dos():
    """Wang-Landau on the whole 4x4 range (levels 0..16, final ln f = 2^-14,
    80% flatness): ln g relative to level 0, averaged over 4 walkers, is
    within 0.1 of the exact ln g on every possible level; the two empty
    levels are never visited."""
    g = exact.ising_dos_enumerated(4)
    N = 16
    ok = g > 0
    est = []
    for w in range(4):
        wk = oracle.Walker(4, 0, N, 13, w)
        wk.wl(400_000, final_stage=14)
        assert wk.stage == 15
        vis = np.array([(wk.visited >> q) & 1 for q in range(wk.K)], bool)
        np.testing.assert_array_equal(vis, ok)
        S = wk.S.astype(np.float64) / 2 ** 32
        est.append(S - S[0])
    lng = np.log(np.where(ok, g, 1.0)) - np.log(g[0])
    diff = np.abs(np.mean(est, axis=0) - lng)[ok]
    assert diff.max() < 0.1, diff


def test_dos_glue_of_exact_windows():
    """Gluing windows that hold the exact ln g plus arbitrary per-window
    offsets returns ln g up to one constant (6x6, windows of 5 levels
    sharing their edge level)."""
    g = exact.ising_dos_transfer(6)
    N = 36
    lng = np.log(np.where(g > 0, g, 1.0))
    klo = np.arange(0, N - 3, 4)
    khi = klo + 4
    rng = np.random.default_rng(5)
    S = np.zeros((len(klo), 5))
    vis = np.zeros(len(klo), np.uint64)
    for w, (a, b) in enumerate(zip(klo, khi)):
        S[w] = lng[a:b + 1] + rng.normal() * 10
        vis[w] = sum(1 << q for q in range(5) if g[a + q] > 0)
    out = oracle.dos_glue(N, klo, khi, S, vis)
    ok = g > 0
    np.testing.assert_allclose((out - out[0])[ok], (lng - lng[0])[ok], atol=1e-9)
    assert np.isnan(out[~ok]).all()


def test_wl_windows_glue_to_exact_dos():
    """Windowed Wang-Landau on 4x4 (four windows of 5 levels sharing edge
    levels, eight walkers each, final ln f = 2^-14), the walkers' estimates
    averaged per window and glued: ln g within 0.15 of the exact values
    (about 0.09 is the bias of 80%-flat stages at window edges)."""
    g = exact.ising_dos_enumerated(4)
    N = 16
    ok = g > 0
    klo = np.arange(0, N - 3, 4)
    khi = klo + 4
    S = np.zeros((len(klo), 5))
    vis = np.zeros(len(klo), np.uint64)
    for w, (a, b) in enumerate(zip(klo, khi)):
        acc = []
        for r in range(8):
            wk = oracle.Walker(4, int(a), int(b), 14, 100 * w + r)
            wk.wl(400_000, final_stage=14)
            assert wk.stage == 15
            Sw = wk.S.astype(np.float64) / 2 ** 32
            acc.append(Sw - Sw[0])
            vis[w] = wk.visited
        S[w] = np.mean(acc, axis=0)
    out = oracle.dos_glue(N, klo, khi, S, vis)
    lng = np.log(np.where(ok, g, 1.0))
    diff = np.abs((out - out[0]) - (lng - lng[0]))[ok]
    assert diff.max() < 0.15, diff
