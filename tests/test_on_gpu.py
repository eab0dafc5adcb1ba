"""GPU parity of the continuous-spin paths (XY angles, Heisenberg vectors;
FP32 spins, FP64 observable totals) against the FP64 oracle.

Accepted spins are fresh proposals, so spin errors do not accumulate: every
component must agree within 1e-5 of the oracle except inside the light cone
of a near-tie that went the other way.  A near-tie is a decision whose
margin |u - p|, p = exp(-beta dE), lies within the error FP32 can make in p.
The oracle reports, for every decision it screens, the margin and a
condition factor K = p (beta (A + |dE|) + 1) (A sums the field components
and the proposal's change against the couplings, see oracle.h): if every
spin component and every FP32 operation errs by at most EPS, p errs by at
most EPS K.  The kernels' spin components differ from the oracle's by at most
2.4e-7 (FP32 storage of fresh proposals and of sin / cos of stored turns,
measured at most 1.4e-7 and 2e-7), and the FP32 sums over 2d neighbours and
the n-term dot product round by at most 2d 2^-24 = 3.6e-7 relative, so
EPS = 1e-6 bounds both with room to spare.  Only a near-tie can go the other
way, and one that did shows at the end of its sweep as an O(1) difference at
its own site: those sites seed the excluded cones, which grow by two lattice
steps per sweep (one colour pass each).  Energies must agree within 1e-5 per
site when no near-tie diverged, and the FP64 energy the kernels track must
match an FP64 recomputation from the final FP32 spins within 1e-4 per site.
The fast-math kernels (hardware sin/cos/exp) have no such bound and keep a
flat screen: every decision within TIE_TOL_FAST counts as a near-tie.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1107_5463_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = 1e-5
EPS = 1e-6           # error bound of an FP32 evaluation of p, in units of K
TIE_SCREEN = 1e-4    # the oracle reports decisions with margins below this (>= EPS K)
TIE_TOL_FAST = 5e-5


@pytest.fixture(scope="module")
def sm():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1107_5463_gb300 import spinmc
    return spinmc


def dilate(mask, d, L, steps):
    """Grow a natural-order site mask by `steps` nearest-neighbour steps on
    the periodic lattice (the Manhattan ball of that radius)."""
    a = mask.reshape((L,) * d)
    for _ in range(steps):
        b = a.copy()
        for ax in range(d):
            b |= np.roll(a, 1, axis=ax) | np.roll(a, -1, axis=ax)
        a = b
    return a.reshape(-1)


def angle_diff(a, b):
    d = np.abs(np.asarray(a, np.float64) - np.asarray(b, np.float64)) % (2 * math.pi)
    return np.minimum(d, 2 * math.pi - d)


def start_state(n, d, L, seed):
    """A start configuration exactly representable in FP32 (both sides use it)."""
    if n == 2:
        return oracle.xy_init(d, L, seed).astype(np.float32)
    return oracle.heis_init(d, L, seed).astype(np.float32)


class Pair:
    """GPU and oracle runs from one FP32 start, compared after every sweep.

    A near-tie decided in sweep t that went the other way makes the two runs
    differ at its site; the difference spreads by at most two lattice steps
    per sweep (one colour pass each), so after sweep t' the sites within
    distance 2 (t' - t) + 2 of it are excluded from the component check.
    tie_tol=None takes the derived near-tie rule (margin < EPS K); a number
    takes a flat screen (margin < tie_tol)."""

    def __init__(self, sm, n, d, L, beta, nsw, seed=3, sweep_seed=11, J=1.0, Jb=None, fast=0,
                 renorm=16, tie_tol=None, kernel=0):
        N = L ** d
        s32 = start_state(n, d, L, seed)
        lat = sm.Lattice(d, L, n=n, J=J, J_bonds=Jb, seed=seed)
        lat.set_option(sm.SL_OPT_FAST_MATH, fast)
        if kernel:
            lat.set_option(sm.SL_OPT_KERNEL, kernel)
        if n == 3:
            lat.set_option(sm.SL_OPT_RENORM_EVERY, renorm)
        lat.set_spins(s32)
        ref = s32.astype(np.float64)
        cone = np.zeros(N, bool)
        self.N, self.nsw, self.ntie, self.ndiverged = N, nsw, 0, 0
        self.compared, self.max_err, self.max_dE_clean, self.max_dm_clean = 0, 0.0, 0.0, 0.0
        self.max_dE = self.max_dm = 0.0
        self.max_diverged_ratio = 0.0   # largest margin / K among decisions that diverged
        screen = TIE_SCREEN if tie_tol is None else tie_tol
        for t in range(nsw):
            E, m = lat.sweep_series(beta, 1, sweep_seed)
            got = lat.get_spins()
            kw = dict(J=J, Jb=Jb, tie_tol=screen, ties_cap=1 << 21, tie_info=True)
            if n == 2:
                Er, mr, tt, nt, info = oracle.xy_sweeps(d, L, ref, beta, sweep_seed, t, 1, **kw)
            else:
                Er, mr, tt, nt, info = oracle.heis_sweeps(d, L, ref, beta, sweep_seed, t, 1,
                                                          renorm_every=renorm, **kw)
            assert nt <= 1 << 21
            if tie_tol is None:
                near = info[:, 0] < EPS * info[:, 1]
            else:
                near = np.ones(len(tt), bool)
            self.ntie += int(near.sum())
            if n == 2:
                err_all = angle_diff(got, ref)
            else:
                err_all = np.abs(got.astype(np.float64) - ref).max(axis=1)
            sites = tt[:, 1]
            # the reach, at the end of this sweep, of earlier divergences
            grown = dilate(cone, d, L, 2)
            diverged = ~grown[sites] & (err_all[sites] > TOL)
            seeds = np.zeros(N, bool)
            seeds[sites[diverged & near]] = True
            self.ndiverged += int((diverged & near).sum())
            cone = grown | dilate(seeds, d, L, 2)
            # a screened decision outside every cone that diverged must be a near-tie
            bad = ~cone[sites] & diverged & ~near
            assert not bad.any(), ("sweep %d: decisions outside the near-tie bound diverged" % t,
                                   sites[bad][:8], info[bad][:8])
            if (diverged & near).any():
                r = info[diverged & near]
                self.max_diverged_ratio = max(self.max_diverged_ratio, float((r[:, 0] / r[:, 1]).max()))
            ok = ~cone
            err = err_all[ok]
            self.compared += int(ok.sum())
            if err.size:
                self.max_err = max(self.max_err, float(err.max()))
            dE = abs(float(E[0].item()) - float(Er[0])) / N
            dm = abs(float(m[0].item()) - float(mr[0]))
            self.max_dE = max(self.max_dE, dE)
            self.max_dm = max(self.max_dm, dm)
            if self.ndiverged == 0:
                self.max_dE_clean = max(self.max_dE_clean, dE)
                self.max_dm_clean = max(self.max_dm_clean, dm)
        lat.close()

    def check(self, min_fraction=0.95):
        """Components within TOL outside the cones of diverged near-ties after
        every sweep; energy per site and |m| within TOL while no near-tie has
        diverged; at least min_fraction of all site-sweeps compared."""
        assert self.max_err <= TOL, (self.max_err, self.ntie, self.ndiverged)
        assert self.max_dE_clean < TOL and self.max_dm_clean < TOL
        assert self.compared >= min_fraction * self.N * self.nsw, \
            ("too many diverged near-ties to compare", self.ntie, self.ndiverged)


@pytest.mark.parametrize("n,d,L", [(2, 2, 2), (2, 2, 6), (2, 2, 32), (2, 3, 4), (2, 3, 8),
                                   (3, 2, 4), (3, 2, 16), (3, 3, 2), (3, 3, 6), (3, 3, 16)])
def test_start_configuration_matches_oracle(sm, n, d, L):
    lat = sm.Lattice(d, L, n=n, seed=21, replica=2)
    got = lat.get_spins()
    lat.close()
    if n == 2:
        ref = oracle.xy_init(d, L, 21, 2)
        assert angle_diff(got, ref).max() < 1e-6
    else:
        ref = oracle.heis_init(d, L, 21, 2)
        assert np.abs(got - ref).max() < 1e-6
        assert np.abs(np.linalg.norm(got.astype(np.float64), axis=1) - 1).max() < 1e-6


@pytest.mark.parametrize("n,d,L,beta", [(2, 2, 16, 1.12), (2, 2, 30, 0.9), (2, 3, 8, 0.5),
                                        (3, 3, 16, 0.693), (3, 2, 32, 1.5), (3, 3, 6, 0.3)])
def test_parity_first_ten_sweeps(sm, n, d, L, beta):
    Pair(sm, n, d, L, beta, 10).check()


@pytest.mark.parametrize("n,d,L,beta", [(3, 3, 64, 0.693), (3, 2, 64, 1.5), (3, 3, 128, 0.693),
                                        (3, 2, 128, 1.5), (2, 2, 128, 1.12), (2, 2, 256, 0.9)])
@pytest.mark.parametrize("kernel", [1, 2])
def test_streaming_and_generic_kernels(sm, n, d, L, beta, kernel):
    """The row-streaming kernels (register window, warp shuffles; Heisenberg
    on single columns for L = 64, on column pairs for L = 128) and the
    per-site kernel both match the oracle on sizes the streaming kernels
    accept; J = -0.8 on the Heisenberg lattices checks the coupling sign."""
    Pair(sm, n, d, L, beta, 6, kernel=kernel, J=-0.8 if n == 3 else 1.0).check()


@pytest.mark.parametrize("L,J,renorm", [(64, 1.0, 16), (128, -0.8, 16), (256, 1.0, 16),
                                        (64, 1.0, 1)])
def test_staged_tiles_match_oracle_and_column_pairs(sm, L, J, renorm):
    """The staged 3D Heisenberg kernel (planes streamed into shared memory by
    bulk asynchronous copies) against the oracle, and spin for spin equal to
    the column-pair and single-column kernels (every rounding of the field,
    dE and renormalisation spelled out in one shared helper); renorm = 1
    renormalises in every sweep."""
    d, beta = 3, 0.693
    Pair(sm, 3, d, L, beta, 6, kernel=4, J=J, renorm=renorm).check()
    spins = []
    for kern in (2, 3, 4):
        lat = sm.Lattice(d, L, n=3, J=J, seed=7)
        lat.set_option(sm.SL_OPT_RENORM_EVERY, renorm)
        lat.set_option(sm.SL_OPT_KERNEL, kern)
        E, _ = lat.sweep_series(beta, 5, 3)
        spins.append((lat.get_spins(), E.cpu().numpy()))
        lat.close()
    for other in spins[1:]:
        np.testing.assert_array_equal(spins[0][0], other[0])
        np.testing.assert_allclose(spins[0][1], other[1], rtol=1e-6)


def test_staged_tiles_refuse_other_lattices(sm):
    for d, L, n, fast in ((3, 96, 3, 0), (2, 128, 3, 0), (3, 64, 3, 1), (3, 64, 2, 0)):
        lat = sm.Lattice(d, L, n=n, seed=1)
        lat.set_option(sm.SL_OPT_FAST_MATH, fast)
        with pytest.raises(sm.SpinMCError):
            lat.set_option(sm.SL_OPT_KERNEL, 4)
        lat.close()


@pytest.mark.parametrize("n,d,L,beta", [(3, 3, 64, 0.693), (2, 2, 128, 1.12)])
def test_streaming_fast_math(sm, n, d, L, beta):
    Pair(sm, n, d, L, beta, 6, fast=1, tie_tol=TIE_TOL_FAST, kernel=2).check()


@pytest.mark.parametrize("n", [2, 3])
def test_parity_with_float_bonds_and_negative_J(sm, n):
    d, L = 3, 8
    jb = inputs.float_bonds(d, L, 5)
    Pair(sm, n, d, L, 0.8, 8, J=-0.6, Jb=jb).check()


@pytest.mark.parametrize("n,d,L,beta", [(2, 2, 32, 1.12), (3, 3, 24, 0.693)])
def test_fast_math_parity(sm, n, d, L, beta):
    Pair(sm, n, d, L, beta, 10, fast=1, tie_tol=TIE_TOL_FAST).check()


def test_sin_cos_of_angles_in_turns(sm):
    """The kernels' sin and cos of an angle stored in turns (exact reduction
    to the nearest quarter turn, Taylor series to degrees 9 and 10) against
    FP64: on the 2 x 2 XY lattice with every spin at one angle, M / 4 is
    exactly the kernel's (cos, sin) of the stored turn; 4001 angles cover
    every quadrant, the octant boundaries and the wrap at one turn."""
    lat = sm.Lattice(2, 2, n=2, seed=1)
    two_pi = np.float32(6.28318530717958647692)
    inv = np.float32(1) / two_pi
    ks = np.arange(4001)
    turns = np.concatenate([ks / 4000.0, [1 / 8, 3 / 8, 5 / 8, 7 / 8, 1 - 2 ** -24]])
    worst = 0.0
    for tt in turns:
        theta = np.float32(tt * 2 * math.pi)
        lat.set_spins(np.full(4, theta, np.float32))
        # the stored turn, as the layout kernel forms it in FP32
        tr = np.float32(theta * inv)
        t = float(tr - np.floor(tr))
        _, M = lat.measure()
        err = max(abs(M[0] / 4 - math.cos(2 * math.pi * t)), abs(M[1] / 4 - math.sin(2 * math.pi * t)))
        worst = max(worst, err)
    lat.close()
    assert worst < 2e-7, worst


def test_heisenberg_renormalisation(sm):
    """Sweep 15 is a renormalising sweep at interval 16: every spin ends at
    unit length even when the start had norm 1.5."""
    d, L = 3, 8
    s = (oracle.heis_init(d, L, 4) * 1.5).astype(np.float32)
    lat = sm.Lattice(d, L, n=3, seed=4)
    lat.set_spins(s)
    lat.set_state(15)
    lat.sweep(0.0 + 1e-9, 1, 7)
    got = lat.get_spins().astype(np.float64)
    lat.close()
    assert np.abs(np.linalg.norm(got, axis=1) - 1).max() < 1e-6


def test_tracked_energy_matches_recomputation(sm):
    """|E_tracked - E_recomputed| / N < 1e-4 after 200 sweeps (FP64 series from
    the fused reduction vs FP64 Eq. 1 on the final FP32 spins)."""
    for n, d, L, beta in ((2, 2, 64, 1.12), (3, 3, 32, 0.693)):
        lat = sm.Lattice(d, L, n=n, seed=9)
        E, m = lat.sweep_series(beta, 200, 10)
        s = lat.get_spins().astype(np.float64)
        E_meas, M_meas = lat.measure()
        lat.close()
        if n == 2:
            E_re, M_re = oracle.xy_measure(d, L, s)
        else:
            E_re, M_re = oracle.heis_measure(d, L, s)
        N = L ** d
        assert abs(float(E[-1].item()) - E_re) / N < 1e-4
        assert abs(E_meas - E_re) / N < 1e-5
        assert np.abs(M_meas[:n] - M_re).max() / N < 1e-5


@pytest.mark.parametrize("n,d,L,beta", [(2, 2, 32, 1.12), (3, 3, 12, 0.693)])
def test_equilibrium_energy_agrees_statistically(sm, n, d, L, beta):
    """Equilibrium <E>/N of the GPU chain and an independent oracle chain agree
    within 3 combined standard errors (no closed form exists here)."""
    nsw, burn = 3000, 300
    lat = sm.Lattice(d, L, n=n, seed=12)
    E, _ = lat.sweep_series(beta, nsw, 13)
    Eg = E.cpu().numpy()[burn:] / L**d
    lat.close()
    if n == 2:
        s = oracle.xy_init(d, L, 99)
        Er, _, _, _ = oracle.xy_sweeps(d, L, s, beta, 98, 0, nsw)
    else:
        s = oracle.heis_init(d, L, 99)
        Er, _, _, _ = oracle.heis_sweeps(d, L, s, beta, 98, 0, nsw)
    Er = Er[burn:] / L**d
    from tests.exact import binned_mean
    mg, eg = binned_mean(Eg, 20)
    mr, er = binned_mean(Er, 20)
    assert abs(mg - mr) < 3 * math.hypot(eg, er), (mg, mr, eg, er)


@pytest.mark.slow
@pytest.mark.parametrize("n,d,L,beta", [(3, 3, 256, 0.693), (2, 2, 4096, 1.12)])
def test_full_size_first_ten_sweeps(sm, n, d, L, beta):
    """The paper-shaped workloads at full size: 3D Heisenberg L = 256 and 2D XY
    L = 4096, first 10 sweeps against the FP64 oracle, at least 95% of all
    site-sweeps compared."""
    p = Pair(sm, n, d, L, beta, 10, seed=inputs.DEFAULT_SEED)
    p.check(min_fraction=0.95)
    # after near-ties the energies differ by a few units per cone
    assert p.max_dE < 1e-4


@pytest.mark.slow
@pytest.mark.parametrize("n,d,L,beta", [(2, 2, 4096, 0.9), (2, 2, 4096, 1.12), (2, 2, 4096, 1.4),
                                        (3, 3, 256, 0.693)])
def test_precision_report(sm, n, d, L, beta, capsys):
    """FP32 kernels against the FP64 oracle per observable on the paper-shaped
    workloads (XY at the three temperatures of the workload, Heisenberg with
    renormalisation every 16 sweeps), first 10 sweeps: the largest spin
    component error outside the cones of diverged near-ties, |dE|/N and
    |d|m|| after every sweep, the number of near-ties and of those that
    diverged, and the largest margin / K of a diverged decision (below EPS by
    the check); printed as one line per workload."""
    p = Pair(sm, n, d, L, beta, 10, seed=inputs.DEFAULT_SEED)
    with capsys.disabled():
        print("\nprecision n=%d d=%d L=%d beta=%g: component %.2e (%s), |dE|/N %.2e, |d|m|| %.2e, "
              "near-ties %d, diverged %d (largest margin/K %.2e), sites compared %.4f"
              % (n, d, L, beta, p.max_err, "rad" if n == 2 else "per component", p.max_dE,
                 p.max_dm, p.ntie, p.ndiverged, p.max_diverged_ratio,
                 p.compared / (p.N * p.nsw)))
    p.check(min_fraction=0.95)
    assert p.max_dE < 1e-4 and p.max_dm < 1e-4


def test_bounded_wait_gives_up_and_the_context_stays_usable(sm):
    """The staged kernels' mbarrier waits are bounded: a wait for bytes that
    never arrive gives up within seconds, the kernel returns, and the device
    runs the next sweep normally."""
    import time
    import torch
    t0 = time.perf_counter()
    assert sm.sl_wait_selftest(torch.cuda.current_stream().cuda_stream) == 1
    assert time.perf_counter() - t0 < 30
    lat = sm.Lattice(3, 64, n=3, seed=1)
    lat.set_option(sm.SL_OPT_KERNEL, 4)
    E, _ = lat.sweep_series(0.693, 2, 3)
    assert np.isfinite(E.cpu().numpy()).all()
    lat.close()
