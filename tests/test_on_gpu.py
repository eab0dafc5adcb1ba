"""GPU parity of the continuous-spin paths (XY angles, Heisenberg vectors;
FP32 spins, FP64 observable totals) against the FP64 oracle.

Accepted spins are fresh proposals, so spin errors do not accumulate: every
component must agree within 1e-5 of the oracle except inside the light cone
of a near-tie, a decision whose margin |u - exp(-beta dE)| is so small that
FP32 rounding may flip it (the oracle logs them; a difference then spreads by
at most two lattice steps per sweep).  Energies must agree within 1e-5 per
site when no near-tie occurred, and the FP64 energy the kernels track must
match an FP64 recomputation from the final FP32 spins within 1e-4 per site.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1107_5463_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = 1e-5
TIE_TOL = 2e-5
TIE_TOL_FAST = 2e-4


@pytest.fixture(scope="module")
def sm():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1107_5463_gb300 import spinmc
    return spinmc


def cone_mask(d, L, ties, nsw, t0=0):
    """True where a site is outside every near-tie's light cone."""
    N = L ** d
    ok = np.ones(N, bool)
    if len(ties) == 0:
        return ok
    idx = np.arange(N)
    coords = [idx % L, (idx // L) % L] + ([idx // (L * L)] if d == 3 else [])
    for t, i in ties:
        ci = [i % L, (i // L) % L] + ([i // (L * L)] if d == 3 else [])
        dist = np.zeros(N, np.int64)
        for a, b in zip(coords, ci):
            dd = np.abs(a - b)
            dist += np.minimum(dd, L - dd)
        radius = 2 * (t0 + nsw - int(t)) + 2
        ok &= dist > radius
    return ok


def angle_diff(a, b):
    d = np.abs(np.asarray(a, np.float64) - np.asarray(b, np.float64)) % (2 * math.pi)
    return np.minimum(d, 2 * math.pi - d)


def start_state(n, d, L, seed):
    """A start configuration exactly representable in FP32 (both sides use it)."""
    if n == 2:
        return oracle.xy_init(d, L, seed).astype(np.float32)
    return oracle.heis_init(d, L, seed).astype(np.float32)


def run_pair(sm, n, d, L, beta, nsw, seed=3, sweep_seed=11, J=1.0, Jb=None, fast=0, renorm=16,
             tie_tol=TIE_TOL):
    s32 = start_state(n, d, L, seed)
    lat = sm.Lattice(d, L, n=n, J=J, J_bonds=Jb, seed=seed)
    lat.set_option(sm.SL_OPT_FAST_MATH, fast)
    if n == 3:
        lat.set_option(sm.SL_OPT_RENORM_EVERY, renorm)
    lat.set_spins(s32)
    E, m = lat.sweep_series(beta, nsw, sweep_seed)
    got = lat.get_spins()
    Eg, mg = E.cpu().numpy(), m.cpu().numpy()
    lat.close()
    ref = s32.astype(np.float64)
    jb = None if Jb is None else Jb
    if n == 2:
        Er, mr, ties, nties = oracle.xy_sweeps(d, L, ref, beta, sweep_seed, 0, nsw, J=J, Jb=jb,
                                               tie_tol=tie_tol, ties_cap=100000)
    else:
        Er, mr, ties, nties = oracle.heis_sweeps(d, L, ref, beta, sweep_seed, 0, nsw, J=J, Jb=jb,
                                                 renorm_every=renorm, tie_tol=tie_tol,
                                                 ties_cap=100000)
    assert nties <= 100000
    return got, Eg, mg, ref, Er, mr, ties


def check_components(n, d, L, got, ref, ties, nsw, min_fraction=0.5):
    mask = cone_mask(d, L, ties, nsw)
    assert mask.mean() >= min_fraction, "too many near-ties to compare"
    if n == 2:
        err = angle_diff(got, ref)[mask]
    else:
        err = np.abs(got.astype(np.float64) - ref)[mask]
    assert err.max() <= TOL, (err.max(), len(ties))
    return mask


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
    nsw = 10
    got, Eg, mg, ref, Er, mr, ties = run_pair(sm, n, d, L, beta, nsw)
    check_components(n, d, L, got, ref, ties, nsw)
    N = L ** d
    if len(ties) == 0:
        assert np.abs(Eg - Er).max() / N < TOL
        assert np.abs(mg - mr).max() < TOL


@pytest.mark.parametrize("n", [2, 3])
def test_parity_with_float_bonds_and_negative_J(sm, n):
    d, L, nsw = 3, 8, 8
    jb = inputs.float_bonds(d, L, 5)
    got, Eg, mg, ref, Er, mr, ties = run_pair(sm, n, d, L, 0.8, nsw, J=-0.6, Jb=jb)
    check_components(n, d, L, got, ref, ties, nsw)


@pytest.mark.parametrize("n,d,L,beta", [(2, 2, 32, 1.12), (3, 3, 16, 0.693)])
def test_fast_math_parity(sm, n, d, L, beta):
    nsw = 10
    got, Eg, mg, ref, Er, mr, ties = run_pair(sm, n, d, L, beta, nsw, fast=1,
                                              tie_tol=TIE_TOL_FAST)
    check_components(n, d, L, got, ref, ties, nsw)


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
    L = 4096, first 10 sweeps against the FP64 oracle."""
    nsw = 10
    got, Eg, mg, ref, Er, mr, ties = run_pair(sm, n, d, L, beta, nsw, seed=inputs.DEFAULT_SEED)
    mask = check_components(n, d, L, got, ref, ties, nsw, min_fraction=0.3)
    N = L ** d
    # energy differs by at most a few units per near-tie cone
    assert np.abs(Eg - Er).max() / N < 1e-4
