"""GPU parity of the windowed multicanonical and Wang-Landau walkers
(Section 4: one system copy per thread in a fixed energy window, flat
histograms, estimates glued afterwards) against the oracle, walker by walker:
start states, spins, level, the fixed-point ln g (exact 64-bit integers),
histograms, visited levels and stages after every run, and the glued S(E).

Wang-Landau decisions compare u with exp(D 2^-32); the kernels decide in FP32
away from the threshold and in FP64 next to it, the oracle always in FP64.
The oracle counts decisions within 1e-12 of the threshold and a test only
compares walkers without such a near-tie (none occur at these sizes)."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sm():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1107_5463_gb300 import spinmc
    return spinmc


def windows(N, width=4, first=0, count=None):
    """Windows of width + 1 levels sharing their edge levels."""
    klo = np.arange(first, N - width + 1, width)
    if count is not None:
        klo = klo[:count]
    return klo.astype(np.int32), (klo + width).astype(np.int32)


def oracle_walkers(L, klo, khi, wpw, seed, pick):
    return {j: oracle.Walker(L, int(klo[j // wpw]), int(khi[j // wpw]), seed, j) for j in pick}


def compare(sm, w, refs, wl=True):
    S, H, lev, st, vis = w.read()
    for j, r in refs.items():
        np.testing.assert_array_equal(w.spins(j), r.s, err_msg="walker %d spins" % j)
        assert lev[j] == r.level, j
        np.testing.assert_array_equal(H[j, :r.K], r.H if wl else r.H_muca, err_msg="H %d" % j)
        if wl:
            np.testing.assert_array_equal(S[j, :r.K], r.S, err_msg="S %d" % j)
            assert int(vis[j]) == r.visited and st[j] == r.stage, j


@pytest.mark.parametrize("L", [4, 8, 16])
def test_walker_start_states(sm, L):
    N = L * L
    klo, khi = windows(N, 4)
    w = sm.Walkers(L, klo, khi, 32, seed=3)
    _, _, lev, st, vis = w.read()
    pick = list(range(0, w.nwalk, 7))
    refs = oracle_walkers(L, klo, khi, 32, 3, pick)
    for j, r in refs.items():
        np.testing.assert_array_equal(w.spins(j), r.s)
        assert lev[j] == r.level and st[j] == 0 and vis[j] == 0
    w.close()


@pytest.mark.parametrize("L,nwin,smem", [(4, None, 1), (8, None, 1), (8, None, 0), (16, 12, 1),
                                          (32, 6, 0)])
def test_wang_landau_parity(sm, L, nwin, smem):
    """Two runs (the sweep counter continues) with stage advances: every
    sampled walker matches the oracle exactly, with the lattices held in
    shared memory or in global memory during a run."""
    N = L * L
    klo, khi = windows(N, 4, first=N // 4 if nwin else 0, count=nwin)
    w = sm.Walkers(L, klo, khi, 32, seed=5)
    w.set_option(sm.SL_WOPT_SPINS_SMEM, smem)
    pick = list(range(0, w.nwalk, 5 if L <= 8 else 9))
    refs = oracle_walkers(L, klo, khi, 32, 5, pick)
    for nsw, fs in ((30, 6), (45, 9)):
        w.wl(nsw, final_stage=fs, flat_percent=80, seed=77)
        ties = sum(r.wl(nsw, fs, 80, tie_tol=1e-12, seed=77) for r in refs.values())
        assert ties == 0
    assert max(r.stage for r in refs.values()) > 1
    compare(sm, w, refs)
    w.close()


def test_wang_landau_wide_windows_and_final_stage(sm):
    """Windows of 17 and 33 levels (larger shared-memory tables), walkers that
    reach the final stage stop moving."""
    L = 8
    klo = np.array([0, 16, 40], np.int32)
    khi = np.array([16, 48, 56], np.int32)
    w = sm.Walkers(L, klo, khi, 32, seed=6)
    pick = list(range(0, w.nwalk, 3))
    refs = oracle_walkers(L, klo, khi, 32, 6, pick)
    w.wl(400, final_stage=4, flat_percent=70, seed=8)
    for r in refs.values():
        assert r.wl(400, 4, 70, tie_tol=1e-12, seed=8) == 0
    assert sum(r.stage == 5 for r in refs.values()) > 0
    compare(sm, w, refs)
    w.close()


def test_multicanonical_parity(sm):
    """Multicanonical sweeps with weights taken from a Wang-Landau run: the
    histograms (restarted by the run), spins and levels match the oracle."""
    L = 8
    N = L * L
    klo, khi = windows(N, 6)
    w = sm.Walkers(L, klo, khi, 32, seed=9)
    w.set_option(sm.SL_WOPT_SPINS_SMEM, 0)
    w.wl(60, final_stage=8, seed=1)
    S, _, _, _, _ = w.read()
    lnW = np.zeros((len(klo), w.kmax))
    for q in range(len(klo)):
        lnW[q, :] = S[q * 32, :].astype(np.float64) / 2 ** 32
    pick = list(range(0, w.nwalk, 4))
    refs = oracle_walkers(L, klo, khi, 32, 9, pick)
    for r in refs.values():
        assert r.wl(60, 8, 80, tie_tol=1e-12, seed=1) == 0
    w.muca(lnW, 40, seed=2)
    for j, r in refs.items():
        win = j // 32
        r.H_muca = r.muca(lnW[win, :r.K], 40, seed=2).astype(np.uint32)
    compare(sm, w, refs, wl=False)
    w.close()


def test_full_size_L64_windows(sm):
    """The 64 x 64 workload (windows of 5 levels sharing edge levels, 64
    walkers each): sampled walkers across the whole energy range match the
    oracle after 3 Wang-Landau sweeps."""
    L = 64
    N = L * L
    klo, khi = windows(N, 4)
    w = sm.Walkers(L, klo, khi, 64, seed=11)
    pick = [j for j in range(0, w.nwalk, 4099)][:16]
    refs = oracle_walkers(L, klo, khi, 64, 11, pick)
    w.wl(3, final_stage=20, seed=4)
    for r in refs.values():
        assert r.wl(3, 20, 80, tie_tol=1e-12, seed=4) == 0
    compare(sm, w, refs)
    w.close()


def test_glue_matches_oracle(sm):
    L = 6
    rng = np.random.default_rng(2)
    klo = np.array([0, 4, 8, 12], np.int32)
    khi = klo + 4
    S = rng.normal(size=(4, 7))
    vis = np.array([0b11101, 0b11111, 0b11111, 0b10111], np.uint64)
    got = sm.sl_dos_glue(L, klo, khi, S, vis)
    ref = oracle.dos_glue(L * L, klo, khi, S, vis)
    np.testing.assert_array_equal(np.isnan(got), np.isnan(ref))
    np.testing.assert_array_equal(got[~np.isnan(got)], ref[~np.isnan(ref)])


def test_walker_argument_checks(sm):
    for L, klo, khi, wpw in ((6, [0], [4], 32), (8, [0], [1], 32), (8, [0], [4], 48),
                             (8, [0], [70], 32), (8, [0, 5], [4, 9], 32)):
        with pytest.raises(sm.SpinMCError):
            w = sm.Walkers(L, klo, khi, wpw)
            # windows that do not share edge levels are legal for sampling;
            # only gluing rejects them
            S, _, _, _, vis = w.read()
            sm.sl_dos_glue(L, w.klo, w.khi, S[::wpw].astype(float), vis[::wpw])


@pytest.mark.parametrize("spins_smem", [0, 1])
def test_checkpoint_resume(sm, spins_smem):
    """2n Wang-Landau sweeps equal n sweeps, a checkpoint (every walker's
    spins, ln g, histogram, stage, visited levels and the sweeps done) loaded
    into a fresh walker set, then n more; the loaded level is recomputed from
    the spins and must lie in the walker's window."""
    L = 8
    klo, khi = windows(L * L, 4)
    a = sm.Walkers(L, klo, khi, 32, seed=6)
    a.set_option(sm.SL_WOPT_SPINS_SMEM, spins_smem)
    a.wl(24, final_stage=12, seed=2)
    b = sm.Walkers(L, klo, khi, 32, seed=6)
    b.set_option(sm.SL_WOPT_SPINS_SMEM, spins_smem)
    b.wl(12, final_stage=12, seed=2)
    ckpt = b.save()
    b.close()
    c = sm.Walkers(L, klo, khi, 32, seed=123)   # another start: the checkpoint replaces it
    c.set_option(sm.SL_WOPT_SPINS_SMEM, spins_smem)
    c.load(ckpt)
    c.wl(12, final_stage=12, seed=2)
    ra, rc = a.read(), c.read()
    for x, y in zip(ra, rc):
        np.testing.assert_array_equal(x, y)
    for j in range(0, a.nwalk, 5):
        np.testing.assert_array_equal(a.spins(j), c.spins(j))
    assert sm.sl_walkers_info(c.h)[2] == 24
    # a configuration whose level is outside walker 0's window is refused
    with pytest.raises(sm.SpinMCError):
        sm.sl_walkers_set_spins(c.h, 0, _far_state(L, klo[0], khi[0]))
    a.close()
    c.close()


def _far_state(L, klo, khi):
    """All up (level 0) unless that lies in [klo, khi]; then a Neel state (level N)."""
    s = np.ones(L * L, np.int8)
    if klo <= 0 <= khi:
        x, y = np.meshgrid(np.arange(L), np.arange(L))
        s = np.where((x + y) % 2 == 0, 1, -1).astype(np.int8).reshape(-1)
    return s
