"""GPU parity of the batched Edwards-Anderson +-J spin glass with replica
exchange (one persistent launch: CTAs take packs of same-size samples from a
queue, every sample's replicas multispin-coded in shared memory) against the
oracle's per-sample, per-replica loops: couplings, start states, every slot's
spins, the slot-to-temperature assignment and the energy series at every
temperature, bit for bit, whatever pack sizes the autotuner picks."""
import numpy as np
import pytest

import oracle
from paper_1107_5463_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sm():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1107_5463_gb300 import spinmc
    return spinmc


def oracle_sample(d, L, nt, betas, seed, run_seed, s, nsw, t0=0, state=None):
    jb = oracle.ea_couplings(d, L, seed, s)
    if state is None:
        spins = np.stack([oracle.ising_init(d, L, seed, s * nt + r) for r in range(nt)])
        perm = np.arange(nt, dtype=np.int32)
    else:
        spins, perm = state
    E = oracle.ea_pt_sweeps(d, L, jb, betas, run_seed, s, t0, nsw, spins, perm)
    return jb, spins, perm, E


def gpu_state(b, s):
    spins, perm = [], np.zeros(b.ntemps, np.int32)
    for r in range(b.ntemps):
        sp, k = b.get(s, r)
        spins.append(sp)
        perm[k] = r
    return np.stack(spins), perm


def check_batch(sm, d, Ls, nt, betas, nsw, seed=5, run_seed=6, samples=None, pack=None):
    b = sm.Batch(d, Ls, nt, betas, seed=seed)
    if pack is not None:
        b.set_option(sm.SL_BOPT_PACK, pack)
    E = b.run(nsw, run_seed, series=True).cpu().numpy()
    for s in (range(len(Ls)) if samples is None else samples):
        jb, spins, perm, Er = oracle_sample(d, Ls[s], nt, betas, seed, run_seed, s, nsw)
        np.testing.assert_array_equal(b.bonds(s), jb)
        gs, gp = gpu_state(b, s)
        np.testing.assert_array_equal(gp, perm)
        np.testing.assert_array_equal(gs, spins)
        np.testing.assert_array_equal(E[s], Er)
    b.close()


def test_start_state_and_couplings(sm):
    d, Ls, nt = 3, [4, 8, 12, 8], 6
    betas = inputs.geometric_betas(nt)
    b = sm.Batch(d, Ls, nt, betas, seed=77)
    for s, L in enumerate(Ls):
        np.testing.assert_array_equal(b.bonds(s), oracle.ea_couplings(d, L, 77, s))
        for r in range(nt):
            sp, k = b.get(s, r)
            assert k == r
            np.testing.assert_array_equal(sp, oracle.ising_init(d, L, 77, s * nt + r))
    b.close()


@pytest.mark.parametrize("d,Ls,nt", [(3, [4, 8, 12], 8), (3, [8, 12, 16, 24, 32], 32),
                                     (2, [8, 16, 32], 16), (3, [8], 2), (2, [4, 12], 5)])
def test_parity_ten_sweeps(sm, d, Ls, nt):
    check_batch(sm, d, Ls, nt, inputs.geometric_betas(nt), 10)


def test_parity_long_run_one_sample_per_size(sm):
    """One sample of every size of the batched workload, 32 temperatures
    geometric in [0.5, 3], 200 sweeps with exchange every sweep."""
    check_batch(sm, 3, [8, 12, 16, 24, 32], 32, inputs.geometric_betas(32), 200)


def test_equal_betas_swap_every_pair(sm):
    check_batch(sm, 3, [8, 8], 7, [0.6] * 7, 12)


def test_runs_compose(sm):
    d, Ls, nt = 3, [8, 12], 8
    betas = inputs.geometric_betas(nt)
    a = sm.Batch(d, Ls, nt, betas, seed=1)
    a.run(12, 2)
    b = sm.Batch(d, Ls, nt, betas, seed=1)
    b.run(5, 2)
    b.run(7, 2)
    assert b.sweeps_done() == 12
    for s in range(2):
        sa, pa = gpu_state(a, s)
        sb, pb = gpu_state(b, s)
        np.testing.assert_array_equal(sa, sb)
        np.testing.assert_array_equal(pa, pb)
    a.close()
    b.close()


def test_bad_arguments(sm):
    for d, Ls, nt, betas in ((3, [6], 4, [0.1] * 4), (3, [36], 4, [0.1] * 4), (3, [8], 1, [0.1]),
                             (3, [8], 33, [0.1] * 33), (4, [8], 4, [0.1] * 4),
                             (3, [8], 4, [0.1, -1.0, 0.2, 0.3])):
        with pytest.raises(sm.SpinMCError):
            sm.Batch(d, Ls, nt, betas)


@pytest.mark.parametrize("pack", [1, 2, 4, 8])
def test_parity_forced_pack_sizes(sm, pack):
    """Every pack size (samples per CTA, each on its own named barrier) gives
    the oracle's chains; uneven classes leave a partial last pack."""
    Ls = [8, 12, 8, 16, 12, 8, 24, 8, 16, 12, 8]
    check_batch(sm, 3, Ls, 12, inputs.geometric_betas(12), 8, pack=pack)


def test_autotuner_reports_and_keeps_the_chain(sm):
    """The tuner times every fitting pack size per class on a copy of the
    state: afterwards the chain is the oracle's, each class has a pack size
    that fits (side 32 alone in a CTA) and a positive measured cost."""
    Ls = [8, 12, 16, 24, 32] * 3
    nt = 32
    betas = inputs.geometric_betas(nt)
    b = sm.Batch(3, Ls, nt, betas, seed=3)
    E = b.run(6, 4, series=True).cpu().numpy()
    tune = b.tuning()
    assert [t[0] for t in tune] == [32, 24, 16, 12, 8]
    assert tune[0][1] == 1 and all(t[1] in (1, 2, 4, 8) for t in tune)
    assert all(t[2] > 0 for t in tune)
    for s in (0, 4, 9):
        jb, spins, perm, Er = oracle_sample(3, Ls[s], nt, betas, 3, 4, s, 6)
        gs, gp = gpu_state(b, s)
        np.testing.assert_array_equal(gs, spins)
        np.testing.assert_array_equal(gp, perm)
        np.testing.assert_array_equal(E[s], Er)
    b.close()
