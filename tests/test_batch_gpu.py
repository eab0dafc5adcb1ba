"""GPU parity of the batched Edwards-Anderson +-J spin glass with replica
exchange (one persistent launch: CTAs take packs of same-size samples from a
queue, every sample's replicas multispin-coded in shared memory) against the
oracle's per-sample, per-replica loops: couplings, start states, every slot's
spins, the slot-to-temperature assignment and the energy series at every
temperature, bit for bit, whatever pack sizes the autotuner picks."""
import json
import os
import hashlib

import numpy as np
import pytest

import oracle
from paper_1107_5463_gb300 import inputs
from tests import oracle_pool

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "ea_long_runs.json")


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
                                     (2, [8, 16, 32], 16), (2, [8, 16, 32, 32], 32),
                                     (3, [8], 2), (2, [4, 12], 5)])
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


def test_split_batches_equal_the_whole_batch(sm):
    """Random numbers are keyed by the global sample index: two batches over
    samples 0..5 and 6..10 (one per GPU, say) hold exactly the samples of one
    batch over 0..10 (couplings, every slot, permutation, energy series)."""
    d, nt = 3, 8
    betas = inputs.geometric_betas(nt)
    Ls = inputs.ea_sample_sizes(11)
    whole = sm.Batch(d, Ls, nt, betas, seed=9)
    Ew = whole.run(7, 3, series=True).cpu().numpy()
    lo = sm.Batch(d, Ls[:6], nt, betas, seed=9, first_sample=0)
    hi = sm.Batch(d, Ls[6:], nt, betas, seed=9, first_sample=6)
    El = lo.run(7, 3, series=True).cpu().numpy()
    Eh = hi.run(7, 3, series=True).cpu().numpy()
    np.testing.assert_array_equal(np.concatenate([El, Eh]), Ew)
    for s in range(11):
        part, q = (lo, s) if s < 6 else (hi, s - 6)
        np.testing.assert_array_equal(part.bonds(q), whole.bonds(s))
        ps, pp = gpu_state(part, q)
        ws, wp = gpu_state(whole, s)
        np.testing.assert_array_equal(ps, ws)
        np.testing.assert_array_equal(pp, wp)
    # and the upper half is the oracle's samples 6..10
    for q in (0, 4):
        jb, spins, perm, Er = oracle_sample(d, Ls[6 + q], nt, betas, 9, 3, 6 + q, 7)
        gs, gp = gpu_state(hi, q)
        np.testing.assert_array_equal(gs, spins)
        np.testing.assert_array_equal(gp, perm)
        np.testing.assert_array_equal(Eh[q], Er)
    for b in (whole, lo, hi):
        b.close()


def test_first_sample_beyond_replica_ids_is_rejected(sm):
    with pytest.raises(sm.SpinMCError):
        sm.Batch(3, [8, 8], 32, inputs.geometric_betas(32), first_sample=(1 << 27) - 1)


def test_checkpoint_resume(sm):
    """2n sweeps equal n sweeps, a checkpoint (every slot, the slot of every
    temperature, the sweeps done) loaded into a fresh batch, then n more."""
    d, nt = 3, 12
    betas = inputs.geometric_betas(nt)
    Ls = [8, 12, 16, 8]
    a = sm.Batch(d, Ls, nt, betas, seed=4)
    Ea = a.run(16, 5, series=True).cpu().numpy()
    b = sm.Batch(d, Ls, nt, betas, seed=4)
    b.run(8, 5)
    ckpt = b.save()
    b.close()
    c = sm.Batch(d, Ls, nt, betas, seed=4)
    c.load(ckpt)
    assert c.sweeps_done() == 8
    Ec = c.run(8, 5, series=True).cpu().numpy()
    np.testing.assert_array_equal(Ec, Ea[:, 8:])
    for s in range(len(Ls)):
        sa, pa = gpu_state(a, s)
        sc, pc = gpu_state(c, s)
        np.testing.assert_array_equal(sc, sa)
        np.testing.assert_array_equal(pc, pa)
    with pytest.raises(sm.SpinMCError):
        sm.sl_batch_set(c.h, 0, ckpt[0][0][0], np.zeros(nt, np.int32))  # not a permutation
    a.close()
    c.close()


@pytest.mark.slow
def test_full_workload_ten_sweeps_every_sample(sm):
    """The batched workload at its full size: 1024 samples of sides
    [8,12,16,24,32][s mod 5] x 32 temperatures geometric in [0.5, 3], 10
    sweeps with exchange, every spin of every slot, every permutation and the
    whole energy series of every sample against the oracle (run sample by
    sample over the host cores)."""
    d, nt, nsw, seed, run_seed = 3, 32, 10, inputs.DEFAULT_SEED, 0x11075463
    betas = inputs.geometric_betas(nt)
    Ls = inputs.ea_sample_sizes(1024)
    b = sm.Batch(d, Ls, nt, betas, seed=seed)
    E = b.run(nsw, run_seed, series=True).cpu().numpy()
    tasks = [(d, L, nt, betas, seed, run_seed, s, nsw) for s, L in enumerate(Ls)]
    checked = 0
    for s, (jb, spins, perm, Er) in enumerate(oracle_pool.imap_spawn(oracle_pool.ea_sample_run,
                                                                     tasks)):
        np.testing.assert_array_equal(E[s], Er, err_msg="energy series, sample %d" % s)
        gs, gp = gpu_state(b, s)
        np.testing.assert_array_equal(gp, perm, err_msg="permutation, sample %d" % s)
        np.testing.assert_array_equal(gs, spins, err_msg="spins, sample %d" % s)
        if s % 97 == 0:
            np.testing.assert_array_equal(b.bonds(s), jb)
        checked += 1
    assert checked == 1024
    b.close()


def _sha(a):
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


@pytest.mark.slow
def test_long_runs_one_sample_per_size(sm):
    """One sample of each side of the batched workload for the full 10^4
    sweeps, 32 temperatures, exchange every sweep: final spins of every slot,
    the permutation and the whole energy series against the oracle's runs
    recorded in tests/golden/ea_long_runs.json (written by
    tests/golden/make_ea_long_runs.py, which calls only the oracle)."""
    with open(GOLDEN) as f:
        g = json.load(f)
    d, nt, nsw = g["d"], g["ntemps"], g["nsweeps"]
    betas = inputs.geometric_betas(nt)
    Ls = [row["L"] for row in g["samples"]]
    assert Ls == list(inputs.EA_SIZES)
    b = sm.Batch(d, Ls, nt, betas, seed=g["create_seed"])
    E = b.run(nsw, g["run_seed"], series=True).cpu().numpy()
    for row in g["samples"]:
        s = row["sample"]
        for t, v in row["E_probe"].items():
            np.testing.assert_array_equal(E[s, int(t)], np.array(v), err_msg="L=%d sweep %s"
                                          % (row["L"], t))
        assert _sha(E[s].astype(np.float64)) == row["E_sha256"], row["L"]
        gs, gp = gpu_state(b, s)
        assert gp.tolist() == row["slot_of_temp"], row["L"]
        assert _sha(gs.astype(np.int8)) == row["spins_sha256"], row["L"]
    b.close()
