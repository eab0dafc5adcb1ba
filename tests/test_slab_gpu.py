"""GPU parity of the domain decomposition (Section 2: the lattice split into
parts that are updated in parallel) with virtual ranks on one GPU: slabs of
one lattice along its slowest axis, each with its own buffer, exchanging the
just-updated colour's boundary planes into their neighbours' halos after
every colour pass (device-to-device copies).  Every split must give the
unsplit lattice's trajectory bit for bit (all spins and the E and |m|
series), and the unsplit lattice is the oracle's, so the slabs are checked
against both: byte and bit storage, 2D and 3D, even and uneven splits, slabs
of one plane, one slab that is its own neighbour, Metropolis and heat-bath,
and the 2D L = 16384 workload split in two."""
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


def make_slabs(sm, d, L, bounds, storage, seed, update=None):
    slabs = []
    z = 0
    for Lz in bounds:
        s = sm.Slab(d, L, z, Lz, seed=seed, storage=storage)
        if update is not None:
            s.set_option(sm.SL_OPT_UPDATE, update)
        slabs.append(s)
        z += Lz
    assert z == L
    return slabs


def split_run(sm, d, L, bounds, storage, beta, nsw, seed=5, sweep_seed=9, update=None,
              calls=1):
    slabs = make_slabs(sm, d, L, bounds, storage, seed, update)
    Es, ms = [], []
    for _ in range(calls):
        E, m = sm.slabs_sweep(slabs, beta, nsw // calls, sweep_seed)
        Es.append(E.cpu().numpy())
        ms.append(m.cpu().numpy())
    spins = np.concatenate([s.get_spins() for s in slabs])
    for s in slabs:
        s.close()
    return spins, np.concatenate(Es), np.concatenate(ms)


def whole_run(sm, d, L, storage, beta, nsw, seed=5, sweep_seed=9, update=None):
    lat = sm.Lattice(d, L, seed=seed, storage=storage)
    if update is not None:
        lat.set_option(sm.SL_OPT_UPDATE, update)
    E, m = lat.sweep_series(beta, nsw, sweep_seed)
    s = lat.get_spins()
    lat.close()
    return s, E.cpu().numpy(), m.cpu().numpy()


CASES = [
    (2, 64, "i8", [32, 32]), (2, 64, "i8", [8, 40, 16]), (2, 64, "i8", [64]),
    (2, 64, "i8", [1, 1, 30, 32]), (2, 96, "i8", [48, 48]), (2, 40, "i8", [8, 24, 8]),
    (3, 32, "i8", [16, 16]), (3, 32, "i8", [3, 7, 22]), (3, 24, "i8", [12, 12]),
    (2, 128, "bits", [64, 64]), (2, 128, "bits", [5, 123]), (3, 64, "bits", [32, 16, 16]),
    (3, 64, "bits", [64]),
]


@pytest.mark.parametrize("d,L,storage,bounds", CASES)
def test_split_equals_whole_and_oracle(sm, d, L, storage, bounds):
    st = sm.SL_STORE_I8 if storage == "i8" else sm.SL_STORE_BITS
    beta = 0.44 if d == 2 else 0.2216546
    nsw = 6
    s_split, E_split, m_split = split_run(sm, d, L, bounds, st, beta, nsw)
    s_whole, E_whole, m_whole = whole_run(sm, d, L, st, beta, nsw)
    np.testing.assert_array_equal(s_split, s_whole)
    np.testing.assert_array_equal(E_split, E_whole)
    np.testing.assert_array_equal(m_split, m_whole)
    s = oracle.ising_init(d, L, 5)
    E_ref, m_ref = oracle.ising_sweeps(d, L, s, beta, 9, 0, nsw)
    np.testing.assert_array_equal(s_split, s)
    np.testing.assert_array_equal(E_split, E_ref)
    np.testing.assert_array_equal(m_split, m_ref)


def test_split_heatbath_and_calls_compose(sm):
    """Heat-bath passes on slabs, and two calls of 4 sweeps equal one of 8."""
    d, L, beta = 2, 64, 0.44
    s_split, E_split, _ = split_run(sm, d, L, [16, 48], sm.SL_STORE_I8, beta, 8,
                                    update=sm.SL_UPDATE_HEATBATH, calls=2)
    s = oracle.ising_init(d, L, 5)
    E_ref, _ = oracle.ising_heatbath_sweeps(d, L, s, beta, 9, 0, 8)
    np.testing.assert_array_equal(s_split, s)
    np.testing.assert_array_equal(E_split, E_ref)


def test_generic_kernel_on_slabs(sm):
    """The per-site kernel (forced) on slabs of a lattice whose rows are too
    short for the streaming kernel."""
    d, L, beta = 2, 24, 0.5
    slabs = make_slabs(sm, d, L, [8, 16], sm.SL_STORE_I8, 5)
    for s in slabs:
        s.set_option(sm.SL_OPT_KERNEL, 1)
    E, _ = sm.slabs_sweep(slabs, beta, 5, 9)
    got = np.concatenate([s.get_spins() for s in slabs])
    s = oracle.ising_init(d, L, 5)
    E_ref, _ = oracle.ising_sweeps(d, L, s, beta, 9, 0, 5)
    np.testing.assert_array_equal(got, s)
    np.testing.assert_array_equal(E.cpu().numpy(), E_ref)
    for sl in slabs:
        sl.close()


def test_single_rank_driver_on_gpu(sm):
    """shard.ShardedLattice without a process group (one rank, its own
    neighbour): the same chain as the whole lattice."""
    from paper_1107_5463_gb300 import shard
    d, L = 2, 64
    local = sm.Slab(d, L, 0, L, seed=5)
    E, m = shard.ShardedLattice(local, L, d).sweep_series(0.44, 5, 9)
    s_whole, E_whole, m_whole = whole_run(sm, d, L, sm.SL_STORE_I8, 0.44, 5)
    np.testing.assert_array_equal(local.get_spins(), s_whole)
    np.testing.assert_array_equal(E.cpu().numpy(), E_whole)
    np.testing.assert_array_equal(m.cpu().numpy(), m_whole)
    local.close()


def test_slab_arguments(sm):
    with pytest.raises(sm.SpinMCError):
        sm.Slab(2, 64, 60, 8)            # beyond the lattice
    with pytest.raises(sm.SpinMCError):
        sm.Slab(2, 60, 0, 30)            # L % 8 != 0
    with pytest.raises(sm.SpinMCError):
        sm.Slab(2, 96, 0, 32, storage=sm.SL_STORE_BITS)   # bits need L % 64 == 0
    a, b = sm.Slab(2, 64, 0, 32), sm.Slab(2, 64, 32, 32)
    with pytest.raises(sm.SpinMCError):
        a.sweep(0.4, 1, 1)               # slabs sweep through passes
    with pytest.raises(sm.SpinMCError):
        sm.sl_slab_pass(a.h, 0.4, 1, 1)  # colour 1 before colour 0
    with pytest.raises(sm.SpinMCError):
        sm.sl_slabs_exchange([b.h, a.h], 0)   # not in order
    with pytest.raises(sm.SpinMCError):
        sm.sl_slabs_exchange([a.h], 0)        # does not reach L
    a.close()
    b.close()


@pytest.mark.slow
def test_full_size_workload_split_in_two(sm):
    """The 2D L = 16384 workload (2.7e8 spins) as two slabs of 8192 rows
    against the unsplit lattice, 5 sweeps: every spin and the series."""
    d, L, beta = 2, 16384, 0.440687
    s_split, E_split, m_split = split_run(sm, d, L, [8192, 8192], sm.SL_STORE_I8, beta, 5,
                                          seed=inputs.DEFAULT_SEED)
    s_whole, E_whole, m_whole = whole_run(sm, d, L, sm.SL_STORE_I8, beta, 5,
                                          seed=inputs.DEFAULT_SEED)
    assert np.array_equal(s_split, s_whole)
    np.testing.assert_array_equal(E_split, E_whole)
    np.testing.assert_array_equal(m_split, m_whole)
