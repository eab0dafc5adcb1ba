"""GPU parity of the Ising heat-bath rule (Section 2: the heat-bath
prescription, a local modification of the Metropolis implementation) against
the oracle, bit for bit: every spin and the per-sweep energy and |m|."""
import numpy as np
import pytest

import oracle
from paper_1107_5463_gb300 import inputs

pytestmark = pytest.mark.gpu

BETA_C = inputs.BETA_C_2D_ISING
GEN, STREAM = 1, 2


@pytest.fixture(scope="module")
def sm():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1107_5463_gb300 import spinmc
    return spinmc


def run_both(sm, d, L, beta, nsw, J=1.0, Jb=None, kernel=0, seed=5, sweep_seed=55):
    lat = sm.Lattice(d, L, n=1, J=J, J_bonds=Jb, seed=seed)
    lat.set_option(sm.SL_OPT_UPDATE, 1)
    if kernel:
        lat.set_option(sm.SL_OPT_KERNEL, kernel)
    E, m = lat.sweep_series(beta, nsw, sweep_seed)
    got = lat.get_spins(), E.cpu().numpy(), m.cpu().numpy()
    lat.close()
    s = oracle.ising_init(d, L, seed)
    Er, mr = oracle.ising_heatbath_sweeps(d, L, s, beta, sweep_seed, 0, nsw, J=J, Jb=Jb)
    np.testing.assert_array_equal(got[0], s)
    np.testing.assert_array_equal(got[1], Er)
    np.testing.assert_array_equal(got[2], mr)


@pytest.mark.parametrize("d,L,kernel", [(2, 2, GEN), (2, 6, GEN), (2, 32, GEN), (2, 32, STREAM),
                                        (2, 96, STREAM), (3, 2, GEN), (3, 6, GEN),
                                        (3, 32, STREAM), (3, 64, STREAM)])
@pytest.mark.parametrize("beta,J", [(BETA_C, 1.0), (0.3, -0.7)])
def test_heatbath_uniform_parity(sm, d, L, kernel, beta, J):
    run_both(sm, d, L, beta, 12, J=J, kernel=kernel)


@pytest.mark.parametrize("d,L,kernel", [(2, 32, STREAM), (3, 32, STREAM), (3, 6, GEN)])
def test_heatbath_pm_bonds_parity(sm, d, L, kernel):
    run_both(sm, d, L, 0.8, 10, Jb=inputs.ising_bonds(d, L, 9), kernel=kernel)


def test_heatbath_zero_bonds_parity(sm):
    run_both(sm, 2, 32, 0.6, 10, J=1.2, Jb=inputs.ising_bonds(2, 32, 10, p_zero=0.3))


def test_heatbath_long_run_2d_L64(sm):
    run_both(sm, 2, 64, BETA_C, 2000, seed=inputs.DEFAULT_SEED, sweep_seed=inputs.DEFAULT_SEED)


def test_heatbath_storage_rules(sm):
    """Bit storage and multi-hit sweeps have no heat-bath rule; byte, angle and
    vector storage accept it."""
    lat = sm.Lattice(2, 64, n=1, storage=sm.SL_STORE_BITS)
    with pytest.raises(sm.SpinMCError):
        lat.set_option(sm.SL_OPT_UPDATE, sm.SL_UPDATE_HEATBATH)
    lat.close()
    lat = sm.Lattice(2, 64, n=1)
    lat.set_option(sm.SL_OPT_MULTIHIT, 4)
    with pytest.raises(sm.SpinMCError):
        lat.set_option(sm.SL_OPT_UPDATE, sm.SL_UPDATE_HEATBATH)
    lat.close()
    for n in (1, 2, 3):
        lat = sm.Lattice(2, 16, n=n)
        lat.set_option(sm.SL_OPT_UPDATE, sm.SL_UPDATE_HEATBATH)
        lat.close()
