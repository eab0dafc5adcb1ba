"""GPU parity of k-fold multi-hit sweeps in big tiles (Section 2: tiles plus
boundary layer in shared memory, k updates of all spins of the tiles of one
colour before the other colour; Table 1 uses k = 100) against the oracle's
tile schedule, bit for bit: spins and per-sweep energy and |m|."""
import numpy as np
import pytest

import oracle
from paper_1107_5463_gb300 import inputs

pytestmark = pytest.mark.gpu

BETA_C = inputs.BETA_C_2D_ISING


@pytest.fixture(scope="module")
def sm():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1107_5463_gb300 import spinmc
    return spinmc


def run_both(sm, d, L, T, k, beta, nsw, J=1.0, seed=4, sweep_seed=44, graph=1):
    lat = sm.Lattice(d, L, n=1, J=J, seed=seed)
    lat.set_option(sm.SL_OPT_TILE, T)
    lat.set_option(sm.SL_OPT_MULTIHIT, k)
    lat.set_option(sm.SL_OPT_GRAPH, graph)
    E, m = lat.sweep_series(beta, nsw, sweep_seed)
    got = lat.get_spins(), E.cpu().numpy(), m.cpu().numpy()
    lat.close()
    s = oracle.ising_init(d, L, seed)
    Er, mr = oracle.ising_multihit_sweeps(d, L, T, k, s, beta, sweep_seed, 0, nsw, J=J)
    np.testing.assert_array_equal(got[0], s)
    np.testing.assert_array_equal(got[1], Er)
    np.testing.assert_array_equal(got[2], mr)


@pytest.mark.parametrize("d,L,T,k", [(2, 16, 8, 1), (2, 32, 8, 3), (2, 64, 16, 2), (2, 96, 16, 2),
                                     (2, 128, 32, 2), (2, 128, 64, 1), (3, 16, 8, 2),
                                     (3, 32, 16, 2), (3, 48, 8, 1)])
@pytest.mark.parametrize("beta,J", [(BETA_C, 1.0), (0.3, -0.7)])
def test_multihit_parity(sm, d, L, T, k, beta, J):
    run_both(sm, d, L, T, k, beta, 4, J=J)


def test_multihit_paper_mode_k100(sm):
    """The paper's benchmark mode: tiles of 16 x 16, k = 100 (Table 1)."""
    run_both(sm, 2, 64, 16, 100, BETA_C, 3)


def test_multihit_graph_replay(sm):
    run_both(sm, 2, 32, 8, 1, BETA_C, 80, graph=1)


def test_multihit_resume(sm):
    lat = sm.Lattice(2, 64, seed=2)
    lat.set_option(sm.SL_OPT_MULTIHIT, 5)
    lat.sweep(0.4, 3, 9)
    lat.sweep(0.4, 4, 9)
    got = lat.get_spins()
    lat.close()
    s = oracle.ising_init(2, 64, 2)
    oracle.ising_multihit_sweeps(2, 64, 16, 5, s, 0.4, 9, 0, 7, series=False)
    np.testing.assert_array_equal(got, s)


def test_multihit_bad_options(sm):
    lat = sm.Lattice(2, 64)
    with pytest.raises(sm.SpinMCError):
        lat.set_option(sm.SL_OPT_TILE, 12)
    with pytest.raises(sm.SpinMCError):
        lat.set_option(sm.SL_OPT_TILE, 64)   # 64 % 128 != 0
    lat.close()
    for kw in (dict(storage=sm.SL_STORE_BITS), dict(J_bonds=inputs.ising_bonds(2, 64, 1))):
        lat = sm.Lattice(2, 64, **kw)
        with pytest.raises(sm.SpinMCError):
            lat.set_option(sm.SL_OPT_MULTIHIT, 2)
        lat.close()
