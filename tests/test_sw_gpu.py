"""GPU parity of the Swendsen-Wang cluster update (Section 3: bonds between
like spins activated with 1 - exp(-2 beta J), clusters joined by active bonds,
each flipped with probability 1/2) against the oracle, bit for bit: every spin
and the energy and |m| after every update.  Cluster names (the smallest site)
and flip bits do not depend on how the GPU schedules its unions, so one
trajectory is correct and the two must agree exactly.

Sizes cover a single tile, several tiles, ragged edge tiles (L not a multiple
of the 64 x 32 / 32 x 16 x 16 tile), the L = 2 multigraph, beta = 0 (no bond
active), a large beta (almost every satisfied bond active), negative J, graph
replays, and one full update of the 8192^2 workload."""
import numpy as np
import pytest

import oracle
from paper_1107_5463_gb300 import inputs

pytestmark = pytest.mark.gpu

BETA_C = inputs.BETA_C_2D_ISING
BETA_3D = inputs.BETA_3D_ISING


@pytest.fixture(scope="module")
def sm():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1107_5463_gb300 import spinmc
    return spinmc


def run_both(sm, d, L, beta, nsw, J=1.0, seed=5, sweep_seed=55, graph=1):
    lat = sm.Lattice(d, L, n=1, J=J, seed=seed)
    lat.set_update(sm.SL_UPDATE_SW)
    lat.set_option(sm.SL_OPT_GRAPH, graph)
    E, m = lat.sweep_series(beta, nsw, sweep_seed)
    got = lat.get_spins(), E.cpu().numpy(), m.cpu().numpy()
    lat.close()
    s = oracle.ising_init(d, L, seed)
    Er, mr = oracle.ising_sw_sweeps(d, L, s, beta, sweep_seed, 0, nsw, J=J)
    np.testing.assert_array_equal(got[0], s)
    np.testing.assert_array_equal(got[1], Er)
    np.testing.assert_array_equal(got[2], mr)


@pytest.mark.parametrize("L", [2, 4, 16, 64, 96, 130])
def test_sw_2d_parity(sm, L):
    run_both(sm, 2, L, BETA_C, 12)


@pytest.mark.parametrize("L", [2, 4, 6, 16, 32, 34])
def test_sw_3d_parity(sm, L):
    run_both(sm, 3, L, BETA_3D, 8)


@pytest.mark.parametrize("d,beta,J", [(2, 0.0, 1.0), (2, 5.0, 1.0), (3, 5.0, 1.0),
                                      (2, BETA_C, -1.0), (3, 0.35, -0.8), (2, 0.9, 1.3)])
def test_sw_special_couplings(sm, d, beta, J):
    run_both(sm, d, 64 if d == 2 else 16, beta, 6, J=J)


def test_sw_graph_replay_matches_plain_launches(sm):
    """70 updates through the captured graph (32 per replay) and through plain
    launches, both against the oracle."""
    run_both(sm, 2, 128, BETA_C, 70, graph=1)
    run_both(sm, 2, 128, BETA_C, 70, graph=0)


def test_sw_interleaves_with_metropolis(sm):
    """Metropolis sweeps, SW updates and Metropolis sweeps again share one
    sweep counter: the same sequence on the oracle gives the same state."""
    d, L, seed, ss = 2, 64, 8, 88
    lat = sm.Lattice(d, L, seed=seed)
    lat.sweep(BETA_C, 5, ss)
    lat.set_update(sm.SL_UPDATE_SW)
    lat.sweep(BETA_C, 4, ss)
    lat.set_option(sm.SL_OPT_UPDATE, sm.SL_UPDATE_METROPOLIS)
    lat.sweep(BETA_C, 3, ss)
    got = lat.get_spins()
    assert lat.state()[1] == 12
    lat.close()
    s = oracle.ising_init(d, L, seed)
    oracle.ising_sweeps(d, L, s, BETA_C, ss, 0, 5, series=False)
    oracle.ising_sw_sweeps(d, L, s, BETA_C, ss, 5, 4, series=False)
    oracle.ising_sweeps(d, L, s, BETA_C, ss, 9, 3, series=False)
    np.testing.assert_array_equal(got, s)


def test_sw_workspace_rules(sm):
    """A caller-owned lattice needs an attached workspace of
    sl_workspace_bytes before SW is selected; SW needs bytes and uniform J."""
    import torch
    d, L = 2, 64
    nb = sm.sl_required_bytes(d, L, 1, sm.SL_J_UNIFORM, sm.SL_STORE_I8)
    buf = torch.empty(nb, dtype=torch.uint8, device="cuda")
    h = sm.sl_create(d, L, 1, sm.SL_J_UNIFORM, sm.SL_STORE_I8, 1.0, None, 1, 0, buf, nb,
                     torch.cuda.current_stream().cuda_stream)
    need = sm.sl_workspace_bytes(h, sm.SL_UPDATE_SW)
    assert need >= 4 * L * L
    assert sm.sl_workspace_bytes(h, sm.SL_UPDATE_METROPOLIS) == 0
    with pytest.raises(sm.SpinMCError):
        sm.sl_set_option(h, sm.SL_OPT_UPDATE, sm.SL_UPDATE_SW)
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    sm.sl_attach_workspace(h, ws, need)
    sm.sl_set_option(h, sm.SL_OPT_UPDATE, sm.SL_UPDATE_SW)
    with pytest.raises(sm.SpinMCError):
        sm.sl_attach_workspace(h, ws, need - 1)
    sm.sl_sweep(h, BETA_C, 3, 9)
    sm.sl_destroy(h)
    for kw in (dict(storage=sm.SL_STORE_BITS), dict(J_bonds=inputs.ising_bonds(2, 64, 3))):
        lat = sm.Lattice(2, 64, **kw)
        with pytest.raises(sm.SpinMCError):
            lat.set_update(sm.SL_UPDATE_SW)
        lat.close()


@pytest.mark.slow
def test_sw_full_size_8192_one_update(sm):
    """The 8192^2 cluster workload (the paper's Table 1 row): one update from
    the random start and one more from its result, compared with the oracle on
    every spin, plus the measured E and |m|."""
    run_both(sm, 2, 8192, BETA_C, 2, seed=inputs.DEFAULT_SEED, sweep_seed=inputs.DEFAULT_SEED)
