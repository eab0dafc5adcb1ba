"""GPU parity of the Ising int8 path (C ABI) against the CPU oracle.

Bit-exact: the start configuration, every spin after the sweeps, and the
per-sweep energy and |m| series (Section 2: Eq. 1, Eq. 2, checkerboard
order).  Sizes span several tiles with ragged tails; both kernels (generic
per-site and row-streaming) are checked, plus the full-size workloads of the
paper's Table 1 (2D L = 16384, 3D L = 512) on their first sweeps.
"""
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


def gpu_run(sm, d, L, beta, seed, sweep_seed, nsw, J=1.0, Jb=None, kernel=0, rows=0, graph=1,
            start=None, replica=0, bits=False):
    lat = sm.Lattice(d, L, n=1, J=J, J_bonds=Jb, seed=seed, replica=replica,
                     storage=sm.SL_STORE_BITS if bits else None)
    if kernel:
        lat.set_option(sm.SL_OPT_KERNEL, kernel)
    if rows:
        lat.set_option(sm.SL_OPT_ROWS, rows)
    lat.set_option(sm.SL_OPT_GRAPH, graph)
    if start is not None:
        lat.set_spins(start)
    E, m = lat.sweep_series(beta, nsw, sweep_seed)
    out = lat.get_spins(), E.cpu().numpy(), m.cpu().numpy()
    lat.close()
    return out


def oracle_run(d, L, beta, seed, sweep_seed, nsw, J=1.0, Jb=None, start=None, replica=0):
    s = oracle.ising_init(d, L, seed, replica) if start is None else start.copy()
    E, m = oracle.ising_sweeps(d, L, s, beta, sweep_seed, 0, nsw, J=J, Jb=Jb, replica=replica)
    return s, E, m


def assert_same(got, ref):
    np.testing.assert_array_equal(got[0], ref[0])
    np.testing.assert_array_equal(got[1], ref[1])
    np.testing.assert_array_equal(got[2], ref[2])


@pytest.mark.parametrize("d,L", [(2, 2), (2, 6), (2, 64), (3, 2), (3, 6), (3, 32)])
def test_start_configuration_matches_oracle(sm, d, L):
    for seed in (1, inputs.DEFAULT_SEED):
        lat = sm.Lattice(d, L, n=1, seed=seed, replica=3)
        np.testing.assert_array_equal(lat.get_spins(), oracle.ising_init(d, L, seed, 3))
        lat.close()


CASES = [
    # d, L, kernel: generic on ragged sizes, streaming where W % 16 == 0
    (2, 2, GEN), (2, 4, GEN), (2, 6, GEN), (2, 10, GEN), (2, 32, GEN), (2, 32, STREAM),
    (2, 64, STREAM), (2, 96, STREAM), (2, 160, STREAM), (2, 1024, STREAM),
    (3, 2, GEN), (3, 4, GEN), (3, 6, GEN), (3, 32, GEN), (3, 32, STREAM), (3, 64, STREAM),
]


@pytest.mark.parametrize("d,L,kernel", CASES)
@pytest.mark.parametrize("beta,J", [(BETA_C, 1.0), (0.25, -0.7)])
def test_uniform_coupling_parity(sm, d, L, kernel, beta, J):
    nsw = 12
    got = gpu_run(sm, d, L, beta, 5, 77, nsw, J=J, kernel=kernel)
    assert_same(got, oracle_run(d, L, beta, 5, 77, nsw, J=J))


@pytest.mark.parametrize("d,L,kernel", [(2, 6, GEN), (2, 32, STREAM), (2, 64, GEN),
                                        (3, 4, GEN), (3, 32, STREAM), (3, 32, GEN)])
def test_pm_bond_parity(sm, d, L, kernel):
    jb = inputs.ising_bonds(d, L, 41)
    got = gpu_run(sm, d, L, 0.9, 6, 78, 10, Jb=jb, kernel=kernel, replica=9)
    assert_same(got, oracle_run(d, L, 0.9, 6, 78, 10, Jb=jb, replica=9))


@pytest.mark.parametrize("d,L", [(2, 4), (2, 32), (3, 6)])
def test_bonds_with_zeros_parity(sm, d, L):
    jb = inputs.ising_bonds(d, L, 42, p_zero=0.3)
    got = gpu_run(sm, d, L, 0.7, 7, 79, 10, J=1.3, Jb=jb)
    assert_same(got, oracle_run(d, L, 0.7, 7, 79, 10, J=1.3, Jb=jb))


def test_2d_L64_full_run_bit_exact(sm):
    """The 2D Ising workload of side 64 at beta_c: 10^4 sweeps, E and |m|
    after every sweep, identical to the oracle."""
    seed = inputs.DEFAULT_SEED
    got = gpu_run(sm, 2, 64, BETA_C, seed, seed, 10_000)
    assert_same(got, oracle_run(2, 64, BETA_C, seed, seed, 10_000))


@pytest.mark.slow
@pytest.mark.parametrize("d,L,beta", [(2, 16384, 0.440687), (3, 512, inputs.BETA_3D_ISING)])
def test_full_size_first_sweeps_bit_exact(sm, d, L, beta):
    """Full-size single-lattice workloads of the paper's Table 1 in the launch
    configuration the bench times (automatic kernel choice, graphs on), with
    byte and bit storage."""
    seed = inputs.DEFAULT_SEED
    ref = oracle_run(d, L, beta, seed, seed + 1, 5)
    assert_same(gpu_run(sm, d, L, beta, seed, seed + 1, 5), ref)
    assert_same(gpu_run(sm, d, L, beta, seed, seed + 1, 5, bits=True), ref)


def sample_sites(d, L, colour, c, n, rng):
    """n random sites of colour c plus every site of colour c on the lattice's
    first and last two columns of the first and last rows (and planes)."""
    N = L ** d
    pick = rng.integers(0, N, 4 * n, dtype=np.int64)
    pick = pick[colour(pick) == c][:n]
    edge = [0, 1, L - 2, L - 1]
    cand = np.array([x + L * y + (L * L * z if d == 3 else 0)
                     for x in edge for y in edge for z in (edge if d == 3 else [0])],
                    np.int64)
    return np.unique(np.concatenate([pick, cand[colour(cand) == c]]))


@pytest.mark.slow
@pytest.mark.parametrize("d,L,bits", [(2, 63232, False), (2, 63230, False), (3, 1568, False),
                                      (2, 63232, True)])
def test_maximum_size_sampled_sites(sm, d, L, bits):
    """Lattices at the library's limit of 4e9 sites (63232^2, the ragged
    63230^2 on the per-site kernel, 1568^3; bytes and bits): one sweep in the
    bench's launch configuration from the Philox start; 8192 sampled sites of
    each colour, every lattice corner among them, against the oracle's
    single-site update from the configuration that colour's pass sees; the
    swept |m| against the final state, and in 2D bytes the energy too."""
    seed, sweep_seed, t = inputs.DEFAULT_SEED, 77, 0
    lat = sm.Lattice(d, L, n=1, seed=seed, storage=sm.SL_STORE_BITS if bits else None)
    before = lat.get_spins()
    E, m = lat.sweep_series(BETA_C if d == 2 else inputs.BETA_3D_ISING, 1, sweep_seed)
    beta = BETA_C if d == 2 else inputs.BETA_3D_ISING
    after = lat.get_spins()
    lat.close()
    N = L ** d

    def colour(i):
        x, y, z = i % L, (i // L) % L, i // (L * L)
        return (x + y + (z if d == 3 else 0)) & 1

    rng = np.random.default_rng(5)
    s0 = sample_sites(d, L, colour, 0, 8192, rng)
    s1 = sample_sites(d, L, colour, 1, 8192, rng)
    ref0 = oracle.ising_site_updates(d, L, before, s0, beta, sweep_seed, t)
    np.testing.assert_array_equal(after[s0], ref0)
    # colour 1 sees the colour-0 result and its own value before the sweep
    got1 = after[s1].copy()
    assert abs(int(after.sum(dtype=np.int64))) / N == pytest.approx(float(m[0].item()), abs=0)
    if d == 2 and not bits:
        from tests.exact import chunked_energy
        assert chunked_energy(after, d, L) == float(E[0].item())
    after[s1] = before[s1]
    ref1 = oracle.ising_site_updates(d, L, after, s1, beta, sweep_seed, t)
    np.testing.assert_array_equal(got1, ref1)


@pytest.mark.parametrize("d,L", [(2, 64), (2, 192), (2, 1024), (3, 64), (3, 128)])
@pytest.mark.parametrize("beta,J", [(BETA_C, 1.0), (0.3, -0.7)])
def test_bit_storage_parity(sm, d, L, beta, J):
    """Multispin (one bit per site) storage: same start state and the same
    trajectory as the oracle, bit for bit."""
    got = gpu_run(sm, d, L, beta, 5, 77, 12, J=J, bits=True)
    assert_same(got, oracle_run(d, L, beta, 5, 77, 12, J=J))


def test_bit_storage_io_and_measure(sm):
    for d, L in ((2, 128), (3, 64)):
        s = inputs.ising_spins(d, L, 3)
        lat = sm.Lattice(d, L, storage=sm.SL_STORE_BITS)
        lat.set_spins(s)
        np.testing.assert_array_equal(lat.get_spins(), s)
        E, M = lat.measure()
        E_ref, M_ref = oracle.ising_measure(d, L, s)
        assert E == E_ref and M[0] == M_ref
        lat.close()


def test_kernels_rows_and_graphs_agree(sm):
    """Decomposition invariance: the random stream is keyed by site and sweep,
    so kernel choice, rows per thread and graph replay cannot change a bit."""
    ref = gpu_run(sm, 2, 128, BETA_C, 3, 4, 100, kernel=GEN, graph=0)
    for kernel, rows, graph in ((STREAM, 0, 1), (STREAM, 1, 1), (STREAM, 4, 0), (STREAM, 128, 1)):
        assert_same(gpu_run(sm, 2, 128, BETA_C, 3, 4, 100, kernel=kernel, rows=rows, graph=graph),
                    ref)


def test_sweeps_compose_and_resume_from_checkpoint(sm):
    d, L, beta = 3, 32, 0.3
    straight = gpu_run(sm, d, L, beta, 8, 9, 90)
    lat = sm.Lattice(d, L, seed=8)
    lat.sweep(beta, 20, 9)
    lat.sweep(beta, 25, 9)
    seed0, done = lat.state()
    assert (seed0, done) == (8, 45)
    snap = lat.get_spins()
    lat.close()
    lat2 = sm.Lattice(d, L, seed=1234)
    lat2.set_spins(snap)
    lat2.set_state(done)
    E, m = lat2.sweep_series(beta, 45, 9)
    np.testing.assert_array_equal(lat2.get_spins(), straight[0])
    np.testing.assert_array_equal(E.cpu().numpy(), straight[1][45:])
    lat2.close()


def test_measure_matches_oracle_on_arbitrary_state(sm):
    for d, L, J, bonds in ((2, 30, 1.0, False), (3, 12, -0.4, True)):
        s = inputs.ising_spins(d, L, 17)
        jb = inputs.ising_bonds(d, L, 18) if bonds else None
        lat = sm.Lattice(d, L, J=J, J_bonds=jb)
        lat.set_spins(s)
        E, M = lat.measure()
        E_ref, M_ref = oracle.ising_measure(d, L, s, J=J, Jb=jb)
        assert E == E_ref and M[0] == M_ref and M[1] == abs(M_ref) / L**d
        lat.close()


def test_beta_zero_flips_every_spin(sm):
    s0 = inputs.ising_spins(2, 64, 5)
    got = gpu_run(sm, 2, 64, 0.0, 1, 2, 1, start=s0)
    np.testing.assert_array_equal(got[0], -s0)


def test_bad_arguments_are_rejected(sm):
    lat = sm.Lattice(2, 16)
    for beta in (-0.1, float("nan"), 1e4):
        with pytest.raises(sm.SpinMCError) as ei:
            lat.sweep(beta, 1, 0)
        assert ei.value.status == sm.SL_EINVAL
    with pytest.raises(sm.SpinMCError):
        lat.set_option(sm.SL_OPT_KERNEL, STREAM)  # W = 8 is not a multiple of 16
    with pytest.raises(sm.SpinMCError):
        lat.set_option(sm.SL_OPT_ROWS, 5)
    lat.sweep(0.3, 0, 0)  # zero sweeps is a no-op
    assert lat.state()[1] == 0
    lat.close()
    jb = inputs.ising_bonds(2, 16, 1)
    jb[0, 3] = 2
    with pytest.raises(sm.SpinMCError) as ei:
        sm.Lattice(2, 16, J_bonds=jb)
    assert ei.value.status == sm.SL_EINVAL
