"""The launch-shape autotuner of the streaming sweep kernels (sl_autotune).

Rows per thread and the grid cap change only which thread updates which site
and when; every random number is keyed by its site, so each shape the tuner
may pick must give the same chain: bit-identical Ising spins and series,
identical FP32 continuous spins.  Their FP64 observable totals may differ:
each thread adds its sites' FP32 terms (up to 64 sites, terms up to 2d in
size) before the FP64 block sums, and the shape decides which sites a thread
adds; an FP32 partial then errs by at most 64 x 2d x 2^-24 (2.3e-5 for E,
3.8e-6 for M), and the totals, sums of about N/64 such partials, by about
sqrt(N/64) times that, so E agrees within 1e-6 relative and |m| within 1e-7
(measured differences: 1.1e-8 relative and 1.2e-9).  Tuning restores the spins
and the sweep counter, so a tuned run continues exactly like an untuned one;
its choice is cached by device and configuration."""
import json

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROWS = (1, 2, 4, 8, 16, 32)
CAPS = (0, 2, 4, 8, 16)


@pytest.fixture(scope="module")
def sm():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1107_5463_gb300 import spinmc
    return spinmc


def make(sm, d, L, n, storage):
    st = None if storage is None else getattr(sm, storage)
    return sm.Lattice(d, L, n=n, seed=4, storage=st)


def run(lat, beta, nsw, seed=8):
    E, m = lat.sweep_series(beta, nsw, seed)
    return lat.get_spins(), E.cpu().numpy(), m.cpu().numpy()


CASES = [(2, 256, 1, None, 0.44), (3, 64, 1, None, 0.2216546), (2, 256, 1, "SL_STORE_BITS", 0.44),
         (3, 64, 1, "SL_STORE_BITS", 0.2216546), (2, 256, 2, None, 1.12), (3, 64, 3, None, 0.693),
         (2, 128, 3, None, 1.5)]


@pytest.mark.parametrize("d,L,n,storage,beta", CASES)
def test_every_shape_gives_the_same_chain(sm, d, L, n, storage, beta):
    ref_lat = make(sm, d, L, n, storage)
    ref = run(ref_lat, beta, 4)
    ref_lat.close()
    for R in ROWS:
        if L % R:
            continue
        for cap in CAPS:
            lat = make(sm, d, L, n, storage)
            lat.set_option(sm.SL_OPT_ROWS, R)
            lat.set_option(sm.SL_OPT_BLOCKS_PER_SM, cap)
            got = run(lat, beta, 4)
            lat.close()
            np.testing.assert_array_equal(got[0], ref[0], err_msg="R=%d cap=%d" % (R, cap))
            if n == 1:
                np.testing.assert_array_equal(got[1], ref[1])
                np.testing.assert_array_equal(got[2], ref[2])
            else:
                np.testing.assert_allclose(got[1], ref[1], rtol=1e-6)   # E
                np.testing.assert_allclose(got[2], ref[2], rtol=0, atol=1e-7)   # |m|


@pytest.mark.parametrize("d,L,n,storage,beta", CASES[:3] + CASES[4:6])
def test_tuning_leaves_the_run_unchanged(sm, d, L, n, storage, beta, tmp_path):
    a = make(sm, d, L, n, storage)
    ra1 = run(a, beta, 3)
    ra2 = run(a, beta, 3)
    a.close()
    b = make(sm, d, L, n, storage)
    rb1 = run(b, beta, 3)
    cache = str(tmp_path / "tune.jsonl")
    R, cap = b.autotune(beta, trial_sweeps=2, cache_path=cache)
    assert L % R == 0 and cap in CAPS
    rb2 = run(b, beta, 3)
    b.close()
    for q, (x, y) in enumerate(zip(ra1 + ra2, rb1 + rb2)):
        if q % 3 == 0 or n == 1:
            np.testing.assert_array_equal(x, y)                     # spins, Ising series
        elif q % 3 == 1:
            np.testing.assert_allclose(x, y, rtol=1e-6)             # E
        else:
            np.testing.assert_allclose(x, y, rtol=0, atol=1e-7)     # |m|
    # the choice is cached: one line, reused by the next lattice of this shape
    lines = open(cache).read().splitlines()
    assert len(lines) == 1
    j = json.loads(lines[0])
    assert (j["d"], j["L"], j["n"], j["rows"], j["blocks_per_sm"]) == (d, L, n, R, cap)
    c = make(sm, d, L, n, storage)
    assert c.autotune(beta, trial_sweeps=2, cache_path=cache) == (R, cap)
    c.close()
    assert len(open(cache).read().splitlines()) == 1


def test_untunable_lattices_keep_their_options(sm):
    lat = sm.Lattice(2, 30, seed=1)   # rows too short for the streaming kernel
    assert lat.autotune(0.4) == (0, 0)
    lat.close()
