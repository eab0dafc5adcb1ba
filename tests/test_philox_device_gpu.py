"""Pins of the oracle's Philox4x32-10 and of its counter readings to cuRAND's
device-API Philox4_32_10 generator (a library routine, built from its header
into a small test kernel and called on the GPU).

curand_init(seed, subsequence, offset) followed by curand4() returns Philox
of the counter (offset/4 low word, offset/4 high word, subsequence low word,
subsequence high word) under the key (seed_lo, seed_hi) for offsets that are
multiples of 4.  Unlike the host generator (whose counters have word 3 = 0),
this reaches word 3, which carries the purpose and colour of every draw the
method makes.  The counter readings themselves (which counter and which
output a site, a bond or a start spin uses) are pinned by drawing them here
from cuRAND and comparing with the oracle's couplings and start states."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
from paper_1107_5463_gb300 import inputs

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def curand_dev():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    out_dir = os.path.join(HERE, "_build")
    os.makedirs(out_dir, exist_ok=True)
    lib = os.path.join(out_dir, "libcurandprobe.so")
    src = os.path.join(HERE, "curand_device_philox.cu")
    if not os.path.exists(lib) or os.path.getmtime(lib) < os.path.getmtime(src):
        subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-shared",
                        "-Xcompiler", "-fPIC", "-o", lib, src], check=True)
    L = ctypes.CDLL(lib)
    L.curand_device_philox.argtypes = [ctypes.c_ulonglong, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_int, ctypes.c_void_p]
    L.curand_device_philox.restype = ctypes.c_int

    def blocks(seed, counters):
        """cuRAND's block for each 4-word counter (words 0, 1 < 2^30 here)."""
        c = np.asarray(counters, np.uint64).reshape(-1, 4)
        sub = np.ascontiguousarray(c[:, 2] | (c[:, 3] << np.uint64(32)))
        off = np.ascontiguousarray((c[:, 0] | (c[:, 1] << np.uint64(32))) * np.uint64(4))
        out = np.zeros((len(c), 4), np.uint32)
        rc = L.curand_device_philox(seed, sub.ctypes.data, off.ctypes.data, len(c),
                                    out.ctypes.data)
        assert rc == 0, rc
        return out
    return blocks


@pytest.mark.parametrize("seed", [0, 1, 0xFFFFFFFF, 1 << 32, inputs.DEFAULT_SEED, 2**64 - 1])
def test_philox_matches_curand_device_api_on_all_counter_words(curand_dev, seed):
    rng = np.random.default_rng(seed % 1000)
    ctrs = np.column_stack([rng.integers(0, 2**30, 64), rng.integers(0, 2**30, 64),
                            rng.integers(0, 2**32, 64), rng.integers(0, 2**32, 64)])
    # the word-3 values the method uses: purpose << 1 | colour, heat-bath attempts
    special = [[5, 7, 3, w3] for w3 in (0, 1, 2, 3, 4, 5, 8, 9, 10, 11, 12, 13, 18, 20, 22,
                                        (31 << 16) | 1)]
    ctrs = np.concatenate([ctrs, np.array(special)]).astype(np.uint64)
    got = curand_dev(seed, ctrs)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for c, g in zip(ctrs, got):
        np.testing.assert_array_equal(oracle.philox4x32_10(c.astype(np.uint32), key), g)


@pytest.mark.parametrize("d,L,sample", [(3, 8, 0), (3, 12, 77), (2, 16, 1023)])
def test_ea_couplings_are_the_documented_draws(curand_dev, d, L, sample):
    """J of the forward bond (i, i + e_mu) of a sample is +1 iff the top bit of
    output 0 of Philox(i, mu, sample, 2 << 1) is set."""
    seed = inputs.DEFAULT_SEED
    jb = oracle.ea_couplings(d, L, seed, sample)
    rng = np.random.default_rng(sample)
    picks = [(int(i), mu) for i in rng.integers(0, L ** d, 40) for mu in range(d)]
    got = curand_dev(seed, [[i, mu, sample, 2 << 1] for i, mu in picks])
    for (i, mu), g in zip(picks, got):
        assert jb[mu, i] == (1 if g[0] >> 31 else -1), (i, mu)


@pytest.mark.parametrize("d,L,replica", [(2, 16, 0), (3, 8, 37)])
def test_ising_start_spins_are_the_documented_draws(curand_dev, d, L, replica):
    """Start spin of site i (colour c, j = i >> 1) is +1 iff the top bit of
    output j & 3 of Philox(j >> 2, 0, replica, 1 << 1 | c) is set."""
    seed = 12345
    s = oracle.ising_init(d, L, seed, replica)
    sites = list(range(0, L ** d, 3))

    def colour(i):
        x, r = i % L, i // L
        return (x + r % L + r // L) & 1
    got = curand_dev(seed, [[(i >> 1) >> 2, 0, replica, (1 << 1) | colour(i)] for i in sites])
    for i, g in zip(sites, got):
        assert s[i] == (1 if g[(i >> 1) & 3] >> 31 else -1), i
