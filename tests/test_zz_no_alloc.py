"""The allocation-free measurement entry point (sl_ising_measure_static).

It serves callers that cannot call cudaMalloc (code under another framework's
device-memory pool, or a latency-critical loop), so it keeps its reduction
scratch in a static device array.  Its results must equal the CPU oracle's
energy and magnetisation of the same configuration, exactly for these integer
sums, and equal those of the regular entry point (sl_measure on a lattice
holding the same spins), on consecutive calls that reuse the shared scratch,
up to the largest lattice the scratch serves (2^28 sites: 2D L = 16384 fills
all of its blocks).  This file is collected last so that a stop at the first
failure has run every other test first; it also passes alone in a fresh
process.
"""
import ctypes

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


def static_measure(sm, d, L, J, dev_s, out, stream):
    import torch
    out.fill_(float("nan"))
    st = sm._lib.sl_ising_measure_static(d, L, J, ctypes.c_void_p(dev_s.data_ptr()),
                                         ctypes.c_void_p(out.data_ptr()),
                                         ctypes.c_void_p(stream.cuda_stream))
    assert st == sm.SL_OK
    torch.cuda.synchronize()
    return out.cpu().numpy()


def test_static_measure_matches_oracle_and_regular_entry_point(sm):
    import torch
    stream = torch.cuda.current_stream()
    out = torch.empty(2, dtype=torch.float64, device="cuda")
    cases = [(2, 256, 1.0, 1), (3, 64, -0.7, 2), (2, 256, 1.0, 1), (3, 38, 0.4, 3), (2, 2, 1.0, 4)]
    for d, L, J, seed in cases:
        s = inputs.ising_spins(d, L, seed)
        E_orc, M_orc = oracle.ising_measure(d, L, s, J=J)
        lat = sm.Lattice(d, L, J=J)
        lat.set_spins(s)
        E_ref, M_ref = lat.measure()
        lat.close()
        dev_s = torch.from_numpy(s).to("cuda")
        for _ in range(2):
            got = static_measure(sm, d, L, J, dev_s, out, stream)
            assert got[0] == E_orc and got[1] == M_orc, (d, L, got, E_orc, M_orc)
            assert got[0] == E_ref and got[1] == M_ref[0], (d, L, got, E_ref, M_ref)


@pytest.mark.parametrize("d,L,J", [(2, 16384, 1.0), (3, 644, -1.0)])
def test_static_measure_at_its_size_limit(sm, d, L, J):
    """2D L = 16384 is exactly 2^28 sites (every scratch block in use) and 3D
    L = 644 the largest cube below it; two calls in a row against the
    oracle."""
    import torch
    stream = torch.cuda.current_stream()
    out = torch.empty(2, dtype=torch.float64, device="cuda")
    s = inputs.ising_spins(d, L, 11)
    E_orc, M_orc = oracle.ising_measure(d, L, s, J=J)
    dev_s = torch.from_numpy(s).to("cuda")
    for _ in range(2):
        got = static_measure(sm, d, L, J, dev_s, out, stream)
        assert got[0] == E_orc and got[1] == M_orc, (d, L, got, E_orc, M_orc)


def test_static_measure_rejects_lattices_beyond_its_scratch(sm):
    import torch
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    dummy = torch.zeros(16, dtype=torch.int8, device="cuda")
    # 2D just above 2^28, 3D just above, and 3D sides whose L^3 overflows
    # 64-bit integers (2^21) or wraps to a small count (2^22 + 2)
    for d, L in ((2, 16386), (3, 646), (3, 1 << 21), (3, (1 << 22) + 2), (3, 1 << 30)):
        with pytest.raises(sm.SpinMCError) as ei:
            sm.sl_ising_measure_static(d, L, 1.0, dummy, out, None)
        assert ei.value.status == sm.SL_EINVAL
        assert "static scratch" in str(ei.value)
