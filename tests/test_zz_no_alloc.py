"""The allocation-free measurement entry point (sl_ising_measure_static).

It serves callers that cannot call cudaMalloc (code under another framework's
device-memory pool, or a latency-critical loop), so it keeps its reduction
scratch in a static device array.  Its results must equal those of the
regular entry point (sl_measure on a lattice holding the same spins), exactly
for these integer sums, on consecutive calls that reuse the shared scratch.
This file is collected last so that a stop at the first failure has run every
other test first; it also passes alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

from paper_1107_5463_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sm():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1107_5463_gb300 import spinmc
    return spinmc


def test_static_measure_matches_regular_entry_point_on_consecutive_calls(sm):
    import torch
    stream = torch.cuda.current_stream()
    out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
    cases = [(2, 256, 1.0, 1), (3, 64, -0.7, 2), (2, 256, 1.0, 1), (3, 38, 0.4, 3)]
    for d, L, J, seed in cases:
        s = inputs.ising_spins(d, L, seed)
        lat = sm.Lattice(d, L, J=J)
        lat.set_spins(s)
        E_ref, M_ref = lat.measure()
        lat.close()
        dev_s = torch.from_numpy(s).to("cuda")
        st = sm._lib.sl_ising_measure_static(d, L, J, ctypes.c_void_p(dev_s.data_ptr()),
                                             ctypes.c_void_p(out.data_ptr()),
                                             ctypes.c_void_p(stream.cuda_stream))
        assert st == sm.SL_OK
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert got[0] == E_ref and got[1] == M_ref[0], (d, L, got, E_ref, M_ref)


def test_static_measure_rejects_lattices_beyond_its_scratch(sm):
    import torch
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    dummy = torch.zeros(16, dtype=torch.int8, device="cuda")
    with pytest.raises(sm.SpinMCError) as ei:
        sm.sl_ising_measure_static(2, 16386, 1.0, dummy, out, None)
    assert ei.value.status == sm.SL_EINVAL
    assert "static scratch" in str(ei.value)
