"""The throughput microbenchmarks the bench composes into measured compute
ceilings: the Philox one computes the real Philox4x32-10 (its per-thread
checksums equal the oracle's Philox on sampled threads), the others run and
report the operations they perform, and bad arguments are rejected."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sm():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1107_5463_gb300 import spinmc
    return spinmc


def run(sm, kind, iters):
    import torch
    n = sm.sl_microbench_threads()
    out = torch.zeros(n, dtype=torch.int32, device="cuda")
    ops = sm.sl_microbench(kind, iters, out, out.numel() * 4,
                           torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return n, ops, out.cpu().numpy()


def test_philox_microbenchmark_computes_philox(sm):
    iters = 5
    n, ops, out = run(sm, sm.SL_MB_PHILOX, iters)
    assert ops == n * iters
    key = [1, 0]
    for g in (0, 1, 31, 4095, n // 2, n - 1):
        acc = 0
        for i in range(iters):
            r = oracle.philox4x32_10([g * iters + i, 7, 0, 0], key)
            acc ^= int(r[0]) ^ int(r[1]) ^ int(r[2]) ^ int(r[3])
        assert np.uint32(out[g]) == np.uint32(acc), g


@pytest.mark.parametrize("kind,per_step", [(1, 16), (2, 8), (3, 8)])
def test_other_microbenchmarks_run(sm, kind, per_step):
    n, ops, out = run(sm, kind, 64)
    assert ops == n * 64 * per_step
    if kind != 1:
        assert np.isfinite(out.view(np.float32)).all()


def test_microbenchmark_argument_checks(sm):
    import torch
    n = sm.sl_microbench_threads()
    out = torch.zeros(n, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for kind, iters, nbytes in ((7, 4, 4 * n), (0, 0, 4 * n), (0, 4, 4 * n - 4),
                                (0, 2 ** 31 - 1, 4 * n)):
        with pytest.raises(sm.SpinMCError):
            sm.sl_microbench(kind, iters, out, nbytes, stream)
