"""Run oracle work in spawned worker processes (test infrastructure).

The oracle is single-threaded C; the largest parity cases (every sample of
the batched spin-glass workload) spread it over the host cores.  Workers are
started with ``spawn``: a process forked after the parent has touched the GPU
can hang.  The functions here only call ``oracle/`` and the seeded inputs.
"""
import multiprocessing as mp
import os

import numpy as np


def ea_sample_run(task):
    """Replica-exchange sweeps of one EA sample from its Philox start state:
    (couplings, spins [slot][N], slot of each temperature, E [sweep][temp])."""
    import oracle
    d, L, nt, betas, seed, run_seed, sample, nsw = task
    jb = oracle.ea_couplings(d, L, seed, sample)
    spins = np.stack([oracle.ising_init(d, L, seed, sample * nt + r) for r in range(nt)])
    perm = np.arange(nt, dtype=np.int32)
    E = oracle.ea_pt_sweeps(d, L, jb, np.asarray(betas, np.float64), run_seed, sample, 0, nsw,
                            spins, perm)
    return jb, spins, perm, E


def imap_spawn(fn, tasks, procs=None):
    """fn over tasks in spawned processes, results in task order (an iterator)."""
    procs = procs or os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    with ctx.Pool(procs) as pool:
        for r in pool.imap(fn, tasks, chunksize=4):
            yield r
