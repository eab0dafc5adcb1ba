"""Write ``ea_long_runs.json``: the oracle's long replica-exchange runs of the
batched Edwards-Anderson workload, one disorder sample of each side.

Weigel & Yavors'kii 2011, Section 2 (spin-glass paragraph): independent
disorder samples; the batched workload runs 3D +-J samples of sides
[8, 12, 16, 24, 32][s mod 5], 32 temperatures geometric in [0.5, 3], replica
exchange after every sweep.  Global samples 0..4 are one sample of each side.
For each, this script runs the oracle for 10^4 sweeps from the sample's Philox
start state and records digests of the final spins of every slot, the
slot-to-temperature map and the whole energy series (plus a few series
values for diagnosis).  It calls only ``oracle/`` and the seeded input
parameters; the CUDA library is compared against the file it writes.

    python tests/golden/make_ea_long_runs.py      # about 15 minutes, 5 processes
"""
import hashlib
import json
import multiprocessing as mp
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

D, NT, NSWEEPS = 3, 32, 10_000
SEED, RUN_SEED = 0x5EED20111107546, 0x11075463
PROBES = (0, 1, 9, 99, 999, 4999, 9999)


def digest(a):
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


def run(sample):
    import oracle
    from paper_1107_5463_gb300 import inputs
    L = inputs.ea_sample_sizes(sample + 1)[sample]
    betas = inputs.geometric_betas(NT)
    jb = oracle.ea_couplings(D, L, SEED, sample)
    spins = np.stack([oracle.ising_init(D, L, SEED, sample * NT + r) for r in range(NT)])
    perm = np.arange(NT, dtype=np.int32)
    E = oracle.ea_pt_sweeps(D, L, jb, betas, RUN_SEED, sample, 0, NSWEEPS, spins, perm)
    return {"sample": sample, "L": L, "spins_sha256": digest(spins.astype(np.int8)),
            "slot_of_temp": perm.tolist(), "E_sha256": digest(E.astype(np.float64)),
            "E_probe": {str(t): E[t].tolist() for t in PROBES}}


def main():
    with mp.get_context("spawn").Pool(5) as pool:
        rows = pool.map(run, range(5))
    out = {"what": "oracle replica-exchange runs of one 3D EA +-J sample of each side",
           "d": D, "ntemps": NT, "betas": "geometric in [0.5, 3]", "nsweeps": NSWEEPS,
           "create_seed": SEED, "run_seed": RUN_SEED,
           "spins": "int8 +-1, array [slot][site], natural order",
           "E": "float64 array [sweep][temperature]", "samples": rows}
    with open(os.path.join(HERE, "ea_long_runs.json"), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
