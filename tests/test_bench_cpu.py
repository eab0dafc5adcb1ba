"""Host-side pieces of bench.py that run without a GPU: the bounded oracle
sample behind `--impl reference` for every workload in the table (it builds
and takes a step, and counts the site updates it makes), the sample sides,
and the table's own consistency."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


@pytest.mark.parametrize("name", sorted(bench.WORKLOADS))
def test_reference_sample_steps_every_workload(name):
    wl = bench.WORKLOADS[name]
    step, n, desc = bench.reference_sample(wl)
    assert n > 0 and isinstance(desc, str) and desc
    step(0)


def test_sample_sides_fit_their_workloads():
    for name, wl in bench.WORKLOADS.items():
        if wl["storage"] in ("walkers", "batch"):
            continue
        Ls = bench.sample_side(wl)
        assert 2 <= Ls <= wl["L"] and Ls % 2 == 0, name
        if wl.get("multihit"):
            assert Ls % (2 * wl["tile"]) == 0, name


def test_workload_table():
    assert bench.HEADLINE in bench.WORKLOADS
    for name, wl in bench.WORKLOADS.items():
        assert wl["d"] in (2, 3) and wl["L"] % 2 == 0, name
        assert wl["storage"] in ("i8", "bits", "vec", "angle", "walkers", "batch"), name
        assert wl["desc"], name
        if wl["storage"] in ("i8", "bits", "vec", "angle"):
            assert wl["n"] == {"i8": 1, "bits": 1, "vec": 3, "angle": 2}[wl["storage"]], name


@pytest.mark.parametrize("world", [1, 2, 3, 4, 8])
def test_batch_sample_ranges_partition_the_batch(world):
    """Each rank's contiguous block of global samples; together they cover
    0..nsamples-1 once, in order (the batch's first_sample is lo)."""
    n = bench.WORKLOADS["ea3d_batch_1024x32"]["samples"]
    got = []
    for r in range(world):
        lo, hi = bench.sample_range(n, r, world)
        assert hi - lo in (n // world, n // world + 1)
        got.extend(range(lo, hi))
    assert got == list(range(n))
