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


def test_profile_records_are_well_formed(tmp_path, monkeypatch):
    """Every committed ncu record names a bench workload, its kernel's
    source files (which exist) and a summary under profiles/; a record whose
    sources changed since the capture is ignored, so no stale DRAM or
    instruction figure reaches a bench line."""
    import json
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
        recs = json.load(f)
    for name, e in recs.items():
        assert name in bench.WORKLOADS, name
        for src in e["source_files"]:
            assert os.path.exists(os.path.join(ROOT, "paper_1107_5463_gb300", "csrc", src)), src
        assert os.path.exists(os.path.join(ROOT, e["summary"])), e["summary"]
        assert len(e["source_hash"]) == 16
        assert e.get("dram_bytes_per_launch") is None or e["dram_bytes_per_launch"] > 0
        assert e.get("thread_instructions_per_site") is None or e["thread_instructions_per_site"] > 0
    # in a scratch tree: a record is used only while its sources hash as recorded
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    (tmp_path / "profiles").mkdir()
    csrc = tmp_path / "paper_1107_5463_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "k.cu").write_text("// kernel\n")
    good = bench.kernel_source_hash(["k.cu"])
    rec = {"a": {"source_files": ["k.cu"], "source_hash": good, "dram_bytes_per_launch": 5},
           "b": {"source_files": ["k.cu"], "source_hash": "0" * 16, "dram_bytes_per_launch": 7},
           "c": {"source_files": ["gone.cu"], "source_hash": good, "dram_bytes_per_launch": 9}}
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(rec))
    assert bench.recorded_traffic("a") == 5
    assert bench.recorded_traffic("b") is None
    assert bench.recorded_traffic("c") is None
    assert bench.recorded_profile("missing") is None
    (csrc / "k.cu").write_text("// kernel, edited\n")
    assert bench.recorded_traffic("a") is None
