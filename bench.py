#!/usr/bin/env python
"""Throughput of the checkerboard Metropolis sweep (Weigel & Yavors'kii 2011,
Section 2, Table 1) on one GB300, in spin flips per nanosecond.

One step = one full sweep (colour 0, colour 1, fused energy and |m|) of the
workload lattice, inputs resident in HBM.  The headline workload is the 2D
Ising ferromagnet of side 16384 (2.7e8 int8 spins, larger than L2) at
beta_c = 0.440687 from a random start.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun every rank runs its own independent replica (weak scaling);
rank 0 prints one JSON line.  ``--impl reference`` times the CPU oracle (the
plain C restatement of the method) on the host cores instead.
"""
import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "spin flips/ns"
UNIT = "flips/ns"

# bytes: algorithmic HBM bytes per site update of one colour pass (read the
# updated colour and the other colour, write the updated colour)
# ops: algorithmic 32-bit lane operations (integer and FP32) per site update:
#   Ising bytes 28: a quarter of a Philox4x32-10 call = 10 rounds x (2 mulhi +
#     2 mullo + 4 xor) / 4 = 20, plus about 8 for the neighbour count,
#     threshold compares and flip (30 in 3D: two more neighbours);
#   Ising bits 26 (2D) / 28 (3D): the quarter call, the d threshold compares
#     with their bit insertion, a share of the word-wide neighbour logic;
#   XY 66: half a call (40), sin/cos of the proposal (and the own and one
#     neighbour angle, computed once per value) and the FP32 field, dE and
#     acceptance (about 26); heat-bath 100 (about 1.3 Best-Fisher attempts of
#     half a call each, the sampler's setup and the new angle);
#   Heisenberg 120 in 3D / 110 in 2D: one call (80), the sphere point, the
#     FP32 field of 2d neighbours and dE, the acceptance; heat-bath 140 (the
#     exponential inverse and the basis around h);
#   spin-glass batch 28 per (site, replica): the quarter call and d threshold
#     compares; the neighbour logic is word-wide over 32 replicas;
#   walkers 40 (Wang-Landau) / 36 (multicanonical) per attempted flip: the
#     quarter call, five lattice words, the level step, the decision and the
#     histogram and ln g updates.
WORKLOADS = {
    "ising2d_L16384_i8": dict(d=2, L=16384, n=1, beta=0.440687, storage="i8", bytes=3.0, ops=28,
                              desc="2D Ising ferromagnet J=1, L=16384 periodic, int8 spins, "
                                   "beta_c=0.440687, random start"),
    "ising3d_L512_i8": dict(d=3, L=512, n=1, beta=0.2216546, storage="i8", bytes=3.0, ops=30,
                            desc="3D Ising ferromagnet J=1, L=512 simple cubic, int8 spins, "
                                 "beta=0.2216546, random start"),
    "ising2d_L16384_i8_heatbath": dict(d=2, L=16384, n=1, beta=0.440687, storage="i8",
                                       bytes=3.0, ops=28, update=1,
                                       desc="2D Ising, L=16384, int8 spins, heat-bath rule"),
    "ising2d_L16384_i8_k100": dict(d=2, L=16384, n=1, beta=0.440687, storage="i8", bytes=0.0,
                                   ops=28, multihit=100, tile=16, paper_flips_per_ns=1 / 0.034,
                                   desc="2D Ising, L=16384, int8 spins, k=100 multi-hit in "
                                        "16x16 tiles (the mode of the paper's Table 1)"),
    "ising2d_L16384_bits": dict(d=2, L=16384, n=1, beta=0.440687, storage="bits", bytes=0.375,
                                ops=26,
                                desc="2D Ising, L=16384, one bit per spin"),
    "ising3d_L512_bits": dict(d=3, L=512, n=1, beta=0.2216546, storage="bits", bytes=0.375,
                              ops=28,
                              desc="3D Ising, L=512, one bit per spin"),
    "ising2d_L8192_sw": dict(d=2, L=8192, n=1, beta=0.440687, storage="i8", bytes=16.0,
                             update=2, paper_flips_per_ns=1 / 4.62,
                             kernels="sw_local, sw_merge, sw_resolve, sw_flip, measurement",
                             desc="2D Ising ferromagnet J=1, L=8192, int8 spins, beta_c, "
                                  "Swendsen-Wang cluster updates (the paper's Table 1 "
                                  "cluster row)"),
    "wl2d_L64_windows": dict(d=2, L=64, n=1, beta=None, storage="walkers", bytes=0.0, ops=40,
                             kind="wl", wpw=128, width=4, paper_flips_per_ns=1 / 0.94,
                             desc="2D Ising L=64, Wang-Landau walkers in 1023 windows of 5 "
                                  "levels (dE = 16) sharing edge levels, 128 walkers each "
                                  "(the paper's Table 1 Wang-Landau row)"),
    "muca2d_L64_windows": dict(d=2, L=64, n=1, beta=None, storage="walkers", bytes=0.0, ops=36,
                               kind="muca", wpw=128, width=4, paper_flips_per_ns=1 / 0.33,
                               desc="2D Ising L=64, multicanonical walkers in 1023 windows of 5 "
                                    "levels sharing edge levels, 128 walkers each, weights from "
                                    "a Wang-Landau run (the paper's Table 1 multicanonical row)"),
    "heis3d_L256_f32": dict(d=3, L=256, n=3, beta=0.693, storage="vec", bytes=36.0, ops=120,
                            desc="3D Heisenberg J=1, L=256, FP32 unit vectors, beta=0.693, "
                                 "renormalised every 16 sweeps"),
    "heis2d_L4096_f32": dict(d=2, L=4096, n=3, beta=0.693, storage="vec", bytes=24.0, ops=110,
                             paper_flips_per_ns=1 / 0.50,
                             desc="2D Heisenberg J=1, L=4096, FP32 unit vectors, FP64 aggregates "
                                  "(the paper's Table 1 single-precision row)"),
    "heis2d_L4096_f32_fast": dict(d=2, L=4096, n=3, beta=0.693, storage="vec", bytes=24.0,
                                  ops=110,
                                  fast=1, paper_flips_per_ns=1 / 0.18,
                                  desc="2D Heisenberg L=4096 with hardware sin/cos/exp "
                                       "intrinsics (the paper's Table 1 fast-math row)"),
    "ising2d_L32_i8_k100": dict(d=2, L=32, n=1, beta=0.440687, storage="i8", bytes=0.0, ops=28,
                                multihit=100, tile=16, paper_flips_per_ns=1 / 1.60,
                                desc="2D Ising L=32, k=100 multi-hit in 16x16 tiles (the paper's "
                                     "Table 1 small-lattice row)"),
    "xy2d_L4096_f32": dict(d=2, L=4096, n=2, beta=1.12, storage="angle", bytes=12.0, ops=66,
                           desc="2D XY J=1, L=4096, FP32 angles, beta=1.12"),
    "heis3d_L256_f32_heatbath": dict(d=3, L=256, n=3, beta=0.693, storage="vec", bytes=36.0,
                                     ops=140,
                                     update=1,
                                     desc="3D Heisenberg L=256, FP32 vectors, heat-bath rule "
                                          "(exponential draws about the local field)"),
    "xy2d_L4096_f32_heatbath": dict(d=2, L=4096, n=2, beta=1.12, storage="angle", bytes=12.0,
                                    ops=100,
                                    update=1,
                                    desc="2D XY L=4096, FP32 angles, heat-bath rule (Best-Fisher "
                                         "von Mises draws)"),
    "ea3d_batch_1024x32": dict(d=3, L=32, n=1, beta=None, storage="batch", bytes=0.0, ops=28,
                               samples=1024, temps=32,
                               desc="3D Edwards-Anderson +-J, 1024 samples of sides "
                                    "[8,12,16,24,32][s mod 5] x 32 temperatures geometric in "
                                    "[0.5, 3], replica exchange every sweep, one persistent graph-captured "
                                    "launch, samples per CTA chosen by the autotuner"),
}
for _name, _wl in WORKLOADS.items():
    _wl["name"] = _name
HEADLINE = "ising2d_L16384_i8"


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            j = json.load(f)
        return j.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


def alu_peak_tops():
    """Integer issue peak of the GPU from its unit counts and clock: every SM
    issues one 32-bit integer operation per clock on each of its 128 lanes
    (152 SMs x 128 x 2.07 GHz = 40.3 T ops/s on GB300)."""
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    mhz = 2070.0
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            mhz = json.load(f).get("sm_max_mhz", mhz)
    return sms * 128 * mhz * 1e6 / 1e12


def kernel_source_hash(files):
    """Hash of the sources a profiled kernel is built from."""
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_1107_5463_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_profile(workload):
    """The committed ncu record of a workload's dominant kernel, only if the
    kernel sources are unchanged since it was taken."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        j = json.load(f)
    e = j.get(workload)
    if not e:
        return None
    try:
        current = kernel_source_hash(e.get("source_files", []))
    except OSError:  # a source file is gone: the record cannot be current
        return None
    return e if e.get("source_hash") == current else None


def recorded_traffic(workload):
    """DRAM bytes per launch of the dominant kernel from a committed ncu
    summary, only if the kernel sources are unchanged since it was taken."""
    e = recorded_profile(workload)
    return e.get("dram_bytes_per_launch") if e else None


def issue_fraction(workload, flips_per_ns):
    """The kernel's issue use on the instructions it actually executes: the
    thread instructions per site update that ncu counted (committed record,
    same sources), at one warp instruction per cycle per scheduler (128
    lanes per SM per clock at the maximum SM clock), against the measured
    rate; None without a current record."""
    e = recorded_profile(workload)
    ipc = e.get("thread_instructions_per_site") if e else None
    peak = alu_peak_tops() if (ipc and torch_cuda()) else None
    if not peak:
        return None
    bound = peak * 1e3 / ipc
    return {"instructions_per_site": ipc, "peak": peak, "unit": "T thread instructions/s",
            "bound_flips_per_ns": bound, "frac": flips_per_ns / bound,
            "source": e.get("summary")}


class Clocks:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        time.sleep(0.2)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 8:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = sorted(float(r[0]) for r in rows if r[0].replace(".", "").isdigit())
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for k, name in enumerate(names):
                if r[4 + k].lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": sm[len(sm) // 2] if sm else None,
                "sm_max_mhz": float(rows[0][1]) if rows[0][1].replace(".", "").isdigit() else None,
                "samples": len(rows), "reasons": sorted(reasons)}


def dist_setup():
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    elif torch.cuda.is_available():
        torch.cuda.set_device(local)
    return world, rank, local


def dist_teardown(world):
    if world > 1:
        import torch.distributed as dist
        if dist.is_initialized():
            dist.destroy_process_group()


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64,
                     device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def batch_sites(wl):
    from paper_1107_5463_gb300 import inputs
    return sum(L ** wl["d"] for L in inputs.ea_sample_sizes(wl["samples"])) * wl["temps"]


def sample_range(nsamples, rank, world):
    """The contiguous block of global sample indices rank `rank` of `world`
    runs: [lo, hi), sizes differing by at most one."""
    return nsamples * rank // world, nsamples * (rank + 1) // world


def time_batch(spinmc, wl, steps, warmup, want_clocks, local, rank=0, world=1):
    """Device-timed K sweeps (with exchange) of the batched spin-glass
    workload; under N ranks each rank takes a contiguous block of the global
    samples, keyed by their global indices (the union is the 1-GPU batch)."""
    import torch
    from paper_1107_5463_gb300 import inputs
    lo, hi = sample_range(wl["samples"], rank, world)
    Ls = inputs.ea_sample_sizes(wl["samples"])[lo:hi]
    b = spinmc.Batch(wl["d"], Ls, wl["temps"], inputs.geometric_betas(wl["temps"]),
                     seed=inputs.DEFAULT_SEED, first_sample=lo)
    b.run(warmup, inputs.DEFAULT_SEED)
    torch.cuda.synchronize()
    clocks = Clocks(local) if want_clocks else None
    if clocks:
        clocks.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(b.stream)
    b.run(steps, inputs.DEFAULT_SEED)
    ev1.record(b.stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    cl = clocks.stop() if clocks else None
    tuning = b.tuning()
    b.close()
    return ms, cl, tuning


def roofline_for(wl, flips_per_ns, launch_ms=None, hbm=None, peak_kind="measured",
                 traffic=None, kernel_name=None, hits=1, N=None):
    """The binding roofline of a workload's dominant kernel: the slower of its
    HBM bound (algorithmic bytes per site update) and its issue bound
    (algorithmic lane operations per site update against 128 lanes per SM
    per clock at the maximum SM clock).  The achieved figure is the measured
    site updates per ns times that bound's unit cost; the other bound is
    reported beside it.  Per launch (one colour pass of N/2 sites) where a
    launch time is given."""
    if hbm is None:
        hbm = peaks()[0]
    ops = wl.get("ops")
    bts = wl.get("bytes") or 0.0
    peak_ops = alu_peak_tops() if torch_cuda() else None
    alu_bound = peak_ops * 1e3 / ops if (ops and peak_ops) else float("inf")
    hbm_bound = hbm / bts if bts else float("inf")
    hbm_obj = {"achieved": flips_per_ns * bts, "peak": hbm, "unit": "GB/s",
               "frac": flips_per_ns * bts / hbm if bts else 0.0, "peak_kind": peak_kind,
               "bytes_per_site": bts, "bound_flips_per_ns": hbm_bound}
    alu_obj = {"achieved": flips_per_ns * ops / 1e3 if ops else None, "peak": peak_ops,
               "unit": "Tops/s",
               "frac": flips_per_ns / alu_bound if alu_bound != float("inf") else None,
               "peak_kind": "unit counts x max SM clock", "ops_per_site": ops,
               "bound_flips_per_ns": alu_bound}
    if hbm_bound <= alu_bound:
        out = {"bound": "hbm"}
        out.update({k: v for k, v in hbm_obj.items() if k != "bound_flips_per_ns"})
        out["alu"] = alu_obj
    else:
        out = {"bound": "alu"}
        out.update({k: v for k, v in alu_obj.items() if k != "bound_flips_per_ns"})
        out["hbm"] = hbm_obj
    out["bound_flips_per_ns"] = min(hbm_bound, alu_bound)
    out["traffic"] = traffic
    if wl.get("name"):
        iss = issue_fraction(wl["name"], flips_per_ns)
        if iss:
            out["issue"] = iss
    if kernel_name:
        out["kernel"] = kernel_name
    if launch_ms is not None and N is not None:
        out["launch_ms"] = launch_ms
        out["sites_per_launch"] = hits * (N // 2)
    return out


def torch_cuda():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def launch_shape(wl):
    """(kernel launches per sweep, name of the dominant kernel) of a workload."""
    d = wl["d"]
    if wl.get("update") == 2:
        return 5, "sw_local<%d> .. sw_flip (Swendsen-Wang)" % d
    if wl.get("multihit"):
        return 3, "ising_tile_kernel<%d,%d>" % (d, wl["tile"])
    # the streaming paths: two colour passes and the one-block kernel that
    # adds the measuring pass's partials
    if wl["storage"] == "bits":
        return 3, "bits_stream<%d,0,0/1>" % d
    hb = 1 if wl.get("update") == 1 else 0
    if wl["storage"] == "vec":
        kern = "heis_pair" if (wl["L"] // 2) % 64 == 0 else "heis_stream"
        return 3, "%s<%d,%d,%d,0/1>" % (kern, d, wl.get("fast", 0), hb)
    if wl["storage"] == "angle":
        return 3, "xy_stream<0,%d,0/1>" % hb
    return 3, "i8_stream<%d,0,0,%d,0/1>" % (d, hb)


def compute_ceilings(spinmc, target_ms=2.0):
    """Measured throughput of the units the sweeps lean on (sl_microbench):
    Philox4x32-10 calls, 32-bit integer multiplies, FP32 FMAs and hardware
    exp2, each timed with CUDA events over one launch of at least target_ms
    after a warm-up launch."""
    import torch
    n = spinmc.sl_microbench_threads()
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    st = torch.cuda.current_stream()
    res = {}
    for name, kind, it in (("philox_calls_per_ns", spinmc.SL_MB_PHILOX, 256),
                           ("imad_per_ns", spinmc.SL_MB_IMAD, 1024),
                           ("ffma_per_ns", spinmc.SL_MB_FFMA, 4096),
                           ("mufu_ex2_per_ns", spinmc.SL_MB_MUFU, 1024)):
        while True:
            spinmc.sl_microbench(kind, it, out, out.numel() * 4, st.cuda_stream)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(st)
            ops = spinmc.sl_microbench(kind, it, out, out.numel() * 4, st.cuda_stream)
            e1.record(st)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            limit = (2 ** 32 - 1) // n if kind == spinmc.SL_MB_PHILOX else 1 << 22
            if ms >= target_ms or 2 * it > limit:
                break
            it *= 2
        res[name] = ops / (ms * 1e6)
    return res


# sites one Philox4x32-10 call serves in a sweep (Metropolis and heat-bath
# Ising: a quarter call per site; XY Metropolis: half; Heisenberg: one)
RNG_SITES_PER_CALL = {"i8": 4, "bits": 4, "angle": 2, "vec": 1}


def configure(spinmc, lat, wl):
    """Apply a workload's update rule, multi-hit and fast-math options."""
    if wl.get("fast"):
        lat.set_option(spinmc.SL_OPT_FAST_MATH, 1)
    if wl.get("update"):
        lat.set_update(wl["update"])
    if wl.get("multihit"):
        lat.set_option(spinmc.SL_OPT_TILE, wl["tile"])
        lat.set_option(spinmc.SL_OPT_MULTIHIT, wl["multihit"])


def time_sweeps(spinmc, wl, steps, warmup, replica, want_clocks, local, shape=None,
                tune_cache=None, fixed_shape=None):
    """Device-timed K sweeps of one lattice, after the launch-shape autotuner
    picked rows per thread and the grid cap (outside the timed region; its
    choice is read from and written to `tune_cache` when one is given, so a
    profiled run can repeat the shape a plain run picked); returns (ms,
    clocks, E of the last sweep) and fills `shape`.  `fixed_shape` = (rows per
    thread, blocks per SM, kernel variant) sets the launch shape instead of
    tuning it (0 keeps the library's default for that option)."""
    import torch
    from paper_1107_5463_gb300 import inputs
    storage = spinmc.SL_STORE_BITS if wl["storage"] == "bits" else None
    lat = spinmc.Lattice(wl["d"], wl["L"], n=wl["n"], seed=inputs.DEFAULT_SEED, replica=replica,
                         storage=storage)
    configure(spinmc, lat, wl)
    if fixed_shape is not None:
        R, cap, kern = fixed_shape
        lat.set_option(spinmc.SL_OPT_ROWS, R)
        lat.set_option(spinmc.SL_OPT_BLOCKS_PER_SM, cap)
        if kern:
            lat.set_option(spinmc.SL_OPT_KERNEL, kern)
        if shape is not None:
            shape.update(rows_per_thread=R, blocks_per_sm=cap, kernel=kern, tuned_by="--shape")
    else:
        R, cap = lat.autotune(wl["beta"], 3, cache_path=tune_cache)
        if shape is not None:
            shape.update(rows_per_thread=R, blocks_per_sm=cap, tuned_by="sl_autotune")
    E = torch.empty(max(steps, warmup, 1), dtype=torch.float64, device="cuda")
    m = torch.empty_like(E)
    spinmc.sl_sweep_series(lat.h, wl["beta"], warmup, inputs.DEFAULT_SEED, E, m)
    torch.cuda.synchronize()
    clocks = Clocks(local) if want_clocks else None
    if clocks:
        clocks.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(lat.stream)
    spinmc.sl_sweep_series(lat.h, wl["beta"], steps, inputs.DEFAULT_SEED, E, m)
    ev1.record(lat.stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    cl = clocks.stop() if clocks else None
    e_last = float(E[steps - 1].item())
    lat.close()
    return ms, cl, e_last


def walkers_run(spinmc, wl, sweeps=10):
    """Windowed Wang-Landau or multicanonical walkers of the 2D Ising model:
    windows of width + 1 levels sharing edge levels over the whole range,
    wpw walkers each; `sweeps` sweeps of every walker timed with CUDA events.
    Multicanonical weights come from a short Wang-Landau run."""
    import numpy as np
    import torch
    L = wl["L"]
    N = L * L
    klo = np.arange(0, N - wl["width"] + 1, wl["width"]).astype(np.int32)
    khi = (klo + wl["width"]).astype(np.int32)
    w = spinmc.Walkers(L, klo, khi, wl["wpw"], seed=1)
    w.wl(3, final_stage=32, seed=2)
    if wl["kind"] == "muca":
        S = w.read()[0]
        lnW = S[::wl["wpw"]].astype(np.float64) / 2 ** 32
        w.muca(lnW, 2, seed=3)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(w.stream)
    if wl["kind"] == "muca":
        w.muca(lnW, sweeps, seed=3)
    else:
        w.wl(sweeps, final_stage=32, seed=2)
    ev1.record(w.stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    flips = w.nwalk * N * sweeps
    w.close()
    return {"value": flips / (ms * 1e6), "unit": UNIT, "ms_per_step": ms / sweeps,
            "walkers": int(len(klo) * wl["wpw"]), "windows": int(len(klo)),
            "paper_gtx480_flips_per_ns": wl["paper_flips_per_ns"],
            "over_paper_gtx480": flips / (ms * 1e6) / wl["paper_flips_per_ns"]}


def batch_run(spinmc, nsamples=1024, ntemps=32, sweeps=100, plain_lattices=32, plain_sweeps=20,
              d=3, sizes=None):
    """The batched Edwards-Anderson workload: nsamples 3D +-J samples of sides
    [8,12,16,24,32][s mod 5], ntemps temperatures geometric in [0.5, 3],
    exchange after every sweep, one run of `sweeps` sweeps timed with CUDA
    events.  The plain comparison runs single lattices (the same couplings,
    one sample x temperature per lattice) through sl_sweep one after another
    for the same number of sweeps per lattice."""
    import torch
    from paper_1107_5463_gb300 import inputs
    Ls = inputs.ea_sample_sizes(nsamples) if sizes is None else list(sizes)
    betas = inputs.geometric_betas(ntemps)
    b = spinmc.Batch(d, Ls, ntemps, betas, seed=inputs.DEFAULT_SEED)
    b.run(2, 1)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(b.stream)
    b.run(sweeps, 7)
    ev1.record(b.stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    flips = sum(L ** d for L in Ls) * ntemps * sweeps
    if plain_lattices == 0:
        b.close()
        return {"value": flips / (ms * 1e6), "unit": UNIT, "ms": ms, "sweeps": sweeps,
                "samples": nsamples, "temps": ntemps}
    # plain path: the samples of side 32, one lattice per (sample, temperature)
    lats = []
    s32 = [s for s, L in enumerate(Ls) if L == 32]
    for q in range(plain_lattices):
        s = s32[q // ntemps % len(s32)]
        lat = spinmc.Lattice(3, 32, J_bonds=b.bonds(s), seed=inputs.DEFAULT_SEED,
                             replica=s * ntemps + q % ntemps)
        lats.append((lat, betas[q % ntemps]))
    for lat, beta in lats:
        lat.sweep(beta, 2, 7)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ev0.record(torch.cuda.current_stream())
    for lat, beta in lats:
        lat.sweep(beta, plain_sweeps, 7)
    ev1.record(torch.cuda.current_stream())
    torch.cuda.synchronize()
    pms = ev0.elapsed_time(ev1)
    for lat, _ in lats:
        lat.close()
    b.close()
    plain_flips = 32 ** 3 * plain_lattices * plain_sweeps
    return {"value": flips / (ms * 1e6), "unit": UNIT, "ms": ms, "sweeps": sweeps,
            "samples": nsamples, "temps": ntemps,
            "plain_value": plain_flips / (pms * 1e6), "plain_sample":
                "%d lattices of side 32 x %d sweeps each, sl_sweep per lattice" % (plain_lattices,
                                                                               plain_sweeps),
            "batched_over_plain": (flips / ms) / (plain_flips / pms)}


def e2e_run(spinmc, wl, jobs, sweeps_per_job, replica):
    """End to end through the public API with host buffers: per job, upload
    the start configuration from pinned host memory, run the sweeps, read the
    E and |m| series back to pinned host memory."""
    import numpy as np
    import torch
    from paper_1107_5463_gb300 import inputs
    d, L = wl["d"], wl["L"]
    N = L ** d
    host = torch.empty(N, dtype=torch.int8, pin_memory=True)
    host.numpy()[:] = inputs.ising_spins(d, L, inputs.DEFAULT_SEED + replica)
    out = torch.empty(2 * sweeps_per_job, dtype=torch.float64, pin_memory=True)
    lat = spinmc.Lattice(d, L, n=1, seed=inputs.DEFAULT_SEED, replica=replica)
    configure(spinmc, lat, wl)
    E = torch.empty(sweeps_per_job, dtype=torch.float64, device="cuda")
    m = torch.empty_like(E)
    # warm: one job
    spinmc.sl_set_spins(lat.h, host.data_ptr())
    spinmc.sl_sweep_series(lat.h, wl["beta"], sweeps_per_job, 99, E, m)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(jobs):
        spinmc.sl_set_spins(lat.h, host.data_ptr())
        spinmc.sl_sweep_series(lat.h, wl["beta"], sweeps_per_job, 99, E, m)
        with torch.cuda.stream(lat.stream):
            out[:sweeps_per_job].copy_(E, non_blocking=True)
            out[sweeps_per_job:].copy_(m, non_blocking=True)
        lat.stream.synchronize()
    dt = time.perf_counter() - t0
    lat.close()
    flips = N * (wl.get("multihit") or 1) * sweeps_per_job * jobs
    return dict(value=flips / (dt * 1e9), unit=UNIT, h2d_bytes_per_step=N,
                d2h_bytes_per_step=2 * 8 * sweeps_per_job, sweeps_per_step=sweeps_per_job,
                steps=jobs)


def oracle_state(wl, L=None):
    """The oracle's start state for a workload (natural order)."""
    import oracle
    from paper_1107_5463_gb300 import inputs
    d, L = wl["d"], L or wl["L"]
    if wl["n"] == 3:
        return oracle.heis_init(d, L, inputs.DEFAULT_SEED)
    if wl["n"] == 2:
        return oracle.xy_init(d, L, inputs.DEFAULT_SEED)
    return oracle.ising_init(d, L, inputs.DEFAULT_SEED)


def oracle_sweep(wl, s, t, L=None):
    """One oracle sweep (with its E/|m| measurement) of the workload's rule."""
    import oracle
    from paper_1107_5463_gb300 import inputs
    d, L, beta, seed = wl["d"], L or wl["L"], wl["beta"], inputs.DEFAULT_SEED
    if wl["n"] == 3:
        oracle.heis_sweeps(d, L, s, beta, seed, t, 1, heatbath=wl.get("update") == 1)
    elif wl["n"] == 2:
        oracle.xy_sweeps(d, L, s, beta, seed, t, 1, heatbath=wl.get("update") == 1)
    elif wl.get("update") == 2:
        oracle.ising_sw_sweeps(d, L, s, beta, seed, t, 1)
    elif wl.get("update") == 1:
        oracle.ising_heatbath_sweeps(d, L, s, beta, seed, t, 1)
    elif wl.get("multihit"):
        oracle.ising_multihit_sweeps(d, L, wl["tile"], wl["multihit"], s, beta, seed, t, 1)
    else:
        oracle.ising_sweeps(d, L, s, beta, seed, t, 1)


def cpu_baseline(wl, target_s=15.0):
    """The oracle (plain C, single thread) on a bounded sample: whole sweeps
    of the full workload lattice, with the per-sweep measurement."""
    d, L = wl["d"], wl["L"]
    N = L ** d
    hits = wl.get("multihit") or 1
    s = oracle_state(wl)
    t0 = time.perf_counter()
    nsw = 0
    while True:
        oracle_sweep(wl, s, nsw)
        nsw += 1
        if time.perf_counter() - t0 > target_s or nsw >= 50:
            break
    dt = time.perf_counter() - t0
    return dict(value=N * hits * nsw / (dt * 1e9), unit=UNIT, cores=1, kind="oracle",
                sample="%d full sweep(s) of the %d^%d lattice incl. per-sweep E/|m|, "
                       "single-threaded C oracle, %.1f s" % (nsw, L, d, dt))


def sample_side(wl):
    """Side of the oracle's sample lattice for a lattice workload: one sweep
    takes a few tens of milliseconds on one core."""
    d = wl["d"]
    if wl.get("multihit"):
        Ls = 64 if d == 2 else 32
    elif wl["n"] > 1:
        Ls = 512 if d == 2 else 64
    else:
        Ls = 1024 if d == 2 else 96
    return min(Ls, wl["L"])


def _oracle_worker(task):
    """One process of the all-cores oracle baseline: sweeps of its own sample
    lattice of the workload until the time budget is spent; returns (site
    updates, seconds)."""
    name, budget_s = task
    wl = WORKLOADS[name]
    Ls = sample_side(wl)
    s = oracle_state(wl, Ls)
    hits = wl.get("multihit") or 1
    t0 = time.perf_counter()
    n = 0
    while True:
        oracle_sweep(wl, s, n, Ls)
        n += 1
        if time.perf_counter() - t0 > budget_s:
            break
    return n * Ls ** wl["d"] * hits, time.perf_counter() - t0


def cpu_baseline_all_cores(name, budget_s=8.0):
    """The oracle as it stands on every host core at once: one spawned process
    per core, each sweeping its own sample lattice (the oracle is
    single-threaded; the processes share nothing), aggregate throughput."""
    import multiprocessing as mp
    wl = WORKLOADS[name]
    cores = os.cpu_count() or 1
    try:
        # spawned (the parent has touched the GPU), bounded in time; leaving
        # the block terminates the workers
        with mp.get_context("spawn").Pool(cores) as pool:
            res = pool.map_async(_oracle_worker, [(name, budget_s)] * cores).get(
                timeout=10 * budget_s + 120)
    except Exception as e:  # the bench line is still printed
        return dict(value=None, unit=UNIT, cores=cores, kind="oracle",
                    error="all-cores run failed: %s" % type(e).__name__)
    sites = sum(r[0] for r in res)
    secs = max(r[1] for r in res)
    Ls = sample_side(wl)
    return dict(value=sites / (secs * 1e9), unit=UNIT, cores=cores, kind="oracle",
                sample="%d processes, each sweeping its own %d^%d sample lattice for %.0f s"
                       % (cores, Ls, wl["d"], budget_s))


def reference_sample(wl):
    """A bounded sample of a workload for the oracle: (step(t), sites updated
    per step, description).  Lattice workloads keep their dimension, model and
    rule on a smaller side; walkers run 8 windows spread over the energy
    range; the spin-glass batch runs one sample of each side with all its
    temperatures and replica exchange."""
    import numpy as np
    import oracle
    from paper_1107_5463_gb300 import inputs
    seed = inputs.DEFAULT_SEED
    st = wl["storage"]
    if st == "walkers":
        L, width = wl["L"], wl["width"]
        N = L * L
        klo = list(range(0, N - width + 1, width))
        pick = klo[::len(klo) // 8][:8]
        walkers = [oracle.Walker(L, k, k + width, seed, i) for i, k in enumerate(pick)]
        flat = np.zeros(width + 1)

        def step(t):
            for w in walkers:
                if wl["kind"] == "wl":
                    w.wl(1, 20)
                else:
                    w.muca(flat, 1)
        return step, len(walkers) * N, ("one sweep of 8 walkers of a %d^2 lattice in windows "
                                        "of %d levels per step" % (L, width + 1))
    if st == "batch":
        d, nt = wl["d"], wl["temps"]
        betas = inputs.geometric_betas(nt)
        samples = []
        for q, Ls in enumerate(inputs.EA_SIZES):
            jb = oracle.ea_couplings(d, Ls, seed, q)
            spins = np.stack([oracle.ising_init(d, Ls, seed, q * nt + r) for r in range(nt)])
            samples.append((Ls, q, jb, spins, np.arange(nt, dtype=np.int32)))

        def step(t):
            for Ls, q, jb, spins, perm in samples:
                oracle.ea_pt_sweeps(d, Ls, jb, betas, seed, q, t, 1, spins, perm)
        n = nt * sum(Ls ** d for Ls in inputs.EA_SIZES)
        return step, n, ("one sweep with exchange of one sample of each side %s x %d "
                         "temperatures per step" % (list(inputs.EA_SIZES), nt))
    d = wl["d"]
    Ls = sample_side(wl)
    s = oracle_state(wl, Ls)
    hits = wl.get("multihit") or 1
    return (lambda t: oracle_sweep(wl, s, t, Ls)), Ls ** d * hits, (
        "one sweep of a %d^%d sample lattice incl. E/|m| per step" % (Ls, d))


def reference_arm(args, world, rank):
    """--impl reference: the CPU oracle as it stands, on a bounded sample of the
    workload (reference_sample), on the host cores; rank 0 alone runs."""
    if rank != 0:
        return
    wl = WORKLOADS[args.workload]
    step, n, sample = reference_sample(wl)
    for k in range(args.warmup):
        step(k)
    t0 = time.perf_counter()
    for k in range(args.steps):
        step(args.warmup + k)
    dt = time.perf_counter() - t0
    v = n * args.steps / (dt * 1e9)
    dtype = {"i8": "int8", "bits": "int8", "vec": "f64", "angle": "f64", "walkers": "int8",
             "batch": "int8"}[wl["storage"]]
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": dtype, "data": "synthetic",
            "config": {"workload": args.workload, "desc": wl["desc"], "sample": sample,
                       "parallelism": "host, 1 thread"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=HEADLINE, choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--e2e-jobs", type=int, default=3)
    ap.add_argument("--shape", default=None,
                    help="ROWS,BLOCKS_PER_SM,KERNEL: fix the launch shape (and for 3D "
                         "Heisenberg the kernel: 2 column pairs, 3 single columns, 4 "
                         "staged tiles) instead of tuning it; 0 keeps a default")
    ap.add_argument("--tune-cache", default=None,
                    help="JSON-lines file the launch-shape autotuner reads and appends "
                         "(lets a profiled run repeat a plain run's shape)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")

    world, rank, local = dist_setup()
    if args.impl == "reference":
        reference_arm(args, world, rank)
        dist_teardown(world)
        return

    import __graft_entry__
    __graft_entry__.build()
    import torch
    from paper_1107_5463_gb300 import spinmc

    wl = WORKLOADS[args.workload]
    d, L = wl["d"], wl["L"]
    hbm, peak_kind = peaks()
    barrier(world)
    if wl["storage"] == "batch":
        ms, clocks, tuning = time_batch(spinmc, wl, args.steps, args.warmup, rank == 0, local,
                                        rank, world)
        ms = max_over_ranks(ms, world)
        flips = batch_sites(wl) * args.steps  # all ranks together
        value = flips / (ms * 1e6)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
            "dtype": "u32 replica planes", "data": "synthetic",
            "config": {"workload": args.workload, "desc": wl["desc"],
                       "step": "one sweep of every replica + energies + exchange",
                       "l2": "shared-memory resident samples; no HBM traffic per sweep",
                       "parallelism": "samples split across ranks" if world > 1 else
                       "single GPU"},
            "roofline": roofline_for(wl, value / world, kernel_name="ea_pt_persistent<3>"),
            "gpu_launches": 1,
            "tuning": [{"L": L, "samples_per_cta": k, "ms_per_sample_sweep": c}
                       for L, k, c in tuning],
            "clocks": clocks,
        }
        if rank == 0:
            print(json.dumps(line), flush=True)
        barrier(world)
        dist_teardown(world)
        return
    if wl["storage"] == "walkers":
        # windowed walkers: every rank runs the full walker set (independent
        # runs), the line reports the sum
        clocks = Clocks(local) if rank == 0 else None
        if clocks:
            clocks.start()
        r = walkers_run(spinmc, wl, sweeps=args.steps)
        cl = clocks.stop() if clocks else None
        ms = max_over_ranks(r["ms_per_step"] * args.steps, world)
        flips = r["walkers"] * L * L * args.steps * world
        line = {
            "metric": METRIC, "value": flips / (ms * 1e6), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u32 walker bit-planes, int64 fixed-point ln g", "data": "synthetic",
            "config": {"workload": args.workload, "desc": wl["desc"],
                       "step": "one sweep of every walker",
                       "l2": "64 MB of walker lattices, L2-resident by design",
                       "parallelism": "replica per GPU" if world > 1 else "single GPU"},
            "roofline": roofline_for(wl, flips / (ms * 1e6) / world,
                                     kernel_name="walk_kernel<%s>" % wl["kind"]),
            "gpu_launches": 1, "clocks": cl,
            "over_paper_gtx480": r["over_paper_gtx480"],
        }
        if rank == 0:
            print(json.dumps(line), flush=True)
        barrier(world)
        dist_teardown(world)
        return
    N = L ** d
    shape = {}
    fixed = tuple(int(v) for v in args.shape.split(",")) if args.shape else None
    if fixed is not None and len(fixed) != 3:
        ap.error("--shape takes ROWS,BLOCKS_PER_SM,KERNEL")
    ms, clocks, e_last = time_sweeps(spinmc, wl, args.steps, args.warmup, rank, rank == 0, local,
                                     shape, args.tune_cache, fixed)
    ms = max_over_ranks(ms, world)
    hits = wl.get("multihit") or 1
    value = N * hits * args.steps * world / (ms * 1e6)

    launches_per_step, kernel_name = launch_shape(wl)
    launch_ms = ms / (args.steps * 2)
    bytes_per_launch = wl["bytes"] * hits * (N // 2)   # half a sweep
    achieved_gbs = bytes_per_launch / (launch_ms * 1e-3) / 1e9
    traffic = recorded_traffic(args.workload)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"i8": "int8", "bits": "u32 bit-planes", "vec": "f32", "angle": "f32"}[
            wl["storage"]], "data": "synthetic",
        "config": {"workload": args.workload, "desc": wl["desc"], "d": d, "L": L,
                   "sites": N, "beta": wl["beta"], "step": "one full sweep + fused E,|m|",
                   "l2": "inputs larger than L2 (%d MB of spins)" % (N // 2**20),
                   "parallelism": "replica per GPU" if world > 1 else "single GPU"},
        "roofline": roofline_for(wl, value / world, launch_ms, hbm, peak_kind, traffic,
                                 kernel_name, hits, N),
        "gpu_launches": args.steps * launches_per_step + 1,
        "launch_shape": shape,
        "clocks": clocks,
        "check": {"E_per_site_last": e_last / N},
    }
    if rank == 0:
        ceil = compute_ceilings(spinmc)
        per_call = RNG_SITES_PER_CALL.get(wl["storage"])
        if per_call and wl.get("update") != 2:
            # no sweep can outrun its random numbers
            ceil["rng_bound_flips_per_ns"] = per_call * ceil["philox_calls_per_ns"]
            ceil["frac_of_rng_bound"] = value / ceil["rng_bound_flips_per_ns"]
        line["compute_ceilings"] = ceil
    if rank == 0:
        if args.e2e_jobs > 0:
            if wl["n"] == 1:
                per_job = 10 if wl.get("multihit") else (100 if wl.get("update") == 2 else 1000)
                line["e2e"] = e2e_run(spinmc, wl, args.e2e_jobs, per_job, rank)
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(wl)
            line["cpu_baseline"]["all_cores"] = cpu_baseline_all_cores(args.workload)
        if not args.no_variants:
            var = {}
            for name, w in WORKLOADS.items():
                if name == args.workload or w["storage"] == "batch":
                    continue
                if w["storage"] == "walkers":
                    var[name] = walkers_run(spinmc, w)
                    var[name]["roofline"] = roofline_for(w, var[name]["value"],
                                                         kernel_name="walk_kernel<%s>" % w["kind"])
                    continue
                n_sites = w["L"] ** w["d"]
                if w.get("multihit"):
                    k = max(10, min(2000, 2 ** 28 // (n_sites * w["multihit"])))
                else:
                    k = 100 if w.get("update") == 2 else 300
                vms, _, _ = time_sweeps(spinmc, w, k, 3 if w.get("multihit") else 5, rank,
                                        False, local)
                n = w["L"] ** w["d"]
                hits = w.get("multihit") or 1
                gbs = w["bytes"] * (n // 2) / (vms / (2 * k) * 1e-3) / 1e9
                var[name] = {"value": n * k * hits / (vms * 1e6), "unit": UNIT,
                             "ms_per_step": vms / k, "achieved_gbs": gbs, "hbm_frac": gbs / hbm}
                var[name]["roofline"] = roofline_for(w, var[name]["value"], hbm=hbm,
                                                     peak_kind=peak_kind,
                                                     traffic=recorded_traffic(name),
                                                     kernel_name=launch_shape(w)[1])
                if w.get("paper_flips_per_ns"):
                    var[name]["paper_gtx480_flips_per_ns"] = w["paper_flips_per_ns"]
                    var[name]["over_paper_gtx480"] = var[name]["value"] / w["paper_flips_per_ns"]
            var["ea3d_batch_1024x32"] = batch_run(spinmc)
            var["ea3d_batch_1024x32"]["roofline"] = roofline_for(
                WORKLOADS["ea3d_batch_1024x32"], var["ea3d_batch_1024x32"]["value"],
                kernel_name="ea_pt_persistent<3>")
            # the paper's 2D spin-glass rows (L = 32; 64-bit multi-spin coding:
            # 0.0023 ns per flip on the GTX 480)
            v2 = batch_run(spinmc, plain_lattices=0, d=2, sizes=[32] * 1024)
            v2["paper_gtx480_flips_per_ns"] = 1 / 0.0023
            v2["over_paper_gtx480"] = v2["value"] / v2["paper_gtx480_flips_per_ns"]
            v2["roofline"] = roofline_for(dict(WORKLOADS["ea3d_batch_1024x32"], d=2, ops=26,
                                               name="ea2d_batch_L32_1024x32"),
                                          v2["value"], kernel_name="ea_pt_persistent<2>")
            var["ea2d_batch_L32_1024x32"] = v2
            line["variants"] = var
        print(json.dumps(line), flush=True)
    barrier(world)
    dist_teardown(world)


if __name__ == "__main__":
    main()
