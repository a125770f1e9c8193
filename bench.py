#!/usr/bin/env python3
"""Throughput of the Vlasov-Hybrid time step on GB300 (marker-steps/s).

Default workload: bump-on-tail 1d3v, the largest single-GPU configuration
(nx = 256, nv = 64^3 over [-8, 8]^3, 2 markers per cell: 134 217 728
markers, dt = 0.05, a 500-step run).  The line's value is the FP64 form
(the paper's precision); the FP32 production form of the same workload is
reported beside it under "fp32".  Each form is timed over K full steps from
the middle of the run (the state after half the run's steps, reached by
untimed steps), so that the timed steps see the re-sorting, grown state of
the run rather than its first steps.  One step is the whole hot path:
gather + push, VHS reconstruction, moment, FP64 Poisson, diagnostics and the
re-sort check.  The adjoint / forward cost of the two-stream adjoint
workload (500 steps) is reported as "adjoint_over_forward".

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload NAME] [--precision auto|fp64|fp32|both]

Prints one JSON line.  --impl reference times the FP64 CPU oracle on the
host cores instead (an x-slab of the same workload per step).  Under
torchrun each rank runs an independent replica (weak scaling, no collective
on the data path).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# per velocity dimension: kernel classes of avl_profile_steps, launches per
# step, algorithmic bytes per marker of the push + deposit kernel (read x,
# v, f and write x, v_x) and the bytes of the stored layout it moves
# ("3B": 1d3v with a magnetic field, whose push + deposit kernel deposits only)
KERNEL_NAMES = {1: ["k_rs1", "k_pd1", "k_fin1", "k_field"],
                3: ["k_sort3", "k_pd3", "k_fin3", "k_field"],
                "3B": ["k_bpush3 + k_src3_tsum + k_src3_scan + k_rs3_scatter + k_src3_flip", "k_pd3", "k_fin3", "k_field"]}
LAUNCHES_PER_STEP = {1: 4,     # k_rs1 (re-sort scatter, exits at once on other steps), k_pd1, k_fin1, k_field
                     3: 4,     # k_pd3, k_fin3, k_field, k_sort3
                     "3B": 8}  # k_bpush3, k_src3_tsum, k_src3_scan, k_rs3_scatter, k_src3_flip (one mobile species), k_pd3, k_fin3, k_field
BYTES_PER_MARKER_ALGO = {(1, "fp32"): 20.0, (1, "fp64"): 40.0,    # 1d1v: read x, v, f; write x, v
                         (3, "fp32"): 28.0, (3, "fp64"): 56.0,    # 1d3v: read x, vx, vy, vz, f; write x, vx
                         ("3B", "fp32"): 24.0, ("3B", "fp64"): 40.0}   # deposit only: read x, v, f
BYTES_PER_MARKER_LAYOUT = {(1, "fp32"): 28.0, (1, "fp64"): 40.0,  # read all fields, write cell, off, dv in place
                           (3, "fp32"): 36.0, (3, "fp64"): 64.0,  # read all fields, write cell, off, vx in place
                           ("3B", "fp32"): 24.0, ("3B", "fp64"): 40.0}
# FP64 floating-point operations per marker of the 1d1v push + deposit (an FMA
# counts 2): field gather (1 - w) E_a + w E_b 4, its CIC weight 2, kick 2,
# drift 2, new CIC weights in x 2 and v 3, the four corner weights 6, the
# numerator and denominator sums 12
FP64_FLOPS_PER_MARKER = {1: 33.0}
# FP64 FMA lanes per clock per SM on the GB300 (a warp's FP64 instruction
# holds its SM sub-partition 64 clocks; four sub-partitions): an in-bounds
# microbenchmark of dependent and independent FMA chains
FP64_FMA_PER_SM_CLK = 2.0
KERNEL_DESC = {1: "k_pd1 (gather + push + VHS deposit, written back in place)",
               3: "k_pd3 (gather + push + x-sorted VHS deposit per pencil, in place)",
               "3B": "k_pd3 mode 2 (x-sorted VHS deposit per pencil of the Boris-pushed, re-sorted markers)"}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", choices=["two_stream", "landau", "bump_on_tail", "bernstein", "two_stream_adjoint",
                                          "ensemble", "landau_paper"],
                   default="bump_on_tail")
    p.add_argument("--precision", choices=["auto", "fp64", "fp32", "both"], default="auto",
                   help="auto: both forms for bump_on_tail (FP64 first), else the workload's own")
    p.add_argument("--start-step", type=int, default=-1,
                   help="untimed steps before the warm-up (-1: half the run, 0: time from t = 0)")
    p.add_argument("--nrun", type=int, default=256, help="runs of the ensemble workload")
    p.add_argument("--no-autotune", action="store_true", help="ensemble: keep the chunk-size heuristic")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--no-adjoint", action="store_true", help="leave out the adjoint / forward cost")
    p.add_argument("--no-ensemble", action="store_true", help="leave out the batched ensemble beside the default line")
    p.add_argument("--nv", type=int, default=0, help="velocity cells (profiling of a smaller case)")
    p.add_argument("--amp", type=float, default=0.0,
                   help="two-stream perturbation amplitude instead of 1e-4 (profiling of the re-sorting, "
                        "strongly driven state from the first step)")
    return p.parse_args()


def workload(name, nv=0, amp=0.0):
    from paper_1804_03901_gb300 import inputs
    if name == "two_stream":
        kw = {"nv": nv} if nv else {}
        if amp:
            kw["amp"] = amp
        return inputs.two_stream(**kw)
    if name == "bump_on_tail":
        return inputs.bump_on_tail(nv=nv) if nv else inputs.bump_on_tail()
    if name == "bernstein":
        return inputs.bernstein(nv=nv) if nv else inputs.bernstein()
    if name == "two_stream_adjoint":
        return inputs.two_stream_adjoint(nv=nv) if nv else inputs.two_stream_adjoint()
    if name == "ensemble":
        return inputs.ensemble()
    if name == "landau_paper":
        return inputs.landau_paper(nv=nv) if nv else inputs.landau_paper()
    return inputs.landau(nv=nv) if nv else inputs.landau()


def with_precision(w, prec):
    """The workload in precision prec, named for it."""
    w2 = dict(w)
    w2["precision"] = prec
    w2["name"] = w["name"].replace("_fp32_", f"_{prec}_").replace("_fp64_", f"_{prec}_")
    if f"_{prec}_" not in w2["name"]:
        w2["name"] = w2["name"] + f"_{prec}"
    return w2


def precisions(args, w):
    if args.precision == "auto":
        return ["fp64", "fp32"] if args.workload == "bump_on_tail" else [w["precision"]]
    if args.precision == "both":
        return ["fp64", "fp32"]
    return [args.precision]


# x-slab of the workload that the CPU oracle times per step: nx / SLAB cells
# (same cell width, markers per cell and velocity grid, so that the markers
# and the grid cells shrink together and the rate per marker is the full
# workload's); the reference arm takes a thinner slab to stay within minutes
SLAB = {"two_stream": 8, "bump_on_tail": 16, "bernstein": 16, "landau": 1, "landau_paper": 8,
        "two_stream_adjoint": 4}
REF_SLAB = {"two_stream": 16, "bump_on_tail": 32, "bernstein": 32, "landau": 1, "landau_paper": 16,
            "two_stream_adjoint": 8}


def host_cpu():
    """Host CPU model and core count (recorded beside every CPU rate)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if model is None:
        try:
            for line in open("/proc/cpuinfo"):
                if line.lower().startswith(("model name", "cpu part")):
                    model = line.split(":", 1)[1].strip()
                    break
        except OSError:
            model = "unknown"
    return model or "unknown", os.cpu_count() or 1


def markers_of(w):
    n = 0
    for sp, lat in zip(w["species"], w["lattice"]):
        n += w["nx"] * int(np.prod(sp["nv"])) * int(np.prod(lat))
    return n


def dist_env():
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local = int(os.environ.get("LOCAL_RANK", 0))
    return rank, world, local


def max_over_ranks(x, world, device="cuda"):
    """The job's time from each rank's: the largest (all-reduce MAX over the
    process group; the value itself for one rank)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(markers_per_rank, world, steps, seconds):
    """Whole-job marker-steps/s of `world` independent replicas, each moving
    markers_per_rank markers for `steps` steps, in the job's time."""
    return markers_per_rank * world * steps / seconds


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


KERNEL_SOURCES = {1: ("k_vhs1.cu", "common.cuh", "resort.cuh", "ptx.cuh", "avl_internal.cuh"),
                  3: ("k_vhs3.cu", "common.cuh", "avl_internal.cuh")}


def kernel_source_hash(nvdim):
    """Hash of the sources the push + deposit kernel of nvdim is built from."""
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[nvdim]:
        h.update(open(os.path.join(ROOT, "paper_1804_03901_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def recorded_traffic(workload_name, prec, nvdim):
    """DRAM bytes per marker of the push + deposit kernel from the committed
    ncu summary, if it was taken on the current kernel source."""
    path = os.path.join(ROOT, "profiles", "pd_traffic.json")
    if not os.path.exists(path):
        return None
    d = json.load(open(path))
    rec = d.get(f"{workload_name}:{prec}")
    if not rec or rec.get("source_hash") != kernel_source_hash(nvdim):
        return None
    return float(rec["dram_bytes_per_marker"])


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev):
        self.dev = dev
        self.proc = None
        self.path = tempfile.mktemp(suffix=".csv")

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.dev), "-lms", "200"], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        self.proc.wait()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def build_sim(A, w, stream, seed_offset=0):
    prec = A.AVL_FP32 if w["precision"] == "fp32" else A.AVL_FP64
    dom = A.make_domain(w["nvdim"], w["nx"], w["L"], w["dt"], 1.0, True, prec)
    sim = A.Simulation(dom, [A.make_species(**sp) for sp in w["species"]], stream=stream)
    init_markers(A, sim, w, seed_offset)
    if "B" in w:
        sim.set_bfield(w["B"])
    return sim


def init_markers(A, sim, w, seed_offset=0):
    for s, (f0, lat) in enumerate(zip(w["f0"], w["lattice"])):
        sim.init_markers(s, lat, A.make_f0(f0["beams"], f0["modes"]), w["seed"] + seed_offset, w["jitter"])


def slab_of(w, slab):
    """The workload restricted to nx / slab cells of the same width."""
    if slab <= 1:
        return w
    w2 = dict(w)
    w2["nx"] = max(4, w["nx"] // slab)
    w2["L"] = w["L"] * w2["nx"] / w["nx"]
    return w2


def cpu_oracle_rate(w, budget_s=12.0, slab=1, steps=None):
    """Marker-steps/s of the FP64 oracle (single thread) on an x-slab of the
    workload: (rate, markers, steps done, seconds)."""
    from oracle import oracle as O
    ws = slab_of(w, slab)
    species = [O.Species(**sp) for sp in ws["species"]]
    sim = O.OracleSim(ws["nvdim"], ws["nx"], ws["L"], ws["dt"], species)
    if "B" in ws:
        sim.B = np.asarray(ws["B"], dtype=np.float64)
    for s, (f0, lat) in enumerate(zip(ws["f0"], ws["lattice"])):
        sim.init_markers(s, lat, O.F0(f0["beams"], f0["modes"]), ws["seed"], ws["jitter"])
    sim.refresh()
    nmark = sum(x.size for x in sim.x)
    done, t0 = 0, time.perf_counter()
    while True:
        sim.step(1)
        done += 1
        el = time.perf_counter() - t0
        if steps is not None and done >= steps:
            break
        if steps is None and (el > budget_s and done >= 2):
            break
    return nmark * done / el, nmark, done, el


def cpu_baseline_entry(w, slab, budget_s=12.0):
    """The oracle's rate on the host cores of this run, with the host CPU and
    the per-core rate times the core count (an ideal-scaling figure: the
    oracle itself runs on one thread)."""
    rate, nm, done, el = cpu_oracle_rate(w, budget_s=budget_s, slab=slab)
    model, cores = host_cpu()
    return {"value": rate, "unit": "marker-steps/s", "cores": 1, "kind": "oracle",
            "sample": f"{done} full steps of an x-slab of the {w['name']} workload (1/{slab} of the x cells: "
                      f"nx = {slab_of(w, slab)['nx']}, same cell width, markers per cell and velocity grid; "
                      f"{nm} markers), FP64 oracle, 1 thread, {el:.1f} s",
            "host_cpu": model, "host_cores": cores,
            "ideal_scaling_all_cores": {"value": rate * cores, "unit": "marker-steps/s",
                                        "note": f"per-core rate x {cores} cores (not measured: the oracle "
                                                f"runs on one thread)"}}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    w = workload(args.workload, args.nv)
    prec = precisions(args, w)[0]
    w = with_precision(w, prec)
    slab = REF_SLAB.get(args.workload, 1)
    cpu_oracle_rate(w, slab=slab, steps=max(1, args.warmup))   # warm-up (page-in)
    rate, nmark, done, el = cpu_oracle_rate(w, slab=slab, steps=args.steps)
    model, cores = host_cpu()
    sample = (f"FP64 oracle, 1 thread, {done} full steps of an x-slab of the {w['name']} workload "
              f"(1/{slab} of the x cells, nx = {slab_of(w, slab)['nx']}, {nmark} markers)")
    line = {"impl": "reference", "metric": "marker_steps_per_s", "value": rate, "unit": "marker-steps/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * el / done, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w["name"], "sample": sample},
            "cpu_baseline": {"value": rate, "unit": "marker-steps/s", "cores": 1, "kind": "oracle",
                             "sample": sample, "host_cpu": model, "host_cores": cores},
            "e2e": {"value": rate, "unit": "marker-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# FP64 floating-point operations per marker of the 1d3v push + deposit k_pd3
# (an FMA counts 2; the weights of the marker's (v_y, v_z) cells are stored
# beside it and not recomputed per step)
def fp64_flops_3d():
    push = 2 + 4 + 2 + 2          # CIC weight of x, field gather, kick, drift
    weights = 2 + 3               # new CIC weight of x; dual row and weight of v_x
    gather = 2 * (5 + 16 * 2)     # per column of the marker (two): ax, a1, a0, a0 f, a1 f; 16 FMAs into the rows
    return float(push + weights + gather)


FP64_FLOPS_PER_MARKER[3] = fp64_flops_3d()


def measure(A, w, args, rank, world, local, stream):
    """Device-timed, profiled and end-to-end rates of one precision form of
    the workload, timed from the state after args.start_step (or half the
    run) untimed steps and W warm-up steps."""
    import torch
    prec = w["precision"]
    sim = build_sim(A, w, stream.cuda_stream, seed_offset=rank)
    nmark = markers_of(w)
    ns = len(w["species"])
    nvd = w["nvdim"]
    for s in range(ns):
        assert sim.marker_count(s) > 0
    start = w["steps"] // 2 if args.start_step < 0 else args.start_step
    if start:
        sim.step(start)
    sim.step(max(3, args.warmup))
    sim.synchronize()
    # the state the timed steps start from, kept on the host for the
    # end-to-end leg and the per-kernel profile
    hx, hv, hf = [], [], []
    if not args.no_e2e:
        for s in range(ns):
            x, v, f = sim.get_markers(s)
            hx.append(torch.from_numpy(x).pin_memory())
            hv.append(torch.from_numpy(np.ascontiguousarray(v[:nvd])).pin_memory())
            hf.append(torch.from_numpy(f).pin_memory())
            del x, v, f

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    try:
        dev_id = "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        dev_id = str(local)
    clocks = Clocks(dev_id)
    barrier()
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sim.step(args.steps)
    e1.record(stream)
    barrier()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    sim.synchronize()
    stats = sim.get_stats()
    ms = max_over_ranks(ms, world)
    value = job_rate(nmark, world, args.steps, ms / 1e3)

    # end to end through the C ABI with host buffers, from the same state
    e2e = None
    if not args.no_e2e:
        nd = 3 + 3 * ns
        diag = torch.zeros((args.steps, nd), dtype=torch.float64).pin_memory()
        h2d = sum(t.numel() * 8 for t in hx + hv + hf)
        barrier()
        t0 = time.perf_counter()
        for s in range(ns):
            sim.set_markers(s, hx[s], hv[s], hf[s])
        for k in range(args.steps):
            sim.step(1)
            sim.get_diag_async(diag[k].data_ptr())
        sim.synchronize()
        rows = diag.numpy()
        if not np.all(np.isfinite(rows)):
            raise RuntimeError("non-finite diagnostics in the end-to-end run")
        barrier()
        el = max_over_ranks(time.perf_counter() - t0, world)
        e2e = {"value": job_rate(nmark, world, args.steps, el), "unit": "marker-steps/s",
               "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": nd * 8,
               "note": "timed: avl_set_markers of the start state (FP64 x, v, f of every marker) from pinned "
                       "host memory, then K x (avl_step + avl_get_diag_async of that step's diagnostics row "
                       "into pinned host memory), avl_synchronize and the host's check of every row; the "
                       "start state's upload is counted once and spread over the K steps"}

    # per-kernel CUDA-event timing over K steps from the same state
    if not args.no_e2e:
        for s in range(ns):
            sim.set_markers(s, hx[s], hv[s], hf[s])
    sim.synchronize()
    kms = sim.profile_steps(args.steps)
    hbm, peak_kind = peaks()
    pd_ms = kms[1] / args.steps
    kind = "3B" if nvd == 3 and any(w.get("B", (0.0, 0.0, 0.0))) else nvd
    algo, lay = BYTES_PER_MARKER_ALGO[(kind, prec)], BYTES_PER_MARKER_LAYOUT[(kind, prec)]
    achieved = nmark * algo / (pd_ms / 1e3) / 1e9
    traffic_pm = recorded_traffic(w["name"], prec, nvd)
    names = KERNEL_NAMES[kind]
    hbm_entry = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                 "traffic": traffic_pm * nmark if traffic_pm else None,
                 "kernel": KERNEL_DESC[kind],
                 "algorithmic_bytes_per_marker": algo,
                 "layout_bytes_per_marker": lay,
                 "frac_layout_bytes": nmark * lay / (pd_ms / 1e3) / 1e9 / hbm,
                 "peak_kind": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured" else peak_kind,
                 "kernel_ms_per_step": {k: float(v / args.steps) for k, v in zip(names, kms)},
                 "kernel_share": {k: float(v / kms.sum()) for k, v in zip(names, kms)}}
    roofline = hbm_entry
    if prec == "fp64" and kind in FP64_FLOPS_PER_MARKER:
        # the FP64 form is bound by the FP64 pipe (a small fraction of the
        # FP32 rate on this GPU): the same kernel against it
        props = torch.cuda.get_device_properties(torch.cuda.current_device())
        mhz = clk.get("sm_max_mhz") or clk.get("sm_mhz") or 2070.0
        fpeak = FP64_FMA_PER_SM_CLK * 2.0 * props.multi_processor_count * mhz * 1e6 / 1e12
        fach = nmark * FP64_FLOPS_PER_MARKER[kind] / (pd_ms / 1e3) / 1e12
        roofline = {"bound": "alu", "achieved": fach, "peak": fpeak, "unit": "TFLOP/s", "frac": fach / fpeak,
                    "traffic": hbm_entry["traffic"], "kernel": KERNEL_DESC[kind],
                    "flops_per_marker": FP64_FLOPS_PER_MARKER[kind],
                    "peak_kind": "FP64 pipe: 2 FMA lanes per clock per SM (in-bounds microbenchmark) x 2 FLOP x "
                                 "SMs x the sampled maximum SM clock",
                    "kernel_ms_per_step": hbm_entry["kernel_ms_per_step"],
                    "kernel_share": hbm_entry["kernel_share"],
                    "hbm": {k: hbm_entry[k] for k in ("achieved", "peak", "unit", "frac", "algorithmic_bytes_per_marker",
                                                      "peak_kind")}}
    sim.close()
    return {"value": value, "ms_per_step": ms / args.steps, "dtype": "f32" if prec == "fp32" else "f64",
            "workload": w["name"], "markers": nmark, "start_step": start, "roofline": roofline, "clocks": clk,
            "e2e": e2e, "kind": kind, "stats": stats}


def adjoint_cost(A, stream, nv=0):
    """Wall time of avl_adjoint over the forward run it differentiates
    (two-stream adjoint workload, 500 steps, checkpoints every 50), FP32 and
    FP64."""
    import torch
    w = workload("two_stream_adjoint", nv)
    out = {"workload": w["name"], "steps": w["steps"], "ckpt_every": w["ckpt"]}
    f0 = w["f0"][0]
    for prec in ("fp32", "fp64"):
        w2 = dict(w)
        w2["precision"] = prec
        sim = build_sim(A, w2, stream.cuda_stream)
        sim.step(3)
        init_markers(A, sim, w2)
        sim.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.step(w["steps"])
        e1.record(stream)
        sim.synchronize()
        fwd = e0.elapsed_time(e1)
        theta = A.make_f0(f0["beams"], f0["modes"])
        sim.adjoint(0, theta, w["steps"], w["ckpt"])   # warm-up (buffers)
        t0 = time.perf_counter()
        sim.adjoint(0, theta, w["steps"], w["ckpt"])
        adj = 1e3 * (time.perf_counter() - t0)
        sim.close()
        out[prec] = {"value": adj / fwd, "forward_ms": fwd, "adjoint_ms": adj}
    out["value"] = out["fp32"]["value"]
    out["unit"] = "x (adjoint wall time / forward wall time, FP32; FP64 beside)"
    return out


def host_near_gpu(dev):
    """Bind this process to the CPUs next to GPU `dev` (the local_cpulist of
    its PCI device, within the CPUs the process may use), so that the pinned
    host buffers of the end-to-end leg are placed in the memory the GPU
    reaches fastest.  Returns the CPU list, or None where the system gives
    none."""
    import torch
    p = torch.cuda.get_device_properties(dev)
    try:
        path = "/sys/bus/pci/devices/%04x:%02x:%02x.0/local_cpulist" % (
            p.pci_domain_id, p.pci_bus_id, p.pci_device_id)
        with open(path) as fh:
            spec = fh.read().strip()
    except (AttributeError, OSError):
        return None
    cpus = set()
    for part in spec.split(","):
        if "-" in part:
            a, b = part.split("-")
            cpus.update(range(int(a), int(b) + 1))
        elif part:
            cpus.add(int(part))
    cpus &= os.sched_getaffinity(0)
    if not cpus:
        return None
    os.sched_setaffinity(0, cpus)
    return ",".join(str(c) for c in sorted(cpus))


def run_ours(args):
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    host_cpus = host_near_gpu(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1804_03901_gb300 import avl as A

    base = workload(args.workload, args.nv, args.amp)
    # a dedicated stream: the library enqueues on it, the timing events too
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    forms = [measure(A, with_precision(base, p), args, rank, world, local, stream) for p in precisions(args, base)]
    main_form = forms[0]

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline_entry(with_precision(base, "fp64"), SLAB.get(args.workload, 1))
    adj = None
    if rank == 0 and world == 1 and not args.no_adjoint:
        adj = adjoint_cost(A, stream)
    ens = None
    if rank == 0 and world == 1 and not args.no_ensemble and args.workload == "bump_on_tail":
        ens = measure_ensemble(A, args, stream)

    l2 = {"two_stream": "inputs larger than L2 (markers 16 B each, 268 MB per step read)",
          "bump_on_tail": "inputs larger than L2 (markers 24 B (FP32) / 40 B (FP64) each, 3.2 / 5.4 GB per step)",
          "bernstein": "inputs larger than L2 (markers 24 B each, 3.2 GB per step read)",
          "landau_paper": "inputs larger than L2 (markers 24 B each, 324 MB per step read)",
          "landau": "small workload (fits in L2)"}[args.workload]
    if rank == 0:
        f = main_form
        kind, nvd = f["kind"], base["nvdim"]
        line = {"metric": "marker_steps_per_s", "value": f["value"], "unit": "marker-steps/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": f["ms_per_step"],
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": f["dtype"], "data": "synthetic",
                "config": {"workload": f["workload"], "markers": f["markers"], "species": len(base["species"]),
                           "steps_in_run": base["steps"],
                           "timed_from": (f"step {f['start_step']} of the {base['steps']}-step run (state reached "
                                          f"by untimed steps), then {max(3, args.warmup)} warm-up steps"
                                          if f["start_step"] else "t = 0"),
                           "l2": l2, "parallelism": "single GPU" if world == 1 else f"{world} independent replicas",
                           "host_cpus": host_cpus or "not bound (no local CPU list)"},
                "roofline": f["roofline"], "clocks": f["clocks"],
                "gpu_launches": LAUNCHES_PER_STEP[kind] * args.steps,
                ("out_of_window_runs_last_step" if nvd == 1 else "movers_last_step"): [int(x) for x in
                                                                                      f["stats"][:, 0]],
                "resort_steps": [int(x) for x in f["stats"][:, 1]], "e2e": f["e2e"], "cpu_baseline": cpu}
        for g in forms[1:]:
            line[g["dtype"].replace("f", "fp")] = {
                "value": g["value"], "unit": "marker-steps/s", "ms_per_step": g["ms_per_step"], "dtype": g["dtype"],
                "workload": g["workload"], "roofline": g["roofline"], "clocks": g["clocks"], "e2e": g["e2e"],
                "cpu_baseline": cpu, "gpu_launches": LAUNCHES_PER_STEP[g["kind"]] * args.steps,
                "resort_steps": [int(x) for x in g["stats"][:, 1]],
                "note": "the same workload in the FP32 production form, timed the same way; cpu_baseline is the "
                        "FP64 oracle (it has no FP32 form)"}
        if adj is not None:
            line["adjoint_over_forward"] = adj
        if ens is not None:
            ens["note"] = ("the batched form: 256 independent 1d1v FP32 runs of uneven sizes (Landau and two-stream) "
                           "advanced together, one launch per kernel class per step in a CUDA graph")
            line["batched_ensemble"] = ens
        line["paper_context"] = ("the paper's performance section reports about 1e7 marker updates per second "
                                 "on one core of an Intel Xeon E5-2650 at 2.6 GHz (dimension, precision and grid "
                                 "not stated) and 1e6-1e7 per CPU in general; context only, no number for this "
                                 "workload")
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def run_adjoint(args):
    """Cost of avl_adjoint over the forward run it differentiates, and its
    gradient against central differences of the FP64 forward run."""
    import torch
    from paper_1804_03901_gb300 import avl as A
    w = workload(args.workload, args.nv)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    nsteps, ckpt = w["steps"], w["ckpt"]
    f0 = w["f0"][0]

    def sim_of(prec, f0e):
        w2 = dict(w)
        w2["precision"] = prec
        w2["f0"] = [f0e] + w["f0"][1:]
        return build_sim(A, w2, stream.cuda_stream)

    def theta(f0e):
        return A.make_f0(f0e["beams"], f0e["modes"])

    res = {}
    for prec in ("fp32", "fp64"):
        sim = sim_of(prec, f0)
        sim.step(3)
        init_markers(A, sim, w)
        sim.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.step(nsteps)
        e1.record(stream)
        sim.synchronize()
        fwd_ms = e0.elapsed_time(e1)
        sim.adjoint(0, theta(f0), nsteps, ckpt)   # warm-up (buffers)
        t0 = time.perf_counter()
        J, ga, gu = sim.adjoint(0, theta(f0), nsteps, ckpt)
        adj_ms = 1e3 * (time.perf_counter() - t0)
        res[prec] = {"J": J, "grad": np.concatenate([ga, gu]), "forward_ms": fwd_ms, "adjoint_ms": adj_ms}
        sim.close()

    # central differences of the FP64 forward run (avl_step), h = 1e-10: the
    # differences carry an O(h) error from markers crossing cloud-in-cell
    # kinks (1e-5 at h = 1e-6) and a roundoff error O(eps J / h) that takes
    # over below 1e-10
    h = 1e-10
    amps = [a for (_, a, _) in f0["modes"]]
    drifts = [u[0] for (_, u, _) in f0["beams"]]

    nfd = nsteps

    def J_of(a, d):
        f0e = {"beams": [(n, (d[b],) + tuple(u[1:]), vth) for b, (n, u, vth) in enumerate(f0["beams"])],
               "modes": [(m, a[k], ph) for k, (m, _, ph) in enumerate(f0["modes"])]}
        sim = sim_of("fp64", f0e)
        sim.step(nfd)
        E = sim.get_E()
        sim.close()
        return 0.5 * float(np.sum(E ** 2)) * (w["L"] / w["nx"])

    def central(hh):
        out = []
        for k in range(len(amps)):
            ap, am = list(amps), list(amps)
            ap[k] += hh
            am[k] -= hh
            out.append((J_of(ap, drifts) - J_of(am, drifts)) / (2 * hh))
        for b in range(len(drifts)):
            dp, dm = list(drifts), list(drifts)
            dp[b] += hh
            dm[b] -= hh
            out.append((J_of(amps, dp) - J_of(amps, dm)) / (2 * hh))
        return np.array(out)

    fd_h, fd_h2 = central(h), central(10 * h)
    fd = fd_h
    scale = float(np.max(np.abs(fd)))
    # the same check over a short horizon in the linear phase (T = 5), where
    # no marker crosses a cloud-in-cell kink under the perturbation
    nfd = nsteps // 5
    lin = {}
    for prec in ("fp64", "fp32"):
        sim = sim_of(prec, f0)
        _, ga, gu = sim.adjoint(0, theta(f0), nfd, ckpt)
        lin[prec] = np.concatenate([ga, gu])
        sim.close()
    fl_h, fl_h2 = central(h), central(10 * h)
    fl = fl_h
    sl = float(np.max(np.abs(fl)))
    linear = {"steps": nfd, "rel_diff_h_vs_10h": float(np.max(np.abs(fl_h2 - fl)) / sl),
              "fp64_adjoint_rel_err": float(np.max(np.abs(lin["fp64"] - fl)) / sl),
              "fp32_adjoint_rel_err": float(np.max(np.abs(lin["fp32"] - fl)) / sl)}
    r32, r64 = res["fp32"], res["fp64"]
    line = {"metric": "adjoint_over_forward", "value": r32["adjoint_ms"] / r32["forward_ms"], "unit": "x",
            "higher_is_better": False, "n_gpus": 1, "steps": nsteps, "dtype": "f32", "data": "synthetic",
            "config": {"workload": w["name"], "electrons": markers_of({"nx": w["nx"], "species": w["species"][:1],
                                                                      "lattice": w["lattice"][:1]}),
                       "ckpt_every": ckpt, "params": len(fd), "ions": "immobile"},
            "fp32": {"forward_ms": r32["forward_ms"], "adjoint_ms": r32["adjoint_ms"], "J": r32["J"],
                     "grad_rel_err_vs_fd64": float(np.max(np.abs(r32["grad"] - fd)) / scale)},
            "fp64": {"forward_ms": r64["forward_ms"], "adjoint_ms": r64["adjoint_ms"], "J": r64["J"],
                     "adjoint_over_forward": r64["adjoint_ms"] / r64["forward_ms"],
                     "grad_rel_err_vs_fd64": float(np.max(np.abs(r64["grad"] - fd)) / scale)},
            "fd": {"h": h, "kind": "central differences of the FP64 avl_step run at h (and 10 h for comparison)",
                   "rel_diff_h_vs_10h": float(np.max(np.abs(fd_h2 - fd)) / scale),
                   "fp64_adjoint_rel_err_vs_10h": float(np.max(np.abs(r64["grad"] - fd_h2)) / scale),
                   "linear_phase": linear},
            "grad_fd64": fd.tolist()}
    print(json.dumps(line), flush=True)


def measure_ensemble(A, args, stream):
    """Marker-steps/s of the batched ensemble: every run advanced by one
    launch per kernel class per step (one CUDA graph per step), chunk size
    chosen by the autotuner; K steps from t = 0 after W warm-up steps."""
    import torch
    from paper_1804_03901_gb300 import inputs
    w = inputs.ensemble(nrun=args.nrun)
    prec = A.AVL_FP32
    doms = [A.make_domain(1, r["nx"], r["L"], r["dt"], 1.0, True, prec) for r in w["runs"]]
    sps = [[A.make_species(**sp) for sp in r["species"]] for r in w["runs"]]
    t0 = time.perf_counter()
    b = A.Batch(doms, sps, stream=stream.cuda_stream)

    def init():
        for i, r in enumerate(w["runs"]):
            f0 = r["f0"][0]
            b.runs[i].init_markers(0, r["lattice"][0], A.make_f0(f0["beams"], f0["modes"]), r["seed"], w["jitter"])

    init()
    nmark = sum(b.runs[i].marker_count(0) for i in range(len(w["runs"])))
    t_init = time.perf_counter() - t0
    best_m = 0 if args.no_autotune else b.autotune(5)
    init()                      # restart from t = 0 with the chosen chunk size
    b.step(max(3, args.warmup))
    b.synchronize()
    init()
    b.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = Clocks("GPU-" + str(torch.cuda.get_device_properties(torch.cuda.current_device()).uuid))
    torch.cuda.synchronize()
    clocks.start()
    e0.record(stream)
    b.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    b.synchronize()
    init()
    b.synchronize()
    kms = b.profile_steps(args.steps)
    b.close()
    hbm, peak_kind = peaks()
    pd_ms = kms[1] / args.steps
    algo = BYTES_PER_MARKER_ALGO[(1, "fp32")]
    achieved = nmark * algo / (pd_ms / 1e3) / 1e9
    traffic_pm = recorded_traffic(w["name"], "fp32", 1)
    names = KERNEL_NAMES[1]
    return {"value": nmark * args.steps / (ms / 1e3), "unit": "marker-steps/s", "ms_per_step": ms / args.steps,
            "dtype": "f32", "workload": w["name"], "runs": len(w["runs"]), "markers": nmark,
            "landau_runs": sum(r["type"] == "landau" for r in w["runs"]), "autotuned_chunk_markers": best_m,
            "init_s": t_init, "timed_from": "t = 0", "launches_per_step": 4,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                         "traffic": traffic_pm * nmark if traffic_pm else None,
                         "kernel": "k_pd1 over all runs (one batched launch)",
                         "algorithmic_bytes_per_marker": algo,
                         "peak_kind": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)",
                         "kernel_ms_per_step": {k: float(v / args.steps) for k, v in zip(names, kms)}},
            "clocks": clk, "gpu_launches": 4 * args.steps}


def run_ensemble(args):
    import torch
    from paper_1804_03901_gb300 import avl as A
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    e = measure_ensemble(A, args, stream)
    line = {"metric": "marker_steps_per_s", "value": e["value"], "unit": "marker-steps/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": e["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": e["workload"], "runs": e["runs"], "markers": e["markers"],
                       "landau_runs": e["landau_runs"], "autotuned_chunk_markers": e["autotuned_chunk_markers"],
                       "init_s": e["init_s"], "timed_from": "t = 0", "launches_per_step": 4,
                       "l2": "inputs larger than L2"},
            "roofline": e["roofline"], "clocks": e["clocks"], "gpu_launches": e["gpu_launches"]}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "two_stream_adjoint":
        run_adjoint(args)
    elif args.workload == "ensemble":
        run_ensemble(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
