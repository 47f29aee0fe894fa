"""Throughput of the moving-grid hybrid LBM step on GB300.

One bench "step" is one lattice step of the whole hot path: relocation and
refill of the patch, lattice classification, eq. 178 feed, stream-collide,
n FV sub-steps with the outer-node feed, and the lamina force.

Metric: MLUPS over both grids, (lattice discretization nodes + patch nodes)
x steps / s / 1e6 (each grid counted once per lattice step); the variant that
counts the patch n times (sub-steps) is reported as ``mlups_subiter``.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
    python bench.py --impl reference ...     # the CPU oracle, bounded sample
Under torchrun every rank runs its own replica of the workload on its GPU
(weak scaling; the instances share nothing).
"""
from __future__ import annotations

import argparse
import math
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MLUPS (both grids)"
UNIT = "MLUPS"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.idx = device_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def run_reference(args):
    """The CPU oracle timed on the host cores, on a bounded sample of the
    same workload (rank 0 only)."""
    world, rank, _ = _dist()
    if rank != 0:
        return 0
    import inputs
    import oracle

    w = inputs.workload(args.workload)
    mesh = w.mesh()
    rho = w.rho_init()
    cores = os.cpu_count() or 1
    o = oracle.Oracle(w, mesh=mesh, rho_init=rho, openmp=True)
    warm = min(args.warmup, 1)
    o.step(warm)
    # bounded sample: as many of the K requested steps as fit in ~60 s of CPU work
    t0 = time.perf_counter()
    o.step(1)
    t1 = time.perf_counter()
    per = t1 - t0
    k = max(0, min(args.steps - 1, int(60.0 / max(per, 1e-3)) - 1))
    if k:
        o.step(k)
    t2 = time.perf_counter()
    steps = k + 1
    secs = t2 - t0
    n_disc = int((o.struct_class() == oracle.DISC).sum())
    units = (n_disc + mesh.n_nodes) * steps
    value = units / secs / 1e6
    sample = (f"{steps} of {args.steps} requested lattice steps of {w.name} after {warm} warm-up, "
              f"FP64 oracle with OpenMP over its node loops on {cores} host threads")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "impl": "reference", "n_gpus": world,
            "steps": steps, "warmup": warm, "ms_per_step": 1e3 * secs / steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "lattice": f"{w.nx}x{w.ny}", "patch_nodes": mesh.n_nodes,
                       "n_sub": w.n_sub},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
                             "cpu_model": _cpu_model()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def _cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu model")):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def cpu_baseline(workload):
    """The oracle timed on the host: its OpenMP build on every host core
    (the same source with its node loops in parallel; identical results),
    two lattice steps of the workload from the initial state."""
    import inputs
    import oracle

    cores = os.cpu_count() or 1
    w = inputs.workload(workload)
    mesh = w.mesh()
    o = oracle.Oracle(w, mesh=mesh, openmp=True)
    t0 = time.perf_counter()
    o.step(2)
    secs = time.perf_counter() - t0
    n_disc = int((o.struct_class() == oracle.DISC).sum())
    return {"value": (n_disc + mesh.n_nodes) * 2 / secs / 1e6, "unit": UNIT, "cores": cores, "kind": "oracle",
            "cpu_model": _cpu_model(),
            "sample": f"2 lattice steps of {w.name} from the initial state, FP64 oracle with OpenMP over its node "
                      f"loops on {cores} host threads"}


# the source sections whose arithmetic and memory access define each
# profiled kernel's DRAM traffic (file, first marker, end marker)
_KERNEL_SOURCES = {
    "stream_collide": [("k_struct.cu", "// ------------------------------------------------------ stream-collide",
                        "// ------------------------------------------------------------- readback"),
                       ("hlbm_dev.cuh", "// ---------------------------------------------------------------- D2Q9",
                        "// ---------------------------------------------------------------- layout"),
                       ("hlbm_dev.cuh", "// ---------------------------------------------------------------- lattice storage",
                        "// ---------------------------------------------------------------- geometry")],
    "fv_deep": [("k_patch.cu", "// ----------------------------------------------------------- FV steps",
                 "// ------------------------------------------------------------- force"),
                ("hlbm_dev.cuh", "// ---------------------------------------------------------------- D2Q9",
                 "// ---------------------------------------------------------------- layout"),
                ("hlbm_dev.cuh", "// ---------------------------------------------------------------- lattice storage",
                 "// ---------------------------------------------------------------- geometry")],
    "fv_tmem": [("k_patch.cu", "// ----------------------------------------------------------- FV steps",
                 "// ------------------------------------------------------------- force"),
                ("hlbm_dev.cuh", "// ---------------------------------------------------------------- D2Q9",
                 "// ---------------------------------------------------------------- layout")],
}


# the share of the lattice rows whose far part the FV launch streams (the
# library's default, stated here because the roofline's byte count uses it)
OVERLAP_SHARE = 0.85


def kernel_source_hash(kernel):
    """Hash of the source sections that define a kernel's traffic."""
    import hashlib

    csrc = os.path.join(ROOT, "paper_2006_13631_gb300", "csrc")
    src = ""
    for name, start, end in _KERNEL_SOURCES[kernel]:
        text = open(os.path.join(csrc, name)).read()
        src += text[text.index(start):text.index(end)]
    return hashlib.sha256(src.encode()).hexdigest()


def kernel_traffic(kernel, workload):
    """DRAM bytes per launch from the committed ncu summary
    profiles/<kernel>_<workload>.md, or None if there is none or the kernel's
    source changed since it was captured."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_{workload}.md")
    try:
        text = open(path).read()
        vals = dict(line.split(":", 1) for line in text.splitlines()
                    if line.startswith(("traffic_bytes_per_launch:", "source_sha256:")))
        if vals["source_sha256"].strip() != kernel_source_hash(kernel):
            return None
        return int(vals["traffic_bytes_per_launch"])
    except Exception:
        return None


def alu_peak_tflops(dtype, device=0):
    """Peak of plain (non-tensor) arithmetic from the device's SM count and
    its maximum SM clock (nvidia-smi clocks.max.sm, else the CUDA attribute):
    SMs x 128 FP32 lanes x 2 FLOP per FMA x clock; FP64 at 1/64 of it on
    this part.  Returns (TFLOP/s, how it was derived)."""
    import torch

    props = torch.cuda.get_device_properties(device)
    sms = props.multi_processor_count
    mhz = None
    try:
        out = subprocess.run(["nvidia-smi", f"--id={device}", "--query-gpu=clocks.max.sm",
                              "--format=csv,noheader,nounits"], capture_output=True, text=True, timeout=10).stdout
        mhz = float(out.strip().splitlines()[0])
    except Exception:
        mhz = None
    if not mhz:
        try:
            mhz = torch.cuda.clock_rate(device)
        except Exception:
            mhz = 2070.0
    fp32 = sms * 128 * 2 * mhz * 1e6 / 1e12
    peak = fp32 if dtype == "f32" else fp32 / 64
    return peak, f"derived: {sms} SMs x 128 FP32 lanes x 2 FLOP x {mhz:.0f} MHz" + ("" if dtype == "f32" else " / 64")
# algorithmic FLOP of one FV sub-step per CSR entry (row P, column k): for each
# of the 9 directions a multiply-add of the streaming term S_ik f_k and one of
# the collision term C_Pk (f - f^eq)_k
FV_FLOP_PER_ENTRY = 9 * 4


def combine_ranks(ms: float, units: float, dist=None, device=None):
    """Whole-job figures over the ranks: the slowest rank's time and the
    units all ranks processed (each rank runs its own replica)."""
    if dist is None:
        return ms, units
    import torch

    t = torch.tensor([ms], dtype=torch.float64, device=device)
    u = torch.tensor([units], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def run_ours(args):
    import numpy as np
    import torch

    import inputs
    from paper_2006_13631_gb300 import Solver, hlbm as H
    from paper_2006_13631_gb300.build import build

    world, rank, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    build()
    w = inputs.workload(args.workload)
    mesh = w.mesh()
    rho = w.rho_init()
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        s = Solver(w, mesh=mesh, rho_init=rho, stream=stream.cuda_stream)
        H.hlbm_set_overlap_share(s.h, OVERLAP_SHARE)
        s.step(args.warmup)
        torch.cuda.synchronize()
        info = s.info()
        # node updates per step: lattice discretization nodes, the patch, and
        # each coarser level's nodes / 2^k (level k steps every 2^k steps)
        n_disc, n_u = info["n_struct_disc"] + int(info["coarse_updates"]), info["n_nodes"]
        sampler = ClockSampler(local)
        sampler.start()
        time.sleep(0.5)
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.profile(True)
        ev0.record(stream)
        s.step(args.steps)
        ev1.record(stream)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        clocks = sampler.stop()
        ms = ev0.elapsed_time(ev1)
        phases = s.profile_read()
        s.profile(False)
        status = s.status
        _, fy = s.force()
        finite = bool(np.isfinite(fy).all())
        # the same solver with the lattice-patch overlap off (each step's
        # stream-collide whole, before its FV launch): the two kernels timed
        # apart, for their own rooflines
        k_iso = max(10, min(args.steps, 100))
        H.hlbm_set_overlap(s.h, False)
        s.step(2)
        torch.cuda.synchronize()
        s.profile(True)
        ev0.record(stream)
        s.step(k_iso)
        ev1.record(stream)
        torch.cuda.synchronize()
        ms_iso = ev0.elapsed_time(ev1)
        phases_iso = s.profile_read()
        s.profile(False)
        H.hlbm_set_overlap(s.h, True)
    ms, units = combine_ranks(ms, float((n_disc + n_u) * args.steps), dist, "cuda")
    value = units / (ms / 1e3) / 1e6
    _, units_sub = combine_ranks(ms, float((n_disc + w.n_sub * n_u) * args.steps), dist, "cuda")
    mlups_subiter = units_sub / (ms / 1e3) / 1e6

    # roofline of the dominant kernel (the FV sub-steps: plain FP32
    # arithmetic on shared-memory tiles) and of the HBM-bound stream-collide
    peak, peak_kind = _peaks()
    bytes_per = 4 if w.dtype == "f32" else 8
    dom = max(phases, key=lambda p: phases[p][0])
    stream_bytes = 18 * bytes_per * n_disc  # 9 populations read + 9 written per discretization node
    # per step: one launch on a single level; with nested levels the phase
    # also holds the coarser levels' launches and the coupling launches
    st_ms, st_n = phases_iso["stream"]
    stream_gbs = stream_bytes / (st_ms / k_iso / 1e3) / 1e9 if st_n else None
    fv_ms, _ = phases["fv"]
    fv_iso_ms, _ = phases_iso["fv"]
    overlapped = phases["stream"][0] < 0.5 * st_ms * args.steps / k_iso  # the far lattice ran in the FV launch
    nnz = info["nnz"]
    # the launch with the next step's far lattice: its stream-collide bytes
    # (the nodes outside the next window) and the FV tile read once
    fused_bytes = (18 * bytes_per * max(0, int(OVERLAP_SHARE * n_disc) - info["box_w"] * info["box_h"]) +
                   112 * (bytes_per // 4) * n_u)
    fv_flop = FV_FLOP_PER_ENTRY * nnz * w.n_sub  # per launch (one lattice step)
    fv_tflops = fv_flop / (fv_ms / args.steps / 1e3) / 1e12 if fv_ms else None
    fv_iso_tflops = fv_flop / (fv_iso_ms / k_iso / 1e3) / 1e12 if fv_iso_ms else None
    alu_peak, alu_src = alu_peak_tflops(w.dtype, local)
    fv_kernel = {1: "k_fv_steps", 2: "k_fv_tiles", 3: "k_fv_tmem", 4: "k_fv_deep"}.get(info["fv_kernel"], "?")
    prof_key = {"k_fv_tmem": "fv_tmem", "k_fv_deep": "fv_deep"}.get(fv_kernel)
    # The dominant kernel's roofline is set by the resource its own work needs
    # longest: its FLOP at the FP32 ALU peak, or its algorithmic bytes at the
    # HBM peak.  FV alone sits far right of the ridge (ALU); the launch with
    # the next step's far lattice moves ~1 GB for 3.2 GFLOP (HBM).
    fv_s = fv_ms / args.steps / 1e3
    alu_part = {"achieved": fv_tflops, "peak": alu_peak, "unit": "TFLOP/s",
                "frac": fv_tflops / alu_peak if fv_tflops else None, "flop_per_launch": fv_flop,
                "peak_source": alu_src}
    hbm_part = None if not overlapped else {
        "achieved": fused_bytes / fv_s / 1e9, "peak": peak, "unit": "GB/s", "frac": fused_bytes / fv_s / 1e9 / peak,
        "bytes_per_launch": fused_bytes, "share_of_rows": OVERLAP_SHARE, "peak_source": peak_kind,
        "bytes_model": "72 B x the lattice discretization nodes of the shared rows outside the next window "
                       "+ 112 B x patch nodes (the FV tile's rows and records once)"}
    hbm_bound = hbm_part is not None and fused_bytes / (peak * 1e9) > fv_flop / (alu_peak * 1e12)
    lead = hbm_part if hbm_bound else alu_part
    roof = {"bound": "hbm" if hbm_bound else "alu", "kernel": fv_kernel, "achieved": lead["achieved"],
            "peak": lead["peak"], "unit": lead["unit"], "frac": lead["frac"],
            "traffic": kernel_traffic(prof_key, w.name) if prof_key else None,
            "peak_source": lead["peak_source"], "fv_depth": info.get("fv_depth"),
            "ms_per_launch": fv_ms / args.steps, "dominant_phase": dom,
            "with_next_step_far_lattice": overlapped, "alu": alu_part, "hbm": hbm_part,
            "isolated": {"ms_per_launch": fv_iso_ms / k_iso, "achieved": fv_iso_tflops, "unit": "TFLOP/s",
                         "frac": fv_iso_tflops / alu_peak if fv_iso_tflops else None,
                         "note": "FV alone (overlap off), against the FP32 ALU peak"},
            "phase_ms_per_step": {p: phases[p][0] / args.steps for p in phases},
            "phase_ms_per_step_overlap_off": {p: phases_iso[p][0] / k_iso for p in phases_iso}}
    roof_stream = {"bound": "hbm", "kernel": "k_stream_collide", "achieved": stream_gbs, "peak": peak, "unit": "GB/s",
                   "frac": stream_gbs / peak if stream_gbs else None,
                   "traffic": kernel_traffic("stream_collide", w.name), "peak_source": peak_kind,
                   "bytes_per_launch": stream_bytes, "ms_per_launch": st_ms / k_iso if st_n else None,
                   "timed": "whole-lattice launches of the overlap-off run"}
    # the whole step against HBM: algorithmic bytes per lattice step of the
    # structured lattice (9 populations read + 9 written per discretization
    # node), the patch (its records and FV rows read once per step, ~112 B
    # per node at FP32) and relocation / donors / feed (~100 B per node),
    # over the device time of a step
    step_bytes = 18 * bytes_per * n_disc + (112 + 100) * (bytes_per // 4) * n_u
    step_gbs = step_bytes / (ms / args.steps / 1e3) / 1e9
    roof_step = {"bound": "hbm", "achieved": step_gbs, "peak": peak, "unit": "GB/s", "frac": step_gbs / peak,
                 "bytes_per_step": step_bytes, "ms_per_step": ms / args.steps, "peak_source": peak_kind,
                 "bytes_model": "18 x bytes per population x lattice discretization nodes + (112 + 100) B x patch "
                                "nodes (FP32; doubled at FP64)",
                 "overlap_off": {"ms_per_step": ms_iso / k_iso,
                                 "frac": step_bytes / (ms_iso / k_iso / 1e3) / 1e9 / peak}}
    launches = sum(v[1] for v in phases.values())

    # end to end through the public API from host buffers: creation from
    # pinned host arrays (timed on its own), then as many steps as the
    # device-timed run, each with the host call and a force read-back to the
    # host, wall-clock over the steps
    e2e = None
    if not args.no_e2e:
        k_e2e = args.steps
        rho_pinned = torch.from_numpy(rho).pin_memory()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            s2 = Solver(w, mesh=mesh, rho_init=rho_pinned.numpy(), stream=stream.cuda_stream)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            for k in range(k_e2e):
                H.hlbm_step(s2.h, 1)
                H.hlbm_force(s2.h, k + 1, 1)
            torch.cuda.synchronize()
            t2 = time.perf_counter()
            s2.close()
        create_s, secs = t1 - t0, t2 - t1
        h2d = rho.nbytes + mesh.xy.nbytes + mesh.tri.nbytes + mesh.kind.nbytes
        e2e = {"value": world * (n_disc + n_u) * k_e2e / secs / 1e6, "unit": UNIT,
               "h2d_bytes_per_step": h2d / k_e2e, "d2h_bytes_per_step": 16,
               "create_s": create_s,
               "value_with_create": world * (n_disc + n_u) * k_e2e / (secs + create_s) / 1e6,
               "note": f"{k_e2e} steps through hlbm_step(1) + hlbm_force (a 16-byte read-back) each, wall clock; "
                       "creation from pinned host arrays timed apart (create_s); h2d counts the creation inputs "
                       "spread over the steps"}
    s.close()
    # the same workload with the lattice populations stored as FP16 / BF16
    # deviations (FP32 arithmetic), each against the FP32 path above
    reduced = {}
    if not args.no_reduced:
        k_red = max(10, min(args.steps, 100))
        for st in ("f16", "bf16"):
            w.dtype = st
            with torch.cuda.stream(stream):
                s3 = Solver(w, mesh=mesh, rho_init=rho, stream=stream.cuda_stream)
                s3.step(args.warmup)
                torch.cuda.synchronize()
                s3.profile(True)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                s3.step(k_red)
                e1.record(stream)
                torch.cuda.synchronize()
                ph = s3.profile_read()
                ms3 = e0.elapsed_time(e1)
                sms, sn = ph["stream"]
                gbs = 18 * 2 * n_disc / (sms / sn / 1e3) / 1e9 if sn else None
                reduced[st] = {"value": (n_disc + n_u) * k_red / (ms3 / 1e3) / 1e6, "unit": UNIT, "steps": k_red,
                               "ms_per_step": ms3 / k_red, "speedup_vs_f32": (ms / args.steps) / (ms3 / k_red),
                               "stream_gbs": gbs, "stream_frac": gbs / peak if gbs else None}
                s3.close()
        w.dtype = "f32"
    # the outer-node and collision-matrix readings of the method on the same
    # workload (FP32): eq. postcollision2_u with its FV sums, lumped C
    variants = {}
    if not args.no_reduced:
        k_var = max(10, min(args.steps, 100))
        for key, attr in (("outer_fv", "outer_fv"), ("lumped", "lumped"), ("induced", "motion")):
            saved = (w.motion, w.A, w.omega)
            if key == "induced":
                # spring-mounted lamina moved by the fluid force (one force read-back per step)
                w.motion, w.A, w.omega = 3, 0.0, 0.0
                w.mass = math.pi / 4 * w.L * w.L
                w.stiffness, w.y0 = w.mass * (2 * math.pi / 2000.0) ** 2, 2.0
            else:
                setattr(w, attr, 1)
            with torch.cuda.stream(stream):
                s4 = Solver(w, mesh=mesh, rho_init=rho, stream=stream.cuda_stream)
                s4.step(args.warmup)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                s4.profile(True)
                e0.record(stream)
                s4.step(k_var)
                e1.record(stream)
                torch.cuda.synchronize()
                ph = s4.profile_read()
                ms4 = e0.elapsed_time(e1)
                variants[key] = {"value": (n_disc + n_u) * k_var / (ms4 / 1e3) / 1e6, "unit": UNIT, "steps": k_var,
                                 "ms_per_step": ms4 / k_var, "fv_ms_per_step": ph["fv"][0] / k_var,
                                 "status": s4.status}
                s4.close()
            if key == "induced":
                w.motion, w.A, w.omega = saved
            else:
                setattr(w, attr, 0)
    refined = None if args.no_refined else run_refined(stream, args, ms / args.steps, w)
    sweep = None if args.no_sweep else run_sweep(stream, args)
    gradient = None if args.no_gradient else run_gradient(stream, args)
    if rank != 0:
        return 0
    cpu = None if (args.no_cpu_baseline or world > 1) else cpu_baseline(args.workload)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": w.dtype, "data": "synthetic",
            "config": {"workload": w.name, "lattice": f"{w.nx}x{w.ny}", "chord": w.L, "patch_nodes": n_u,
                       "lattice_disc_nodes": n_disc, "n_sub": w.n_sub, "parallelism": f"replicas{world}",
                       "l2": "inputs larger than L2 (two lattice buffers of %.0f MB)"
                             % (9 * bytes_per * (w.nx * w.ny + sum(a * b for a, b, _, _ in w.levels)) / 1e6)},
            "mlups_subiter": mlups_subiter, "roofline": roof, "roofline_stream": roof_stream, "roofline_step": roof_step,
            "cpu_baseline": cpu, "e2e": e2e,
            "reduced_storage": reduced or None, "variants": variants or None, "refined": refined, "sweep": sweep,
            "gradient": gradient,
            "gpu_launches": launches, "clocks": clocks, "status": status, "force_finite": finite}
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def run_refined(stream, args, uniform_ms_per_step, uniform):
    """The headline domain on nested structured levels (Sec. 5): two levels
    (a 2048^2 lattice of spacing 2 and a 1025^2 box) and the paper's four
    (513^2 boxes of spacing 1, 2, 4 and a 512^2 lattice of spacing 8),
    against the uniform 4096^2 lattice step timed above.  Node updates per
    step: level-0 discretization nodes + each coarser level's nodes / 2^k +
    the patch; fine-equivalent MLUPS counts the uniform lattice's nodes."""
    import torch

    import inputs
    from paper_2006_13631_gb300 import Solver

    if uniform.name != "lamina-4096-f32":
        return None
    out = {}
    for name in ("lamina-4096-refined-f32", "lamina-4096-levels4-f32"):
        w = inputs.workload(name)
        period = 2 ** len(w.levels)
        k = period * max(1, min(args.steps, 320) // period)
        with torch.cuda.stream(stream):
            s = Solver(w, stream=stream.cuda_stream)
            s.step(period * max(1, -(-args.warmup // period)))
            torch.cuda.synchronize()
            info = s.info()
            s.profile(True)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            s.step(k)
            e1.record(stream)
            torch.cuda.synchronize()
            ph = s.profile_read()
            s.profile(False)
            ms = e0.elapsed_time(e1)
            status = s.status
            s.close()
        updates = info["n_struct_disc"] + info["coarse_updates"] + info["n_nodes"]
        out[name] = {"levels": [f"{w.nx}x{w.ny}"] + [f"{a}x{b}" for a, b, _, _ in w.levels], "steps": k,
                     "ms_per_step": ms / k, "speedup_vs_uniform": uniform_ms_per_step / (ms / k),
                     "mlups": updates * k / (ms / 1e3) / 1e6,
                     "mlups_fine_equivalent": (uniform.nx * uniform.ny + info["n_nodes"]) * k / (ms / 1e3) / 1e6,
                     "phase_ms_per_step": {p: ph[p][0] / k for p in ph}, "status": status}
    return out


def run_sweep(stream, args):
    """The 64-instance KC/beta study stepped as one batch (hlbm_sweep_*),
    FV tiles chosen per instance by the tuner; against the same instances
    stepped one after another on one stream."""
    import torch

    import inputs
    from paper_2006_13631_gb300 import Solver, Sweep

    ws = inputs.sweep_workloads()
    with torch.cuda.stream(stream):
        solvers = [Solver(w, stream=stream.cuda_stream) for w in ws]
        infos = [s.info() for s in solvers]
        lat = sum(i["n_struct_disc"] for i in infos)
        pat = sum(i["n_nodes"] for i in infos)
        sub = sum(w.n_sub * i["n_nodes"] for w, i in zip(ws, infos))
        sw = Sweep(solvers, stream=stream.cuda_stream)
        picks = sw.tune(trial_steps=1)
        # solvers of similar sub-step counts share FV launches (the others keep the tuned tiles)
        n_packs = sw.pack()
        sw.step(args.warmup)
        k = max(1, args.sweep_steps)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sw.step(k)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        fv = sw.fv_time(1)
        # the same instances one after another, each a plain hlbm_step
        k_serial = max(1, min(k, 3))
        e0.record(stream)
        for s in solvers:
            s.step(k_serial)
        e1.record(stream)
        torch.cuda.synchronize()
        ms_serial = e0.elapsed_time(e1) / k_serial
        bad = sum(1 for s in solvers if s.status != 0)
        sw.close()
        for s in solvers:
            s.close()
    hist = {str(c): picks.count(c) for c in sorted(set(picks))}
    return {"instances": len(ws), "value": (lat + pat) * k / (ms / 1e3) / 1e6, "unit": UNIT, "steps": k,
            "ms_per_step": ms / k, "mlups_subiter": (lat + sub) * k / (ms / 1e3) / 1e6,
            "serial_ms_per_step": ms_serial, "speedup_vs_serial": ms_serial / (ms / k),
            "fv_ms_per_step": float(fv.sum()), "lattice_nodes": lat, "patch_nodes": pat,
            "fv_node_substeps_per_step": sub, "n_sub_range": [min(w.n_sub for w in ws), max(w.n_sub for w in ws)],
            "throughput_only": sum(1 for w in ws if w.throughput_only), "tile_nodes_chosen": hist,
            "fv_packs": n_packs,
            "instances_with_status": bad}


def run_gradient(stream, args):
    """Theta and its gradient in (A, omega, tau_s) on the 1024^2 gradient case
    (chord 32, KC 0.5, beta 800, tau_s 0.506, n 96, FP32, 4 periods): by the
    adjoint of the discrete step (checkpoints every 256 steps; one reverse
    sweep per output, Re and Im), and by central differences over seven
    solvers stepped as one sweep, each against one forward solve."""
    import torch

    import inputs
    from paper_2006_13631_gb300 import Solver, hlbm_theta_adjoint, hlbm_theta_gradient, workload_inputs

    w = inputs.workload("lamina-1024-gradient")
    mesh, rho = w.mesh(), w.rho_init()
    with torch.cuda.stream(stream):
        s = Solver(w, mesh=mesh, rho_init=rho, stream=stream.cuda_stream)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.step(w.steps)
        e1.record(stream)
        torch.cuda.synchronize()
        fwd_ms = e0.elapsed_time(e1)
        th_f = s.gamma(1.0, 3.0)
        s.close()
        grid, patch, motion = workload_inputs(w, mesh, rho)
        th_a, g_re, fwd_ck, bwd_re = hlbm_theta_adjoint(grid, patch, w.tau_s, motion, w.steps, 1.0, 3.0, 1.0, 0.0, 256,
                                                         stream.cuda_stream)
        _, g_im, _, bwd_im = hlbm_theta_adjoint(grid, patch, w.tau_s, motion, w.steps, 1.0, 3.0, 0.0, 1.0, 256,
                                                stream.cuda_stream)
        th, grad, ms = hlbm_theta_gradient(grid, patch, w.tau_s, motion, w.steps, 1.0, 3.0, 1e-4,
                                           stream.cuda_stream)
    return {"workload": w.name, "steps": w.steps, "theta": [th_a.real, th_a.imag], "forward_ms": fwd_ms,
            "forward_theta": [th_f[0], th_f[1]],
            "adjoint": {"dRe_dA_domega_dtau": list(g_re), "dIm_dA_domega_dtau": list(g_im),
                        "checkpointed_forward_ms": fwd_ck, "reverse_ms_per_output": [bwd_re, bwd_im],
                        "backward_over_forward": bwd_re / fwd_ms,
                        "method": "reverse sweep of the discrete step, decisions held fixed, checkpoints every 256 "
                                  "steps (FP32 adjoint)"},
            "central_differences": {"dtheta_dA": [grad[0].real, grad[0].imag],
                                    "dtheta_domega": [grad[1].real, grad[1].imag],
                                    "dtheta_dtau": [grad[2].real, grad[2].imag], "gradient_ms": ms,
                                    "gradient_over_forward": ms / fwd_ms,
                                    "method": "central differences, rel step 1e-4, 7 solves in one sweep"}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="lamina-4096-f32")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-reduced", action="store_true", help="skip the FP16/BF16 lattice-storage runs")
    ap.add_argument("--no-sweep", action="store_true", help="skip the 64-instance KC/beta sweep")
    ap.add_argument("--no-refined", action="store_true", help="skip the nested-level lattice runs")
    ap.add_argument("--sweep-steps", type=int, default=10)
    ap.add_argument("--no-gradient", action="store_true", help="skip the Theta-gradient case")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
