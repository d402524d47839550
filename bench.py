#!/usr/bin/env python
"""MPDATA step throughput on one or more GB300s.

Workload (default): 2D solid-body rotation of a cone, 1024^2 periodic cells,
G = 1, FCT limiter, two passes, FP32 -- the rotating-cone test of the paper
(Sect. 3.6) scaled to 1024^2, one revolution = 6434 steps.  A benchmark step
is one MPDATA time step (all sub-steps fused in one kernel launch).  Inputs are
resident in HBM when timing starts; the 129 MB L2 is flushed (256 MiB write)
before every timed step because the 16 MB working set would otherwise stay in
L2.  Each step is timed with CUDA events on the launching stream; the value is
cells x steps / summed step time.

  python bench.py [--steps K] [--warmup W] [--dtype f32|f64] [--impl ours|reference]
  torchrun --nproc-per-node N bench.py --gpus N ...   (independent replicas, weak scaling)

Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "MPDATA Gcell-steps/s & %HBM roofline, FP32 vs FP64 at stated err; adjoint/fwd"
UNIT = "Gcell-steps/s"
N_SIDE = 1024
REV_STEPS = 6434  # steps per revolution of the 1024^2 rotation workload


def parse_args():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=REV_STEPS)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--dtype", choices=["f32", "f64"], default="f32")
    ap.add_argument("--state", choices=["compensated", "plain"], default="compensated",
                    help="FP32 state of the timed path: compensated (hi + lo, the path that keeps the FP32 "
                         "error bars over a revolution) or plain")
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=N_SIDE, help="side length of the rotation workload")
    ap.add_argument("--no-extras", action="store_true", help="skip the FP64 / staged / e2e / oracle legs")
    ap.add_argument("--no-tune", action="store_true",
                    help="skip the autotuner and time the library's automatic kernel choice")
    ap.add_argument("--n3d", type=int, default=256, help="side length of the deform3d workload")
    ap.add_argument("--kernel", choices=["warp", "band", "warp2"], default=None,
                    help="time this fused kernel family (skips the autotuner)")
    ap.add_argument("--tile-rows", type=int, default=0, help="tile / band rows with --kernel (0 = automatic)")
    ap.add_argument("--workload", choices=["rotation", "ensemble", "deform3d", "adjoint"], default="rotation",
                    help="rotation: 1024^2 rotating cone (default); ensemble: 512 fields of 64^2..512^2, "
                         "split over the ranks by cell count; deform3d: 256^3 deformational flow, "
                         "n_iters = 3 + tot + fct, G != 1 (replicas under torchrun); adjoint: the 512^2 "
                         "adjoint workload alone (one GPU; --no-extras skips its finite-difference check)")
    return ap.parse_args()


def config(args, extra=None):
    c = {"workload": f"2d_solid_body_rotation_{args.n}x{args.n}_fct_n_iters2", "grid": [args.n, args.n],
         "opts": "fct", "n_iters": 2, "G": 1, "boundary": "periodic", "steps_per_revolution": REV_STEPS,
         "l2": "flushed (256 MiB write) before every timed step", "parallelism": f"replicas{args.gpus}"}
    if extra:
        c.update(extra)
    return c


# ----------------------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.idx = device_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        try:
            with open(self.path) as f:
                for line in f:
                    parts = [p.strip() for p in line.split(",")]
                    if len(parts) >= 9:
                        rows.append(parts)
        finally:
            os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ----------------------------------------------------------------------------------- helpers

def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


KERNEL_NAMES = {1: "k_fused2d", 2: "k_band2d", 3: "k_fused2d_nc2"}
KERNEL_SOURCES = {"k_fused2d": ("fused2d.cu", "stencil2d.cuh"), "k_band2d": ("band2d.cu", "stencil2d.cuh"),
                  "k_fused2d_comp": ("fused2d.cu", "stencil2d.cuh"), "k_fused2d_nc2": ("fused2d.cu", "stencil2d.cuh"),
                  "k_fused2d_comp_nc2": ("fused2d.cu", "stencil2d.cuh")}


def kernel_sources_sha256(kernel):
    """SHA-256 of the code of the kernel's sources, comments and white space left out (a stamp
    taken on the code stays valid across edits of comments only)."""
    import hashlib
    import re
    h = hashlib.sha256()
    for name in KERNEL_SOURCES.get(kernel, ()):
        with open(os.path.join(ROOT, "paper_1407_1309_gb300", "csrc", name), encoding="utf-8") as f:
            src = f.read()
        src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
        src = re.sub(r"//[^\n]*", " ", src)
        h.update(" ".join(src.split()).encode())
    return h.hexdigest()


def traffic_from_profiles(kernel, n, dtype, key="bytes_per_launch"):
    """Per-launch DRAM bytes (read + write) of the timed kernel from the committed ncu summary
    (or another per-launch counter stored there, by `key`); None when there is none or when the
    kernel's sources changed since it was taken."""
    path = os.path.join(ROOT, "profiles", f"traffic_{kernel}_rotation{n}_{dtype}.json")
    try:
        with open(path) as f:
            d = json.load(f)
        if d.get("sources_sha256") != kernel_sources_sha256(kernel):
            return None
        return d.get(key)
    except Exception:
        return None


# Algorithmic FP32 instructions per cell-step of the 2D step (n_iters = 2, FCT, G = 1), counted
# from the scheme with every quantity computed once: pass 1 (Eq. 4-5) 12, pseudo-velocities with
# the cross term (Eq. 6 and its 2D form) 19 per face, FCT bounds, in/out sums and factors 32,
# limited pseudo-velocities 10, pass 2 12; each of the 6 divisions is a reciprocal + multiply.
# The compensated state adds, per donor pass, an error-free two-sum of psi + divergence (6
# instructions instead of one add), the error's addition to lo (2) and the renormalisation (6),
# and in pass 1 the low parts' own fluxes (8) and their sum (1): 104 + 2 x 13 + 9 = 139.
ALU_INST_PER_CELL_STEP = {"plain": 104, "compensated": 139}


def alu_roofline(cells, seconds_per_step, kernel, n, dtype, sm_max_mhz, sm_count, state="plain"):
    """The second bound of the step: FP32 lane-instructions against the SMs' issue rate
    (4 schedulers x 32 lanes per SM per clock at the highest SM clock)."""
    if dtype != "f32" or not sm_max_mhz:
        return None
    peak = sm_count * 128 * sm_max_mhz * 1e6 / 1e12
    inst = ALU_INST_PER_CELL_STEP[state]
    achieved = inst * cells / seconds_per_step / 1e12
    warp_inst = traffic_from_profiles(kernel, n, dtype, "smsp__inst_executed.sum")
    out = {"bound": "alu", "achieved": round(achieved, 3), "peak": round(peak, 2), "unit": "Tinst/s",
           "frac": round(achieved / peak, 4), "algorithmic_inst_per_cell_step": inst,
           "peak_source": f"{sm_count} SMs x 128 lanes x {sm_max_mhz:.0f} MHz",
           "executed_lane_slots_per_cell_step": None, "issue_frac_of_executed": None}
    if warp_inst:
        per_cell = warp_inst * 32 / cells
        out["executed_lane_slots_per_cell_step"] = round(per_cell, 1)
        out["issue_frac_of_executed"] = round(per_cell * cells / seconds_per_step / 1e12 / peak, 4)
    return out


# FP64 arithmetic per cell-step (adds, multiplies and fused multiply-adds, one each: the work of
# the FP64 pipe, in the unit of the measured FMA rate; comparisons and selections not counted, a
# division being the Newton-Raphson division with remainder correction, 7):
#   2D (n_iters = 2, FCT, G = 1), 94, counted from the formulas: pass 1 6 (two face fluxes, three
#   flux differences, the update), pseudo-velocities 29 per face (A and B 9 each, V_q 3, the
#   combination 7, the flux 1), FCT 24 (in/out sums 8, two factors 8 each), limited fluxes 2,
#   pass 2 4 (the 2D kernels execute 118 per cell-step at 1024^2, their recomputed halo included);
#   3D (n_iters = 3 + tot + FCT + G), 992, counted by ncu as the DADD + DMUL + DFMA instructions of
#   one step of the staged FP64 kernels at 128^3 (no recomputed halo): pass 1 46, the bounds 0,
#   per corrective pass 473 (pseudo-advector with the cross and third-order terms 376, factors 42,
#   limiter 9, donor pass 46).  (A hand tally of the 3D formulas, 1164, counted multiply-add
#   pairs the compiler fuses.)
FP64_OPS_PER_CELL_STEP = {"2d": 94, "3d": 992}


def measure_fma_rates(dev):
    """FMA lane operations per second of this GPU in FP32 and FP64 (mpdata_selftest_fma_rate:
    every SM full of independent FMA chains), best of three launches of ~30 ms each."""
    import torch

    from paper_1407_1309_gb300 import capi
    out = {}
    for name, code, dt in (("f32", capi.F32, torch.float32), ("f64", capi.F64, torch.float64)):
        sink = torch.zeros(1, dtype=dt, device=dev)
        stream = torch.cuda.current_stream(dev)

        def timed(iters):
            e0, e1 = _events()
            e0.record(stream)
            n = capi.mpdata_selftest_fma_rate(code, iters, sink, stream)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            return n, e0.elapsed_time(e1) / 1e3

        n, secs = timed(256)
        iters = max(256, int(256 * 0.03 / max(secs, 1e-6)))
        best = max(n / s for n, s in (timed(iters) for _ in range(3)))
        out[name] = best
    return {"f32_fma_per_s": out["f32"], "f64_fma_per_s": out["f64"],
            "how": "mpdata_selftest_fma_rate: 8 x 256 threads per SM, 8 independent FMA chains each, "
                   "CUDA events, best of 3"}


def fp64_roofline(cell_steps_per_s, case, rates):
    """The FP64 path against the measured FP64 FMA issue rate (one FP64 operation per lane slot)."""
    ops = FP64_OPS_PER_CELL_STEP[case]
    achieved = ops * cell_steps_per_s / 1e12
    peak = rates["f64_fma_per_s"] / 1e12
    return {"bound": "alu_fp64", "achieved": round(achieved, 4), "peak": round(peak, 4), "unit": "Top/s",
            "frac": round(achieved / peak, 4), "algorithmic_fp64_ops_per_cell_step": ops,
            "peak_source": "measured in this run (" + rates["how"] + ")"}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ----------------------------------------------------------------------------------- multi-rank helpers

def max_over_ranks(seconds, device=None):
    """Largest value of `seconds` over all ranks (the job finishes with its slowest rank)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(seconds)
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(cells_per_rank, steps, world_size, max_seconds):
    """Whole-job throughput in Gcell-steps/s: every rank advanced cells_per_rank cells by
    `steps` steps (weak scaling), the job took the slowest rank's time."""
    return cells_per_rank * steps * world_size / max_seconds / 1e9


def partition_fields(sizes, world_size):
    """Split ensemble fields over ranks by cell count (largest first onto the least loaded
    rank); returns one list of field indices per rank, each in ascending order."""
    loads = [0] * world_size
    parts = [[] for _ in range(world_size)]
    for f in sorted(range(len(sizes)), key=lambda k: (-sizes[k], k)):
        r = min(range(world_size), key=lambda q: (loads[q], q))
        parts[r].append(f)
        loads[r] += sizes[f]
    return [sorted(p) for p in parts]


# ----------------------------------------------------------------------------------- ours

def _split(x):
    """FP64 field -> FP32 pair (hi, lo) with hi + lo = x to ~1e-14 relative."""
    import numpy as np
    hi = x.astype(np.float32)
    return hi, (x - hi.astype(np.float64)).astype(np.float32)


def one_revolution_errors(n, psi_np, gc_np, dev, steps):
    """Both FP32 states over `steps` steps (one revolution) against the FP64 GPU path from the
    same input (which matches the FP64 oracle to 1e-12): relative L2 error and relative mass
    drift of each, with the same inputs rounded to FP32 for the FP32 paths."""
    import numpy as np
    import torch

    from paper_1407_1309_gb300 import capi
    from paper_1407_1309_gb300.solver import Mpdata
    out = {"steps": steps, "vs": "FP64 GPU path from the same input (equal to the FP64 oracle to 1e-12)"}
    with Mpdata((n, n), dtype=torch.float64, n_iters=2, opts=capi.FCT, device=dev) as m64:
        a = torch.tensor(psi_np, dtype=torch.float64, device=dev)
        b = torch.empty_like(a)
        m64.advance(a, b, [torch.tensor(v, dtype=torch.float64, device=dev) for v in gc_np], n_steps=steps)
        ref = b.cpu().numpy()
    m0 = psi_np.sum()
    g32 = [torch.tensor(v.astype(np.float32), device=dev) for v in gc_np]
    with Mpdata((n, n), dtype=torch.float32, n_iters=2, opts=capi.FCT, device=dev) as m:
        a = torch.tensor(psi_np.astype(np.float32), device=dev)
        b = torch.empty_like(a)
        m.advance(a, b, g32, n_steps=steps)
        plain = b.double().cpu().numpy()
        hi, lo = (torch.tensor(x, device=dev) for x in _split(psi_np))
        ho, lo2 = torch.empty_like(hi), torch.empty_like(lo)
        m.advance_compensated(hi, lo, ho, lo2, g32, n_steps=steps)
        comp = ho.double().cpu().numpy() + lo2.double().cpu().numpy()
    for name, x in (("compensated", comp), ("plain", plain)):
        out[name] = {"rel_l2": float(np.linalg.norm(x - ref) / np.linalg.norm(ref)),
                     "rel_mass_drift": float(abs(x.sum() - m0) / abs(m0)),
                     "meets_fp32_bars": bool(np.linalg.norm(x - ref) <= 1e-5 * np.linalg.norm(ref) and
                                             abs(x.sum() - m0) <= 1e-6 * abs(m0))}
    return out


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_1407_1309_gb300 import capi, workloads
    from paper_1407_1309_gb300.solver import Mpdata

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=dev)
    dtype = torch.float32 if args.dtype == "f32" else torch.float64
    comp = dtype == torch.float32 and args.state == "compensated"
    state = "compensated" if comp else "plain"
    esize = 4 if dtype == torch.float32 else 8
    n = args.n
    cells = n * n
    psi_np, gc_np, _ = workloads.rotation_2d(n, REV_STEPS if n == N_SIDE else None)
    psi0 = torch.tensor(psi_np, dtype=dtype, device=dev)
    gc = [torch.tensor(v, dtype=dtype, device=dev) for v in gc_np]
    if comp:
        hi_np, lo_np = _split(psi_np)
        hi0, lo0 = torch.tensor(hi_np, device=dev), torch.tensor(lo_np, device=dev)
        a, al = hi0.clone(), lo0.clone()
        b, bl = torch.empty_like(a), torch.empty_like(al)
    else:
        a, b = psi0.clone(), torch.empty_like(psi0)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    m = Mpdata((n, n), dtype=dtype, n_iters=2, opts=capi.FCT, device=dev)
    stream = torch.cuda.current_stream(dev)
    if args.kernel:
        choice = ({"warp": 1, "band": 2, "warp2": 3}[args.kernel] if not comp or args.kernel != "band" else 1,
                  args.tile_rows)
        m.tune(capi.TUNE_KERNEL, choice[0])
        m.tune(capi.TUNE_TILE_ROWS, choice[1])
    elif args.no_tune:
        choice = None
    else:  # kernel family and tile height for this workload, timed on these buffers (not cached)
        from paper_1407_1309_gb300 import autotune
        # one step per timed launch (the fusion depths, never faster here, are compared in the
        # fusion_depth leg)
        one_step = tuple(c for c in autotune.CANDIDATES if c[2] == 1)
        choice, _, _ = autotune.autotune(m, a, gc, candidates=one_step, steps=8, use_cache=False,
                                         lo=al if comp else None)
    if comp:
        kname = "k_fused2d_comp_nc2" if choice and choice[0] == 3 else "k_fused2d_comp"
    else:
        kname = KERNEL_NAMES[choice[0]] if choice else "automatic"
    tuned = {"kernel": kname, "tile_rows": choice[1] if choice else 0,
             "chosen_by": "command line" if args.kernel else ("autotuner" if choice else "library default")}

    def timed(K, flush_l2=True):
        # arguments marshalled once per direction, so the host enqueues a step faster than the
        # device runs flush + step and no host gap falls between the events
        nonlocal a, b
        if comp:
            nonlocal al, bl
            calls = {a.data_ptr(): capi.prepare_advance_compensated(m.h, a, al, b, bl, gc),
                     b.data_ptr(): capi.prepare_advance_compensated(m.h, b, bl, a, al, gc)}
        else:
            calls = {a.data_ptr(): capi.prepare_advance(m.h, a, b, gc),
                     b.data_ptr(): capi.prepare_advance(m.h, b, a, gc)}
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
        for e0, e1 in evs:
            if flush_l2:
                flush.zero_()
            e0.record(stream)
            calls[a.data_ptr()]()
            e1.record(stream)
            a, b = b, a
            if comp:
                al, bl = bl, al
        torch.cuda.synchronize(dev)
        return sum(e0.elapsed_time(e1) for e0, e1 in evs) / 1e3

    for _ in range(args.warmup):
        if comp:
            m.advance_compensated(a, al, b, bl, gc)
            al, bl = bl, al
        else:
            m.advance(a, b, gc)
        a, b = b, a
    if comp:
        a.copy_(hi0)
        al.copy_(lo0)
    else:
        a.copy_(psi0)
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    clocks = ClockSampler(local)
    clocks.start()
    t_wall0 = time.perf_counter()
    secs = timed(args.steps)
    torch.cuda.synchronize(dev)
    wall = time.perf_counter() - t_wall0
    clk = clocks.stop()
    secs = max_over_ranks(secs, dev)
    if ws > 1:
        dist.barrier()
    result_after_K = a.double().cpu().numpy() + (al.double().cpu().numpy() if comp else 0.0)
    value = job_value(cells, args.steps, ws, secs)
    ms_per_step = secs / args.steps * 1e3

    peaks, how = measured_peaks()
    # read psi (and lo), gc0, gc1; write psi (and lo)
    bytes_per_cell = (6 if comp else 4) * esize
    achieved = bytes_per_cell * cells / (secs / args.steps) / 1e9
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": round(achieved / peaks["hbm_gbs"], 4),
                "traffic": traffic_from_profiles(kname, n, args.dtype),
                "peak_source": f"{how} (MEASURED_PEAKS.json hbm_gbs, burst copy)" if how == "measured" else "fallback",
                "algorithmic_bytes_per_cell_step": bytes_per_cell, "kernel": kname}

    out = {"metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": round(ms_per_step, 5), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": args.dtype,
           "data": "synthetic (seeded rotating-cone workload, no dataset)",
           "config": config(args, {"wall_s_timed_region_incl_flushes": round(wall, 3), "kernel": tuned,
                                   "fp32_state": ("compensated: psi = hi + lo, both FP32 arrays; every quantity "
                                                  "of the step in FP32" if comp else
                                                  ("plain FP32" if dtype == torch.float32 else "FP64"))}),
           "roofline": roofline,
           "alu_roofline": alu_roofline(cells, secs / args.steps, kname, n, args.dtype, clk.get("sm_max_mhz"),
                                        torch.cuda.get_device_properties(dev).multi_processor_count, state),
           "gpu_launches": args.steps, "clocks": clk}

    if rank == 0 and not args.no_extras:
        extras = {}
        # accuracy of the headline arithmetic over one full revolution (independent of --steps),
        # and of this run's K steps against the FP64 GPU path
        if dtype == torch.float32 and n == N_SIDE:
            out["err_one_revolution"] = one_revolution_errors(n, psi_np, gc_np, dev, REV_STEPS)
        with Mpdata((n, n), dtype=torch.float64, n_iters=2, opts=capi.FCT, device=dev) as m64:
            p64 = torch.tensor(psi_np, dtype=torch.float64, device=dev)
            g64 = [torch.tensor(v, dtype=torch.float64, device=dev) for v in gc_np]
            t0 = torch.cuda.Event(enable_timing=True)
            t1 = torch.cuda.Event(enable_timing=True)
            q = torch.empty_like(p64)
            k64 = min(args.steps, 1000)
            t0.record(stream)
            for s_ in range(args.steps):
                m64.advance(p64, q, g64)
                p64, q = q, p64
                if s_ + 1 == k64:
                    t1.record(stream)
            torch.cuda.synchronize(dev)
            s64 = t0.elapsed_time(t1) / 1e3
            ref64 = p64.cpu().numpy()
        e = result_after_K - ref64
        out["err_vs_fp64_gpu_after_K_steps"] = {
            "rel_l2": float(np.linalg.norm(e) / np.linalg.norm(ref64)),
            "max_abs": float(np.abs(e).max()),
            "rel_mass_drift": float(abs(result_after_K.sum() - psi_np.sum()) / abs(psi_np.sum()))}
        rates = measure_fma_rates(dev)
        extras["fma_rates"] = rates
        extras["fp64_path"] = {"value": round(cells * k64 / s64 / 1e9, 3), "unit": UNIT, "steps": k64,
                               "l2": "not flushed (ALU-bound: FP64 arithmetic, not HBM, limits it)",
                               "roofline": fp64_roofline(cells * k64 / s64, "2d", rates)}
        if comp:
            # the plain FP32 state, timed like the headline (autotuned family and tile height)
            from paper_1407_1309_gb300 import autotune
            with Mpdata((n, n), dtype=torch.float32, n_iters=2, opts=capi.FCT, device=dev) as mp:
                x = psi0.clone()
                pchoice, _, _ = autotune.autotune(mp, x, gc, candidates=tuple(c for c in autotune.CANDIDATES
                                                                              if c[2] == 1),
                                                  steps=8, use_cache=False)
                kp = min(args.steps, 1000)
                sp = autotune.time_steps(mp, x, gc, steps=kp)
                pk = KERNEL_NAMES[pchoice[0]]
            extras["fp32_plain_state"] = {
                "value": round(cells / sp / 1e9, 3), "unit": UNIT, "steps_timed": kp,
                "kernel": {"kernel": pk, "tile_rows": pchoice[1]}, "bytes_per_cell_step": 16,
                "roofline": {"bound": "hbm", "achieved": round(16 * cells / sp / 1e9, 1), "peak": peaks["hbm_gbs"],
                             "unit": "GB/s", "frac": round(16 * cells / sp / 1e9 / peaks["hbm_gbs"], 4),
                             "traffic": traffic_from_profiles(pk, n, "f32")},
                "alu_roofline": alu_roofline(cells, sp, pk, n, "f32", clk.get("sm_max_mhz"),
                                             torch.cuda.get_device_properties(dev).multi_processor_count),
                "note": "fails the FP32 bars over a revolution (err_one_revolution.plain): the background of "
                        "1.0 sits on a binade edge, where the rounding of psi + flux divergence is biased"}
        # staged path (one kernel per sub-step) for comparison
        with Mpdata((n, n), dtype=dtype, n_iters=2, opts=capi.FCT | capi.STAGED, device=dev) as ms:
            x, y = psi0.clone(), torch.empty_like(psi0)
            ks = min(args.steps, 300)
            evs = []
            for _ in range(ks):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                ms.advance(x, y, gc)
                e1.record(stream)
                evs.append((e0, e1))
                x, y = y, x
            torch.cuda.synchronize(dev)
            st = sum(e0.elapsed_time(e1) for e0, e1 in evs) / 1e3
            extras["staged_path"] = {"value": round(cells * ks / st / 1e9, 3), "unit": UNIT, "steps": ks,
                                     "kernels_per_step": 6}
        extras["abs_variable_sign"] = bench_abs(psi_np, gc_np, dtype, dev, stream, flush, min(args.steps, 300))
        extras["dfl_divergent_flow"] = bench_dfl(n, dtype, dev, stream, flush, min(args.steps, 300))
        out["e2e"] = run_e2e(m, psi_np, gc_np, dtype, dev, stream, min(args.steps, 1000), ws, comp)

        def gpu_steps(k):  # this build's headline step from the same input, for the oracle leg's comparison
            with Mpdata((n, n), dtype=dtype, n_iters=2, opts=capi.FCT, device=dev) as mm:
                if comp:
                    h0, l0 = hi0.clone(), lo0.clone()
                    h1, l1 = torch.empty_like(h0), torch.empty_like(l0)
                    mm.advance_compensated(h0, l0, h1, l1, gc, n_steps=k)
                    return h1.double().cpu().numpy() + l1.double().cpu().numpy()
                x, y = psi0.clone(), torch.empty_like(psi0)
                mm.advance(x, y, gc, n_steps=k)
                return y.double().cpu().numpy()

        out["cpu_baseline"] = cpu_baseline(psi_np if comp else psi0.double().cpu().numpy(),
                                           [v.double().cpu().numpy() for v in gc], gpu_steps=gpu_steps)
        out["extras"] = extras
        configs = {}
        for name, fn in (("1d", bench_config1), ("3d", bench_config3), ("ensemble", bench_config4),
                         ("adjoint", bench_config5), ("next_rows", bench_next_rows),
                         ("fusion_depth", bench_fusion_depth)):
            try:
                configs[name] = fn(dev)
            except Exception as ex:  # one failing leg must not sink the headline line
                configs[name] = {"error": f"{type(ex).__name__}: {str(ex)[:300]}"}
        out["other_configs"] = configs
    elif not args.no_extras:
        run_e2e(m, psi_np, gc_np, dtype, dev, stream, min(args.steps, 1000), ws, comp)
    m.close()
    if ws > 1:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(out), flush=True)


def _events():
    import torch
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def bench_abs(psi_np, gc_np, dtype, dev, stream, flush, steps):
    """The variable-sign option (abs, Sect. 3.1.5) on the rotation workload shifted to cross zero
    (cone top +1.5 over a background of -1.5), FCT, on the staged kernels (the fused ones
    decline it): each step timed between CUDA events after an L2 flush, and 10 steps against
    the same option in FP64 on the GPU (whose parity with the oracle the tests check)."""
    import numpy as np
    import torch

    from paper_1407_1309_gb300 import capi
    from paper_1407_1309_gb300.solver import Mpdata
    n = psi_np.shape[0]
    psi_v = psi_np - 2.5
    opts = capi.ABS | capi.FCT
    with Mpdata((n, n), dtype=dtype, n_iters=2, opts=opts, device=dev) as m:
        x = torch.tensor(psi_v, dtype=dtype, device=dev)
        y = torch.empty_like(x)
        gc = [torch.tensor(v, dtype=dtype, device=dev) for v in gc_np]
        m.advance(x, y, gc, n_steps=3)
        evs = []
        for _ in range(steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            m.advance(x, y, gc)
            e1.record(stream)
            evs.append((e0, e1))
            x, y = y, x
        torch.cuda.synchronize(dev)
        secs = sum(e0.elapsed_time(e1) for e0, e1 in evs) / 1e3
        res = {"value": round(n * n * steps / secs / 1e9, 3), "unit": UNIT, "steps": steps,
               "workload": f"2d_rotation_{n}x{n}_variable_sign_abs_fct", "path": "staged kernels"}
        p0 = torch.tensor(psi_v, dtype=dtype, device=dev)
        q = torch.empty_like(p0)
        m.advance(p0, q, gc, n_steps=10)
        got = q.double().cpu().numpy()
    with Mpdata((n, n), dtype=torch.float64, n_iters=2, opts=opts, device=dev) as m64:
        p64 = p0.double()
        q64 = torch.empty_like(p64)
        m64.advance(p64, q64, [v.double() for v in gc], n_steps=10)
        ref = q64.cpu().numpy()
    res["err_vs_fp64_gpu_10_steps"] = {"rel_l2": float(np.linalg.norm(got - ref) / np.linalg.norm(ref)),
                                       "max_abs": float(np.abs(got - ref).max())}
    return res


def bench_dfl(n, dtype, dev, stream, flush, steps):
    """The divergent-flow option (dfl, Sect. 3.1.3) on an n^2 field in the steady separable
    divergent flow u = 1 + 0.5 sin(2 pi x), v = 0.7 (1 + 0.4 cos(2 pi y)) at max |C| 0.25 (the
    flow of its convergence pin), two passes, on the staged kernels: each step timed between
    CUDA events after an L2 flush, and 10 steps against FP64 on the GPU."""
    import numpy as np
    import torch

    from paper_1407_1309_gb300 import capi
    from paper_1407_1309_gb300.solver import Mpdata
    x = (np.arange(n) + 0.5) / n
    f = (np.arange(n) + 1.0) / n
    psi = 2.0 + np.sin(2 * np.pi * x)[None, :] * np.cos(2 * np.pi * x)[:, None]
    u, v = 1.0 + 0.5 * np.sin(2 * np.pi * f), 0.7 * (1.0 + 0.4 * np.cos(2 * np.pi * f))
    c = 0.25 / max(u.max(), v.max())
    gc_np = [np.broadcast_to((c * v)[:, None], (n, n)).copy(), np.broadcast_to((c * u)[None, :], (n, n)).copy()]
    opts = capi.DFL
    res = {"workload": f"2d_divergent_separable_{n}x{n}_dfl_n_iters2", "path": "staged kernels"}
    outs = {}
    for dt in (dtype, torch.float64):
        with Mpdata((n, n), dtype=dt, n_iters=2, opts=opts, device=dev) as m:
            a = torch.tensor(psi, dtype=dt, device=dev)
            b = torch.empty_like(a)
            gc = [torch.tensor(g, dtype=dt, device=dev) for g in gc_np]
            m.advance(a, b, gc, n_steps=10)
            outs[dt] = b.double().cpu().numpy()
            if dt == dtype:
                evs = []
                for _ in range(steps):
                    flush.zero_()
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    m.advance(a, b, gc)
                    e1.record(stream)
                    evs.append((e0, e1))
                    a, b = b, a
                torch.cuda.synchronize(dev)
                secs = sum(e0.elapsed_time(e1) for e0, e1 in evs) / 1e3
                res.update({"value": round(n * n * steps / secs / 1e9, 3), "unit": UNIT, "steps": steps})
    got, ref = outs[dtype], outs[torch.float64]
    res["err_vs_fp64_gpu_10_steps"] = {"rel_l2": float(np.linalg.norm(got - ref) / np.linalg.norm(ref)),
                                       "rel_mass_drift": float(abs(got.sum() - ref.sum()) / abs(ref.sum()))}
    return res


def bench_config1(dev):
    """1D: N = 500, C = 0.5, box + Gaussian, two passes, FP64, 1000 steps = one transit."""
    import numpy as np
    import torch

    from paper_1407_1309_gb300 import workloads
    from paper_1407_1309_gb300.solver import Mpdata
    psi, gc = workloads.hello_1d()
    with Mpdata((500,), dtype=torch.float64, n_iters=2, device=dev) as m:
        a = torch.tensor(psi, device=dev)
        b = torch.empty_like(a)
        g = [torch.tensor(gc[0], device=dev)]
        m.advance(a, b, g, n_steps=10)
        e0, e1 = _events()
        e0.record()
        m.advance(a, b, g, n_steps=1000)
        e1.record()
        torch.cuda.synchronize(dev)
        secs = e0.elapsed_time(e1) / 1e3
        out = b.cpu().numpy()
    return {"workload": "1d_box_gaussian_n500_c0.5_n_iters2_f64", "steps": 1000, "time_ms": round(secs * 1e3, 3),
            "value": round(500 * 1000 / secs / 1e9, 4), "unit": UNIT,
            "one_transit_rms_err_vs_initial": float(np.sqrt(np.mean((out - psi) ** 2))),
            "path": "one launch of one block for all steps (field and intermediates in shared memory; FP64 rate of one SM)"}


def bench_config3(dev, n=256, steps=20, oracle_steps=1):
    """3D deformational flow, n^3, G != 1, FP32; n_iters = 3 + tot + fct, and the infinite-gauge
    variant (n_iters = 2, tot, fct, blobs of +/-1).  Each variant: FP32 and FP64 timed over
    `steps` steps; both compared with the FP64 oracle after its first `oracle_steps` steps
    (every cell), and FP32 with FP64 after all steps."""
    import numpy as np
    import torch

    import oracle
    from paper_1407_1309_gb300 import capi, workloads
    from paper_1407_1309_gb300.solver import Mpdata
    out = {}
    peaks, _ = measured_peaks()
    rates = measure_fma_rates(dev)
    oracle.set_threads(0)
    for label, iga in (("n_iters3_tot_fct", False), ("iga_n_iters2_tot_fct", True)):
        psi, gc, G = workloads.deformational_3d(n, iga=iga)
        K = 2 if iga else 3
        opts = capi.TOT | capi.FCT | capi.NUG | (capi.IGA if iga else 0)
        scales = [workloads.deformational_scale(s) for s in range(steps)]
        res, first = {}, {}
        for dt in (torch.float32, torch.float64):
            t = lambda x: torch.tensor(x, dtype=dt, device=dev)
            with Mpdata((n, n, n), dtype=dt, n_iters=K, opts=opts, device=dev) as m:
                a, b, g, Gt = t(psi), torch.empty(n, n, n, dtype=dt, device=dev), [t(v) for v in gc], t(G)
                m.advance(a, b, g, Gt, None, 0.0, oracle_steps, scales[:oracle_steps])
                torch.cuda.synchronize(dev)
                first[dt] = b.double().cpu().numpy()
                m.advance(a, b, g, Gt, None, 0.0, 2, scales[:2])
                e0, e1 = _events()
                e0.record()
                m.advance(a, b, g, Gt, None, 0.0, steps, scales)
                e1.record()
                torch.cuda.synchronize(dev)
                res[dt] = (e0.elapsed_time(e1) / 1e3, b.double().cpu().numpy())
        # the oracle from the FP64 inputs (FP64 path) and from the FP32-rounded inputs (FP32 path)
        errs = {}
        for dt in (torch.float64, torch.float32):
            r = (lambda x: x.astype(np.float32).astype(np.float64)) if dt == torch.float32 else (lambda x: x)
            ref = r(psi)
            for s_ in scales[:oracle_steps]:
                ref = oracle.step(ref, [r(v) * s_ for v in gc], g=r(G), n_iters=K, opts=int(opts) & ~capi.NUG)
            got = first[dt]
            key = "f64" if dt == torch.float64 else "f32"
            errs[key] = {"max_rel": float(np.abs(got - ref).max() / np.abs(ref).max()),
                         "rel_l2": float(np.linalg.norm(got - ref) / np.linalg.norm(ref)),
                         "rel_mass_drift": float(abs(got.sum() - ref.sum()) / np.abs(ref).sum())}
        secs32, o32 = res[torch.float32]
        o64 = res[torch.float64][1]
        cells = n ** 3
        bpc = 24  # psi, gc0..2, G read; psi written
        achieved = bpc * cells * steps / secs32 / 1e9
        v64 = cells * steps / res[torch.float64][0]
        out[label] = {"workload": f"3d_deformational_{n}^3_{label}_G", "steps": steps,
                      "value": round(cells * steps / secs32 / 1e9, 3), "unit": UNIT,
                      "fp64_value": round(v64 / 1e9, 3),
                      "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peaks["hbm_gbs"],
                                   "unit": "GB/s", "frac": round(achieved / peaks["hbm_gbs"], 4),
                                   "algorithmic_bytes_per_cell_step": bpc},
                      "err_vs_oracle_first_steps": {"steps": oracle_steps, **errs},
                      "err_fp32_vs_fp64_gpu": {"rel_l2": float(np.linalg.norm(o32 - o64) / np.linalg.norm(o64)),
                                               "rel_mass_drift": float(abs(o32.sum() - o64.sum()) / np.abs(o64).sum())},
                      "path": ("z-march kernels: pass 1 + bounds, then per corrective pass the pseudo-advector "
                               "and the limited donor pass (5 launches per step)" if not iga else
                               "z-march kernels: pass 1 + bounds, the pseudo-advector, the limited donor pass "
                               "(3 launches per step)")}
        if not iga:
            out[label]["fp64_roofline"] = fp64_roofline(v64, "3d", rates)
    return out


def bench_fusion_depth(dev, sizes=(1024, 4096)):
    """Temporal blocking against one step per launch: the rotation workload (FCT, two passes,
    plain FP32 state) at each size, timed by the autotuner over every candidate (L2 flushed before
    each launch; a launch at depth S runs S steps and its time counts for S steps), with the
    oracle-checked parity of every depth in the GPU tests.  Reports Gcell-steps/s of the best
    one-step-per-launch kernel and of each depth, and the autotuner's pick."""
    import torch

    from paper_1407_1309_gb300 import autotune, capi, workloads
    from paper_1407_1309_gb300.solver import Mpdata
    out = {"how": "autotune.time_steps: per launch after a 256 MiB L2 flush, CUDA events, 12 launches"}
    for n in sizes:
        psi_np, gc_np, _ = workloads.rotation_2d(n)
        psi = torch.tensor(psi_np, dtype=torch.float32, device=dev)
        gc = [torch.tensor(v, dtype=torch.float32, device=dev) for v in gc_np]
        with Mpdata((n, n), dtype=torch.float32, n_iters=2, opts=capi.FCT, device=dev) as m:
            best, sec, timings = autotune.autotune(m, psi, gc, steps=12, use_cache=False)
        one = min((v, c) for c, v in timings.items() if c[2] == 1)
        rate = lambda s_: round(n * n / s_ / 1e9, 2)
        out[f"{n}x{n}"] = {"one_step_per_launch": {"value": rate(one[0]), "kernel": KERNEL_NAMES.get(one[1][0], "auto"),
                                                   "tile_rows": one[1][1]},
                           "depth": {str(d): rate(timings[(0, 0, d)]) for d in (2, 3, 4) if (0, 0, d) in timings},
                           "autotuner_pick": {"kernel": best[0], "tile_rows": best[1], "steps_per_launch": best[2]},
                           "unit": UNIT}
    return out


def bench_next_rows(dev):
    """The scope table's later rows on their paper workloads, FP64, each against the oracle:
    open edges (the hello world of Sect. 3.3: 101 points, 100 steps, the default options), the
    trapezoidal sources (the translating oscillator of Sect. 4.2: 1000 cells, 1400 steps) and the
    prognosed-velocity shallow-water system (the 1D drop of Sect. 5.3 to t = 3, and the 2D drop of
    Sect. 5.4 on 320^2 cells to t = 3 against the paper's closed form).  These workloads are small:
    their times are launch latency, reported for completeness."""
    import math

    import numpy as np
    import torch

    import oracle
    from paper_1407_1309_gb300 import capi, workloads
    from paper_1407_1309_gb300.solver import Mpdata
    out = {}
    f64 = lambda a: torch.tensor(a, dtype=torch.float64, device=dev)

    def timed(fn):
        e0, e1 = _events()
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1) / 1e3

    # open edges: Sect. 3.3
    psi, gc = workloads.agnesi_1d()
    opts = capi.FCT | capi.IGA | capi.KAHAN | capi.OPEN0
    ref = oracle.step(psi, gc, n_iters=2, opts=int(opts), n_steps=100)
    with Mpdata((101,), dtype=torch.float64, n_iters=2, opts=opts, device=dev) as m:
        a, b = f64(psi), torch.empty(101, dtype=torch.float64, device=dev)
        g = [f64(gc[0])]
        secs = timed(lambda: m.advance(a, b, g, n_steps=100))
        got = b.cpu().numpy()
    out["open_edges_hello_world"] = {"cells": 101, "steps": 100, "time_ms": round(secs * 1e3, 3),
                                     "max_rel_err_vs_oracle": float(np.abs(got - ref).max() / np.abs(ref).max())}
    # trapezoidal sources: Sect. 4.2
    psi0, phi0, gc, omega = workloads.oscillator_1d()
    A = [[0.0, omega], [-omega, 0.0]]
    opts = capi.FCT | capi.IGA | capi.KAHAN | capi.RHS_TRAPEZ
    ref = np.stack(oracle.step_trapez([psi0, phi0], gc, A, dt=1.0, n_iters=2, opts=int(opts & ~capi.RHS_TRAPEZ),
                                      n_steps=1400))
    with Mpdata([(1000,), (1000,)], dtype=torch.float64, n_iters=2, opts=opts, device=dev) as m:
        st = torch.cat([f64(psi0), f64(phi0)])
        o = torch.empty_like(st)
        g = [torch.cat([f64(gc[0])] * 2)]
        m.set_rhs_linear(A)
        secs = timed(lambda: m.advance(st, o, g, dt=1.0, n_steps=1400))
        got = o.cpu().numpy().reshape(2, 1000)
    out["trapez_oscillator"] = {"cells": 1000, "equations": 2, "steps": 1400, "time_ms": round(secs * 1e3, 3),
                                "max_rel_err_vs_oracle": float(np.abs(got - ref).max() / np.abs(ref).max()),
                                "phase_after_one_period": {"max_abs_phi": float(np.abs(got[1]).max())}}
    # shallow water: Sect. 5.3 (1D) and 5.4 (2D)
    for nd, n, dx, dt, steps in ((1, 320, 0.05, 0.01, 300), (2, 320, 0.05, 0.01, 300)):
        c = -0.5 * n * dx + (np.arange(n) + 0.5) * dx
        if nd == 1:
            h0 = np.where(np.abs(c) <= 1.0, 1.0 - c ** 2, 0.0)
        else:
            X, Y = np.meshgrid(c, c, indexing="ij")
            h0 = np.maximum(1.0 - X ** 2 - Y ** 2, 0.0)
        opts = capi.ABS | capi.FCT | capi.DFL | sum(capi.OPEN0 << d for d in range(nd))
        with Mpdata([h0.shape] * (nd + 1), dtype=torch.float64, n_iters=2, opts=opts | capi.SW, device=dev) as m:
            state = torch.cat([f64(h0).flatten()] + [torch.zeros(h0.size, dtype=torch.float64, device=dev)] * nd)
            secs = timed(lambda: m.sw_advance(state, dt, dx, n_steps=steps))
            got = state.cpu().numpy().reshape(nd + 1, *h0.shape)
        res = {"cells": int(h0.size), "steps": steps, "time_ms": round(secs * 1e3, 3),
               "value": round(h0.size * steps / secs / 1e9, 4), "unit": UNIT}
        if nd == 1:
            h, qs, _ = oracle.step_shallow_water(h0, [np.zeros_like(h0)], dt, dx, n_iters=2, opts=int(opts),
                                                 n_steps=steps)
            want = np.stack([h] + qs)
            res["max_rel_err_vs_oracle"] = float(np.abs(got - want).max() / np.abs(want).max())
        else:
            lam = math.sqrt(2 * (steps * dt) ** 2 + 1)
            ha = np.maximum(1 / lam ** 2 - (X ** 2 + Y ** 2) / lam ** 4, 0.0)
            res["rel_l2_err_h_vs_closed_form"] = float(np.linalg.norm(got[0] - ha) / np.linalg.norm(ha))
            res["depth_conservation_rel"] = float(abs(got[0].sum() - h0.sum()) / h0.sum())
        out[f"shallow_water_{nd}d_drop"] = res
    return out


def bench_config4(dev, n_fields=512, steps=500, fp64_steps=5):
    """Ensemble: n_fields 2D fields, sides uniform in {64, ..., 512}, FCT, two passes, FP32;
    the step loop captured in one CUDA graph; compared with one FP64 handle per field."""
    import numpy as np
    import torch

    from paper_1407_1309_gb300 import capi, workloads
    from paper_1407_1309_gb300.solver import Mpdata
    ens = workloads.ensemble_2d(n_fields, seed=0)
    shapes = [p.shape for p, _ in ens]
    cells = sum(int(np.prod(s)) for s in shapes)
    cat = lambda arrs, dt: torch.tensor(np.concatenate([x.ravel() for x in arrs]), dtype=dt, device=dev)
    psi = cat([p for p, _ in ens], torch.float32)
    gc = [cat([g[d] for _, g in ens], torch.float32) for d in range(2)]
    with Mpdata(shapes, dtype=torch.float32, n_iters=2, opts=capi.FCT, device=dev) as m:
        from paper_1407_1309_gb300 import autotune
        # lane width and tile height of the persistent kernel for this ensemble (not cached)
        choice, _, _ = autotune.autotune(m, psi, gc, steps=8, use_cache=False, flush_bytes=0)
        src, out = psi.clone(), torch.empty_like(psi)
        graph = m.capture(src, out, gc, steps)
        graph.replay()
        torch.cuda.synchronize(dev)
        e0, e1 = _events()
        e0.record()
        graph.replay()
        e1.record()
        torch.cuda.synchronize(dev)
        secs = e0.elapsed_time(e1) / 1e3
        short = torch.empty_like(psi)
        m.advance(psi, short, gc, n_steps=fp64_steps)
        torch.cuda.synchronize(dev)
        short = short.double().cpu().numpy()
    # plain per-field FP64 GPU path: one handle and one launch sequence per field
    handles, ins, outs, gcs = [], [], [], []
    for p, g in ens:
        handles.append(Mpdata(p.shape, dtype=torch.float64, n_iters=2, opts=capi.FCT, device=dev))
        ins.append(torch.tensor(p, device=dev))
        outs.append(torch.empty(p.shape, dtype=torch.float64, device=dev))
        gcs.append([torch.tensor(v, device=dev) for v in g])
    e0, e1 = _events()
    e0.record()
    for h, a, b, g in zip(handles, ins, outs, gcs):
        h.advance(a, b, g, n_steps=fp64_steps)
    e1.record()
    torch.cuda.synchronize(dev)
    secs64 = e0.elapsed_time(e1) / 1e3
    ref = np.concatenate([b.cpu().numpy().ravel() for b in outs])
    for h in handles:
        h.close()
    return {"workload": f"ensemble_{n_fields}_fields_64..512_fct_n_iters2_f32", "fields": n_fields,
            "cells_per_step": cells, "steps": steps, "value": round(cells * steps / secs / 1e9, 3), "unit": UNIT,
            "path": "one persistent fused launch per step, 500-step loop captured in one CUDA graph",
            "kernel": {"lanes_columns": 2 if choice[0] == 3 else 4, "tile_rows": choice[1], "chosen_by": "autotuner"},
            "roofline": {"bound": "hbm", "achieved": round(16 * cells * steps / secs / 1e9, 1),
                         "peak": measured_peaks()[0]["hbm_gbs"], "unit": "GB/s",
                         "frac": round(16 * cells * steps / secs / 1e9 / measured_peaks()[0]["hbm_gbs"], 4),
                         "algorithmic_bytes_per_cell_step": 16},
            "per_field_fp64_value": round(cells * fp64_steps / secs64 / 1e9, 3),
            "err_fp32_batched_vs_fp64_per_field": {
                "steps": fp64_steps, "rel_l2": float(np.linalg.norm(short - ref) / np.linalg.norm(ref)),
                "rel_mass_drift": float(abs(short.sum() - ref.sum()) / np.abs(ref).sum())}}


def bench_config5(dev, n=512, steps=200, every=20, n_dirs=64):
    """Adjoint: 512^2, FCT, two passes; time of one adjoint step vs one forward step (FP32),
    the checkpointed backward of a 200-step rollout vs its forward, and the FP64 FD check."""
    import numpy as np
    import torch

    from paper_1407_1309_gb300 import capi, workloads
    from paper_1407_1309_gb300 import autograd
    from paper_1407_1309_gb300.autograd import rollout
    from paper_1407_1309_gb300.solver import Mpdata
    psi0, gc_np, pert = workloads.adjoint_2d(n)
    res = {"workload": f"adjoint_{n}^2_fct_n_iters2_{steps}_steps_checkpoint_{every}"}
    for dt in (torch.float32, torch.float64):
        t = lambda x: torch.tensor(x, dtype=dt, device=dev)
        with Mpdata((n, n), dtype=dt, n_iters=2, opts=capi.FCT, device=dev) as m:
            a, b, g = t(psi0), torch.empty(n, n, dtype=dt, device=dev), [t(v) for v in gc_np]
            pb, gb = torch.ones_like(a), [torch.zeros_like(a), torch.zeros_like(a)]
            tape = torch.empty(m.tape_numel(), dtype=dt, device=dev)
            for _ in range(3):
                m.advance(a, b, g)
                m.adjoint_step(a, g, pb, gc_bar=gb)
                m.adjoint_record(a, g, tape, psi_next=b)
                m.adjoint_replay(a, g, tape, pb, gc_bar=gb)
            e0, e1 = _events()
            e2 = torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(50):
                m.advance(a, b, g)
            e1.record()
            for _ in range(50):
                m.adjoint_step(a, g, pb, gc_bar=gb)
            e2.record()
            # the split reverse step of the taped rollout backward: tape + result, then the sweep
            e3, e4 = _events()
            for _ in range(50):
                m.adjoint_record(a, g, tape, psi_next=b)
            e3.record()
            for _ in range(50):
                m.adjoint_replay(a, g, tape, pb, gc_bar=gb)
            e4.record()
            torch.cuda.synchronize(dev)
            fwd, adj = e0.elapsed_time(e1) / 50, e1.elapsed_time(e2) / 50
            rec, rep = e2.elapsed_time(e3) / 50, e3.elapsed_time(e4) / 50
            # whole rollout: forward vs backward (recompute + adjoint)
            p0 = t(psi0).requires_grad_(True)
            gg = [v.clone().requires_grad_(True) for v in g]
            with torch.no_grad():
                target = rollout(m, t(psi0 + 0.05 * pert), g, steps, every)
            # untimed warm-up rollout: captures the backward segment graphs once
            warm = rollout(m, p0, gg, steps, every)
            (0.5 * ((warm.double() - target.double()) ** 2).sum()).backward()
            p0.grad = None
            for x in gg:
                x.grad = None
            torch.cuda.synchronize(dev)
            fw, bw = [], []
            for trial in range(3):  # wall-clock medians of three rollouts (forward, then backward)
                if trial:
                    p0.grad = None
                    for x in gg:
                        x.grad = None
                tf0 = time.perf_counter()
                outT = rollout(m, p0, gg, steps, every)
                torch.cuda.synchronize(dev)
                tf1 = time.perf_counter()
                loss = 0.5 * ((outT.double() - target.double()) ** 2).sum()
                loss.backward()
                torch.cuda.synchronize(dev)
                tb1 = time.perf_counter()
                fw.append(tf1 - tf0)
                bw.append(tb1 - tf1)
            tf0, tf1, tb1 = 0.0, statistics.median(fw), statistics.median(fw) + statistics.median(bw)
            key = "f32" if dt == torch.float32 else "f64"
            res[key] = {"forward_step_ms": round(fwd, 4), "adjoint_step_ms": round(adj, 4),
                        "adjoint_over_forward_step": round(adj / fwd, 2),
                        "record_step_ms": round(rec, 4), "replay_step_ms": round(rep, 4),
                        "backward_records_tapes": autograd._tapes_fit(m, every, a),
                        "rollout_forward_ms": round((tf1 - tf0) * 1e3, 2),
                        "rollout_backward_ms": round((tb1 - tf1) * 1e3, 2),
                        "backward_over_forward": round((tb1 - tf1) / (tf1 - tf0), 2)}
            if dt == torch.float64 and n_dirs > 0:
                rng = np.random.default_rng(1)
                errs = []
                for _ in range(n_dirs):
                    d = [workloads.low_modes(rng, (n, n), 4) for _ in range(3)]
                    d = [x / np.sqrt(np.mean(x ** 2)) for x in d]
                    dp, dg = t(d[0]), [t(d[1]) * 0.05, t(d[2]) * 0.05]
                    eps = 1e-7
                    with torch.no_grad():
                        lp = 0.5 * ((rollout(m, p0 + eps * dp, [x + eps * y for x, y in zip(g, dg)], steps, every)
                                     - target) ** 2).sum()
                        lm = 0.5 * ((rollout(m, p0 - eps * dp, [x - eps * y for x, y in zip(g, dg)], steps, every)
                                     - target) ** 2).sum()
                    fd = float((lp - lm) / (2 * eps))
                    an = float((p0.grad * dp).sum() + sum((x.grad * y).sum() for x, y in zip(gg, dg)))
                    errs.append(abs(fd - an) / abs(fd))
                res["fd_check_f64"] = {"directions": n_dirs, "eps": 1e-7, "max_rel_err": max(errs),
                                       "note": "FCT is piecewise smooth; eps = 1e-3 crosses limiter switches"}
    return res


def run_ensemble(args):
    """Ensemble workload as the headline: 512 fields (sides 64..512), FCT, two passes, FP32;
    under torchrun each rank advances its share of the fields (partition_fields), no collective
    on the data path; every timed step is one persistent launch, L2 flushed before it."""
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_1407_1309_gb300 import capi, workloads
    from paper_1407_1309_gb300.solver import Mpdata
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=dev)
    ens = workloads.ensemble_2d(512, seed=0)
    sizes = [int(np.prod(p.shape)) for p, _ in ens]
    mine = partition_fields(sizes, ws)[rank]
    fields = [ens[f] for f in mine]
    shapes = [p.shape for p, _ in fields]
    cells = sum(sizes[f] for f in mine)
    cat = lambda arrs: torch.tensor(np.concatenate([x.ravel() for x in arrs]), dtype=torch.float32, device=dev)
    a = cat([p for p, _ in fields])
    b = torch.empty_like(a)
    gc = [cat([g[d] for _, g in fields]) for d in range(2)]
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    with Mpdata(shapes, dtype=torch.float32, n_iters=2, opts=capi.FCT, device=dev) as m:
        for _ in range(args.warmup):
            m.advance(a, b, gc)
            a, b = b, a
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)
        clocks = ClockSampler(local)
        clocks.start()
        evs = []
        for _ in range(args.steps):
            flush.zero_()
            e0, e1 = _events()
            e0.record(stream)
            m.advance(a, b, gc)
            e1.record(stream)
            evs.append((e0, e1))
            a, b = b, a
        torch.cuda.synchronize(dev)
        clk = clocks.stop()
        secs = sum(e0.elapsed_time(e1) for e0, e1 in evs) / 1e3
    # every rank reports its total cells; the job value is their sum over the slowest time
    secs = max_over_ranks(secs, dev)
    total = cells
    if ws > 1:
        t = torch.tensor([float(cells)], dtype=torch.float64, device=dev)
        dist.all_reduce(t)
        total = float(t.item())
        dist.barrier()
        dist.destroy_process_group()
    value = total * args.steps / secs / 1e9
    peaks, how = measured_peaks()
    achieved = 16 * total / ws * args.steps / secs / 1e9
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(secs / args.steps * 1e3, 5), "higher_is_better": True,
            "scaling": "weak" if ws == 1 else "strong", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded ensemble workload, no dataset)",
            "config": {"workload": "ensemble_512_fields_64..512_fct_n_iters2", "fields_per_rank": len(mine),
                       "l2": "flushed (256 MiB write) before every timed step", "parallelism": f"fields{ws}"},
            "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peaks["hbm_gbs"], "unit": "GB/s",
                         "frac": round(achieved / peaks["hbm_gbs"], 4), "traffic": None,
                         "algorithmic_bytes_per_cell_step": 16, "kernel": "k_fused2d_batched"},
            "gpu_launches": args.steps, "clocks": clk}), flush=True)


def run_e2e(m, psi_np, gc_np, dtype, dev, stream, K, ws, comp=False):
    """Same metric through the public API with host buffers: every step copies its inputs
    (psi -- hi and lo for the compensated state --, gc0, gc1) from pinned host memory and reads
    its result (psi, or hi and lo) back into pinned host memory.  The copies of neighbouring
    steps overlap the step in between: host-to-device copies, steps and device-to-host copies
    run on three streams over two buffer sets, ordered by events (a buffer set is refilled only
    after the step and the read-back that used it two steps earlier have finished)."""
    import torch
    if comp:
        hi_np, lo_np = _split(psi_np)
        hstate = [torch.tensor(hi_np).pin_memory(), torch.tensor(lo_np).pin_memory()]
    else:
        hstate = [torch.tensor(psi_np, dtype=dtype).pin_memory()]
    hg = [torch.tensor(v, dtype=dtype).pin_memory() for v in gc_np]
    ho = [[torch.empty_like(h).pin_memory() for h in hstate] for _ in range(2)]
    dp = [[torch.empty(h.shape, dtype=h.dtype, device=dev) for h in hstate] for _ in range(2)]
    dq = [[torch.empty_like(x) for x in dp[0]] for _ in range(2)]
    dg = [[torch.empty(v.shape, dtype=dtype, device=dev) for v in hg] for _ in range(2)]
    s_in, s_out = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    ev = lambda: torch.cuda.Event()
    copied, stepped, read = [ev(), ev()], [ev(), ev()], [ev(), ev()]
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s_in)
    stream.wait_stream(s_in)
    s_out.wait_stream(s_in)
    for k in range(K):
        b = k % 2
        with torch.cuda.stream(s_in):
            if k >= 2:
                s_in.wait_event(stepped[b])     # step k-2 no longer reads dp[b], dg[b]
            for d, h in zip(dp[b], hstate):
                d.copy_(h, non_blocking=True)
            for d, h in zip(dg[b], hg):
                d.copy_(h, non_blocking=True)
            copied[b].record(s_in)
        stream.wait_event(copied[b])
        if k >= 2:
            stream.wait_event(read[b])          # read-back k-2 no longer reads dq[b]
        if comp:
            m.advance_compensated(dp[b][0], dp[b][1], dq[b][0], dq[b][1], dg[b])
        else:
            m.advance(dp[b][0], dq[b][0], dg[b])
        stepped[b].record(stream)
        with torch.cuda.stream(s_out):
            s_out.wait_event(stepped[b])
            for h, d in zip(ho[b], dq[b]):
                h.copy_(d, non_blocking=True)
            read[b].record(s_out)
    s_out.wait_stream(stream)
    s_out.wait_stream(s_in)
    e1.record(s_out)
    torch.cuda.synchronize(dev)
    secs = e0.elapsed_time(e1) / 1e3
    cells = hstate[0].numel()
    state_bytes = sum(h.numel() * h.element_size() for h in hstate)
    gc_bytes = sum(h.numel() * h.element_size() for h in hg)
    return {"value": round(cells * K * ws / secs / 1e9, 4), "unit": UNIT, "steps": K,
            "h2d_bytes_per_step": state_bytes + gc_bytes, "d2h_bytes_per_step": state_bytes,
            "overlap": "copies of neighbouring steps overlap the step (3 streams, 2 buffer sets)"}


def cpu_baseline(psi_np, gc_np, budget_s=12.0, gpu_steps=None):
    """The oracle as it stands on this host's cores, on a bounded sample of the workload.
    With gpu_steps (k -> this build's result after k steps from the same input), the oracle's
    timed result is also the reference of the GPU run's error."""
    import numpy as np

    import oracle
    cores = oracle.set_threads(0)
    t0 = time.perf_counter()
    oracle.step(psi_np, gc_np, n_iters=2, opts=oracle.FCT, n_steps=1)
    one = time.perf_counter() - t0
    k = max(1, min(40, int(budget_s / max(one, 1e-3))))
    t0 = time.perf_counter()
    ref = oracle.step(psi_np, gc_np, n_iters=2, opts=oracle.FCT, n_steps=k)
    secs = time.perf_counter() - t0
    err = None
    if gpu_steps is not None:
        got = gpu_steps(k)
        err = {"steps": k, "rel_l2": float(np.linalg.norm(got - ref) / np.linalg.norm(ref)),
               "max_rel": float(np.abs(got - ref).max() / np.abs(ref).max())}
    cells = psi_np.size
    # the same oracle on one thread (the plain sweep), on a smaller bounded sample
    oracle.set_threads(1)
    try:
        t0 = time.perf_counter()
        oracle.step(psi_np, gc_np, n_iters=2, opts=oracle.FCT, n_steps=1)
        one1 = time.perf_counter() - t0
        k1 = max(1, min(10, int(budget_s / 3 / max(one1, 1e-3))))
        t0 = time.perf_counter()
        oracle.step(psi_np, gc_np, n_iters=2, opts=oracle.FCT, n_steps=k1)
        secs1 = time.perf_counter() - t0
    finally:
        oracle.set_threads(0)
    return {"value": round(cells * k / secs / 1e9, 6), "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{k} steps of the full {psi_np.shape[0]}x{psi_np.shape[1]} workload, FP64, OpenMP over rows",
            "single_thread": {"value": round(cells * k1 / secs1 / 1e9, 6), "unit": UNIT, "cores": 1,
                              "sample": f"{k1} steps of the same workload, one thread"},
            "gpu_fp32_err_vs_this_run": err}


# ----------------------------------------------------------------------------------- reference arm

def run_reference(args):
    """The oracle (plain FP64 CPU MPDATA) on the host cores, on the same workload as this build's
    arm: each timed step advances the full rotation field by one MPDATA step (FCT, two passes)."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    from paper_1407_1309_gb300 import workloads
    psi, gc, _ = workloads.rotation_2d(args.n, REV_STEPS if args.n == N_SIDE else None)
    cores = oracle.set_threads(0)
    for _ in range(args.warmup):
        psi = oracle.step(psi, gc, n_iters=2, opts=oracle.FCT)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        psi = oracle.step(psi, gc, n_iters=2, opts=oracle.FCT)
    secs = time.perf_counter() - t0
    value = psi.size * args.steps / secs / 1e9
    sample = (f"one MPDATA step of the full {args.n}x{args.n} rotation workload per timed step "
              f"(FP64, OpenMP over rows)")
    out = {"impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": UNIT, "n_gpus": ws,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(secs / args.steps * 1e3, 4),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic (seeded rotating-cone workload, no dataset)",
           "config": config(args, {"same_config": True, "l2": "not applicable (the oracle runs on the host cores)"}),
           "cpu_baseline": {"kind": "oracle", "cores": cores, "sample": sample, "value": round(value, 6), "unit": UNIT},
           "e2e": {"value": round(value, 6), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_deform3d(args, n=256):
    """The 3D configuration on its own: every step timed with CUDA events (the five input
    arrays, 335 MB in FP32, exceed the L2, so no flush is needed), one JSON line."""
    import torch
    import torch.distributed as dist

    from paper_1407_1309_gb300 import capi, workloads
    from paper_1407_1309_gb300.solver import Mpdata
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=dev)
    dtype = torch.float32 if args.dtype == "f32" else torch.float64
    psi, gc, G = workloads.deformational_3d(n)
    t = lambda x: torch.tensor(x, dtype=dtype, device=dev)
    K = args.warmup + args.steps
    scales = [workloads.deformational_scale(s) for s in range(K)]
    opts = capi.TOT | capi.FCT | capi.NUG
    with Mpdata((n, n, n), dtype=dtype, n_iters=3, opts=opts, device=dev) as m:
        a, b, g, Gt = t(psi), torch.empty(n, n, n, dtype=dtype, device=dev), [t(v) for v in gc], t(G)
        for s in range(args.warmup):
            m.advance(a, b, g, Gt, None, 0.0, 1, scales[s:s + 1])
            a, b = b, a
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)
        clocks = ClockSampler(local)
        clocks.start()
        evs = []
        for s in range(args.warmup, K):
            e0, e1 = _events()
            e0.record()
            m.advance(a, b, g, Gt, None, 0.0, 1, scales[s:s + 1])
            e1.record()
            evs.append((e0, e1))
            a, b = b, a
        torch.cuda.synchronize(dev)
        clk = clocks.stop()
    secs = max_over_ranks(sum(e0.elapsed_time(e1) for e0, e1 in evs) / 1e3, dev)
    peaks, how = measured_peaks()
    cells = n ** 3
    esize = 4 if dtype == torch.float32 else 8
    bpc = 6 * esize  # psi, gc0..2, G read; psi written
    achieved = bpc * cells * args.steps / secs / 1e9
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": round(job_value(cells, args.steps, ws, secs), 3), "unit": UNIT,
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(secs / args.steps * 1e3, 4), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": args.dtype, "data": "synthetic (seeded deformational flow, no dataset)",
            "config": {"workload": f"3d_deformational_{n}^3_n_iters3_tot_fct_G", "grid": [n, n, n],
                       "l2": "inputs larger than L2 (no flush)", "parallelism": f"replicas{ws}",
                       "path": "z-march kernels: pass 1 + bounds, then per corrective pass the pseudo-advector "
                               "and the limited donor pass"},
            "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peaks["hbm_gbs"], "unit": "GB/s",
                         "frac": round(achieved / peaks["hbm_gbs"], 4), "traffic": None,
                         "algorithmic_bytes_per_cell_step": bpc},
            "gpu_launches": (5 if dtype == torch.float32 else 10) * args.steps, "clocks": clk}), flush=True)
    if ws > 1:
        dist.barrier()
        dist.destroy_process_group()


def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "ensemble":
        run_ensemble(args)
    elif args.workload == "deform3d":
        run_deform3d(args, args.n3d)
    elif args.workload == "adjoint":
        import torch
        res = bench_config5(torch.device("cuda", 0), n_dirs=0 if args.no_extras else 64)
        print(json.dumps({"metric": "adjoint rollout backward / forward (512^2, fct, n_iters 2, 200 steps)",
                          "value": res["f64"]["backward_over_forward"], "unit": "x (FP64)",
                          "higher_is_better": False, "data": "synthetic", **res}), flush=True)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
