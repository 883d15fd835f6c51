"""Benchmark: CCZ4 RK4 substeps on a 96^3 periodic patch (cell-updates/s).

One "step" is one full RK4 step (four fused RHS + stage-update launches)
of the conformal Z4 system (25 fields, 1+log slicing, Gamma-driver shift,
KO sigma = 0.1, dt = 0.25 dx) on Minkowski data plus seeded uniform noise
of amplitude 1e-10.  The headline value is the FP32-bulk path; the plain
FP64 path is timed on the same data and reported beside it.

Metric: cell-updates per second per RK substep = 96^3 * 4 * steps / time.
Every array of the working set (5 ghosted arrays of 25 x 102^3 values) is
larger than the 129 MB L2, so no flush is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun each rank advances its own independent 96^3 patch (weak
scaling, no collective on the data path); rank 0 prints one JSON line with
the max time over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import threading
import time

import numpy as np

N = 96
GHOST = 3
NF = 25
WORKLOAD = "ccz4_96cubed_rk4_periodic"
# Algorithmic operations of one CCZ4 cell-update (right-hand side of the
# plain formulation, counted by instantiating the oracle's per-cell function
# on a counting scalar: 3680 add + 3970 mul + 164 div + 1 log; the RK
# combination adds two or three per field and is left out), and the ALU
# peaks they are set against: FP32 from the unit counts and the maximum SM
# clock, FP64 as measured with an FMA probe on this GPU.
FLOPS_PER_CELL_UPDATE = 3680 + 3970 + 164 + 1
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
FP64_PEAK_TFLOPS = 1.20
# Row pitch of the float arrays: 104 floats (416 bytes) puts every row, plane
# and field on a 16-byte boundary, which the TMA-staged CCZ4 kernel needs;
# FP64 keeps the dense pitch (its kernel reads stencils from global memory).
FLOAT_PITCH = 104
METRIC = "cell-updates/s per RK substep (Z4 96^3, FP32-bulk; FP64 beside it)"
UNIT = "cell-updates/s"
ROOT = os.path.dirname(os.path.abspath(__file__))


def bytes_per_cell_update(precision: str) -> float:
    """Algorithmic HBM bytes per interior cell and RK substep, as the kernels
    move them (every array pass of one RK4 step, divided by its four
    substeps).  FP64: stage 0 reads U^n and writes acc, U(2) (3 passes);
    stages 1-2 read U(i), U^n, acc and write acc, U(i+1) (5 each); stage 3
    reads U(4), acc and writes U^{n+1} (3): 16 passes.  FP32-bulk adds the
    Kahan array (read and written once per step) and one read of U^n in
    stage 3, since its accumulator holds the increment alone and the
    compensated sum adds it to U^n there: 19 passes."""
    if precision == "fp64":
        return 16 / 4 * NF * 8
    return 19 / 4 * NF * 4


def contract_bytes_per_cell_update(precision: str) -> float:
    """The measurement contract's algorithmic bytes: FP64 4 nf s = 800 B;
    FP32-bulk (16 + 2) / 4 nf s = 450 B (the 16 RK4 passes plus the Kahan
    array's read and write; it does not count the U^n read of stage 3)."""
    if precision == "fp64":
        return 4 * NF * 8
    return (16 + 2) / 4 * NF * 4


STAGE_PASSES = {"fp64": [3, 5, 5, 3], "fp32": [3, 5, 5, 6], "fp32dw": [3, 5, 5, 6]}


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines: list[str] = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()
        time.sleep(0.3)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=5)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


class NvmlSampler:
    """Read-only NVML samples (SM clock, clock-event reasons) every ~2 ms
    between mark_start() and mark_stop(): the timed region of the headline is
    tens of milliseconds, shorter than nvidia-smi's sampling interval.  Loads
    libnvidia-ml through ctypes; without it (no driver) it reports nothing."""

    # nvmlClocksEventReasons bits
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}

    def __init__(self, index: int, period_s: float = 0.002):
        import ctypes
        self.period = period_s
        self.samples: list[tuple[float, int, int]] = []
        self.max_mhz = None
        self.lib = None
        self.window = [None, None]
        self._stop = threading.Event()
        self.thread = None
        try:
            lib = ctypes.CDLL("libnvidia-ml.so.1")
            if lib.nvmlInit_v2() != 0:
                return
            h = ctypes.c_void_p()
            if lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(index), ctypes.byref(h)) != 0:
                return
            self.h = h
            self.reasons_fn = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
                lib.nvmlDeviceGetCurrentClocksThrottleReasons
            m = ctypes.c_uint()
            if lib.nvmlDeviceGetMaxClockInfo(h, ctypes.c_int(1), ctypes.byref(m)) == 0:
                self.max_mhz = m.value
            self.lib = lib
        except (OSError, AttributeError):
            self.lib = None

    def _poll(self):
        import ctypes
        mhz, rs = ctypes.c_uint(), ctypes.c_ulonglong()
        while not self._stop.is_set():
            t = time.perf_counter()
            if (self.lib.nvmlDeviceGetClockInfo(self.h, ctypes.c_int(1), ctypes.byref(mhz)) == 0 and
                    self.reasons_fn(self.h, ctypes.byref(rs)) == 0):
                self.samples.append((t, mhz.value, rs.value))
            time.sleep(self.period)

    def start(self):
        if self.lib is not None:
            self.thread = threading.Thread(target=self._poll, daemon=True)
            self.thread.start()

    def mark_start(self):
        self.window[0] = time.perf_counter()

    def mark_stop(self):
        self.window[1] = time.perf_counter()

    def stop(self) -> dict | None:
        if self.lib is None:
            return None
        self._stop.set()
        self.thread.join(timeout=5)
        return self.summary(self.samples, self.window, self.max_mhz)

    @classmethod
    def summary(cls, samples, window, max_mhz) -> dict:
        """Samples taken inside [window[0], window[1]]: median SM clock and the
        reasons active in any of them."""
        lo, hi = window
        inside = [s for s in samples if lo is not None and hi is not None and lo <= s[0] <= hi]
        reasons = sorted({nm for _, _, r in inside for bit, nm in cls.REASONS.items() if r & bit})
        return {"source": "NVML, ~2 ms polling, host-clock window from the first timed launch to "
                          "the synchronize after the last",
                "samples_in_timed_region": len(inside),
                "sm_mhz": statistics.median([m for _, m, _ in inside]) if inside else None,
                "sm_mhz_min": min([m for _, m, _ in inside]) if inside else None,
                "sm_max_mhz": max_mhz, "reasons": reasons}


# ---------------------------------------------------------------- traffic
# DRAM traffic and the instruction count of the headline kernel come from one
# ncu capture, recorded in a JSON file beside its summary under profiles/;
# they are reported only while the kernel sources still hash to the value
# recorded there (null once the kernel has changed).
PROFILE = os.path.join(ROOT, "profiles", "z4_pair_fp32dw_96cubed.json")
KERNEL_SOURCES = ["sf_common.cuh", "sf_dw.cuh", "sf_f2.cuh", "sf_mbar.cuh", "sf_pair.cuh", "sf_z4.cuh",
                  "sf_z4.cu", "sf_z4_pair.cu"]


def kernel_source_hash() -> str:
    """Hash of the headline kernel's sources with // comments, trailing blanks
    and empty lines removed, so that comment edits keep the profiled counters."""
    import hashlib
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1806_04182_gb300", "csrc", name)) as f:
            for line in f:
                code = line.split("//", 1)[0].rstrip()
                if code:
                    h.update(code.encode() + b"\n")
    return h.hexdigest()[:16]


def profiled_traffic():
    """(bytes per launch, source hash) from the profile record, or (None, None)."""
    v = profiled_values()
    return v.get("traffic_bytes_per_launch"), v.get("kernel_source_sha256_16")


def profiled_values() -> dict:
    """The ncu figures of the headline kernel (profiles/*.json), or {}."""
    if not os.path.exists(PROFILE):
        return {}
    with open(PROFILE) as f:
        return json.load(f)


# ---------------------------------------------------------------- ranks
def max_over_ranks(v: float, device=None) -> float:
    """Max of v over the ranks of the default process group (v itself if none)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return v
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world: int, cells: int, substeps: int, max_ms: float) -> float:
    """Cell-updates/s of the whole job: every rank advances its own patch."""
    return world * cells * substeps / (max_ms * 1e-3)


# ---------------------------------------------------------------- GPU arm
def make_state(precision: str, seed: int, device, float_pitch: int = FLOAT_PITCH,
               x_offset: int = 1):
    import torch
    from paper_1806_04182_gb300 import capi, inputs
    from paper_1806_04182_gb300.state import PatchState
    U0, dx = inputs.z4_minkowski_noise((N, N, N), seed=seed, amp=1e-10)
    prec = {"fp64": capi.SF_FP64, "fp32": capi.SF_FP32_BULK,
            "fp32dw": capi.SF_FP32_BULK_DW}[precision]
    st = PatchState(capi.SF_Z4, (N, N, N), dx, 0.25 * dx[0], precision=prec,
                    prm=capi.params(), device=device,
                    x_pitch=None if precision == "fp64" else float_pitch,
                    x_offset=0 if precision == "fp64" else x_offset)
    st.upload(U0)
    torch.cuda.synchronize()
    return st


def time_device(st, steps: int, warmup: int, marks=None):
    """Per-launch CUDA-event durations (ms) of `steps` RK4 steps after warm-up
    (`marks`: mark_start() / mark_stop() around the timed region)."""
    import torch
    from paper_1806_04182_gb300 import capi
    stream = torch.cuda.current_stream()
    h = stream.cuda_stream
    patches = [st.stage_patch(s) for s in range(4)]
    for _ in range(warmup):
        for s in range(4):
            capi.sf_substep(st.prm, patches[s], s, h)
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4 * steps + 1)]
    c0 = capi.sf_launch_count()
    if marks:
        marks.mark_start()
    ev[0].record(stream)
    for k in range(steps):
        for s in range(4):
            capi.sf_substep(st.prm, patches[s], s, h)
            ev[4 * k + s + 1].record(stream)
    torch.cuda.synchronize()
    if marks:
        marks.mark_stop()
    launches = capi.sf_launch_count() - c0
    per = np.array([ev[q].elapsed_time(ev[q + 1]) for q in range(4 * steps)]).reshape(steps, 4)
    total = ev[0].elapsed_time(ev[-1])
    return total, per, launches


def time_e2e(st, steps: int, warmup: int, chained: bool):
    """The same steps through host buffers, by the C-ABI call sf_step_host
    (state.HostPipeline): every step uploads its input state from pinned
    host memory, runs the four stages and downloads U^{n+1}.  The chained
    evolution moves interior host images (SF_HOST_INTERIOR: 18% fewer bytes
    over the host link, whose copies are serial with its stages; the
    periodic ghost shell is rebuilt on the device); the independent states
    move full state images (their copies hide behind the stages, and the
    device-side spreading and gathering of interior images would lengthen
    the stage stream).
    chained: one evolution kept in host memory (each step's input is the
    previous step's output, one pinned buffer updated in place, one device
    slot whose Kahan compensation carries over): the copies and the stages
    of a step are serial.  Otherwise: independent states (the same input
    every step, outputs alternating between two pinned buffers), three
    device slots, the copies of other steps overlapping the stages on copy
    streams of their own.  The timed region spans all three streams."""
    import torch
    from paper_1806_04182_gb300.state import HostPipeline
    pipe = HostPipeline(st.system, st.n, st.dx, st.dt, precision=st.precision, prm=st.prm,
                        ghost=st.g, x_pitch=st.pitch, x_offset=st.xo, slots=1 if chained else 3,
                        interior=chained)
    host_in = pipe.host_buffer()
    host_in.copy_(pipe.image(st.A).cpu())
    if chained:
        ins, outs = [host_in] * steps, [host_in] * steps
        wins, wouts = [host_in] * warmup, [host_in] * warmup
    else:
        o = [pipe.host_buffer(), pipe.host_buffer()]
        ins, outs = [host_in] * steps, [o[k % 2] for k in range(steps)]
        wins, wouts = [host_in] * warmup, [o[k % 2] for k in range(warmup)]
    pipe.run(wins, wouts, reset_kahan=not chained)
    pipe.synchronize()
    torch.cuda.synchronize()
    cur = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(cur)
    pipe.start(cur)
    pipe.run(ins, outs, reset_kahan=not chained)
    pipe.join(cur)
    e1.record(cur)
    torch.cuda.synchronize()
    nbytes = host_in.numel() * host_in.element_size()
    del pipe
    return e0.elapsed_time(e1), nbytes, nbytes


def gpu_arm(args):
    import torch
    import torch.distributed as dist
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    from paper_1806_04182_gb300 import build as sfbuild
    sfbuild.build()
    peaks = {}
    pk = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk):
        peaks = json.load(open(pk))
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    cells = N ** 3
    res = {}
    clocks = None
    precisions = ("fp32dw", "fp32", "fp64") if args.only is None else (args.only,)
    for precision in precisions:
        # native FP64 islands run best on the one-point TMA kernel (no row
        # offset): their FP64 arithmetic needs the 12 warps' latency hiding
        xo = 0 if precision == "fp32" else args.x_offset
        st = make_state(precision, seed=rank, device=device, float_pitch=args.pitch, x_offset=xo)
        barrier()
        sampler = ClockSampler(local) if precision == "fp32dw" else None
        nvml = NvmlSampler(local) if precision == "fp32dw" else None
        if sampler:
            sampler.start()
            nvml.start()
        total_ms, per, launches = time_device(st, args.steps, args.warmup, marks=nvml)
        if sampler:
            fine = nvml.stop()
            clocks = sampler.stop()
            if fine is not None:
                clocks["timed_region_nvml"] = fine
        barrier()
        total_ms = max_over_ranks(total_ms, device)
        substeps = 4 * args.steps
        value = whole_job_rate(world, cells, substeps, total_ms)
        # dominant kernel: the stage kernel; average launch duration
        avg_launch_ms = float(per.mean())
        bpc = bytes_per_cell_update(precision)
        achieved = cells * bpc / (avg_launch_ms * 1e-3) / 1e9
        bpc_c = contract_bytes_per_cell_update(precision)
        achieved_c = cells * bpc_c / (avg_launch_ms * 1e-3) / 1e9
        per_stage_ms = per.mean(axis=0).tolist()
        stage_gbs = [cells * p * NF * (8 if precision == "fp64" else 4) / (ms * 1e-3) / 1e9
                     for p, ms in zip(STAGE_PASSES[precision], per_stage_ms)]
        res[precision] = dict(value=value, ms_per_step=total_ms / args.steps, launches=launches,
                              avg_launch_ms=avg_launch_ms, achieved_gbs=achieved_c,
                              achieved_gbs_kernel_passes=achieved, contract_bytes=bpc_c,
                              per_stage_ms=per_stage_ms, per_stage_gbs=stage_gbs,
                              bytes_per_cell_update=bpc, state=st)
    if args.only is not None:
        if world > 1:
            dist.destroy_process_group()
        r = res[args.only]
        return None if rank else {"profiling_run": args.only, "value": r["value"],
                                  "ms_per_step": r["ms_per_step"], "achieved_gbs": r["achieved_gbs"]}
    # end to end through host buffers (FP32-bulk, double-word islands)
    st = res["fp32dw"]["state"]
    barrier()
    e2e_ms, bi, bo = time_e2e(st, args.steps, args.warmup, chained=True)
    barrier()
    ind_ms, ibi, ibo = time_e2e(st, args.steps, args.warmup, chained=False)
    barrier()
    e2e_ms = max_over_ranks(e2e_ms, device)
    ind_ms = max_over_ranks(ind_ms, device)
    e2e_value = whole_job_rate(world, cells, 4 * args.steps, e2e_ms)
    ind_value = whole_job_rate(world, cells, 4 * args.steps, ind_ms)
    if world > 1:
        dist.destroy_process_group()
    if rank != 0:
        return None
    r32, r32n, r64 = res["fp32dw"], res["fp32"], res["fp64"]
    traffic, traffic_src = profiled_traffic()
    line = {
        "metric": METRIC,
        "value": r32["value"],
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": r32["ms_per_step"],
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic: Minkowski + seeded uniform noise 1e-10 on all 25 fields",
        "config": {"workload": WORKLOAD, "n": N, "ghost": GHOST, "fields": NF, "rk": "RK4",
                   "substeps_per_step": 4,
                   "precision": "fp32_bulk: float storage and stencils, Kahan RK accumulation, "
                                "det/inverse/ln det/trace removals in double-word (FP64-class) "
                                "arithmetic on the FP32 pipe",
                   "slicing": "1+log", "shift": "Gamma-driver", "sigma_ko": 0.1,
                   "dt_over_dx": 0.25, "l2": "inputs larger than L2 (5 arrays x 106 MB fp32)",
                   "parallelism": f"replicas x{world}",
                   "forms": {
                       "fp32_bulk_dw": {"value": r32["value"], "precision":
                                        "float storage and stencils; det, inverse, ln det and trace "
                                        "removals in double-word floats (relative error a few 2^-48 "
                                        "per operation), Kahan RK accumulation (the headline)"},
                       "fp32_bulk_fp64_islands": {"value": r32n["value"], "precision":
                                                  "float storage and stencils; det, inverse, ln det "
                                                  "and trace removals in native FP64, Kahan RK "
                                                  "accumulation"},
                       "fp64": {"value": r64["value"], "precision": "FP64 throughout (the paper's precision)"}}},
        "roofline": {"bound": "hbm", "achieved": r32["achieved_gbs"], "peak": hbm_peak,
                     "unit": "GB/s", "frac": r32["achieved_gbs"] / hbm_peak,
                     "traffic": traffic if traffic_src == kernel_source_hash() else None,
                     "traffic_unit": "bytes per launch (ncu dram__bytes_read+write, mean of the 4 stages)",
                     "peak_source": peak_src,
                     "cells_per_launch": cells, "avg_launch_ms": r32["avg_launch_ms"],
                     "bytes_per_cell_update_kernel_passes": r32["bytes_per_cell_update"],
                     "achieved_kernel_passes": r32["achieved_gbs_kernel_passes"],
                     "frac_kernel_passes": r32["achieved_gbs_kernel_passes"] / hbm_peak,
                     "kernel": headline_kernel(args),
                     "bytes_per_cell_update": r32["contract_bytes"],
                     "per_stage_ms": r32["per_stage_ms"], "per_stage_gbs": r32["per_stage_gbs"]},
        "alu_roofline": {
            "bound": "alu", "flops_per_cell_update": FLOPS_PER_CELL_UPDATE,
            "achieved": r32["value"] * FLOPS_PER_CELL_UPDATE / 1e12, "unit": "TFLOP/s",
            "peak": FP32_PEAK_TFLOPS, "frac": r32["value"] * FLOPS_PER_CELL_UPDATE / 1e12 / FP32_PEAK_TFLOPS,
            "peak_source": "152 SMs x 128 FP32 lanes x 2 flops x 2.07 GHz",
            "fp64_frac": r64["value"] * FLOPS_PER_CELL_UPDATE / 1e12 / FP64_PEAK_TFLOPS,
            "fp64_peak": FP64_PEAK_TFLOPS,
            "fp64_peak_source": "measured FMA probe, 1/58 of the FP32 rate",
            "note": "flops counted on the oracle's plain formulation (unfused, symmetric sums "
                    "expanded); the kernels evaluate a factored form with fewer operations, so "
                    "the FP64 fraction can exceed 1 (ncu: FP64 pipe 86% busy)"},
        "issue_roofline": issue_roofline(r32, clocks),
        "fp32_bulk_fp64_islands": {
            "value": r32n["value"], "ms_per_step": r32n["ms_per_step"],
            "layout": "row pitch 104, no row offset: the one-point TMA kernel z4_tma_kernel<double,12,8>",
            "achieved_gbs": r32n["achieved_gbs"], "hbm_frac": r32n["achieved_gbs"] / hbm_peak,
            "per_stage_ms": r32n["per_stage_ms"]},
        "fp64": {"value": r64["value"], "ms_per_step": r64["ms_per_step"],
                 "achieved_gbs": r64["achieved_gbs"], "hbm_frac": r64["achieved_gbs"] / hbm_peak,
                 "bytes_per_cell_update": r64["contract_bytes"],
                 "per_stage_ms": r64["per_stage_ms"]},
        "speedup_fp32_bulk_over_fp64": r32["value"] / r64["value"],
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": bi,
                "d2h_bytes_per_step": bo,
                "path": "C-ABI sf_step_host (state.HostPipeline, interior host images): one evolution "
                        "kept in pinned host memory, every step uploads U^n's interior, rebuilds the "
                        "ghost shell on the device, runs the four stages and downloads U^{n+1}'s "
                        "interior into the buffer the next step uploads; copies in eight pieces, the "
                        "next upload beside the rest of the download, stages serial with the copies",
                "independent_states": {
                    "value": ind_value, "unit": UNIT, "h2d_bytes_per_step": ibi,
                    "d2h_bytes_per_step": ibo,
                    "path": "sf_step_host with three device slots and full state images: a new state "
                            "every step (same input), the copies of other steps overlapping the stages "
                            "on copy streams"}},
        "gpu_launches": int(r32["launches"]),
        "clocks": clocks,
    }
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(seconds=args.cpu_seconds)
    return line


def headline_kernel(args) -> str:
    if args.pitch % 4 == 0 and args.x_offset == 1:
        return "z4_pair_kernel<DW2,8,7> (two points per thread on f32x2, TMA-staged stencils)"
    if args.pitch % 4 == 0 and args.x_offset == 0:
        return "z4_tma_kernel<dw,12,8> (TMA-staged stencils)"
    return "z4_stage_kernel<float,dw> (global-load stencils)"


def issue_roofline(r32, clocks) -> dict | None:
    """The bound the float CCZ4 kernel actually meets: instruction issue.
    achieved = warp instructions per launch (ncu count of the same kernel
    source, from the profile summary) / mean CUDA-event stage time; peak = one
    warp instruction per cycle on each of the 4 schedulers of the 152 SMs at
    the median SM clock sampled during the timed region."""
    v = profiled_values()
    inst = v.get("warp_instructions_per_launch")
    if inst is None or v.get("kernel_source_sha256_16") != kernel_source_hash():
        return None
    mhz = clocks.get("sm_mhz") or 2070.0
    t = statistics.fmean(r32["per_stage_ms"]) * 1e-3
    peak = 152 * 4 * mhz * 1e6
    return {"bound": "issue", "warp_instructions_per_launch": inst, "achieved": inst / t,
            "peak": peak, "unit": "warp instructions/s", "frac": inst / t / peak,
            "peak_source": f"152 SMs x 4 schedulers x 1 instruction/cycle x {mhz:.0f} MHz "
                           "(median sampled SM clock)"}


# ---------------------------------------------------------------- other rows
def _events_time(fn, steps: int, warmup: int) -> float:
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def suite(args, hbm_peak: float) -> list[dict]:
    """The remaining workloads, each timed on the device with CUDA events."""
    import torch
    from paper_1806_04182_gb300 import adjoint, capi, inputs
    from paper_1806_04182_gb300.state import PatchState
    rows = set(args.rows.split(",")) if args.rows else {"wave", "mhd", "batch", "adjoint"}
    out = []
    # wave 64^3 FP64 and FP32, RK4, CFL 0.25
    for prec, name, bpc in (() if "wave" not in rows else ((capi.SF_FP64, "fp64", 16 / 4 * 5 * 8),
                            (capi.SF_FP32_BULK, "fp32", 19 / 4 * 5 * 4))):
        n = (64, 64, 64)
        U0, dx = inputs.wave_plane(n, seed=0)
        st = PatchState(capi.SF_WAVE, n, dx, 0.25 * dx[0], precision=prec)
        st.upload(U0)
        ms = _events_time(lambda: st.step(1), 20, 3)
        cells = 64 ** 3
        rate = cells * 4 * 20 / (ms * 1e-3)
        out.append({"workload": f"wave_64cubed_rk4_{name}", "value": rate, "unit": UNIT,
                    "ms_per_step": ms / 20, "bytes_per_cell_update": bpc,
                    "hbm_frac": rate * bpc / 1e9 / hbm_peak})
    if "mhd" in rows:
        out += _mhd_row(hbm_peak)
    if "batch" in rows or "batch_graph" in rows:
        out += _batch_rows(hbm_peak, npatch=args.npatch, per_patch="batch" in rows)
    if "adjoint" in rows:
        out += _adjoint_rows()
    if "variants" in rows:
        out += _variant_rows(hbm_peak)
    if "amr" in rows:
        out += _amr_rows(hbm_peak)
    if "puncture" in rows:
        out += _puncture_rows(hbm_peak)
    return out


def _puncture_rows(hbm_peak: float) -> list[dict]:
    """Second workload (Sec. V): a spinning, boosted puncture on a 96^3
    non-periodic box with radiative boundaries (interior stage kernel +
    radiative ghost-shell kernel per stage)."""
    import numpy as np
    from paper_1806_04182_gb300 import capi, inputs
    from paper_1806_04182_gb300.state import PatchState
    out = []
    n = (N, N, N)
    U, dx, x0 = inputs.z4_puncture(n, length=16.0, ghost=GHOST)
    speed = np.ones(NF)
    for prec, name, pitch in ((capi.SF_FP32_BULK_DW, "fp32dw", FLOAT_PITCH), (capi.SF_FP64, "fp64", None)):
        st = PatchState(capi.SF_Z4, n, dx, 0.25 * dx[0], precision=prec,
                        prm=capi.params(ghosts=capi.SF_GHOSTS_NONE), x_pitch=pitch)
        st.upload_ghosted(U)
        steps = 10 if prec != capi.SF_FP64 else 3
        ms = _events_time(lambda: st.step_radiative(1, x0, inputs.Z4_UINF, speed), steps, 2)
        rate = N ** 3 * 4 * steps / (ms * 1e-3)
        out.append({"workload": f"ccz4_puncture_96cubed_radiative_{name}", "value": rate, "unit": UNIT,
                    "ms_per_step": ms / steps, "hbm_frac": rate * (475 if prec != capi.SF_FP64 else 800)
                    / 1e9 / hbm_peak,
                    "note": "interior cells; 1+log slicing, Gamma-driver, radiative ghost shell"})
    return out


def _variant_rows(hbm_peak: float) -> list[dict]:
    """Reconstruction and advection variants: CCZ4 with one-sided advection,
    MHD with WENO5-Z and WENO3."""
    from paper_1806_04182_gb300 import capi, inputs
    from paper_1806_04182_gb300.state import PatchState
    out = []
    U0, dx = inputs.z4_minkowski_noise((N, N, N), seed=0, amp=1e-10)
    st = PatchState(capi.SF_Z4, (N, N, N), dx, 0.25 * dx[0], precision=capi.SF_FP32_BULK_DW,
                    prm=capi.params(lopsided=1))
    st.upload(U0)
    steps = 10
    ms = _events_time(lambda: st.step(1), steps, 3)
    rate = N ** 3 * 4 * steps / (ms * 1e-3)
    out.append({"workload": "ccz4_96cubed_rk4_fp32dw_lopsided_advection", "value": rate,
                "unit": UNIT, "ms_per_step": ms / steps, "bytes_per_cell_update": 475,
                "hbm_frac": rate * 475 / 1e9 / hbm_peak,
                "note": "one-sided advection stencils (runtime-stride global-load kernel)"})
    n = (128, 128, 128)
    U0, dx = inputs.mhd_blast(n, seed=0)
    for variant, split, name in ((1, 0, "weno5z"), (2, 0, "weno3"), (0, 1, "weno5_lf_split")):
        prm = capi.params(rk=capi.SF_SSPRK3, weno_variant=variant, flux_split=split)
        st = PatchState(capi.SF_MHD, n, dx, 1e-3, precision=capi.SF_FP64, prm=prm)
        st.upload(U0)
        steps = 10
        ms = _events_time(lambda: st.step_cfl(1, cfl=0.3), steps, 3)
        rate = 128 ** 3 * 3 * steps / (ms * 1e-3)
        bpc = 8 / 3 * 8 * 8
        out.append({"workload": f"mhd_128cubed_{name}_ssprk3_fp64", "value": rate, "unit": UNIT,
                    "ms_per_step": ms / steps, "bytes_per_cell_update": bpc,
                    "hbm_frac": rate * bpc / 1e9 / hbm_peak})
    return out


def _amr_rows(hbm_peak: float) -> list[dict]:
    """Inter-patch steps of the level loop (Sec. III): same-level ghost
    synchronisation, quintic prolongation, BOR prolongation, and a sub-cycled
    two-level CCZ4 step."""
    import torch
    from paper_1806_04182_gb300 import amr, capi, inputs
    from paper_1806_04182_gb300.state import PatchState
    out = []
    h = torch.cuda.current_stream().cuda_stream
    # ghost synchronisation of a 96^3 CCZ4 box split into 2 x 2 x 2 patches of 48^3 (float)
    m = (48, 48, 48)
    dx = (1 / 96,) * 3
    grid = {}
    for a in range(2):
        for b in range(2):
            for c in range(2):
                st = PatchState(capi.SF_Z4, m, dx, 0.25 * dx[0], precision=capi.SF_FP32_BULK_DW,
                                prm=capi.params(ghosts=capi.SF_GHOSTS_NONE))
                grid[(a, b, c)] = st
    boxes = amr.halo_boxes(grid, "A")
    moved = sum(bx.ext[0] * bx.ext[1] * bx.ext[2] * bx.nf for bx in boxes) * 4
    ms = _events_time(lambda: capi.sf_copy_boxes(boxes, capi.SF_FP32_BULK_DW, h), 50, 3)
    gbs = 2 * moved * 50 / (ms * 1e-3) / 1e9
    out.append({"workload": "halo_sync_8_patches_48cubed_ccz4_fp32", "value": gbs, "unit": "GB/s",
                "ms_per_call": ms / 50, "bytes_per_call": 2 * moved, "hbm_frac": gbs / hbm_peak,
                "note": f"{len(boxes)} box copies (26 per patch), read + write counted"})
    # the same 96^3 CCZ4 box as a level of 2 x 2 x 2 patches stepped as ONE batch: every
    # stage's TMA tile launch ends with the halo copies of the buffer it wrote, and one RK4
    # step of the level (stages + synchronisation) is one captured graph
    Ub, dxb = inputs.z4_minkowski_noise((96, 96, 96), seed=0, amp=1e-10)
    for lname, lay, kern in (("rows56", dict(x_pitch=56), "one-point TMA tile launch"),
                             ("two_point_layout", dict(x_pitch=56, x_offset=1),
                              "two-point tile launch (32 x 16 tiles, the second in x half used)")):
        level = {}
        for a in range(2):
            for b_ in range(2):
                for c in range(2):
                    st = PatchState(capi.SF_Z4, m, dxb, 0.25 * dxb[0], precision=capi.SF_FP32_BULK_DW,
                                    prm=capi.params(ghosts=capi.SF_GHOSTS_NONE), **lay)
                    st.upload(np.ascontiguousarray(Ub[:, c * 48:(c + 1) * 48, b_ * 48:(b_ + 1) * 48,
                                                      a * 48:(a + 1) * 48]))
                    level[(a, b_, c)] = st
        gs = torch.cuda.Stream()
        gs.wait_stream(torch.cuda.current_stream())
        lb = amr.level_batch(level)
        try:
            with torch.cuda.stream(gs):
                capi.sf_copy_boxes(amr.halo_boxes(level, "A"), capi.SF_FP32_BULK_DW, gs.cuda_stream)
                capi.sf_batch_capture(lb, gs.cuda_stream)
                nlevel = 20
                ms = _events_time(lambda: capi.sf_batch_launch(lb, gs.cuda_stream), nlevel, 3)
            out.append({"workload": f"level_8_patches_48cubed_ccz4_fp32dw_batch_halo_graph_{lname}",
                        "value": 96 ** 3 * 4 * nlevel / (ms * 1e-3), "unit": UNIT,
                        "ms_per_step": ms / nlevel,
                        "launches_per_step": capi.sf_batch_launches_per_step(lb), "layout": lay,
                        "note": f"96^3 CCZ4 box as 2x2x2 patches of 48^3: per stage one {kern} over "
                                "all patches + one launch of the 208 halo box copies, one graph per "
                                "RK4 step (amr.level_batch)"})
        finally:
            capi.sf_batch_destroy(lb)
        del level
    # prolongation of a 96^3 fine box (ratio 2) from a 48^3 coarse CCZ4 patch, and the BOR form
    cst = PatchState(capi.SF_Z4, m, (2 / 96,) * 3, 0.5 / 96, precision=capi.SF_FP32_BULK_DW)
    U0, _ = inputs.z4_perturbed(m, seed=1, amp=0.02)
    cst.upload(U0)
    ext = (90, 90, 90)
    fine = torch.zeros((25, ext[2], ext[1], ext[0]), dtype=torch.float32, device="cuda")
    p = cst.patch(cst.A, cst.A, cst.B)
    pts = ext[0] * ext[1] * ext[2]
    states = [cst.A.data_ptr(), cst.B.data_ptr(), cst.C.data_ptr(), cst.D.data_ptr(), cst.E.data_ptr()]
    for name, fn, narr in (
            ("prolong", lambda: capi.sf_prolong(p, cst.A.data_ptr(), 25, 2, (3, 3, 3), ext,
                                                fine.data_ptr(), ext[0], ext[0] * ext[1], pts, h), 1),
            ("bor_prolong", lambda: capi.sf_bor_prolong(p, capi.SF_RK4, states, 25, 2, 1, 2, (3, 3, 3),
                                                        ext, fine.data_ptr(), ext[0], ext[0] * ext[1],
                                                        pts, h), 5)):
        ms = _events_time(fn, 20, 3)
        rate = pts * 20 / (ms * 1e-3)
        alg = pts * 25 * 4 + narr * (ext[0] // 2 + 6) ** 3 * 25 * 4
        out.append({"workload": f"{name}_ratio2_fine_90cubed_ccz4_fp32", "value": rate,
                    "unit": "fine points/s", "ms_per_call": ms / 20,
                    "achieved_gbs": alg * 20 / (ms * 1e-3) / 1e9,
                    "hbm_frac": alg * 20 / (ms * 1e-3) / 1e9 / hbm_peak,
                    "note": "6x6x6 Lagrange taps per fine point and field; algorithmic bytes = "
                            "fine writes + one read of each coarse array region"})
    # sub-cycled two-level CCZ4 step: periodic 64^3 coarse, 64^3 fine patch (ratio 2) inside,
    # on two layouts: rows of 72 floats (16-byte rows: the one-point TMA-staged kernel) and
    # the two-point kernel's layout (rows of 104 floats with one float before each row,
    # planes of 102 rows)
    nc = (64, 64, 64)
    nf = (64, 64, 64)
    Uc, dxc = inputs.z4_minkowski_noise(nc, seed=0, amp=1e-10)
    Uf, _ = inputs.z4_minkowski_noise(nf, seed=1, amp=1e-10)
    for lname, lay in (("rows72", dict(x_pitch=72)),
                       ("two_point_layout", dict(x_pitch=104, x_offset=1, plane_rows=102))):
        coarse = PatchState(capi.SF_Z4, nc, dxc, 0.25 * dxc[0], precision=capi.SF_FP32_BULK_DW, **lay)
        coarse.upload(Uc)
        fine = PatchState(capi.SF_Z4, nf, tuple(v / 2 for v in dxc), 0.125 * dxc[0],
                          precision=capi.SF_FP32_BULK_DW, prm=capi.params(ghosts=capi.SF_GHOSTS_NONE),
                          **lay)
        fine.upload(Uf)
        pair = amr.SubcycledPair(coarse, fine, 2, (16, 16, 16))
        steps = 5
        ms_launch = _events_time(lambda: pair.step(1), steps, 2)
        pair.capture(1)
        ms = _events_time(pair.replay, steps, 2)
        cells = 64 ** 3 * 4 + 64 ** 3 * 4 * 2
        out.append({"workload": f"subcycled_bor_ccz4_fp32dw_coarse64_fine64_ratio2_{lname}", "value":
                    cells * steps / (ms * 1e-3), "unit": UNIT, "ms_per_coarse_step": ms / steps,
                    "ms_per_coarse_step_python_driver": ms_launch / steps,
                    "layout": lay,
                    "note": "one coarse RK4 step + 2 fine RK4 steps with BOR ghost fills before every "
                            "fine stage (6 prolongation boxes each, on a second stream beside the "
                            "fine stage before) and restriction, replayed as one CUDA graph "
                            "(amr.SubcycledPair.capture)"})
        del pair, coarse, fine
    return out


def _mhd_row(hbm_peak: float) -> list[dict]:
    from paper_1806_04182_gb300 import capi, inputs
    from paper_1806_04182_gb300.state import PatchState
    out = []
    # MHD 128^3, SSP-RK3, CFL 0.3 with the rate fused into each step's last stage
    n = (128, 128, 128)
    U0, dx = inputs.mhd_blast(n, seed=0)
    prm = capi.params(rk=capi.SF_SSPRK3)
    for prec, name, es in ((capi.SF_FP64, "fp64", 8), (capi.SF_FP32_BULK, "fp32", 4)):
        st = PatchState(capi.SF_MHD, n, dx, 1e-3, precision=prec, prm=prm)
        st.upload(U0)
        steps = 10 if prec == capi.SF_FP64 else 50
        ms = _events_time(lambda: st.step_cfl(1, cfl=0.3), steps, 3)
        rate = 128 ** 3 * 3 * steps / (ms * 1e-3)
        bpc = 8 / 3 * 8 * es
        out.append({"workload": f"mhd_128cubed_weno5_llf_ssprk3_{name}", "value": rate,
                    "unit": UNIT, "ms_per_step": ms / steps, "bytes_per_cell_update": bpc,
                    "hbm_frac": rate * bpc / 1e9 / hbm_peak,
                    "note": "dt = 0.3 / max signal rate: sf_mhd_max_rate once, then the rate "
                            "fused into each step's last stage, read back every step"})
    return out


def _batch_rows(hbm_peak: float, npatch: int = 512, per_patch: bool = True) -> list[dict]:
    import torch
    from paper_1806_04182_gb300 import capi, inputs
    from paper_1806_04182_gb300.state import PatchState
    out = []
    # batched AMR step: npatch patches, one persistent launch per stage in a CUDA graph
    table = inputs.amr_patch_table(npatch, seed=0)

    def states(precision, tma_pitch=False, pair=False):
        # tma_pitch: float CCZ4 rows padded to a multiple of 4 floats, which
        # sends those patches to the TMA-staged kernel inside the batch; pair:
        # the same with one float before each row (the two-point kernel); the
        # other run keeps every CCZ4 row off that multiple (persistent only)
        sts = []
        for q, t in enumerate(table):
            h = t["dx"]
            system = capi.SF_WAVE if t["system"] == "wave" else capi.SF_Z4
            if system == capi.SF_WAVE:
                U0, _ = inputs.wave_plane(t["n"], seed=q, length=t["n"][0] * h)
            else:
                U0, _ = inputs.z4_minkowski_noise(t["n"], seed=q)
            pitch, xo = None, 0
            if system == capi.SF_Z4:
                # a multiple of 4 floats for the TMA-staged kernel; otherwise a
                # pitch that is not, so every CCZ4 patch takes the persistent kernel
                row = t["n"][0] + 6
                pitch = (row + 3) // 4 * 4 if tma_pitch else (row + 1 if row % 4 == 0 else row)
                if pair:
                    pitch, xo = (row + 1 + 3) // 4 * 4, 1
            sts.append(PatchState(system, t["n"], (h, h, h), t["dt"], precision=precision,
                                  x_pitch=pitch, x_offset=xo))
            sts[-1].upload(U0)
        return sts

    cells = sum(t["n"][0] * t["n"][1] * t["n"][2] for t in table)
    bytes_step = sum(t["n"][0] * t["n"][1] * t["n"][2] * (19 * (25 if t["system"] == "z4" else 5) * 4)
                     for t in table)
    batch_rate = None
    for name, tma, pair in (("pair_ccz4_tiles_plus_persistent", True, True),
                            ("tma_ccz4_tiles_plus_persistent", True, False),
                            ("persistent_only", False, False)):
        sts = states(capi.SF_FP32_BULK_DW, tma_pitch=tma, pair=pair)
        stream = torch.cuda.Stream()
        b = capi.sf_batch_create(capi.params(), [s_.patch(s_.B, s_.A, s_.C) for s_ in sts])
        with torch.cuda.stream(stream):
            capi.sf_batch_tune(b, stream.cuda_stream)
            capi.sf_batch_capture(b, stream.cuda_stream)
            ms = _events_time(lambda: capi.sf_batch_launch(b, stream.cuda_stream), 10, 3)
        launches = capi.sf_batch_launches_per_step(b)
        tuned = capi.sf_batch_tuned(b)
        capi.sf_batch_destroy(b)
        rate = cells * 4 * 10 / (ms * 1e-3)
        batch_rate = rate if batch_rate is None else batch_rate
        out.append({"workload": f"amr_batch_{npatch}_patches_fp32_bulk_dw_graph_{name}",
                    "value": rate, "unit": UNIT, "ms_per_step": ms / 10, "cells": cells,
                    "launches_per_step": launches, "launches_per_stage": launches / 4,
                    "tuned": tuned,
                    "hbm_frac": bytes_step * 10 / (ms * 1e-3) / 1e9 / hbm_peak})
        del sts
    if not per_patch:
        return out
    sts = states(capi.SF_FP64)
    z4p = [s_ for s_ in sts if s_.system == capi.SF_Z4]
    wvp = [s_ for s_ in sts if s_.system == capi.SF_WAVE]

    def per_patch_step():
        h = torch.cuda.current_stream().cuda_stream
        for stg in range(4):
            capi.sf_substep(z4p[0].prm, [s_.stage_patch(stg) for s_ in z4p], stg, h)
            capi.sf_substep(wvp[0].prm, [s_.stage_patch(stg) for s_ in wvp], stg, h)

    ms = _events_time(per_patch_step, 3, 1)
    pp_rate = cells * 4 * 3 / (ms * 1e-3)
    out.append({"workload": f"amr_{npatch}_patches_fp64_per_patch_launches", "value": pp_rate,
                "unit": UNIT, "ms_per_step": ms / 3,
                "batched_fp32_speedup": batch_rate / pp_rate})
    return out


def _adjoint_rows() -> list[dict]:
    import torch
    from paper_1806_04182_gb300 import adjoint, capi, inputs
    out = []
    # adjoint: 128^3 wave, 200 RK4 steps, 64 observers, checkpoints every 20 steps
    for prec, name in ((capi.SF_FP64, "fp64"), (capi.SF_FP32_BULK, "fp32")):
        n = (128, 128, 128)
        U0, dx = inputs.wave_plane(n, seed=0)
        dt = 0.25 * dx[0]
        dtype = torch.float64 if prec == capi.SF_FP64 else torch.float32
        phi0 = torch.tensor(U0[0], device="cuda", dtype=dtype)
        Pi0 = torch.tensor(U0[1], device="cuda", dtype=dtype)
        obs = torch.tensor(inputs.observers(n, 64, seed=1), device="cuda")
        bump = torch.tensor(1e-3 * inputs.smooth_bump(n, seed=2), device="cuda", dtype=dtype)
        ref = adjoint.observe(phi0 + bump, Pi0, obs, dx, dt, 200, precision=prec)

        def grad_eval():
            p = phi0.clone().requires_grad_(True)
            q = Pi0.clone().requires_grad_(True)
            adjoint.misfit(p, q, obs, ref, dx, dt, 200, precision=prec, checkpoint_every=20).backward()

        ms = _events_time(grad_eval, 1, 1)
        out.append({"workload": f"wave_adjoint_128cubed_200steps_{name}", "value": 1e3 / ms,
                    "unit": "gradients/s", "ms_per_gradient": ms,
                    "cell_updates_per_s": 128 ** 3 * 4 * 200 * 3 / (ms * 1e-3),
                    "note": "forward + recompute + adjoint = 3 x 200 RK4 steps"})
    return out


# ---------------------------------------------------------------- oracle arm
# The oracle's sample: a 96 x 96 x 16 periodic slab of the 96^3 workload (same
# spacing, data distribution and parameters).  Its right-hand-side sweep is
# parallel over the slab's 16 x 96 = 1536 (z, y) rows, so every host core has
# work; the CCZ4 cell cost does not depend on the slab's depth.
ORACLE_NZ = 16


def host_cpu() -> str:
    """CPU model of this host (lscpu's model name, else the platform string)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    import platform
    return platform.machine()


def _oracle_slab(nz: int):
    import oracle
    from paper_1806_04182_gb300 import inputs
    oracle.build()
    U0, _ = inputs.z4_minkowski_noise((N, N, nz), seed=0, amp=1e-10)
    dx = (1.0 / N,) * 3
    return oracle, oracle.ghosted(U0), dx, oracle.params(), 0.25 * dx[0]


def _oracle_rate(threads: int, seconds: float, nz: int) -> tuple[float, int, float, int]:
    """Cell-updates/s of RK4 steps of the slab on `threads` threads, stepping
    until `seconds` have passed (at least one step).  Returns (rate, steps,
    seconds, threads in effect)."""
    oracle, G, dx, p, dt = _oracle_slab(nz)
    used = oracle.set_threads(threads)
    t0 = time.perf_counter()
    steps = 0
    while True:
        oracle.rk4_step(oracle.Z4, G, dx, dt, p)
        steps += 1
        el = time.perf_counter() - t0
        if el > seconds or steps >= 1000:
            break
    return N * N * nz * 4 * steps / el, steps, el, used


def cpu_baseline(seconds: float = 15.0, nz: int = ORACLE_NZ) -> dict:
    """The FP64 oracle as it stands on a bounded sample of the same workload,
    on every host core and on one core."""
    cores = os.cpu_count() or 1
    rate, steps, el, used = _oracle_rate(cores, seconds, nz)
    rate1, steps1, el1, _ = _oracle_rate(1, seconds / 2, nz)
    import oracle
    oracle.set_threads(cores)
    p = min(used, N * nz)
    speedup = rate / rate1
    # Amdahl's serial share of the single-thread step implied by the speed-up
    serial = (1.0 / speedup - 1.0 / p) / (1.0 - 1.0 / p) if p > 1 else 1.0
    return {"value": rate, "unit": UNIT, "cores": p, "kind": "oracle",
            "sample": f"{steps} RK4 steps of a 96x96x{nz} periodic slab of the 96^3 workload "
                      f"(same dx, data, params), {el:.1f} s, OpenMP over its {N * nz} (z, y) rows",
            "cpu": host_cpu(), "nproc": cores,
            "single_thread": {"value": rate1, "unit": UNIT, "cores": 1,
                              "sample": f"{steps1} RK4 steps of the same slab, {el1:.1f} s"},
            "parallel_speedup": speedup,
            "serial_share": serial,
            "parallel_note": "the oracle's right-hand-side sweep runs in parallel over the slab's "
                             "(z, y) rows; its RK combinations, periodic ghost fills and the "
                             "zero-filled stage arrays it allocates every step run on one thread. "
                             "serial_share is that part of the single-thread step as implied by "
                             "Amdahl's law from the two rates, and it caps the speed-up below "
                             "the thread count"}


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return None
    nz = ORACLE_NZ
    oracle, G, dx, p, dt = _oracle_slab(nz)
    cores = os.cpu_count() or 1
    used = oracle.set_threads(cores)
    for _ in range(args.warmup):
        oracle.rk4_step(oracle.Z4, G, dx, dt, p)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.rk4_step(oracle.Z4, G, dx, dt, p)
    el = time.perf_counter() - t0
    value = N * N * nz * 4 * args.steps / el
    sample = (f"each step: one RK4 step of a 96x96x{nz} periodic slab of the 96^3 workload, "
              f"OpenMP over its {N * nz} (z, y) rows")
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic: Minkowski + seeded uniform noise 1e-10",
            "config": {"workload": WORKLOAD, "n": N, "sample_nz": nz},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": min(used, N * nz), "kind": "oracle",
                             "sample": sample, "cpu": host_cpu(), "nproc": cores},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--suite", action="store_true",
                    help="time every workload row (one JSON line each) instead of the headline")
    ap.add_argument("--rows", default=None,
                    help="comma-separated subset of wave,mhd,batch,batch_graph,adjoint,variants,amr,puncture "
                         "for --suite")
    ap.add_argument("--npatch", type=int, default=512, help="patches of the batch rows")
    ap.add_argument("--pitch", type=int, default=FLOAT_PITCH,
                    help="row pitch of the float arrays (102 = dense: global-load kernel)")
    ap.add_argument("--x-offset", type=int, default=1,
                    help="floats before each row's first ghost point of the float arrays (1: the "
                         "two-point CCZ4 kernel; 0: the one-point TMA kernel)")
    ap.add_argument("--only", choices=["fp32dw", "fp32", "fp64"], default=None,
                    help="time one precision only (profiling runs)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.suite:
        import torch
        from paper_1806_04182_gb300 import build as sfbuild
        sfbuild.build()
        torch.cuda.set_device(0)
        pk = os.path.join(ROOT, "MEASURED_PEAKS.json")
        hbm = json.load(open(pk)).get("hbm_gbs", 6800.0) if os.path.exists(pk) else 6800.0
        for row in suite(args, hbm):
            print(json.dumps(row), flush=True)
        return
    line = reference_arm(args) if args.impl == "reference" else gpu_arm(args)
    if line is not None:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
