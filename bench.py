"""Benchmark of the fused coupled LB step on GB300 (one JSON line on stdout).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl {gb300,reference}]
                    [--workload NAME] [--precision fp64]

Workload (default): the single sessile droplet freezing on a cold wall, 512 x 512,
N = 2, FP64 (the second problem of Section 4; inputs synthetic, built by
paper_2603_22902_gb300.workloads).  A step is one fused time step over the lattice.
Timing: W untimed warm-up steps, then K steps, each timed with CUDA events on the
launching stream and preceded by an untimed L2 flush (a 256 MiB write, then a 256 MiB
read, so that L2 holds none of the state and no dirty line of the flush), bracketed by
a barrier + device synchronise; the max over ranks is reported.  With N > 1 every rank
runs its own replica of the workload (replicas only: the single-lattice step has no
multi-GPU path here), so the scaling is weak.

With --precision fp64 (the default) and one GPU, the line also carries, for each
--compare policy, its throughput timed the same way on the same workload and its
freezing-front position against FP64 after --front-steps steps from the same initial
state (the error bound is 0.5 lattice units): "reduced_precision" for FP16 storage and
"double_word" for the double-word policy (FP32 pairs on the FP32 pipes, held to the
FP64 parity bar by the tests).

The reference arm (--impl reference) times the CPU oracle (oracle/) as it stands on
the host cores, one oracle time step of the same workload per step.
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
sys.path.insert(0, ROOT)

METRIC = "coupled-step MLUPS and % HBM roofline at 1 GB300; reduced-precision vs FP64 at stated error"
# Algorithmic bytes per lattice update of the fused step: every population read and
# written once, every lagged plane read and written once:
# 2 [ (N + 2) rest + 8 (N + 2) moving populations + (3 + 2 N) lagged planes ],
# with (rest, moving, lagged) element sizes of (8, 8, 8) for FP64 (688 B at N = 2),
# (4, 4, 4) for FP32 and (4, 2, 4) for the 16-bit storage policies.
ELEM = {"fp64": (8, 8, 8), "df64": (8, 8, 8), "fp32": (4, 4, 4), "fp16s": (4, 2, 4), "bf16s": (4, 2, 4)}


def bytes_per_lu(N: int, precision: str = "fp64") -> int:
    er, em, ea = ELEM[precision]
    return 2 * ((N + 2) * er + 8 * (N + 2) * em + (3 + 2 * N) * ea)


# The FP64 step is bound by the FP64 pipe, not by HBM.  Its roofline is the issue rate
# of that pipe: 152 SMs x 2 FP64 lanes per clock x 2.07 GHz = 629.3 G thread-instructions
# per second (x 2 flop per FMA = 1.259 TFLOP/s).
FP64_PIPE_PEAK_GINST = 152 * 2 * 2.070
# Instruction issue: 152 SMs x 4 schedulers x 1 warp-instruction per clock x 2.07 GHz.
# The double-word step runs ~4400 FP32 instructions per lattice update on the FP32 pipes
# and is bound by this issue rate rather than by any one pipe or by HBM.
ISSUE_PEAK_GWINST = 152 * 4 * 2.070
# Per lattice update of the fused step kernel, from one ncu capture of the kernel built
# from the kernel sources with digest `digest` (build.kernel_digest; sessile drop 512^2,
# N = 2, 32 x 8 tiles):
# FP64-pipe thread-instructions, FP64 flop (DFMA = 2, DADD / DMUL = 1), warp-instructions
# issued, FP32 thread-instructions (FADD + FMUL + FFMA; the packed FADD2 of the double-word
# sums is not among them) and DRAM bytes.
# A changed kernel has another digest, and then these counts are not reported.
# (DRAM bytes are what ncu saw during the launch: part of the writes of a launch is
# still in L2 when it ends and reaches DRAM during the next one.)
_D = "61f9297197c4bb8f09a6f9210f730158592671151ccc04797480a1b3f5077d6c"
NCU_COUNTS = {
    ("fp64", 2): {"digest": _D, "fp64_inst": 487.0, "fp64_flop": 660.8, "warp_inst": 101.6, "dram_bytes": 539.8},
    ("df64", 2): {"digest": _D, "fp64_inst": 0.08, "warp_inst": 175.0, "fp32_inst": 4089.1, "dram_bytes": 665.9},
    # the FP16-storage step is the TMA-staged kernel (staged_tile_kernel) where it applies
    ("fp16s", 2): {"digest": _D, "fp64_inst": 0.06, "fp64_flop": 0.03, "warp_inst": 45.0, "dram_bytes": 108.5},
}


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


def kernel_digest():
    from paper_2603_22902_gb300 import build as B
    return B.kernel_digest()


def ncu_counts(precision, N):
    c = NCU_COUNTS.get((precision, N))
    if c and c["digest"] == kernel_digest():
        return c
    return None


def case_params(case):
    """Physical and numerical parameters of a workload, for the line's config."""
    m = case.meta
    out = {"eps": case.eps, "mobility": case.mobility, "T0": float(case.T.flat[0])}
    for k in ("R", "R_core", "R_shell", "ste", "rho_ratio", "theta", "T_wall", "h0"):
        if k in m:
            out[k] = m[k]
    sig = [float(case.sigma[p, q]) for p in range(case.N) for q in range(p + 1, case.N)]
    out["sigma"] = sig if len(sig) > 1 else sig[0]
    out["rho_l"] = [ph["rho_l"] for ph in case.phases]
    return out


def make_case(name):
    from paper_2603_22902_gb300 import workloads as W
    if name == "sessile_drop_512":
        return W.sessile_drop()
    if name == "film_16x256":
        return W.film()
    if name == "compound_drop_1024":
        return W.compound_drop()
    raise SystemExit(f"unknown workload {name}")


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    def __init__(self, index=0, directory=None):
        self.proc = None
        self.index = index
        # the raw samples go to `directory` (--clocks-dir) when given, else to a temporary
        # directory; the JSON line carries their summary either way
        self.path = os.path.join(directory or tempfile.gettempdir(), f"clocks_rank{index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                parts = [s.strip() for s in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx = max(mx, float(parts[2]))
                except ValueError:
                    continue
                for n, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        import torch
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend)
    return world, rank, local


def reduce_max(value: float, world: int) -> float:
    """Max of a float over all ranks (identity for one process)."""
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def host_info():
    """CPU model and the number of cores this process may run on."""
    model = None
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                key = line.split(":")[0].strip().lower()
                if key in ("model name", "cpu model", "hardware") and ":" in line:
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    if not model:
        try:  # Arm hosts: /proc/cpuinfo has no model name, lscpu maps the part number
            out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
            for line in out.splitlines():
                if line.lower().startswith("model name:"):
                    model = line.split(":", 1)[1].strip()
                    break
        except (OSError, subprocess.SubprocessError):
            pass
    if not model:
        import platform
        model = platform.processor() or platform.machine()
    try:
        cores = len(os.sched_getaffinity(0))
    except AttributeError:
        cores = os.cpu_count() or 1
    return model, cores


def time_oracle(case, steps, budget_s=20.0, warmup=1, omp=False):
    """The CPU oracle as it stands: oracle time steps of the case after `warmup` untimed
    steps, one thread (or, with omp=True, its -fopenmp build on every core this process
    may use); stops early when the budget is spent."""
    import oracle
    o = oracle.Oracle(case, omp=omp)
    o.step(warmup)  # warm (page-in, caches)
    done, t0 = 0, time.perf_counter()
    while done < steps:
        o.step(1)
        done += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    return case.cells * done / dt / 1e6, done, dt


def run_reference(args):
    world, rank, _ = dist_setup()
    if rank != 0:
        return 0
    case = make_case(args.workload)
    mlups, done, dt = time_oracle(case, args.steps, budget_s=args.ref_budget, warmup=args.warmup)
    cores = 1
    model, avail = host_info()
    line = {
        "impl": "reference", "metric": METRIC, "value": round(mlups, 4), "unit": "MLUPS",
        "n_gpus": args.gpus, "steps": done, "warmup": args.warmup, "ms_per_step": round(1e3 * dt / done, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": case.name, "nx": case.nx, "ny": case.ny, "N": case.N,
                                        "params": case_params(case)},
        "cpu_baseline": {"value": round(mlups, 4), "unit": "MLUPS", "cores": cores, "kind": "oracle",
                         "cpu_model": model, "cores_available": avail,
                         "sample": f"{done} timed oracle steps of {case.name} (of {args.steps} requested, after "
                                   f"{args.warmup} untimed; {args.ref_budget:.0f} s budget), one host thread"},
        "e2e": {"value": round(mlups, 4), "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_gpu(args):
    import numpy as np
    import torch

    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    from paper_2603_22902_gb300 import build as B
    if rank == 0:
        B.build()
    barrier(world)
    from paper_2603_22902_gb300 import lbm

    case = make_case(args.workload)
    N = case.N
    stream = torch.cuda.current_stream()
    s = lbm.Solver(case, precision=args.precision, tile=tuple(args.tile) if args.tile else None)
    s.set_fields()
    flush = L2Flush(torch)

    for _ in range(args.warmup):
        s.step(1)
    torch.cuda.synchronize()
    barrier(world)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    clocks = ClockSampler(local, args.clocks_dir)
    clocks.start()
    torch.cuda.synchronize()
    barrier(world)
    t_wall0 = time.perf_counter()
    for k in range(args.steps):
        flush()                           # untimed: evict L2 between timed steps
        starts[k].record(stream)
        s.step(1)
        ends[k].record(stream)
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall0
    barrier(world)
    clk = clocks.stop()
    per_step_ms = [a.elapsed_time(b) for a, b in zip(starts, ends)]
    t_ms = sum(per_step_ms)
    t_ms_max = reduce_max(t_ms, world)
    diag = s.diagnostics()
    if diag["nonfinite"]:
        raise SystemExit("non-finite state during the benchmark")

    cells = case.cells
    value = world * cells * args.steps / (t_ms_max * 1e-3) / 1e6          # MLUPS, all ranks
    mlups_rank = cells * args.steps / (t_ms * 1e-3) / 1e6
    hbm_peak, peak_kind = load_peaks()
    bpl = bytes_per_lu(N, args.precision)
    gbs = bpl * mlups_rank * 1e6 / 1e9
    counts = ncu_counts(args.precision, N)
    traffic = round(counts["dram_bytes"] * cells) if counts else None
    fp64_peak, fp64_peak_kind = FP64_PIPE_PEAK_GINST, "derived: 152 SMs x 2 FP64 lanes/clock x 2.07 GHz"
    if args.precision == "fp64":
        try:
            r, ms = lbm.lbm_measure_fp64_rate()
            fp64_peak = r
            fp64_peak_kind = (f"measured: FP64 FMA loop (lbm_measure_fp64_rate, best of 5 launches of {ms:.2f} ms "
                              f"after 3 untimed); derived {FP64_PIPE_PEAK_GINST:.1f}")
        except lbm.LBMError:
            pass
    roof_hbm = {"bound": "hbm", "achieved": round(gbs, 1), "peak": hbm_peak, "unit": "GB/s",
                "frac": round(gbs / hbm_peak, 4), "traffic": traffic,
                "peak_kind": f"{peak_kind} (copy bandwidth)", "bytes_per_lu": bpl, "lu_per_launch": cells}
    roofline = roof_hbm
    if args.precision == "fp64":
        roof_hbm["fp64_rate"] = {"peak": round(fp64_peak, 1), "unit": "G FP64-pipe inst/s", "peak_kind": fp64_peak_kind}
    if counts and args.precision == "fp64":
        gi = counts["fp64_inst"] * mlups_rank * 1e6 / 1e9
        roofline = {"bound": "alu", "achieved": round(gi, 1), "peak": round(fp64_peak, 1),
                    "unit": "G FP64-pipe inst/s", "frac": round(gi / fp64_peak, 4), "traffic": traffic,
                    "peak_kind": fp64_peak_kind,
                    "fp64_inst_per_lu": counts["fp64_inst"], "lu_per_launch": cells,
                    "tflops": round(counts["fp64_flop"] * mlups_rank * 1e6 / 1e12, 4),
                    "hbm": {k: roof_hbm[k] for k in ("achieved", "peak", "unit", "frac", "bytes_per_lu")}}

    # ---- end to end through the C ABI with host buffers ------------------------------
    e2e = None
    if args.e2e_steps > 0:
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).pin_memory()
        h_in = [pin(case.phi), pin(case.T), pin(case.ux), pin(case.uy)]
        h_out = [torch.empty((N, case.ny, case.nx), dtype=torch.float64).pin_memory()] + \
                [torch.empty((case.ny, case.nx), dtype=torch.float64).pin_memory() for _ in range(6)]
        torch.cuda.synchronize()
        barrier(world)
        t0 = time.perf_counter()
        lbm.lbm_set_fields(s.h, h_in[0], h_in[1], h_in[2], h_in[3], lbm.LBM_HOST)
        lbm.lbm_step(s.h, args.e2e_steps)
        lbm.lbm_get_fields(s.h, *h_out, lbm.LBM_HOST)
        torch.cuda.synchronize()
        dt = reduce_max(time.perf_counter() - t0, world)
        h2d = sum(t.numel() * 8 for t in h_in)
        d2h = sum(t.numel() * 8 for t in h_out)
        e2e = {"value": round(world * cells * args.e2e_steps / dt / 1e6, 2), "unit": "MLUPS",
               "h2d_bytes_per_step": int(h2d / args.e2e_steps), "d2h_bytes_per_step": int(d2h / args.e2e_steps),
               "steps_per_call": args.e2e_steps}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        model, avail = host_info()
        mlups_cpu, done, dt = time_oracle(case, 10 ** 6, budget_s=args.cpu_budget)
        cpu = {"value": round(mlups_cpu, 4), "unit": "MLUPS", "cores": 1, "kind": "oracle",
               "sample": f"{done} oracle time steps of {case.name} ({dt:.1f} s), one host thread",
               "cpu_model": model, "cores_available": avail}
        if avail > 1:
            mlups_omp, done_o, dt_o = time_oracle(case, 10 ** 6, budget_s=args.cpu_budget, omp=True)
            cpu["openmp"] = {"value": round(mlups_omp, 4), "unit": "MLUPS", "cores": avail,
                             "sample": f"{done_o} oracle time steps of {case.name} ({dt_o:.1f} s), the -fopenmp build "
                                       f"of the same source (per-cell loops over {avail} threads)"}

    s.close()
    rp = None
    if world == 1 and args.precision == "fp64" and args.compare and args.compare != "none":
        rp = compare_precision(case, args.compare.split(","), mlups_rank, args.front_steps, stream, flush)
    extra = {}
    if world == 1 and args.precision == "fp64" and args.workload == "sessile_drop_512" and args.extras != "none":
        extra = extra_workloads(args, lbm, stream, flush)
    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 2), "unit": "MLUPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(t_ms_max / args.steps, 5),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp64": "f64", "df64": "df64 (f32 pair)", "fp32": "f32", "fp16s": "f16-storage/f32",
                      "bf16s": "bf16-storage/f32"}[args.precision],
            "data": "synthetic",
            "config": {"workload": case.name, "nx": case.nx, "ny": case.ny, "N": N, "precision": args.precision,
                       "params": case_params(case),
                       "l2": "flushed (256 MiB write, then 256 MiB read) before every timed step", "timing": "CUDA events per step",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": args.steps,
            "clocks": clk, "wall_s_timed_loop": round(t_wall, 4),
        }
        if rp is not None:
            # "reduced_precision": FP16 storage (the reduced-precision form of the step);
            # "double_word": FP64-class accuracy on the FP32 pipes (parity-tested to 1e-10)
            if "fp16s" in rp:
                line["reduced_precision"] = rp.pop("fp16s")
            if "df64" in rp:
                line["double_word"] = rp.pop("df64")
            line.update({f"compare_{k}": v for k, v in rp.items()})
        line.update(extra)
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


class L2Flush:
    """Evicts L2 (129 MB on GB300) between timed steps: a 256 MiB write, then a 256 MiB
    read.  After the write alone L2 is full of the flush's dirty lines, and the timed step
    would pay for writing them back to HBM (~3 us of a 28 us FP16 step at 512 x 512); after
    the read L2 holds only clean lines of the read buffer, none of the state."""

    def __init__(self, torch):
        n = 256 * 1024 * 1024 // 4
        self.w = torch.empty(n, dtype=torch.float32, device="cuda")
        self.r = torch.ones(n, dtype=torch.float32, device="cuda")
        self.out = torch.zeros((), dtype=torch.float32, device="cuda")
        self.torch = torch

    def __call__(self):
        self.w.zero_()
        self.torch.sum(self.r, dim=0, out=self.out)


def timed_mlups(lbm, case, precision, steps, stream, flush, staged=None):
    """Same protocol as the headline: L2 flushed before every timed step, CUDA events.
    staged: None for the library's default form, else force the TMA-staged form on / off."""
    import torch
    s = lbm.Solver(case, precision=precision, staged=staged).set_fields()
    s.step(5)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    torch.cuda.synchronize()
    for k in range(steps):
        flush()
        starts[k].record(stream)
        s.step(1)
        ends[k].record(stream)
    torch.cuda.synchronize()
    s.close()
    t_ms = sum(a.elapsed_time(b) for a, b in zip(starts, ends))
    return case.cells * steps / (t_ms * 1e-3) / 1e6


def compare_precision(case, precisions, mlups_fp64, front_steps, stream, flush):
    """Other policies against FP64 on the same GPU: throughput timed like the headline,
    and the freezing-front position after front_steps steps from the same initial state."""
    from paper_2603_22902_gb300 import lbm
    from paper_2603_22902_gb300.metrics import front_height, front_integral
    hbm_peak, _ = load_peaks()
    out = {}
    fronts, integrals = {}, {}
    for prec in ["fp64"] + list(precisions):
        if front_steps > 0:
            s = lbm.Solver(case, precision=prec).set_fields()
            s.step(front_steps)
            F = s.fields_numpy()
            fronts[prec] = front_height(F, case.nx)
            integrals[prec] = front_integral(F, case.nx)
            s.close()
        if prec == "fp64":
            continue
        mlups = timed_mlups(lbm, case, prec, 300, stream, flush)
        bpl = bytes_per_lu(case.N, prec)
        r = {"precision": prec, "value": round(mlups, 2), "unit": "MLUPS",
             "speedup_vs_fp64": round(mlups / mlups_fp64, 3), "bytes_per_lu": bpl,
             "hbm_frac": round(bpl * mlups * 1e6 / 1e9 / hbm_peak, 4)}
        if front_steps > 0:
            r.update({"front_steps": front_steps, "front_fp64_lu": round(fronts["fp64"], 4),
                      "front_err_lu": float(f"{abs(fronts[prec] - fronts['fp64']):.3g}"), "front_err_bound_lu": 0.5,
                      "front_integral_fp64_lu": round(integrals["fp64"], 4),
                      "front_integral_err_lu": float(f"{abs(integrals[prec] - integrals['fp64']):.3g}")})
        counts = ncu_counts(prec, case.N)
        if counts:
            wi = counts["warp_inst"] * mlups * 1e6 / 1e9
            r["issue"] = {"achieved": round(wi, 1), "peak": round(ISSUE_PEAK_GWINST, 1), "unit": "G warp-inst/s",
                          "frac": round(wi / ISSUE_PEAK_GWINST, 4), "warp_inst_per_lu": counts["warp_inst"],
                          "peak_kind": "derived: 152 SMs x 4 schedulers x 1 warp-inst/clock x 2.07 GHz"}
            fi = counts["fp64_inst"] * mlups * 1e6 / 1e9
            r["fp64_pipe"] = {"achieved": round(fi, 1), "peak": round(FP64_PIPE_PEAK_GINST, 1),
                              "unit": "G FP64-pipe inst/s", "frac": round(fi / FP64_PIPE_PEAK_GINST, 4),
                              "fp64_inst_per_lu": counts["fp64_inst"]}
            if "fp32_inst" in counts:
                r["issue"]["fp32_inst_per_lu"] = counts["fp32_inst"]
            r["traffic"] = round(counts["dram_bytes"] * case.cells)
        out[prec] = r
    return out


def extra_workloads(args, lbm, stream, flush):
    """The other single-GPU configurations, timed by this same run:
    - compound_drop_1024: 1024 x 1024, N = 3, each policy timed like the headline (L2
      flushed before every timed step, CUDA events per step), FP16 storage in its staged and
      one-launch forms;
    - staged_fp16s: the FP16-storage step of the 512^2 and 1024^2 sessile drops in its
      TMA-staged form and in the one-launch form, timed the same way;
    - batch_sweep_256: the 256-drop sweep in one batch (FP16 storage), autotuned plan,
      CUDA events per call of --batch-chunk steps (state far larger than L2);
    - adjoint_impurity_512: one call of the hand-written adjoint on the 512 x 512 pool with
      24 impurity disks (N = 4), 4000 steps, checkpoint every 200: seconds per call (CUDA
      events on the handle's stream) and the share of a plain forward run of the same
      length; and the loss of that run's FP64 forward beside the loss of an FP32 forward."""
    import numpy as np
    import torch
    from paper_2603_22902_gb300 import workloads as W
    hbm_peak, _ = load_peaks()
    out = {}
    parts = args.extras.split(",")
    if "compound" in parts:
        case = W.compound_drop()
        r = {"workload": case.name, "N": case.N, "params": case_params(case), "steps": 200}
        for prec in ("fp64", "df64", "fp32", "fp16s"):
            mlups = timed_mlups(lbm, case, prec, 200, stream, flush)
            bpl = bytes_per_lu(case.N, prec)
            r[prec] = {"value": round(mlups, 2), "unit": "MLUPS", "bytes_per_lu": bpl,
                       "hbm_frac": round(bpl * mlups * 1e6 / 1e9 / hbm_peak, 4)}
        # FP16 storage runs the TMA-staged step by default (N = 3); the one-launch form beside it
        r["fp16s"]["form"] = "staged"
        r["fp16s"]["one_launch"] = round(timed_mlups(lbm, case, "fp16s", 200, stream, flush, staged=False), 2)
        out["compound_drop_1024"] = r
    if "staged" in parts:
        # the FP16-storage step with its inputs staged by tensor copies against the one-launch form
        r = {}
        for n, R in ((512, 100.0), (1024, 200.0)):
            case = W.sessile_drop(n=n, R=R)
            a = timed_mlups(lbm, case, "fp16s", 200, stream, flush, staged=False)
            b = timed_mlups(lbm, case, "fp16s", 200, stream, flush, staged=True)
            r[case.name] = {"one_launch": round(a, 2), "staged": round(b, 2), "unit": "MLUPS",
                            "hbm_frac_staged": round(bytes_per_lu(2, "fp16s") * b * 1e6 / 1e9 / hbm_peak, 4)}
        out["staged_fp16s"] = r
    if "batch" in parts:
        out["batch_sweep_256"] = batch_measure(args, lbm, stream, steps=200, warmup=20)
    if "adjoint" in parts:
        from paper_2603_22902_gb300.grad import final_liquid_fraction, pcm_liquid_fraction
        nsteps, K = 4000, 200
        case = W.impurity_freeze(T_wall=-1.0)
        target = final_liquid_fraction(W.impurity_freeze(T_wall=-1.3), nsteps)
        d = lambda a: np.ascontiguousarray(a, dtype=np.float64)
        s = lbm.Solver(case, precision="fp64")
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        torch.cuda.synchronize()
        ev[0].record(stream)
        g = lbm.lbm_adjoint_fl_loss(s.h, d(case.phi), d(case.T), d(case.ux), d(case.uy), d(target), None,
                                    lbm.LBM_HOST, nsteps, K)
        ev[1].record(stream)
        torch.cuda.synchronize()
        s.set_fields()
        ev[2].record(stream)
        s.step(nsteps)
        ev[3].record(stream)
        torch.cuda.synchronize()
        F64 = s.fields_numpy()
        s.close()
        t_call, t_fwd = ev[0].elapsed_time(ev[1]) * 1e-3, ev[2].elapsed_time(ev[3]) * 1e-3
        s = lbm.Solver(case, precision="fp32").set_fields()
        s.step(nsteps)
        F32 = s.fields_numpy()
        s.close()
        loss64 = float(((pcm_liquid_fraction(case, F64) - target) ** 2).sum())
        loss32 = float(((pcm_liquid_fraction(case, F32) - target) ** 2).sum())
        out["adjoint_impurity_512"] = {
            "workload": case.name, "N": case.N, "steps": nsteps, "checkpoint_every": K,
            "seconds_per_call": round(t_call, 3), "forward_s": round(t_fwd, 3),
            "forward_share": round(t_fwd / t_call, 4), "loss_fp64": g.loss, "loss_fp64_forward_check": loss64,
            "loss_fp32_forward": loss32, "grad_T_wall": g.T_wall[2],
            "timing": "CUDA events on the handle's stream around one lbm_adjoint_fl_loss call"}
    return out


def batch_measure(args, lbm, stream, steps, warmup):
    """Throughput of the 256-drop sweep in one batch (FP16 storage), autotuned plan."""
    import torch
    from paper_2603_22902_gb300 import workloads as W
    prec = "fp16s"
    cases = W.batch_sweep()
    cells = sum(c.cells for c in cases)
    solvers = [lbm.Solver(c, precision=prec).set_fields() for c in cases]
    batch = lbm.Batch(solvers)
    t0 = time.perf_counter()
    batch.autotune(trial_steps=args.batch_chunk)
    tune_s = time.perf_counter() - t0
    chunk = args.batch_chunk
    calls = max(1, steps // chunk)
    for _ in range(max(1, warmup // chunk)):
        batch.step(chunk)
    batch.sync()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(calls)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(calls)]
    torch.cuda.synchronize()
    for k in range(calls):
        starts[k].record(stream)
        batch.step(chunk)
        ends[k].record(stream)
    batch.sync()
    t_ms = sum(a.elapsed_time(b) for a, b in zip(starts, ends))
    nonfinite = sum(s.diagnostics()["nonfinite"] for s in solvers)
    plan = batch.plan.as_dict()
    batch.close()
    for s in solvers:
        s.close()
    if nonfinite:
        raise SystemExit("non-finite state during the batch measurement")
    hbm_peak, _ = load_peaks()
    mlups = cells * calls * chunk / (t_ms * 1e-3) / 1e6
    bpl = bytes_per_lu(2, prec)
    return {"workload": f"batch_sweep_256 ({len(cases)} sessile drops, sides 128-512, seed 4)", "cells": cells,
            "precision": prec, "value": round(mlups, 2), "unit": "MLUPS", "steps": calls * chunk,
            "steps_per_call": chunk, "hbm_frac": round(bpl * mlups * 1e6 / 1e9 / hbm_peak, 4), "bytes_per_lu": bpl,
            "plan": plan, "autotune_s": round(tune_s, 2),
            "timing": "CUDA events per call; the state is far larger than L2 (no flush)"}


def run_batch(args):
    """The batched droplet sweep: 256 independent sessile drops of sides 128..512 in one
    batch (FP16 storage unless --precision says otherwise).  A timed call advances every
    case by --batch-chunk steps; MLUPS = sum of cells x steps / time.  The state (~6 GB)
    is far larger than L2, so no flush is needed between calls."""
    import numpy as np
    import torch
    from paper_2603_22902_gb300 import build as B
    from paper_2603_22902_gb300 import workloads as W
    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    if rank == 0:
        B.build()
    barrier(world)
    from paper_2603_22902_gb300 import lbm
    prec = args.precision if args.precision != "fp64" or args.batch_fp64 else "fp16s"
    cases = W.batch_sweep()
    cells = sum(c.cells for c in cases)
    stream = torch.cuda.current_stream()
    solvers = [lbm.Solver(c, precision=prec).set_fields() for c in cases]
    batch = lbm.Batch(solvers)
    t0 = time.perf_counter()
    if args.batch_mode:
        batch.set_plan(mode=args.batch_mode, tiles=[(32, 8)] * lbm.BATCH_CLASSES)
        plan = batch.plan.as_dict()
    else:
        plan = batch.autotune(trial_steps=args.batch_chunk) if args.autotune else batch.plan.as_dict()
    tune_s = time.perf_counter() - t0
    chunk = args.batch_chunk
    calls = max(1, args.steps // chunk)
    for _ in range(max(1, args.warmup // chunk)):
        batch.step(chunk)
    batch.sync()
    barrier(world)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(calls)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(calls)]
    clocks = ClockSampler(local, args.clocks_dir)
    clocks.start()
    torch.cuda.synchronize()
    barrier(world)
    t_wall0 = time.perf_counter()
    for k in range(calls):
        starts[k].record(stream)
        batch.step(chunk)
        ends[k].record(stream)
    batch.sync()
    t_wall = time.perf_counter() - t_wall0
    barrier(world)
    clk = clocks.stop()
    t_ms = sum(a.elapsed_time(b) for a, b in zip(starts, ends))
    t_ms_max = reduce_max(t_ms, world)
    steps = calls * chunk
    nonfinite = sum(s.diagnostics()["nonfinite"] for s in solvers)
    if nonfinite:
        raise SystemExit("non-finite state during the batch benchmark")
    value = world * cells * steps / (t_ms_max * 1e-3) / 1e6
    mlups_rank = cells * steps / (t_ms * 1e-3) / 1e6
    hbm_peak, peak_kind = load_peaks()
    bpl = bytes_per_lu(2, prec)
    gbs = bpl * mlups_rank * 1e6 / 1e9
    final_plan = batch.plan.as_dict()
    kinds_used = {tuple(final_plan["tile"][_class(c)]) for c in cases}
    launches = calls * len(kinds_used) if final_plan["mode"] == "persistent" else steps * len(kinds_used)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        small = next(c for c in cases if c.nx == 128)
        mlups_cpu, done, dt = time_oracle(small, 10 ** 6, budget_s=args.cpu_budget)
        cpu = {"value": round(mlups_cpu, 4), "unit": "MLUPS", "cores": 1, "kind": "oracle",
               "sample": f"{done} oracle time steps of {small.name} (FP64, {dt:.1f} s), one host thread"}
    for s in solvers:
        s.close()
    batch.close()
    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 2), "unit": "MLUPS", "n_gpus": world, "steps": steps,
            "warmup": args.warmup, "ms_per_step": round(t_ms_max / steps, 5), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp64": "f64", "fp32": "f32", "fp16s": "f16-storage/f32", "bf16s": "bf16-storage/f32"}[prec],
            "data": "synthetic",
            "config": {"workload": f"batch_sweep_256 ({len(cases)} sessile drops, sides 128-512, seed 4)",
                       "cells": cells, "N": 2, "precision": prec, "steps_per_call": chunk,
                       "l2": "not flushed: the state (%.1f GB) is far larger than L2" % (2 * cells * bpl / 2 / 1e9),
                       "timing": "CUDA events per call", "parallelism": "replicas" if world > 1 else "single GPU"},
            "plan": final_plan, "autotune_s": round(tune_s, 2),
            "roofline": {"bound": "hbm", "achieved": round(gbs, 1), "peak": hbm_peak, "unit": "GB/s",
                         "frac": round(gbs / hbm_peak, 4), "traffic": None, "peak_kind": f"{peak_kind} (copy bandwidth)",
                         "bytes_per_lu": bpl, "lu_per_call": cells * chunk},
            "cpu_baseline": cpu, "e2e": None, "gpu_launches": launches, "clocks": clk,
            "wall_s_timed_loop": round(t_wall, 4),
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def _class(case):
    n = case.cells
    return 0 if n <= 128 * 128 else 1 if n <= 256 * 256 else 2 if n <= 384 * 384 else 3


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="sessile_drop_512")
    ap.add_argument("--precision", default="fp64")
    ap.add_argument("--tile", type=int, nargs=2, default=None)
    ap.add_argument("--e2e-steps", type=int, default=100)
    ap.add_argument("--compare", default="fp16s,df64",
                    help="comma-separated policies timed beside fp64 ('none' to skip)")
    ap.add_argument("--front-steps", type=int, default=20000)
    ap.add_argument("--batch-chunk", type=int, default=10, help="steps per batch call (batch_sweep_256)")
    ap.add_argument("--batch-fp64", action="store_true", help="run the batch sweep in FP64")
    ap.add_argument("--no-autotune", dest="autotune", action="store_false")
    ap.add_argument("--batch-mode", default=None, choices=["persistent", "per_step", "staged"],
                    help="batch_sweep_256: this launch form with 32x8 tiles instead of the autotuner's plan")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--ref-budget", type=float, default=120.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--extras", default="compound,staged,batch,adjoint",
                    help="other configurations timed beside the headline ('none' to skip)")
    ap.add_argument("--clocks-dir", default=None, help="directory for the raw nvidia-smi clock samples")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch_sweep_256":
        return run_batch(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
