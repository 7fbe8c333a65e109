#!/usr/bin/env python3
"""LES cell-steps/s on one GB300 (arXiv 2301.04698 hot path), as one JSON line.

A step is one full time step of the iterative predictor-corrector scheme:
thermodynamics, K = 3 sub-iterations of (scalar predictor, momentum predictor
and Poisson right side, Poisson solve, correction).  Default workload: the
largest single-GPU configuration, the dry Taylor-Green box tiled to
1536 x 1536 x 256 nodes (604 M cells), FP32 fields with FP64 reductions, CG to
1e-6 relative residual.

Legs of one run:
  value    device time of exactly --steps steps (CUDA events on the library's
           stream; L2 flushed by a 256 MiB write before every timed step,
           outside the events; the large workload's fields are each larger
           than L2 anyway), inputs resident in HBM;
  e2e      steps through the C ABI with host buffers: every step starts from
           the state held in pinned host memory, uploaded on a copy stream
           while the step before runs (les_prefetch_states), and reads the
           FP64 diagnostics back;
  roofline the kernel with the largest share of device time in a profiled
           pass of the same steps (event pair around every launch):
           algorithmic bytes per launch / mean launch time vs measured HBM
           peak; every kernel's fraction is in `kernels`;
  second_record  the moist capped boundary layer 128 x 128 x 96 (its rate over
           --steps steps and over its whole 1000-step run from the seeded
           state);
  cpu_baseline (rank 0, N = 1) the FP64 oracle on a bounded sample.
--impl reference times the oracle alone (the reference arm of this build).
--poisson-only times single Poisson solves on a chosen grid (for profiling a
CG kernel).  Under torchrun each rank runs an independent replica (different
seed): weak scaling with no collective on the data path; timing is max over
ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "LES cell-steps/s on 1 GB300; Poisson ms/step at fixed residual, learned vs plain"
UNIT = "cell-steps/s"


def workload(name: str, seed: int, grid=None):
    from paper_2301_04698_gb300 import inputs
    if name == "cbl128":
        return inputs.cbl(128, 128, 96, seed=seed, precision=32)
    if name == "tgv32":
        return inputs.tgv(32, seed=seed)
    if name == "tgv_large":
        return inputs.tgv(32, nxyz=grid or (1536, 1536, 256), seed=seed, precision=32, steps_tol=1e-6)
    if name == "ensemble16":
        return inputs.ensemble(16, seed=seed)
    raise SystemExit(f"unknown workload {name}")


WORKLOAD_DESC = {
    "cbl128": "moist capped boundary layer 128x128x96, dx=35 m, dz=10 m, FP32 (FP64 reductions), "
              "K=3, CG to 1e-6",
    "tgv32": "dry triply periodic Taylor-Green 32^3, FP64, K=3, CG to 1e-10",
    "tgv_large": "dry triply periodic Taylor-Green 1536x1536x256, FP32 (FP64 reductions), K=3, CG to 1e-6",
    "ensemble16": "uneven ensemble of 16 moist capped boundary layers, 64^2..192^2 x 64..128, FP32 (FP64 "
                  "reductions), seeded inversions, surface fluxes and subsidence, K=3, CG to 1e-6",
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--workload", default="tgv_large", choices=sorted(WORKLOAD_DESC))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample", default="auto", help="oracle sample: auto | full | NXxNY")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-vs-plain Poisson leg")
    ap.add_argument("--long-run", type=int, default=-1,
                    help="steps of the untimed-in-value long-run leg from the seeded state (cbl128: 1000 by "
                         "default, the configuration's run length; 0 skips it)")
    ap.add_argument("--warm", default="zero", choices=("zero", "prev"),
                    help="first guess of every Poisson solve of the timed workload")
    ap.add_argument("--advection", default="quick", choices=("quick", "weno3"),
                    help="advection scheme of the timed workload")
    ap.add_argument("--no-autotune", action="store_true", help="ensemble workload: keep the default tuning")
    ap.add_argument("--ensemble-share", type=int, default=1,
                    help="ensemble workload: cap each member's persistent CG at 1/share of the SMs so that up to "
                         "share members solve at once (1: one at a time)")
    ap.add_argument("--learned-seeds", type=int, default=20, help="training runs for the learned leg")
    ap.add_argument("--learned-train-steps", type=int, default=1500)
    ap.add_argument("--no-second-record", action="store_true",
                    help="skip the 128x128x96 capped-boundary-layer record")
    ap.add_argument("--aux-steps", type=int, default=-1,
                    help="steps of the stage-breakdown, profiled and end-to-end legs (default: --steps, at most 3 / "
                         "3 / 5 on grids above 100 M cells)")
    ap.add_argument("--fma-peak", action="store_true",
                    help="measure the device's FP32 and FP64 FMA rates (the ALU bounds)")
    # single Poisson solves (profiling a CG kernel)
    ap.add_argument("--poisson-only", action="store_true",
                    help="time single Poisson solves of a seeded right side instead of steps")
    ap.add_argument("--grid", default=None,
                    help="NXxNYxNZ: the --poisson-only grid (walls in z, default 512x512x64), or another grid for "
                         "--workload tgv_large (profiling a smaller tiling of the same box)")
    ap.add_argument("--variant", type=int, default=0, help="--poisson-only: les_tuning.cg_variant")
    ap.add_argument("--resident", type=int, default=1,
                    help="--poisson-only: les_tuning.cg_resident (0: on chip when the grid fits, 1: streams, "
                         "2: on chip with every vector in shared memory)")
    ap.add_argument("--iters", type=int, default=20, help="--poisson-only: CG iterations (tolerance unreachable)")
    ap.add_argument("--repeat", type=int, default=2, help="--poisson-only: solves")
    ap.add_argument("--fp64", action="store_true", help="--poisson-only: FP64 fields")
    ap.add_argument("--max-blocks", type=int, default=0,
                    help="--poisson-only: les_tuning.cg_max_blocks (0: the library's choice, all SMs)")
    ap.add_argument("--stencil-path", type=int, default=-1,
                    help="les_tuning.stencil_path of the timed workload (-1: the library's default)")
    ap.add_argument("--oracle-one-thread", type=int, default=0, metavar="SIDE",
                    help="internal: time one oracle step of a SIDE x SIDE full-column sample in this process and "
                         "print {value, secs} (the single-thread leg of cpu_baseline runs it with OMP_NUM_THREADS=1)")
    return ap.parse_args()


# ---------------------------------------------------------------------------
def dist_setup(n):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    elif torch.cuda.is_available():
        torch.cuda.set_device(0)
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def allmax(world, x: float, device: str = "cuda") -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class Clocks:
    """nvidia-smi clock / throttle sampling during the timed region.  The
    sampler is started, and its first sample awaited, before the region;
    mark() brackets the region and stop() keeps the samples stamped inside
    it (or the one nearest to it when the region is shorter than the
    sampling interval)."""

    def __init__(self, gpu_index: int):
        self.proc = None
        self.t = [None, None]
        fd, self.path = tempfile.mkstemp(prefix="les_clocks_", suffix=".csv")
        os.close(fd)
        q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={gpu_index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
            return
        t_end = time.time() + 5.0
        while time.time() < t_end and os.path.getsize(self.path) == 0 and self.proc.poll() is None:
            time.sleep(0.02)

    def mark(self, which: int) -> None:
        self.t[which] = time.time()

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        import datetime
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 10:
                continue
            try:
                ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                rows.append((ts, float(parts[2]), float(parts[3]), parts[6:10]))
            except ValueError:
                continue
        try:
            os.remove(self.path)
        except OSError:
            pass
        if not rows:
            return None
        t0, t1 = self.t
        inside = [r for r in rows if t0 is not None and t1 is not None and t0 <= r[0] <= t1]
        if not inside and t0 is not None and t1 is not None:
            mid = 0.5 * (t0 + t1)
            inside = [min(rows, key=lambda r: abs(r[0] - mid))]
        use = inside or rows
        sm = [r[1] for r in use]
        mx = max(r[2] for r in use)
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({names[i] for r in use for i, v in enumerate(r[3]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": reasons, "samples": len(use),
                "samples_in_region": len([r for r in use if t0 is not None and t1 is not None and t0 <= r[0] <= t1])}


# the source files whose change invalidates a kernel's DRAM-traffic record
TRAFFIC_SOURCES = {
    "cg_wave": ("les_cg_wave.cu", "les_gridsync.cuh", "les_common.cuh"),
    "cg_regs": ("les_cg_regs.cu", "les_gridsync.cuh", "les_common.cuh"),
    "scalar": ("les_predict_col.cu", "les_common.cuh"),
    "momentum": ("les_predict_col.cu", "les_common.cuh"),
    "rhs": ("les_stencil_col.cu",),
    "correct": ("les_stencil_col.cu",),
}


def src_hash(files) -> str:
    h = hashlib.sha256()
    cs = os.path.join(ROOT, "paper_2301_04698_gb300", "csrc")
    for f in files:
        h.update(open(os.path.join(cs, f), "rb").read())
    return h.hexdigest()[:16]


def traffic_for(kernel: str, units: float):
    """DRAM bytes of one launch of `kernel` processing `units` (cells, or
    cell-iterations for a CG solve), from the per-unit figure of an ncu
    capture in profiles/traffic.json -- None when there is no record or the
    kernel's source has changed since it was taken."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    try:
        d = json.load(open(p))
        ent = d.get(kernel)
        if not ent or ent.get("src") != src_hash(ent["files"]):
            return None
        return float(ent["dram_bytes_per_unit"]) * float(units)
    except Exception:
        return None


def traffic_capture(kernel: str) -> str:
    """Where the per-unit DRAM figure of `kernel` comes from (the captured grid)."""
    try:
        ent = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))[kernel]
        grid = "x".join(str(v) for v in ent["capture"]["grid"])
        return (f"profiles/traffic.json: DRAM bytes per {ent['per']} of an ncu capture on {grid}, scaled to this "
                "launch's units")
    except Exception:
        return "no record"


# ---------------------------------------------------------------------------
def oracle_sample(case, args, budget=2.0e6, side=None):
    """A bounded sample of the workload for the FP64 oracle: the same physics
    on the full column height over a horizontal sub-domain of at most
    `budget` cells (or `side` x `side` columns).  Sides are halved from the
    full grid, so a Taylor-Green tiling keeps whole periods."""
    if args.cpu_sample == "full":
        return case, "full domain"
    if args.cpu_sample not in ("auto",):
        sx, sy = (int(v) for v in args.cpu_sample.lower().split("x"))
    elif side is not None:
        sx, sy = min(side, case.nx), min(side, case.ny)
    else:
        sx, sy = case.nx, case.ny
        while sx * sy * case.nz > budget and sx > 16:
            sx //= 2
            sy //= 2
    if sx == case.nx and sy == case.ny:
        return case, "full domain"
    sub = case.replace(nx=sx, ny=sy, name=case.name + f"_sub{sx}x{sy}")
    return sub, f"{sx}x{sy}x{case.nz} horizontal sub-domain (full columns) of the same workload"


def time_oracle(case, steps: int, warm: int):
    from oracle import Oracle
    from paper_2301_04698_gb300 import inputs
    o = Oracle(case, inputs.initial_state(case))
    if warm:
        o.step(warm)
    t0 = time.perf_counter()
    o.step(steps)
    dt = time.perf_counter() - t0
    return case.n * steps / dt, dt


def oracle_one_thread(args, side: int):
    """The oracle on one host core: a child process with OMP_NUM_THREADS=1
    times one step of a side x side full-column sample; (value, secs, desc)."""
    import subprocess
    env = dict(os.environ, OMP_NUM_THREADS="1")
    cmd = [sys.executable, os.path.abspath(__file__), "--workload", args.workload, "--oracle-one-thread", str(side)]
    out = subprocess.run(cmd, env=env, capture_output=True, text=True, timeout=600)
    if out.returncode != 0:
        return None
    r = json.loads(out.stdout.strip().splitlines()[-1])
    return r["value"], r["secs"], r["sample"]


def cores():
    n = os.environ.get("OMP_NUM_THREADS")
    return int(n) if n else (os.cpu_count() or 1)


def reference_arm(args, rank, world):
    if rank != 0:
        return 0
    case = workload(args.workload, 1)
    if args.warm != case.warm:
        case = case.replace(warm=args.warm)
    if args.advection != case.advection:
        case = case.replace(advection=args.advection)
    # each of the W + K oracle steps is a bounded sample so the arm ends in
    # minutes: 64 x 64 full columns of the large box (1 M cells), ~0.4 M cells
    # of the others
    if case.n > 1e8:
        sample, desc = oracle_sample(case, args, side=64)
    else:
        sample, desc = oracle_sample(case, args, budget=4.0e5)
    val, secs = time_oracle(sample, args.steps, args.warmup)
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / max(args.steps, 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD_DESC[args.workload], "sample": desc},
        "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores(), "kind": "oracle", "sample": desc},
        "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def fma_peak(args):
    """The FP32 and FP64 FMA rates of the device (les_measure_fma), three
    times each, with the FP32 issue rate they imply: one warp instruction
    retires 32 FMAs."""
    import torch

    from paper_2301_04698_gb300 import build as B
    from paper_2301_04698_gb300 import les
    B.build()
    les.load_library()
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    nsm = props.multi_processor_count
    clk = (json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))).get("sm_max_mhz")
           if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else None) or 2070.0
    clocks = Clocks(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.mark(0)
    fp32 = [les.measure_fma(32, 10000) for _ in range(3)]
    fp64 = [les.measure_fma(64, 200) for _ in range(3)]
    clocks.mark(1)
    b32 = max(r["tflops"] for r in fp32)
    b64 = max(r["tflops"] for r in fp64)
    print(json.dumps({"fp32_fma_tflops": b32, "fp64_fma_tflops": b64, "fp32_runs": fp32, "fp64_runs": fp64,
                      "sms": nsm, "sm_max_mhz": clk,
                      "fp32_fma_per_sm_per_clk_at_max": b32 * 1e12 / 2 / nsm / (clk * 1e6),
                      "fp32_warp_instr_per_sm_per_clk_at_max": b32 * 1e12 / 2 / 32 / nsm / (clk * 1e6),
                      "fp64_fma_per_sm_per_clk_at_max": b64 * 1e12 / 2 / nsm / (clk * 1e6),
                      "clocks": clocks.stop()}), flush=True)
    return 0


def poisson_only(args):
    """Single Poisson solves of a seeded uniform right side through the public
    API (Sec. 2.4: L_c psi = b, CG), one JSON line per solve: iterations, the
    relative residual reached and the CUDA-event time.  Walls in z; the
    tolerance is unreachable so every solve runs --iters iterations."""
    import torch

    from paper_2301_04698_gb300 import build as B
    from paper_2301_04698_gb300 import inputs, les
    B.build()
    les.load_library()
    nx, ny, nz = (int(v) for v in (args.grid or "512x512x64").lower().split("x"))
    prec = 64 if args.fp64 else 32
    case = inputs.Case(name="poisson", nx=nx, ny=ny, nz=nz, dx=35.0, dy=35.0, dz=10.0, walls=True,
                       precision=prec, init="zero", physics=())
    sim = les.Simulation(case)
    sim.set_tuning(cg_variant=args.variant, cg_resident=args.resident)
    if args.max_blocks > 0:
        sim.set_tuning(cg_max_blocks=args.max_blocks)
    dt = torch.float64 if prec == 64 else torch.float32
    b = torch.from_numpy(inputs.uniform(1, 0, case.n, -1, 1).reshape(case.shape)).to("cuda", dt)
    for _ in range(args.repeat):
        x = torch.zeros_like(b)
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record()
        rc, it, rel = sim.poisson_solve(b, x, 1e-30, args.iters, allow_not_converged=True)
        t1.record()
        t1.synchronize()
        print(json.dumps({"grid": [nx, ny, nz], "precision": prec, "variant": args.variant,
                          "resident": args.resident, "max_blocks": args.max_blocks, "iters": it, "rel": rel,
                          "ms": t0.elapsed_time(t1)}),
              flush=True)
    sim.close()
    return 0


# ---------------------------------------------------------------------------
def bench_ensemble(args, rank, world, local):
    """The uneven ensemble: every member tuned by the autotuner, the
    ensemble's mode (members stepped together through les_ensemble_step, or
    one after another) chosen by timing both; whole-job cell-steps/s over
    wall time bracketed by device synchronisation (the members run on their
    own streams)."""
    import torch

    from paper_2301_04698_gb300 import inputs, les
    cases = workload(args.workload, seed=1 + rank)
    ens = les.Ensemble(cases, share=args.ensemble_share)
    ens.set_states([inputs.initial_state(c) for c in cases])
    tuned = []
    for m in ens.members:
        if args.no_autotune:
            tuned.append(None)
        else:
            tuned.append(les.autotune(m)["tuning"])
        if args.ensemble_share > 1:   # the share's cap wins over a tuned one
            nsm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
            m.set_tuning(cg_max_blocks=max(1, nsm // args.ensemble_share))
    # stepped together or one member after another, whichever is faster
    mode = None if args.no_autotune else ens.tune()
    for _ in range(args.warmup):
        ens.step(1, allow_not_converged=True)
    torch.cuda.synchronize()
    # the members' states at the start of the timed steps, so that the steps
    # one member after another below start from the same states
    fields = ("u", "v", "w", "p", "theta_l", "q_t")
    snaps = [({k: m.view(k).clone() for k in fields}, m.dt) for m in ens.members]
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    clocks = Clocks(local)
    launches0 = sum(m.launch_count() for m in ens.members)
    total_s = 0.0
    iters = 0
    barrier(world)
    clocks.mark(0)
    for s in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st = ens.step(1, allow_not_converged=True)
        torch.cuda.synchronize()
        total_s += time.perf_counter() - t0
        iters += sum(x["iters_total"] for x in st)
    clocks.mark(1)
    barrier(world)
    clk = clocks.stop()
    total_s = allmax(world, total_s)
    launches = sum(m.launch_count() for m in ens.members) - launches0
    # the same steps member after member from the same states, for the gain of
    # stepping them together
    torch.cuda.synchronize()
    for m, (snap, dt) in zip(ens.members, snaps):
        for k in fields:
            m.view(k).copy_(snap[k])
        if dt:
            m.dt = dt
    torch.cuda.synchronize()
    seq_s = 0.0
    for s in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for m in ens.members:
            m.step(1, allow_not_converged=True)
        torch.cuda.synchronize()
        seq_s += time.perf_counter() - t0
    value = world * ens.cells * args.steps / total_s
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD_DESC[args.workload], "members": [c.name for c in cases],
                       "cells": ens.cells, "K": cases[0].K, "tol": cases[0].tol,
                       "timing": "wall clock between device synchronisations (members on their own streams)",
                       "l2": "flushed (256 MiB write) before every timed step", "autotuned": tuned,
                       "mode": "together" if ens.together else "one after another",
                       "share": args.ensemble_share},
            "roofline": None, "cpu_baseline": None, "e2e": None, "gpu_launches": launches, "clocks": clk,
            "poisson": {"iters_per_step": iters / args.steps},
            "one_after_another_ms_per_step": 1e3 * seq_s / args.steps,
            "ensemble_mode": ("together" if ens.together else "one after another"),
            "mode_choice": mode,
        }
        print(json.dumps(line), flush=True)
    ens.close()
    return 0


def timed_steps(sim, case, steps, flush, stream, world, local):
    """Exactly `steps` steps bracketed by CUDA events on the library's stream,
    L2 flushed before each (outside the events); clocks sampled meanwhile."""
    import torch
    launches0 = sim.launch_count()
    clocks = Clocks(local)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    iters = nc = 0
    barrier(world)
    torch.cuda.synchronize()
    clocks.mark(0)
    wall0 = time.perf_counter()
    with torch.cuda.stream(stream):
        for s in range(steps):
            flush.zero_()
            ev[s][0].record(stream)
            r = sim.step(1, allow_not_converged=True)
            ev[s][1].record(stream)
            iters += r["iters_total"]
            nc += r["not_converged"]
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    clocks.mark(1)
    barrier(world)
    clk = clocks.stop()
    dev_ms = allmax(world, sum(a.elapsed_time(b) for a, b in ev))
    return {"dev_ms": dev_ms, "iters": iters, "not_converged": nc, "wall": wall, "clocks": clk,
            "launches": sim.launch_count() - launches0}


def long_run(case, nlong, chunk=50):
    """The configuration's whole run from the seeded state, CUDA events around
    chunks of steps (no L2 flush): mean cell-steps/s and CG iterations."""
    import torch

    from paper_2301_04698_gb300 import inputs, les
    lsim = les.Simulation(case)
    lsim.set_state(inputs.initial_state(case))
    done, iters_l, nc_l, ms_l = 0, 0, 0, 0.0
    while done < nlong:
        n = min(chunk, nlong - done)
        ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ea.record(lsim.stream)
        st = lsim.step(n, allow_not_converged=True)
        eb.record(lsim.stream)
        eb.synchronize()
        ms_l += ea.elapsed_time(eb)
        iters_l += st["iters_total"]
        nc_l += st["not_converged"]
        done += n
    d = lsim.diagnostics()
    lsim.close()
    return {"steps": nlong, "value": case.n * nlong / (ms_l / 1e3), "unit": UNIT, "ms_per_step": ms_l / nlong,
            "iters_per_step": iters_l / nlong, "not_converged": nc_l, "nonfinite": d["nonfinite"],
            "max_cfl_end": d["max_cfl"],
            "note": f"every step from the seeded state, CUDA events around chunks of {chunk} steps, no L2 flush"}


def second_record(args, rank, world, local, flush):
    """The moist capped boundary layer (128 x 128 x 96, FP32): its rate over
    the timed steps after the warm-up, and over its whole 1000-step run."""
    import torch

    from paper_2301_04698_gb300 import inputs, les
    case = workload("cbl128", seed=1 + rank)
    sim = les.Simulation(case)
    sim.set_state(inputs.initial_state(case))
    with torch.cuda.stream(sim.stream):
        for _ in range(args.warmup):
            sim.step(1, allow_not_converged=True)
    torch.cuda.synchronize()
    steps = max(args.steps, 10)
    t = timed_steps(sim, case, steps, flush, sim.stream, world, local)
    sim.close()
    rec = {"workload": WORKLOAD_DESC["cbl128"], "steps": steps, "warmup": args.warmup,
           "value": world * case.n * steps / (t["dev_ms"] / 1e3), "unit": UNIT,
           "ms_per_step": t["dev_ms"] / steps, "iters_per_step": t["iters"] / steps}
    if world == 1 and args.long_run != 0:
        rec["long_run"] = long_run(case, args.long_run if args.long_run > 0 else 1000)
    return rec


def main():
    args = parse()
    if args.poisson_only:
        return poisson_only(args)
    if args.fma_peak:
        return fma_peak(args)
    if args.oracle_one_thread:
        case = workload(args.workload, 1)
        sample, desc = oracle_sample(case, args, side=args.oracle_one_thread)
        val, secs = time_oracle(sample, 1, 0)
        print(json.dumps({"value": val, "secs": secs, "sample": desc}), flush=True)
        return 0
    rank, world, local = dist_setup(args.gpus)
    if args.impl == "reference":
        rc = reference_arm(args, rank, world)
        barrier(world)
        return rc

    import torch

    from paper_2301_04698_gb300 import build as B
    from paper_2301_04698_gb300 import inputs, les
    if rank == 0:
        B.build()
    barrier(world)
    les.load_library()

    if args.workload == "ensemble16":
        return bench_ensemble(args, rank, world, local)

    grid = tuple(int(v) for v in args.grid.lower().split("x")) if args.grid else None
    if grid is not None and args.workload != "tgv_large":
        raise SystemExit("--grid applies to --workload tgv_large (or --poisson-only)")
    case = workload(args.workload, seed=1 + rank, grid=grid)
    if args.warm != case.warm:
        case = case.replace(warm=args.warm)
    if args.advection != case.advection:
        case = case.replace(advection=args.advection)
    big = case.n > 1e8
    aux = args.aux_steps if args.aux_steps > 0 else None
    aux_prof = aux or (min(args.steps, 3) if big else args.steps)
    aux_e2e = aux or (min(args.steps, 3) if big else args.steps)
    st0 = inputs.initial_state(case)
    sim = les.Simulation(case)
    if args.stencil_path >= 0:
        sim.set_tuning(stencil_path=args.stencil_path)
    sim.set_state(st0)
    del st0
    stream = sim.stream
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")   # 256 MiB > L2

    # warm-up (also fixes dt when it comes from the Courant number)
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            sim.step(1, allow_not_converged=True)
    torch.cuda.synchronize()
    names = ("u", "v", "w", "p", "theta_l", "q_t")
    snap = {k: sim.view(k).clone() for k in names}

    # ---- timed region: exactly --steps steps ------------------------------
    t = timed_steps(sim, case, args.steps, flush, stream, world, local)
    dev_ms = t["dev_ms"]
    value = world * case.n * args.steps / (dev_ms / 1e3)

    # ---- stage breakdown (Poisson ms / step) -------------------------------
    for k in names:
        sim.view(k).copy_(snap[k])
    stage_ms = {"begin": 0.0, "scalar": 0.0, "momentum": 0.0, "solve": 0.0, "correct": 0.0}
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        for s in range(aux_prof):
            flush.zero_()
            for stg in ["begin"] + ["scalar", "momentum", "solve", "correct"] * case.K + ["end"]:
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                sim.stage(stg, allow_not_converged=True)
                b.record(stream)
                b.synchronize()
                if stg in stage_ms:
                    stage_ms[stg] += a.elapsed_time(b)
    stage_ms = {k: v / aux_prof for k, v in stage_ms.items()}

    # ---- per-kernel profile of the same steps -------------------------------
    for k in names:
        sim.view(k).copy_(snap[k])
    sim.profile_reset()
    sim.profile(True)
    torch.cuda.synchronize()
    prof_iters = 0
    with torch.cuda.stream(stream):
        for s in range(aux_prof):
            flush.zero_()
            prof_iters += sim.step(1, allow_not_converged=True)["iters_total"]
    kstats = sim.profile_read()
    sim.profile(False)
    total_k = sum(k["total_ms"] for k in kstats) or 1.0
    top = max(kstats, key=lambda k: k["total_ms"])
    hbm, peak_kind = peaks()
    mean_ms = top["total_ms"] / max(top["timed"], 1)
    achieved = top["bytes_per_launch"] / (mean_ms / 1e3) / 1e9
    # units of one launch of the top kernel for its traffic record: cells, or
    # cell-iterations for a CG solve (the profiled steps' mean per solve)
    top_units = case.n * (prof_iters / max(top["launches"], 1) if top["name"].startswith("cg") else 1.0)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                "traffic": traffic_for(top["name"], top_units), "kernel": top["name"],
                "share": top["total_ms"] / total_k, "mean_launch_us": mean_ms * 1e3,
                "bytes_per_launch": top["bytes_per_launch"], "peak_source": f"{peak_kind} (MEASURED_PEAKS.json)"
                if peak_kind == "measured" else "fallback 6.8 TB/s",
                "frac_of_8tbs": achieved / 8000.0, "profiled_steps": aux_prof,
                "traffic_source": traffic_capture(top["name"])}
    if top["name"] in ("cg_regs", "cg_resident"):
        roofline["note"] = ("an on-chip CG: achieved counts the solve's algorithmic bytes, which stay in registers "
                            "and shared memory; its DRAM bytes are `traffic`, and the iteration time is set by the "
                            "grid sums' latency, not by HBM")
    kernels = {}
    for k in kstats:
        mean = k["total_ms"] / max(k["timed"], 1)
        gbs = k["bytes_per_launch"] / (mean / 1e3) / 1e9 if k["total_ms"] > 0 else None
        units = case.n * (prof_iters / max(k["launches"], 1) if k["name"].startswith("cg") else 1.0)
        tr = traffic_for(k["name"], units)
        kernels[k["name"]] = {"launches": k["launches"], "ms": round(k["total_ms"], 4),
                              "share": round(k["total_ms"] / total_k, 4), "mean_us": round(mean * 1e3, 2),
                              "gbs": round(gbs, 1) if gbs else None,
                              "frac": round(gbs / hbm, 4) if gbs else None,
                              "bytes_per_launch": k["bytes_per_launch"],
                              "traffic_per_launch": round(tr) if tr else None}

    # ---- end to end through the C ABI with host buffers ----------------------
    # The same steps as the timed region, each from its input state held in
    # pinned host memory (gathered beforehand by stepping from the snapshot):
    # every upload (les_prefetch_states, pinned host -> staging buffer on a
    # copy stream) is enqueued before the previous step runs and overlaps it;
    # BEGIN takes the staged state; the diagnostics come back after every step.
    for k in names:
        sim.view(k).copy_(snap[k])
    del snap
    hosts = []
    for s in range(aux_e2e):
        torch.cuda.synchronize()
        hosts.append({k: sim.view(k).cpu().pin_memory() for k in names})
        if s + 1 < aux_e2e:
            with torch.cuda.stream(stream):
                sim.step(1, allow_not_converged=True)
    h2d = sum(h.numel() * h.element_size() for h in hosts[0].values())
    staging = [torch.empty(h2d, dtype=torch.uint8, device="cuda") for _ in range(2)]
    copy_stream = torch.cuda.Stream()
    torch.cuda.synchronize()
    barrier(world)
    parts = [0.0, 0.0, 0.0]  # enqueue the upload, step, diagnostics read-back (host clocks)
    e2e_iters = 0
    eva = [torch.cuda.Event(enable_timing=True) for _ in range(aux_e2e)]
    evb = [torch.cuda.Event(enable_timing=True) for _ in range(aux_e2e)]
    cpa = [torch.cuda.Event(enable_timing=True) for _ in range(aux_e2e)]
    cpb = [torch.cuda.Event(enable_timing=True) for _ in range(aux_e2e)]

    def upload(s):
        cpa[s].record(copy_stream)
        sim.prefetch_from_host(hosts[s], staging[s % 2], copy_stream)
        cpb[s].record(copy_stream)

    t0 = time.perf_counter()
    upload(0)
    for s in range(aux_e2e):
        ta = time.perf_counter()
        if s + 1 < aux_e2e:
            upload(s + 1)
        tb = time.perf_counter()
        with torch.cuda.stream(stream):
            eva[s].record(stream)
            e2e_iters += sim.step(1, allow_not_converged=True)["iters_total"]
            evb[s].record(stream)
        tc = time.perf_counter()
        sim.diagnostics()
        td = time.perf_counter()
        parts[0] += tb - ta
        parts[1] += tc - tb
        parts[2] += td - tc
    torch.cuda.synchronize()
    e2e_s = allmax(world, time.perf_counter() - t0)
    copy_ms = sum(x.elapsed_time(y) for x, y in zip(cpa, cpb))
    e2e = {"value": world * case.n * aux_e2e / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d,
           "d2h_bytes_per_step": les.NDIAG * 8, "steps": aux_e2e,
           "upload": "the input state of each of the first timed steps, from pinned host memory to a device "
                     "staging buffer on a copy stream (les_prefetch_states), each upload overlapping the step "
                     "before it; the first one is not overlapped",
           "ms_per_step": {"enqueue_upload": 1e3 * parts[0] / aux_e2e, "step": 1e3 * parts[1] / aux_e2e,
                           "diagnostics": 1e3 * parts[2] / aux_e2e,
                           "step_on_device": sum(x.elapsed_time(y) for x, y in zip(eva, evb)) / aux_e2e,
                           "upload_on_copy_stream": copy_ms / aux_e2e},
           "h2d_gbs": h2d * aux_e2e / max(copy_ms / 1e3, 1e-12) / 1e9,
           "iters_per_step": e2e_iters / aux_e2e}
    del hosts, staging
    sim.close()
    del flush
    torch.cuda.empty_cache()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")

    # ---- Poisson ms/step at a fixed residual: learned vs plain first guesses ----
    learned = None
    if rank == 0 and not args.no_learned:
        from paper_2301_04698_gb300 import learned as L
        t0 = time.perf_counter()
        Bp, Pp = L.generate_pairs(list(range(100, 100 + args.learned_seeds)), 50, n=32)
        nval = 16
        model = les.UNet(32, max_batch=16)
        model.set_weights(L.init_weights(0))
        model.set_loss("energy")
        model.out_scale = L.output_scale(Bp[nval:], Pp[nval:])
        hist, t_train = L.train(model, Bp[nval:], Pp[nval:], steps=args.learned_train_steps, batch=16)
        ev = L.evaluate(model, [1, 2], steps=10, n=32, tol=1e-6)
        learned = {"workload": "Taylor-Green 32^3, FP64, K=3, CG to 1e-6 relative residual, held-out seeds 1-2",
                   "loss": "energy norm of the error", "pairs": int(Bp.shape[0]),
                   "train_steps": args.learned_train_steps, "train_s": t_train,
                   "leg_s": time.perf_counter() - t0, "val_rel_err": L.relative_error(model, Bp[:nval], Pp[:nval]),
                   **ev}
        del Bp, Pp, model

    # ---- the configuration's full run from the seeded state (on request) ------
    long_main = None
    nlong = args.long_run if args.long_run >= 0 else (1000 if args.workload == "cbl128" else 0)
    if rank == 0 and world == 1 and nlong > 0:
        long_main = long_run(case, nlong)

    # ---- second record: the moist capped boundary layer ------------------------
    second = None
    if args.workload != "cbl128" and not args.no_second_record:
        second = second_record(args, rank, world, local, flush)

    # ---- CPU oracle baseline ---------------------------------------------------
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # the large box: 128 x 128 full columns (4 x 4 x 8 Taylor-Green
        # periods, 4.2 M cells, ~15 s on 16 cores); others: at most 2 M cells
        sample, desc = oracle_sample(case, args, side=128) if big else oracle_sample(case, args)
        val, secs = time_oracle(sample, 1, 0)
        cpu = {"value": val, "unit": UNIT, "cores": cores(), "kind": "oracle",
               "sample": f"1 step of the {desc} (FP64, {secs:.1f} s)"}
        # and on one core (a smaller sample of about the same time)
        one = oracle_one_thread(args, 32 if big else 16)
        if one is not None:
            cpu["one_core"] = {"value": one[0], "cores": 1,
                               "sample": f"1 step of the {one[2]} (FP64, {one[1]:.1f} s)"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dev_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32" if case.precision == 32 else "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD_DESC[args.workload] if grid is None else
                       f"dry triply periodic Taylor-Green {case.nx}x{case.ny}x{case.nz}, FP32 (FP64 reductions), K=3, "
                       "CG to 1e-6", "grid": [case.nx, case.ny, case.nz],
                       "cells": case.n, "K": case.K, "solver": case.solver, "tol": case.tol,
                       "warm_start": case.warm, "advection": case.advection,
                       "l2": "flushed (256 MiB write) before every timed step"
                             + ("; every field (2.4 GB) is also larger than L2" if big else ""),
                       "replicas": world, "seed": 1},
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": t["launches"],
            "clocks": t["clocks"],
            "poisson": {"ms_per_step": stage_ms["solve"], "iters_per_step": t["iters"] / args.steps,
                        "not_converged": t["not_converged"], "warm_start": case.warm, "tol": case.tol,
                        "learned_vs_plain": learned},
            "stage_ms_per_step": stage_ms,
            "long_run": long_main,
            "kernels": kernels,
            "second_record": second,
            "wall_s_timed": t["wall"],
        }
        print(json.dumps(line), flush=True)
    barrier(world)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
