#!/usr/bin/env python
"""Benchmark of the SCR-FGMRES + AMG path on one GB300 (or N replicas).

One step = the whole linear-solver path of one Newton step:

  scr_setup  (upload of A, B, C, D into the solver layout, Shat = D - C
              diag(A)^{-1} B, AMG hierarchies of A and Shat)
  scr_solve  (FGMRES + SCR to ||b - calA x|| / ||b|| <= 1e-8, FP64 check)
  mm_setup + mm_solve  (mesh-motion AMG hierarchy, CG to 1e-8)

Lines of the default run (all on one GPU, inputs resident in HBM):

- headline `value`: the refined straight tube (96 circ x (11 lumen + 5 wall)
  rings x 400 axial layers: 616,337 nodes, 2,503,844 block unknowns, 423,857
  mesh nodes) with the FP64 preconditioner, --steps timed steps;
- `mixed`: the same step with the FP32 / BF16 preconditioner (FP64 outer);
- `e2e`: the FP64 step through host pinned buffers (every matrix and
  right-hand side copied in, both solutions copied out);
- `stenosis`: the stenosed tube (160 x (13 + 7) x 600, 50% area at
  mid-length: 1,923,801 nodes, 7,791,364 unknowns), FP64 and mixed steps;
- `bifurcation`: the bifurcation (about 4M nodes, 16M unknowns) with eight
  right-hand sides (inflow peaks U(0, 60) cm/s) solved as one 8-column
  mixed-precision block solve (scr_setup + scr_solve_multi per step);
- `cpu_baseline`: the CPU oracle, timed on the host cores after the GPU legs.

Every step's matrices (1.5 GB and more) exceed the 129 MB L2, so no flush is
needed between steps.  Multi-GPU: the path does not partition a single
solve; with N ranks each rank solves its own copy of the workload
(independent problems, no collective on the data path), `scaling` = "weak".
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "tube_large"
METRIC = "SCR-FGMRES+AMG solves/s to rel-res 1e-8 (mixed vs FP64) on 1 GB300; % HBM peak"
UNIT = "solves/s"


def describe_workload(name: str) -> str:
    """Geometry of a generator preset in words (circumferential x (lumen +
    wall rings) x axial layers for the tubes; core, rings and layers for the
    bifurcation)."""
    import fsi_inputs as F
    p = F.PRESETS[name]
    kind = p.get("kind", 0)
    if kind == 2:
        return (f"bifurcation, O-grid core {p['n_circ']}x{p['n_circ']}, ({p['n_rad_f']}+{p['n_rad_s']}) rings, "
                f"{p['n_ax']} layers, daughters at +-35 degrees")
    shape = "stenosed tube" if kind == 1 else "straight tube"
    return f"{shape} {p['n_circ']}x({p['n_rad_f']}+{p['n_rad_s']})x{p['n_ax']}"


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["fp64", "mixed"], default="fp64")
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--legs", default="stenosis,bifurcation",
                    help="comma-separated larger configurations timed after the headline: stenosis (FP64 and "
                         "mixed), bifurcation (8 right-hand sides, mixed); 'none' for the headline only")
    ap.add_argument("--big-steps", type=int, default=1,
                    help="timed steps of each larger leg (after one warm-up step)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--skip-mixed", action="store_true")
    ap.add_argument("--tune-file", default=None,
                    help="autotuner decisions: loaded before the first set-up when the file exists, "
                         "written after the run otherwise (replays one run's kernel choices in another, "
                         "e.g. under a profiler whose instrumentation distorts the autotuner's timings)")
    ap.add_argument("--multi-rhs", action="store_true",
                    help="also time eight right-hand sides (inflow peaks U(0, 60) cm/s, one Jacobian) on the "
                         "headline tube solved as one 8-column block solve in mixed precision against the same "
                         "eight solved one by one")
    ap.add_argument("--assembly", action="store_true",
                    help="also time the GPU residual assembly (element loop) and one multi-corrector iteration "
                         "(residual, FP64 solve, updates) on the workload's mesh, with and without the mesh motion "
                         "solved inside it")
    ap.add_argument("--batched", action="store_true",
                    help="also time the 64-tube batched form against the same 64 tubes solved one by one, "
                         "FP64 against FP64 and mixed against mixed")
    return ap.parse_args(argv)


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


# FP64 FMA rate of GB300: 2 FP64 FMA per SM per clock (152 SMs); measured
# 0.600 TFMA/s at 1995 MHz with an independent-chain FMA loop
FP64_FMA_PER_SM_CLK = 2
N_SM = 152
# dram bytes / algorithmic bytes of the level-0 A products, from one ncu
# capture each of the scalar-row kernel with the Chebyshev-step epilogue on
# the 309k-node tube (2 lanes per scalar row; FP64 396.7 / 403.6 MB, FP32
# 206.5 / 211.4 MB: see profiles/)
TRAFFIC_RATIO = {"fp64": 396.7 / 403.6, "fp32": 206.5 / 211.4}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons every 200 ms during a timed region."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def stop(self) -> dict:
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        os.unlink(self.path)
        sm.sort()
        med = sm[len(sm) // 2] if sm else None
        return {"sm_mhz": med, "sm_max_mhz": smax, "reasons": sorted(reasons), "samples": len(sm)}


def dist_init(backend: str | None = None):
    """One process per GPU (torchrun's RANK / LOCAL_RANK / WORLD_SIZE): NCCL
    on GPUs, gloo otherwise (CPU tests of the multi-process logic)."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch
        import torch.distributed as dist
        if backend is None:
            backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend)
        pg = dist
    return world, rank, local, pg


def barrier(pg):
    if pg is not None:
        pg.barrier()


def allmax(pg, v: float, device):
    if pg is None:
        return v
    import torch
    t = torch.tensor([v], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def job_value(pg, ms_local: float, world: int, device) -> tuple[float, float]:
    """Whole-job throughput: every rank solves its own replica in its timed
    step; the job's step time is the slowest rank's, and the job completes
    `world` solves per step.  Returns (ms per step, solves per second)."""
    ms = allmax(pg, ms_local, device)
    return ms, world * 1000.0 / ms


def split_members(sizes, world: int) -> list[list[int]]:
    """Balanced split of independent problems (sizes in unknowns) over
    `world` ranks: largest first, each to the rank with the least work so
    far (ties to the lowest rank).  Returns the member indices per rank, in
    increasing order."""
    load = [0] * world
    out = [[] for _ in range(world)]
    for i in sorted(range(len(sizes)), key=lambda j: (-sizes[j], j)):
        r = min(range(world), key=lambda q: (load[q], q))
        out[r].append(i)
        load[r] += sizes[i]
    return [sorted(o) for o in out]


def roofline(kprof: dict | None, fp64: bool, clocks: dict, ms_step: float, hbm: float, peak_kind: str,
             kernel: str, kernel_code: int, captured: bool = True) -> dict | None:
    """Roofline of the level-0 A product from the library's event profiler:
    algorithmic bytes (stored values and indices once, source vector once,
    destination and epilogue vectors) and flops (2 per stored scalar) of the
    profiled launches over their summed event time.  FP64: one FMA per stored
    value binds the FP64 pipe before HBM, so the bound is "alu" against 2 FMA
    per SM per clock at the sampled SM clock, with the HBM fraction beside
    it; FP32: HBM against the measured copy bandwidth.  `traffic` scales the
    ncu DRAM/algorithmic ratio of the captured kernel (null for a kernel no
    capture covers)."""
    if not kprof or kprof["timed"] <= 0:
        return None
    per_launch_s = kprof["ms"] * 1e-3 / kprof["timed"]
    bytes_pl = kprof["bytes"] / kprof["timed"]
    flops_pl = kprof["flops"] / kprof["timed"]
    achieved_gbs = bytes_pl / per_launch_s * 1e-9
    roof = None
    if fp64:
        clk = (clocks.get("sm_mhz") or 1995.0) * 1e6
        fma_peak = FP64_FMA_PER_SM_CLK * N_SM * clk
        if flops_pl / 2.0 / fma_peak > bytes_pl / (hbm * 1e9):
            roof = {"bound": "alu", "achieved": flops_pl / per_launch_s * 1e-12, "peak": 2.0 * fma_peak * 1e-12,
                    "unit": "TFLOP/s", "frac": (flops_pl / per_launch_s) / (2.0 * fma_peak),
                    "hbm_achieved_gbs": achieved_gbs, "hbm_frac": achieved_gbs / hbm,
                    "peak_note": f"FP64 pipe: {FP64_FMA_PER_SM_CLK} FMA/SM/clk x {N_SM} SMs at the median sampled "
                                 f"SM clock; HBM {peak_kind} {hbm:.0f} GB/s"}
    if roof is None:
        roof = {"bound": "hbm", "achieved": achieved_gbs, "peak": hbm, "unit": "GB/s", "frac": achieved_gbs / hbm,
                "peak_note": f"{peak_kind} HBM copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"}
    ratio = TRAFFIC_RATIO["fp64" if fp64 else "fp32"]
    roof.update({"kernel": kernel, "kernel_code": kernel_code, "launches_per_step": kprof["launches"],
                 "timed_launches": kprof["timed"], "bytes_per_launch": bytes_pl, "us_per_launch": per_launch_s * 1e6,
                 "share_of_step": kprof["ms"] / ms_step,
                 "traffic": ratio * bytes_pl if (captured and ratio and kernel_code in (0, 102)) else None})
    if roof["traffic"] is not None:
        roof["traffic_note"] = ("ncu dram__bytes_read.sum + dram__bytes_write.sum of the same kernel on a smaller tube, "
                                "scaled to this launch by its algorithmic bytes")
    return roof


# ------------------------------------------------------------------ CPU oracle
# the oracle's timed samples: the bench tube's 96 x (11 + 5) cross-section
# with 25 layers has the full tube's outer and inner iteration counts (3 /
# about 405), so its cost per unknown is the full tube's; 10 layers serve
# the all-core run (shorter tubes need more iterations)
CPU_SAMPLE = ("tube_large", {"n_ax": 25})
CPU_SAMPLE_SMALL = ("tube_large", {"n_ax": 10})
_BLAS_ENV = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS")


def _oracle_sample(name: str, overrides: dict, want_x: bool = False):
    """One full oracle step (set-up, SCR-FGMRES, mesh AMG-CG) on a generator
    preset; returns (seconds, unknowns, outer, inner iterations) and, with
    want_x, the oracle's block solution."""
    import fsi_inputs as F
    from oracle import scr as oscr
    s = F.tube_system(name, **overrides)
    t0 = time.perf_counter()
    out = oscr.solve_system(s)
    dt = time.perf_counter() - t0
    assert out["info"].converged
    c = out["counters"]
    res = (dt, s.n, out["info"].iters, c.a_iters + c.s_iters + c.i_iters)
    return res + (out["x"],) if want_x else res


def _pool_sample(args):
    return _oracle_sample(*args)


def _oracle_in_processes(sample, nproc: int):
    """`nproc` spawned processes, each one oracle step on `sample`, at the
    same time; each process's BLAS pools are capped at one thread (set in
    the environment before the child imports numpy), so nproc processes use
    nproc cores.  Returns the per-process results."""
    import multiprocessing as mp
    saved = {k: os.environ.get(k) for k in _BLAS_ENV}
    for k in _BLAS_ENV:
        os.environ[k] = "1"
    try:
        with mp.get_context("spawn").Pool(nproc) as pool:
            return pool.map(_pool_sample, [sample] * nproc)
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


def cpu_baseline(n_full: int) -> dict:
    """The oracle on the host cores, measured in this run (every sample in
    spawned processes with one BLAS thread each, after the GPU work):
    - single thread: one oracle step on the bench tube's cross-section with
      25 layers, which needs the full tube's outer and inner iteration
      counts; the full workload's time is that time x the unknown ratio;
    - all cores: os.cpu_count() processes at once, each one oracle step on
      the 10-layer tube, against one such process alone: the aggregate
      speed-up of the host over one thread;
    `value` = the single-thread full-workload rate x that aggregate speed-up
    (independent problems on every core, as the GPU runs replicas)."""
    cores = os.cpu_count() or 1
    t1, n1, o1, i1, x1 = _oracle_in_processes(CPU_SAMPLE + (True,), 1)[0]
    t_full = t1 * n_full / n1
    ts, ns, _, _ = _oracle_in_processes(CPU_SAMPLE_SMALL, 1)[0]
    t0 = time.perf_counter()
    res = _oracle_in_processes(CPU_SAMPLE_SMALL, cores)
    wall = time.perf_counter() - t0
    per = sorted(r[0] for r in res)
    t_med = per[len(per) // 2]
    speedup = cores * ts / t_med
    return {
        "value": speedup / t_full, "unit": UNIT, "cores": cores, "kind": "oracle",
        "sample": (f"oracle steps (set-up + SCR-FGMRES + mesh CG, FP64 numpy/scipy, one BLAS thread per process): "
                   f"{n1} unknowns (the bench tube's cross-section, 25 layers; {o1} outer / {i1} inner iterations) in "
                   f"{t1:.2f} s on one thread, scaled by the unknown ratio to the {n_full}-unknown workload; "
                   f"{cores} processes at once on {ns} unknowns took {t_med:.2f} s each (median; one alone {ts:.2f} "
                   f"s, {wall:.1f} s wall): aggregate {speedup:.2f}x one thread"),
        "extrapolated": True,
        "single_thread": {"value": 1.0 / t_full, "unit": UNIT, "cores": 1, "seconds_per_solve": t_full},
        "all_core_speedup": speedup,
        "_x_sample": x1,
    }


def run_reference(args):
    """Reference arm: the CPU oracle as it stands, on the host cores.  Each
    of the --warmup + --steps steps is one oracle step on the tube_small
    preset (24,764 unknowns, one thread); after them cpu_baseline measures
    the bench tube's cost per unknown and the all-core aggregate, and the
    line's value is the all-core throughput on the workload (extrapolated by
    the unknown ratio from the 25-layer sample).  Under torchrun only rank 0
    runs it; the other ranks exit without work."""
    if int(os.environ.get("RANK", "0")) != 0:
        return
    import fsi_inputs as F
    m = F.build_mesh(F.make_params(**F.PRESETS[args.workload]))
    n_full = 3 * m.n_nodes + m.n_p
    small = ("tube_small", {})
    for _ in range(args.warmup):
        _oracle_sample(*small)
    times = []
    for _ in range(args.steps):
        times.append(_oracle_sample(*small)[0])
    cb = cpu_baseline(n_full)
    cb.pop("_x_sample", None)
    line = {
        "impl": "reference", "metric": METRIC, "value": cb["value"], "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 / cb["value"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"{args.workload}: {describe_workload(args.workload)}, {n_full} unknowns "
                               f"(extrapolated by the unknown ratio from a measured 25-layer sample)",
                   "precision": "fp64",
                   "timed_steps": f"{args.steps} oracle steps on tube_small, {sum(times) / len(times):.2f} s each "
                                  f"(one thread)"},
        "cpu_baseline": cb,
        "e2e": {"value": cb["value"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


# ------------------------------------------------------------------ GPU arm
def main(argv=None):
    args = parse(argv)
    if args.impl == "reference":
        run_reference(args)
        return
    world, rank, local, pg = dist_init()
    import numpy as np
    import torch

    import fsi_inputs as F
    import paper_2206_06996_gb300 as pkg

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pkg.load_library()
    tune_loaded = bool(args.tune_file) and os.path.exists(args.tune_file)
    if tune_loaded:
        pkg.tune_load(args.tune_file)
    stream = torch.cuda.current_stream(dev)
    hbm, peak_kind = peaks()
    legs = [x for x in args.legs.split(",") if x and x != "none"]

    def events():
        return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(sol, fn, k):
        """k steps of fn between two CUDA events on the launching stream, a
        barrier and a device synchronisation on both sides; returns (ms per
        step, library launches per step)."""
        barrier(pg)
        torch.cuda.synchronize(dev)
        l0 = sol.stats()["kernel_launches"]
        e0, e1 = events()
        e0.record(stream)
        for _ in range(k):
            fn(sol)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        barrier(pg)
        return e0.elapsed_time(e1) / k, (sol.stats()["kernel_launches"] - l0) // k

    def block_leg(name, s, prec, steps, warmup, with_mesh=True, profile=True, resetup=False):
        """FP64 or mixed steps (set-up + solve [+ mesh set-up + solve]) on
        system s; returns the leg's record and the solution of the last step."""
        Ad, Bd, Cd, Dd = (pkg.DeviceBSR.from_host(M, device=dev) for M in (s.A, s.B, s.C, s.D))
        bd = torch.as_tensor(s.b, device=dev)
        xd = torch.empty_like(bd)
        Ld = gd = ud = None
        if with_mesh:
            Ld = pkg.DeviceBSR.from_host(s.L, device=dev)
            gd = torch.as_tensor(s.mesh_b, device=dev)
            ud = torch.empty_like(gd)
        sol = pkg.BlockSolver(precision=prec)

        def step(sol_):
            sol_.setup(Ad, Bd, Cd, Dd)
            sol_.solve(bd, xd)
            if with_mesh:
                sol_.mesh_setup(Ld)
                sol_.mesh_solve(gd, ud)

        for _ in range(warmup):
            step(sol)
        sampler = ClockSampler(local).start()
        barrier(pg)
        torch.cuda.synchronize(dev)
        l0 = sol.stats()["kernel_launches"]
        e0, e1 = events()
        e0.record(stream)
        kprof = None
        for i in range(steps):
            sol.setup(Ad, Bd, Cd, Dd)
            if i == 0 and profile:
                sol.profile_begin(pkg.abi.SCR_PROF_SPMV_A, 40000)
            sol.solve(bd, xd)
            if i == 0 and profile:
                kprof = sol.profile_end()
            if with_mesh:
                sol.mesh_setup(Ld)
                sol.mesh_solve(gd, ud)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        barrier(pg)
        clocks = sampler.stop()
        ms = e0.elapsed_time(e1) / steps
        launches = (sol.stats()["kernel_launches"] - l0) // steps
        st = sol.stats()
        upd = None
        if resetup:
            # the same step with the numeric re-set-up (scr_update_values on the
            # first set-up's patterns) in place of the full scr_setup: what a
            # Newton step whose Jacobian keeps its pattern pays
            def step_upd(sol_):
                sol_.update_values(Ad, Bd, Cd, Dd)
                sol_.solve(bd, xd)
                if with_mesh:
                    sol_.mesh_setup(Ld)
                    sol_.mesh_solve(gd, ud)

            sol.setup(Ad, Bd, Cd, Dd)
            step_upd(sol)
            msu, _ = timed(sol, step_upd, min(steps, 5))
            stu = sol.stats()
            upd = {"ms_per_step": msu, "value": world * 1000.0 / allmax(pg, msu, dev), "update_ms": stu["setup_ms"],
                   "setup_ms": st["setup_ms"], "outer_iters": stu["outer_iters"],
                   "inner_iters": stu["a_iters"] + stu["s_iters"] + stu["i_iters"], "rel_res": stu["rel_res"],
                   "steps": min(steps, 5),
                   "step": "scr_update_values + scr_solve + mm_setup + mm_solve (aggregates, truncation positions "
                           "and product patterns of the first set-up reused; every numeric phase and the value "
                           "upload inside the timed step)"}
        sol.close()
        fp64 = prec == pkg.SCR_FP64
        rec = {"precision": "fp64" if fp64 else "mixed", "steps": steps, "warmup": warmup, "ms_per_step": ms,
               "value": world * 1000.0 / allmax(pg, ms, dev), "unit": UNIT,
               "rel_res": st["rel_res"], "outer_iters": st["outer_iters"],
               "inner_iters": st["a_iters"] + st["s_iters"] + st["i_iters"],
               "setup_ms": st["setup_ms"], "solve_ms": st["solve_ms"],
               "dofs_iters_per_s": s.n * st["outer_iters"] * 1000.0 / st["solve_ms"],
               "gpu_launches": int(launches), "clocks": clocks,
               "kernel_A": st["kernel_A"], "kernel_Shat": st["kernel_Shat"],
               "host_waits_per_solve": st["syncs"], "pc_from_device_loop_graph": st["pc_graph_runs"]}
        if with_mesh:
            rec.update({"mesh_iters": st["mm_iters"], "mesh_rel_res": st["mm_rel_res"],
                        "mm_setup_ms": st["mm_setup_ms"], "mm_solve_ms": st["mm_solve_ms"]})
        if profile:
            rec["roofline"] = roofline(kprof, fp64, clocks, ms, hbm, peak_kind,
                                       f"level-0 A product ({'FP64' if fp64 else 'FP32'} values)", st["kernel_A"])
        if upd is not None:
            rec["numeric_resetup"] = upd
        del Ad, Bd, Cd, Dd, Ld
        return rec, xd, ud

    # ---------------------------------------------------------- headline
    t_in = time.perf_counter()
    s = F.tube_system(args.workload)
    t_in = time.perf_counter() - t_in
    prec = pkg.SCR_MIXED if args.precision == "mixed" else pkg.SCR_FP64
    head, x_head, _ = block_leg(args.workload, s, prec, args.steps, args.warmup, resetup=True)
    ms, value = job_value(pg, head["ms_per_step"], world, dev)

    mixed = None
    if prec == pkg.SCR_FP64 and not args.skip_mixed:
        x64 = x_head.clone()
        mixed, xm, _ = block_leg(args.workload, s, pkg.SCR_MIXED, args.steps, max(1, args.warmup), resetup=True)
        mixed["speedup_vs_fp64"] = ms / mixed["ms_per_step"]
        mixed["rel_error_vs_fp64_gpu"] = float(torch.linalg.vector_norm(xm - x64) / torch.linalg.vector_norm(x64))
        del x64, xm
    torch.cuda.empty_cache()

    # end to end through the public API with host pinned buffers
    e2e = None
    if not args.no_e2e:
        Ah, Bh, Ch, Dh, Lh = (pkg.DeviceBSR.pinned(M) for M in (s.A, s.B, s.C, s.D, s.L))
        bh = torch.as_tensor(s.b).pin_memory()
        gh = torch.as_tensor(s.mesh_b).pin_memory()
        xh = torch.empty_like(bh).pin_memory()
        uh = torch.empty_like(gh).pin_memory()
        sol = pkg.BlockSolver(precision=prec)

        def step_host(sol_):
            sol_.setup(Ah, Bh, Ch, Dh)
            sol_.solve(bh, xh)
            sol_.mesh_setup(Lh)
            sol_.mesh_solve(gh, uh)

        step_host(sol)
        k_e2e = min(args.steps, 5)
        mse, _ = timed(sol, step_host, k_e2e)
        sol.close()
        mse = allmax(pg, mse, dev)
        h2d = sum(M.nbytes() for M in (Ah, Bh, Ch, Dh, Lh)) + bh.numel() * 8 + gh.numel() * 8
        d2h = xh.numel() * 8 + uh.numel() * 8
        e2e = {"value": world * 1000.0 / mse, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "ms_per_step": mse, "steps": k_e2e,
               "precision": args.precision}
        del Ah, Bh, Ch, Dh, Lh, bh, gh, xh, uh

    # ---------------------------------------------------------- optional legs on the headline tube
    batched = None
    if args.batched:
        batched = batched_leg(args, pkg, F, torch, dev, timed, pg, world, rank)
    assembly = None
    if args.assembly:
        assembly = assembly_leg(args, pkg, F, torch, dev, stream, s)
    multi = None
    if args.multi_rhs:
        multi = multi_rhs_leg(args, pkg, F, torch, np, dev, timed, s)
    n_head, nv_head, nm_head = s.n, s.n_v, s.L.nb_rows
    del s
    torch.cuda.empty_cache()

    # ---------------------------------------------------------- larger configurations
    sten = None
    if "stenosis" in legs:
        t0 = time.perf_counter()
        ss = F.tube_system("stenosis")
        t_build = time.perf_counter() - t0
        r64, x64, _ = block_leg("stenosis", ss, pkg.SCR_FP64, args.big_steps, 1)
        x64 = x64.clone()
        torch.cuda.empty_cache()
        rmx, xm, _ = block_leg("stenosis", ss, pkg.SCR_MIXED, args.big_steps, 1)
        rmx["speedup_vs_fp64"] = r64["ms_per_step"] / rmx["ms_per_step"]
        rmx["rel_error_vs_fp64_gpu"] = float(torch.linalg.vector_norm(xm - x64) / torch.linalg.vector_norm(x64))
        sten = {"workload": f"stenosis: {describe_workload('stenosis')}, {ss.n_v} nodes, {ss.n} unknowns, "
                            f"{ss.L.nb_rows} mesh nodes",
                "step": "scr_setup + scr_solve + mm_setup + mm_solve", "inputs_build_s": t_build,
                "fp64": r64, "mixed": rmx}
        del ss, x64, xm
        torch.cuda.empty_cache()

    bif = None
    if "bifurcation" in legs:
        bif = bifurcation_leg(args, pkg, F, torch, np, dev, stream, events, barrier, pg, allmax, world, hbm,
                              peak_kind, local)
        torch.cuda.empty_cache()

    if rank != 0:
        return
    cpu = None
    oracle_check = None
    if not args.no_cpu_baseline and world == 1:
        try:
            cpu = cpu_baseline(n_head)
        except Exception as e:  # pragma: no cover
            cpu = {"value": None, "unit": UNIT, "cores": 0, "kind": "oracle", "sample": f"failed: {e}"}
        x_or = cpu.pop("_x_sample", None)
        if x_or is not None:
            # the GPU's FP64 and mixed answers on the oracle's timed sample,
            # against the oracle's own SCR-FGMRES answer (both at 1e-8)
            so = F.tube_system(CPU_SAMPLE[0], **CPU_SAMPLE[1])
            oracle_check = {"workload": f"{CPU_SAMPLE[0]} with {CPU_SAMPLE[1]}, {so.n} unknowns",
                            "reference": "the oracle's SCR-FGMRES at rel-res 1e-8 (the cpu_baseline sample)"}
            for nm, pr in (("fp64", pkg.SCR_FP64), ("mixed", pkg.SCR_MIXED)):
                with pkg.BlockSolver(precision=pr) as so_sol:
                    so_sol.setup(so.A, so.B, so.C, so.D)
                    xg = so_sol.solve(so.b.copy())
                    rr = so_sol.residual()
                oracle_check[nm] = {"rel_difference": float(np.linalg.norm(xg - x_or) / np.linalg.norm(x_or)),
                                    "rel_res": rr}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if prec == pkg.SCR_FP64 else "f64+f32",
        "data": "synthetic",
        "config": {"workload": f"{args.workload}: {describe_workload(args.workload)}, {nv_head} nodes, {n_head} "
                               f"unknowns, {nm_head} mesh nodes", "precision": args.precision,
                   "step": "scr_setup + scr_solve + mm_setup + mm_solve", "l2": "inputs > L2 (no flush)",
                   "parallelism": f"replicas x{world}",
                   "autotune": "decisions loaded from --tune-file" if tune_loaded else "timed at set-up",
                   "larger_legs": f"{args.big_steps} timed steps each after 1 warm-up" if legs else "none"},
        "rel_res": head["rel_res"], "outer_iters": head["outer_iters"], "inner_iters": head["inner_iters"],
        "mesh_iters": head["mesh_iters"], "mesh_rel_res": head["mesh_rel_res"], "setup_ms": head["setup_ms"],
        "solve_ms": head["solve_ms"], "dofs_iters_per_s": head["dofs_iters_per_s"],
        "mm_setup_ms": head["mm_setup_ms"], "mm_solve_ms": head["mm_solve_ms"],
        "gpu_launches": head["gpu_launches"], "host_waits_per_solve": head["host_waits_per_solve"],
        "pc_from_device_loop_graph": head["pc_from_device_loop_graph"],
        "roofline": head["roofline"], "cpu_baseline": cpu, "e2e": e2e,
        "numeric_resetup": head.get("numeric_resetup"),
        "mixed": mixed, "oracle_check": oracle_check, "stenosis": sten, "bifurcation": bif,
        "batched": batched, "multi_rhs": multi, "assembly": assembly,
        "clocks": head["clocks"], "inputs_build_s": t_in,
    }
    if args.tune_file and not tune_loaded and rank == 0:
        pkg.tune_save(args.tune_file)
    print(json.dumps(line))


def bifurcation_leg(args, pkg, F, torch, np, dev, stream, events, barrier, pg, allmax, world, hbm, peak_kind,
                    local):
    """The bifurcation (about 16M unknowns): eight right-hand sides -R at
    inflow peaks drawn U(0, 60) cm/s (seed 2206) on the Jacobian at 30 cm/s,
    one step = scr_setup + scr_solve_multi (8-column block solve, mixed
    precision, FP64 outer)."""
    t0 = time.perf_counter()
    s = F.tube_system("bifurcation")
    peaks_u = np.random.default_rng(2206).uniform(0.0, 60.0, 8)
    rhs = [torch.as_tensor(F.rhs_only("bifurcation", u_max=float(u)), device=dev) for u in peaks_u]
    t_build = time.perf_counter() - t0
    Ad, Bd, Cd, Dd = (pkg.DeviceBSR.from_host(M, device=dev) for M in (s.A, s.B, s.C, s.D))
    xs = [torch.empty_like(b) for b in rhs]
    sol = pkg.BlockSolver(precision=pkg.SCR_MIXED, nrhs=8)
    rel = None

    def step(sol_):
        nonlocal rel
        sol_.setup(Ad, Bd, Cd, Dd)
        _, rel = sol_.solve_multi(rhs, xs)

    step(sol)
    sampler = ClockSampler(local).start()
    barrier(pg)
    torch.cuda.synchronize(dev)
    l0 = sol.stats()["kernel_launches"]
    e0, e1 = events()
    e0.record(stream)
    kprof = None
    for i in range(args.big_steps):
        if i == 0:
            sol.setup(Ad, Bd, Cd, Dd)
            sol.profile_begin(pkg.abi.SCR_PROF_SPMV_A, 40000)
            _, rel = sol.solve_multi(rhs, xs)
            kprof = sol.profile_end()
        else:
            step(sol)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    barrier(pg)
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1) / args.big_steps
    st = sol.stats()
    launches = (st["kernel_launches"] - l0) // args.big_steps
    sol.close()
    ms = allmax(pg, ms, dev)
    out = {"workload": f"bifurcation: {describe_workload('bifurcation')}, {s.n_v} nodes, {s.n} unknowns",
           "step": "scr_setup + scr_solve_multi (8 right-hand sides, one Jacobian)", "precision": "mixed",
           "rhs": 8, "inflow_peaks_cm_s": [round(float(u), 3) for u in peaks_u], "steps": args.big_steps,
           "warmup": 1, "ms_per_step": ms, "rhs_solves_per_s": world * 8 * 1000.0 / ms,
           "solves_per_s": world * 1000.0 / ms, "outer_iters": st["outer_iters"],
           "inner_iters": st["a_iters"] + st["s_iters"] + st["i_iters"], "setup_ms": st["setup_ms"],
           "solve_ms": st["solve_ms"], "max_rel_res": float(np.max(rel)), "gpu_launches": int(launches),
           "roofline": roofline(kprof, False, clocks, ms, hbm, peak_kind,
                                "level-0 A product, FP32 values, 8 interleaved right-hand sides", st["kernel_A"],
                                captured=False),
           "clocks": clocks, "inputs_build_s": t_build}
    del Ad, Bd, Cd, Dd, rhs, xs, s
    return out


def gather_members(pg, world: int, mine: list[int], values: list, n: int) -> list:
    """Per-member results of every rank, in member order: rank r holds the
    members `mine` (its part of split_members) with `values`; returns the n
    values on every rank (all_gather of the (index, value) pairs)."""
    pairs = list(zip(mine, values))
    if pg is None or world == 1:
        got = [pairs]
    else:
        got = [None] * world
        pg.all_gather_object(got, pairs)
    out = [None] * n
    for part in got:
        for i, v in part:
            out[i] = v
    return out


def batched_leg(args, pkg, F, torch, dev, timed, pg=None, world=1, rank=0):
    """The 64-tube batch: one block-diagonal set-up + solve of all members
    against the same members set up and solved one after another, in the
    same precision (FP64 and mixed).  The one-by-one runs reuse the
    autotuner's decisions of a first pass (the members' shapes are
    distinct, so without the cache every member would time its kernels),
    with set-up and solve times reported apart.  With N ranks the members
    are split by unknowns (split_members) and each rank solves its own part
    as one union; the per-member residuals are gathered in member order and
    the job time is the slowest rank's (no collective on the data path)."""
    import numpy as np
    params = [F.batch_member_params(i) for i in range(64)]
    # nodes of a member: a centre node plus n_circ x (lumen + wall rings) per
    # section, n_ax + 1 sections (the unknowns grow in proportion)
    sizes = [(1 + p["n_circ"] * (p["n_rad_f"] + p["n_rad_s"])) * (p["n_ax"] + 1) for p in params]
    mine = split_members(sizes, world)[rank]
    members = [F.tube_system("batch", **params[i]) for i in mine]
    devm = [tuple(pkg.DeviceBSR.from_host(M, device=dev) for M in (m.A, m.B, m.C, m.D)) for m in members]
    bsd = [torch.as_tensor(m.b, device=dev) for m in members]
    xsd = [torch.empty_like(b) for b in bsd]
    out = {"members": 64, "members_this_rank": len(mine), "split": "by unknowns over ranks" if world > 1 else "none",
           "nodes_this_rank": int(sum(m.n_v for m in members)),
           "unknowns_this_rank": int(sum(m.n for m in members))}
    for name, prec in (("fp64", pkg.SCR_FP64), ("mixed", pkg.SCR_MIXED)):
        solb = pkg.BlockSolver(precision=prec)

        def step_batch(sol_):
            sol_.setup_batch(devm)
            sol_.solve_batch(bsd, xsd)

        step_batch(solb)
        msb, _ = timed(solb, step_batch, max(1, min(args.steps, 3)))
        relb = gather_members(pg, world, mine, [float(r) for r in solb.batch_residuals()], 64)
        stb = solb.stats()
        solb.close()
        sols = pkg.BlockSolver(precision=prec)
        setup_ms = solve_ms = 0.0
        outer = inner = 0

        def step_seq(sol_):
            nonlocal setup_ms, solve_ms, outer, inner
            setup_ms = solve_ms = 0.0
            outer = inner = 0
            for (Am, Bm, Cm, Dm), b, x in zip(devm, bsd, xsd):
                sol_.setup(Am, Bm, Cm, Dm)
                sol_.solve(b, x)
                st = sol_.stats()
                setup_ms += st["setup_ms"]
                solve_ms += st["solve_ms"]
                outer += st["outer_iters"]
                inner += st["a_iters"] + st["s_iters"] + st["i_iters"]

        step_seq(sols)  # first pass: the autotuner times each member's shapes once
        mss, _ = timed(sols, step_seq, 1)
        sols.close()
        msb_job = allmax(pg, msb, dev)
        out[name] = {"batched_ms": msb_job, "members_per_s": 64 * 1000.0 / msb_job, "one_by_one_ms": allmax(pg, mss, dev),
                     "one_by_one_setup_ms": setup_ms, "one_by_one_solve_ms": solve_ms,
                     "batched_outer_iters": stb["outer_iters"],
                     "batched_inner_iters": stb["a_iters"] + stb["s_iters"] + stb["i_iters"],
                     "one_by_one_outer_iters": outer, "one_by_one_inner_iters": inner,
                     "speedup_vs_one_by_one": mss / msb, "max_member_rel_res": float(np.max(relb))}
    return out


def assembly_leg(args, pkg, F, torch, dev, stream, s_head):
    sm = F.tube_system(args.workload, keep_mesh=True)
    asm_h = F.Assembler(F.make_params(**F.PRESETS[args.workload]))
    v0, p0 = asm_h.initial_state()
    L_raw = asm_h.mesh_laplacian()
    asm_h.close()
    Ad, Bd, Cd, Dd = (pkg.DeviceBSR.from_host(M, device=dev) for M in (sm.A, sm.B, sm.C, sm.D))
    sola = pkg.BlockSolver()
    sola.assembly_setup(sm.mesh, sm.params)
    vd0 = torch.zeros(3 * sm.mesh.n_nodes, dtype=torch.float64, device=dev)
    vt, pt = torch.as_tensor(v0, device=dev), torch.as_tensor(p0, device=dev)
    for _ in range(3):
        sola.assemble_residual(vt, pt, vdot=vd0, u=vd0)
    torch.cuda.synchronize(dev)
    ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ea.record(stream)
    for _ in range(10):
        sola.assemble_residual(vt, pt, vdot=vd0, u=vd0)
    eb.record(stream)
    torch.cuda.synchronize(dev)
    ms_res = ea.elapsed_time(eb) / 10
    sola.setup(Ad, Bd, Cd, Dd)
    vc, pc, vdc, uc = vt.clone(), pt.clone(), vd0.clone(), vd0.clone()
    sola.corrector(vc, pc, vdc, uc, 1)  # warm-up
    vc, pc, vdc, uc = vt.clone(), pt.clone(), vd0.clone(), vd0.clone()
    torch.cuda.synchronize(dev)
    ea.record(stream)
    norms = sola.corrector(vc, pc, vdc, uc, 1)
    eb.record(stream)
    torch.cuda.synchronize(dev)
    ms_corr = ea.elapsed_time(eb)
    sola.mesh_setup(sm.L)
    sola.mesh_coupling(L_raw, sm.mesh.fluid_id, sm.mesh.dir_m, F.interface_follow(sm.mesh))
    zf = torch.zeros(3 * sm.mesh.n_fluid, dtype=torch.float64, device=dev)
    vc, pc, vdc, uc = vt.clone(), pt.clone(), vd0.clone(), vd0.clone()
    sola.corrector_ale(vc, pc, vdc, uc, zf, 1)  # warm-up
    vc, pc, vdc, uc = vt.clone(), pt.clone(), vd0.clone(), vd0.clone()
    torch.cuda.synchronize(dev)
    ea.record(stream)
    norms_ale, _ = sola.corrector_ale(vc, pc, vdc, uc, zf, 1)
    eb.record(stream)
    torch.cuda.synchronize(dev)
    ms_ale = ea.elapsed_time(eb)
    mesh_it, _ = sola.mesh_iters()
    sola.close()
    # the tangent on the GPU (element tangents + per-block sums) followed by
    # the set-up of the solve on it, and one full-Newton corrector iteration
    # (tangent re-assembled at the iteration's state)
    solt = pkg.BlockSolver(newton=1)
    solt.setup(Ad, Bd, Cd, Dd)
    solt.assembly_setup(sm.mesh, sm.params)
    solt.assemble_tangent(vt, pt)
    torch.cuda.synchronize(dev)
    ea.record(stream)
    solt.setup(Ad, Bd, Cd, Dd)
    eb.record(stream)
    torch.cuda.synchronize(dev)
    setup_tan = ea.elapsed_time(eb)
    solt.assemble_tangent(vt, pt)  # the pattern captured again after the caller's set-up
    torch.cuda.synchronize(dev)
    ea.record(stream)
    solt.assemble_tangent(vt, pt)
    eb.record(stream)
    torch.cuda.synchronize(dev)
    ms_tan = ea.elapsed_time(eb)
    vc, pc, vdc, uc = vt.clone(), pt.clone(), vd0.clone(), vd0.clone()
    solt.corrector(vc, pc, vdc, uc, 1)  # warm-up
    vc, pc, vdc, uc = vt.clone(), pt.clone(), vd0.clone(), vd0.clone()
    torch.cuda.synchronize(dev)
    ea.record(stream)
    norms_nt = solt.corrector(vc, pc, vdc, uc, 2)
    eb.record(stream)
    torch.cuda.synchronize(dev)
    ms_nt = ea.elapsed_time(eb) / 2
    solt.close()
    return {"elements": int(sm.mesh.n_elem), "residual_ms": ms_res, "elements_per_s": sm.mesh.n_elem * 1000.0 / ms_res,
            "tangent_and_setup_ms": ms_tan, "setup_ms": setup_tan, "tangent_ms": ms_tan - setup_tan,
            "newton_iteration_ms": ms_nt, "newton_residuals": [float(x) for x in norms_nt],
            "corrector_iteration_ms": ms_corr, "corrector_residual_drop": float(norms[1] / norms[0]),
            "corrector_ale_iteration_ms": ms_ale,
            "corrector_ale_residual_drop": float(norms_ale[1] / norms_ale[0]),
            "corrector_ale_mesh_cg_iters": int(mesh_it)}


def multi_rhs_leg(args, pkg, F, torch, np, dev, timed, s):
    Ad, Bd, Cd, Dd = (pkg.DeviceBSR.from_host(M, device=dev) for M in (s.A, s.B, s.C, s.D))
    peaks_u = np.random.default_rng(2206).uniform(0.0, 60.0, 8)
    rhs = [torch.as_tensor(F.rhs_only(args.workload, u_max=float(u)), device=dev) for u in peaks_u]
    xs8 = [torch.empty_like(b) for b in rhs]
    solk = pkg.BlockSolver(precision=pkg.SCR_MIXED, nrhs=8)
    rel8 = None

    def step_multi(sol_):
        nonlocal rel8
        sol_.setup(Ad, Bd, Cd, Dd)
        _, rel8 = sol_.solve_multi(rhs, xs8)

    step_multi(solk)
    msk, _ = timed(solk, step_multi, max(1, min(args.steps, 3)))
    stk = solk.stats()
    solk.close()
    sol1 = pkg.BlockSolver(precision=pkg.SCR_MIXED)

    def step_single(sol_):
        sol_.setup(Ad, Bd, Cd, Dd)
        for b, x in zip(rhs, xs8):
            sol_.solve(b, x)

    step_single(sol1)
    ms1, _ = timed(sol1, step_single, max(1, min(args.steps, 3)))
    sol1.close()
    return {"rhs": 8, "inflow_peaks_cm_s": [float(u) for u in peaks_u], "precision": "mixed",
            "block_ms": msk, "rhs_solves_per_s": 8 * 1000.0 / msk, "one_by_one_ms": ms1,
            "speedup_vs_one_by_one": ms1 / msk, "block_outer_iters": stk["outer_iters"],
            "max_rel_res": float(np.max(rel8))}


if __name__ == "__main__":
    main()
