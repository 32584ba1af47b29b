#!/usr/bin/env python
"""Benchmark of the SCR-FGMRES + AMG path on one GB300 (or N replicas).

One step = the whole linear-solver path of one Newton step on the refined
straight tube (96 circ x (11 lumen + 5 wall) rings x 400 axial layers:
616,337 nodes, 2,503,844 block unknowns, 423,857 mesh nodes):

  scr_setup  (upload of A, B, C, D into the solver layout, Shat = D - C
              diag(A)^{-1} B, AMG hierarchies of A and Shat)
  scr_solve  (FGMRES + SCR to ||b - calA x|| / ||b|| <= 1e-8, FP64 check)
  mm_setup + mm_solve  (mesh-motion AMG hierarchy, CG to 1e-8)

The matrices (about 1.5 GB) exceed the 129 MB L2, so no flush is needed
between steps.  `value` is solves per second over the device-resident
timed region; `e2e` repeats the step through host pinned buffers (every
matrix and right-hand side copied in, both solutions copied out).

Multi-GPU: the path does not partition a single solve; with N ranks each
rank solves its own copy of the workload (independent problems, no
collective on the data path), `scaling` = "weak".
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "tube_large"


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
METRIC = "SCR-FGMRES+AMG solves/s to rel-res 1e-8 (mixed vs FP64) on 1 GB300; % HBM peak"
UNIT = "solves/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["fp64", "mixed"], default="fp64")
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--skip-mixed", action="store_true")
    ap.add_argument("--tune-file", default=None,
                    help="autotuner decisions: loaded before the first set-up when the file exists, "
                         "written after the run otherwise (replays one run's kernel choices in another, "
                         "e.g. under a profiler whose instrumentation distorts the autotuner's timings)")
    ap.add_argument("--multi-rhs", action="store_true",
                    help="also time eight right-hand sides (inflow peaks U(0, 60) cm/s, one Jacobian) solved as one "
                         "8-column block solve in mixed precision against the same eight solved one by one")
    ap.add_argument("--assembly", action="store_true",
                    help="also time the GPU residual assembly (element loop) and one multi-corrector iteration "
                         "(residual, FP64 solve, updates) on the workload's mesh, with and without the mesh motion "
                         "solved inside it")
    ap.add_argument("--batched", action="store_true",
                    help="also time the 64-tube batched form (mixed, one block-diagonal solve) against the "
                         "same 64 tubes solved one by one in FP64")
    return ap.parse_args()


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


# FP64 FMA rate of GB300: 2 FP64 FMA per SM per clock (152 SMs); measured
# 0.600 TFMA/s at 1995 MHz with an independent-chain FMA loop
FP64_FMA_PER_SM_CLK = 2
# dram bytes / algorithmic bytes of the FP64 level-0 product (ncu, 154k-node tube)
TRAFFIC_OVER_ALGORITHMIC_FP64 = 181.0 / 180.0
N_SM = 152


class ClockSampler:
    """nvidia-smi clocks and throttle reasons every 200 ms during the timed region."""

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


def bytes_of_system(s) -> int:
    n = 0
    for M in (s.A, s.B, s.C, s.D, s.L):
        n += M.row_ptr.nbytes + M.col.nbytes + M.val.nbytes
    return n


# ------------------------------------------------------------------ CPU oracle
def oracle_step_sample(sample_name: str = "tube_small"):
    """Time one full oracle step (setup, SCR-FGMRES, mesh AMG-CG) on the
    coarser member of the tube family; returns (seconds, unknowns)."""
    import fsi_inputs as F
    from oracle import scr as oscr
    s = F.tube_system(sample_name)
    t0 = time.perf_counter()
    out = oscr.solve_system(s)
    dt = time.perf_counter() - t0
    assert out["info"].converged
    return dt, s.n


def cpu_threads() -> int:
    try:
        import threadpoolctl
        info = threadpoolctl.threadpool_info()
        return max([i.get("num_threads", 1) for i in info] + [1])
    except Exception:
        return 1


def run_reference(args):
    """Reference arm: the CPU oracle as it stands, on the host cores.  Under
    torchrun only rank 0 runs it (no process group is needed); the other
    ranks exit without work."""
    if int(os.environ.get("RANK", "0")) != 0:
        return
    import fsi_inputs as F
    m = F.build_mesh(F.make_params(**F.PRESETS[args.workload]))
    n_large = 3 * m.n_nodes + m.n_p
    for _ in range(args.warmup):
        oracle_step_sample()
    times = []
    n_small = None
    for _ in range(args.steps):
        dt, n_small = oracle_step_sample()
        times.append(dt)
    sec = sum(times) / len(times)
    scaled = 1.0 / (sec * n_large / n_small)
    cores = cpu_threads()
    line = {
        "impl": "reference", "metric": METRIC, "value": scaled, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * n_large / n_small * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": f"{args.workload} ({n_large} unknowns); each step one full oracle step on "
                               f"tube_small ({n_small} unknowns), scaled by the unknown ratio",
                   "precision": "fp64"},
        "cpu_baseline": {"value": scaled, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"one oracle step (setup + SCR-FGMRES + mesh CG) on tube_small "
                                   f"({n_small} unknowns) per bench step, {sec:.2f} s each, scaled "
                                   f"x{n_small / n_large:.5f} to the {n_large}-unknown workload"},
        "e2e": {"value": scaled, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


# ------------------------------------------------------------------ GPU arm
def main():
    args = parse()
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
    t_in = time.perf_counter()
    s = F.tube_system(args.workload)
    t_in = time.perf_counter() - t_in
    prec = pkg.SCR_MIXED if args.precision == "mixed" else pkg.SCR_FP64

    Ad, Bd, Cd, Dd, Ld = (pkg.DeviceBSR.from_host(M, device=dev) for M in (s.A, s.B, s.C, s.D, s.L))
    bd = torch.as_tensor(s.b, device=dev)
    gd = torch.as_tensor(s.mesh_b, device=dev)
    xd = torch.empty_like(bd)
    ud = torch.empty_like(gd)
    stream = torch.cuda.current_stream(dev)

    def make_solver(p):
        return pkg.BlockSolver(precision=p)

    def step_device(sol):
        sol.setup(Ad, Bd, Cd, Dd)
        sol.solve(bd, xd)
        sol.mesh_setup(Ld)
        sol.mesh_solve(gd, ud)

    def timed(sol, fn, k, profile=False):
        barrier(pg)
        torch.cuda.synchronize(dev)
        launches0 = sol.stats()["kernel_launches"]
        prof = None
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for i in range(k):
            fn(sol)
            if profile and i == 0:
                pass
        e1.record(stream)
        torch.cuda.synchronize(dev)
        barrier(pg)
        ms = e0.elapsed_time(e1) / k
        launches = (sol.stats()["kernel_launches"] - launches0) // k
        return ms, launches, prof

    sol = make_solver(prec)
    for _ in range(args.warmup):
        step_device(sol)
    # timed region with the dominant kernel's launches bracketed by events
    sampler = ClockSampler(local)
    sampler.start()
    barrier(pg)
    torch.cuda.synchronize(dev)
    launches0 = sol.stats()["kernel_launches"]
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    kprof = None
    for i in range(args.steps):
        sol.setup(Ad, Bd, Cd, Dd)
        if i == 0:
            sol.profile_begin(pkg.abi.SCR_PROF_SPMV_A, 40000)
        sol.solve(bd, xd)
        if i == 0:
            kprof = sol.profile_end()
        sol.mesh_setup(Ld)
        sol.mesh_solve(gd, ud)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    barrier(pg)
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1) / args.steps
    launches = (sol.stats()["kernel_launches"] - launches0) // args.steps
    st = sol.stats()
    ms, value = job_value(pg, ms, world, dev)
    # residual check of the timed answer by the same FP64 operator
    rel_res = st["rel_res"]

    # mixed precision, same step (reported beside the FP64 headline)
    mixed = None
    if prec == pkg.SCR_FP64 and not args.skip_mixed:
        x64 = xd.clone()  # the FP64 answer; the mixed steps overwrite xd
        solm = make_solver(pkg.SCR_MIXED)
        for _ in range(max(1, args.warmup)):
            step_device(solm)
        msm, _, _ = timed(solm, step_device, args.steps)
        stm = solm.stats()
        msm = allmax(pg, msm, dev)
        torch.cuda.synchronize(dev)
        err = float(torch.linalg.vector_norm(xd - x64) / torch.linalg.vector_norm(x64))
        mixed = {"value": world * 1000.0 / msm, "ms_per_step": msm, "outer_iters": stm["outer_iters"],
                 "rel_res": stm["rel_res"], "speedup_vs_fp64": ms / msm,
                 "solve_ms": stm["solve_ms"], "setup_ms": stm["setup_ms"],
                 "dofs_iters_per_s": s.n * stm["outer_iters"] * 1000.0 / stm["solve_ms"],
                 "rel_error_vs_fp64": err}
        solm.close()

    # end to end through the public API with host pinned buffers
    e2e = None
    if not args.no_e2e:
        Ah, Bh, Ch, Dh, Lh = (pkg.DeviceBSR.pinned(M) for M in (s.A, s.B, s.C, s.D, s.L))
        bh = torch.as_tensor(s.b).pin_memory()
        gh = torch.as_tensor(s.mesh_b).pin_memory()
        xh = torch.empty_like(bh).pin_memory()
        uh = torch.empty_like(gh).pin_memory()

        def step_host(sol_):
            sol_.setup(Ah, Bh, Ch, Dh)
            sol_.solve(bh, xh)
            sol_.mesh_setup(Lh)
            sol_.mesh_solve(gh, uh)

        step_host(sol)
        mse, _, _ = timed(sol, step_host, args.steps)
        mse = allmax(pg, mse, dev)
        h2d = sum(M.nbytes() for M in (Ah, Bh, Ch, Dh, Lh)) + bh.numel() * 8 + gh.numel() * 8
        d2h = xh.numel() * 8 + uh.numel() * 8
        e2e = {"value": world * 1000.0 / mse, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "ms_per_step": mse}

    batched = None
    if args.batched:
        members = [F.tube_system("batch", **F.batch_member_params(i)) for i in range(64)]
        devm = [tuple(pkg.DeviceBSR.from_host(M, device=dev) for M in (m.A, m.B, m.C, m.D)) for m in members]
        bsd = [torch.as_tensor(m.b, device=dev) for m in members]
        xsd = [torch.empty_like(b) for b in bsd]
        solb = pkg.BlockSolver(precision=pkg.SCR_MIXED)

        def step_batch(sol_):
            sol_.setup_batch(devm)
            sol_.solve_batch(bsd, xsd)

        step_batch(solb)
        msb, _, _ = timed(solb, step_batch, max(1, args.steps))
        relb = solb.batch_residuals()
        solb.close()
        sols = pkg.BlockSolver()

        def step_seq(sol_):
            for (Am, Bm, Cm, Dm), b, x in zip(devm, bsd, xsd):
                sol_.setup(Am, Bm, Cm, Dm)
                sol_.solve(b, x)

        step_seq(sols)
        mss, _, _ = timed(sols, step_seq, 1)
        sols.close()
        batched = {"members": 64, "nodes": int(sum(m.n_v for m in members)),
                   "unknowns": int(sum(m.n for m in members)),
                   "mixed_batched_ms": msb, "members_per_s": 64 * 1000.0 / msb,
                   "fp64_one_by_one_ms": mss, "speedup_vs_fp64_one_by_one": mss / msb,
                   "max_member_rel_res": float(relb.max())}

    assembly = None
    if args.assembly:
        sm = F.tube_system(args.workload, keep_mesh=True)
        asm_h = F.Assembler(F.make_params(**F.PRESETS[args.workload]))
        v0, p0 = asm_h.initial_state()
        L_raw = asm_h.mesh_laplacian()
        asm_h.close()
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
        torch.cuda.synchronize(dev)
        ea.record(stream)
        norms = sola.corrector(vc, pc, vdc, uc, 1)
        eb.record(stream)
        torch.cuda.synchronize(dev)
        ms_corr = ea.elapsed_time(eb)
        # the same iteration with the mesh motion solved inside it (interface
        # displacement -> mesh CG + AMG -> mesh velocity in the residual)
        sola.mesh_setup(sm.L)
        sola.mesh_coupling(L_raw, sm.mesh.fluid_id, sm.mesh.dir_m, F.interface_follow(sm.mesh))
        zf = torch.zeros(3 * sm.mesh.n_fluid, dtype=torch.float64, device=dev)
        vc, pc, vdc, uc = vt.clone(), pt.clone(), vd0.clone(), vd0.clone()
        torch.cuda.synchronize(dev)
        ea.record(stream)
        norms_ale, _ = sola.corrector_ale(vc, pc, vdc, uc, zf, 1)
        eb.record(stream)
        torch.cuda.synchronize(dev)
        mesh_it, _ = sola.mesh_iters()
        sola.close()
        assembly = {"elements": int(sm.mesh.n_elem), "residual_ms": ms_res,
                    "elements_per_s": sm.mesh.n_elem * 1000.0 / ms_res,
                    "corrector_iteration_ms": ms_corr,
                    "corrector_residual_drop": float(norms[1] / norms[0]),
                    "corrector_ale_iteration_ms": ea.elapsed_time(eb),
                    "corrector_ale_residual_drop": float(norms_ale[1] / norms_ale[0]),
                    "corrector_ale_mesh_cg_iters": int(mesh_it)}
        del sm

    multi = None
    if args.multi_rhs:
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
        msk, _, _ = timed(solk, step_multi, max(1, args.steps))
        stk = solk.stats()
        solk.close()
        sol1 = pkg.BlockSolver(precision=pkg.SCR_MIXED)

        def step_single(sol_):
            sol_.setup(Ad, Bd, Cd, Dd)
            for b, x in zip(rhs, xs8):
                sol_.solve(b, x)

        step_single(sol1)
        ms1, _, _ = timed(sol1, step_single, max(1, args.steps))
        sol1.close()
        multi = {"rhs": 8, "inflow_peaks_cm_s": [float(u) for u in peaks_u], "precision": "mixed",
                 "block_ms": msk, "rhs_solves_per_s": 8 * 1000.0 / msk, "one_by_one_ms": ms1,
                 "speedup_vs_one_by_one": ms1 / msk, "block_outer_iters": stk["outer_iters"],
                 "max_rel_res": float(np.max(rel8))}

    if rank != 0:
        return
    hbm, peak_kind = peaks()
    roof = None
    if kprof and kprof["timed"] > 0:
        per_launch_s = kprof["ms"] * 1e-3 / kprof["timed"]
        bytes_pl = kprof["bytes"] / kprof["timed"]
        flops_pl = kprof["flops"] / kprof["timed"]
        achieved_gbs = bytes_pl / per_launch_s * 1e-9
        if prec == pkg.SCR_FP64:
            # one FP64 FMA per stored value: the FP64 pipe binds before HBM
            clk = (clocks.get("sm_mhz") or 1995.0) * 1e6
            fma_peak = FP64_FMA_PER_SM_CLK * N_SM * clk
            t_alu = flops_pl / 2.0 / fma_peak
            t_hbm = bytes_pl / (hbm * 1e9)
            if t_alu > t_hbm:
                roof = {"bound": "alu", "achieved": flops_pl / per_launch_s * 1e-12,
                        "peak": 2.0 * fma_peak * 1e-12, "unit": "TFLOP/s",
                        "frac": (flops_pl / per_launch_s) / (2.0 * fma_peak),
                        "hbm_achieved_gbs": achieved_gbs, "hbm_frac": achieved_gbs / hbm,
                        "peak_note": f"FP64 pipe: {FP64_FMA_PER_SM_CLK} FMA/SM/clk x {N_SM} SMs at the median "
                                     f"sampled SM clock; HBM {peak_kind} {hbm:.0f} GB/s"}
        if roof is None:
            roof = {"bound": "hbm", "achieved": achieved_gbs, "peak": hbm, "unit": "GB/s",
                    "frac": achieved_gbs / hbm, "peak_note": f"{peak_kind} HBM copy bandwidth"}
        roof.update({"kernel": "k_spmv<3,3,1> (level-0 A product)", "launches_per_step": kprof["launches"],
                     "timed_launches": kprof["timed"], "bytes_per_launch": bytes_pl,
                     "us_per_launch": per_launch_s * 1e6,
                     "share_of_step": kprof["ms"] / ms, "traffic": None})
        if prec == pkg.SCR_FP64:
            # DRAM bytes per launch: the ncu capture of this kernel on the
            # 154k-node tube measured dram read + write = 181.0 MB against
            # 180.0 MB of algorithmic bytes per launch (x gathers hit L1/L2, no
            # re-reads); traffic grows with the stored blocks, so the full
            # launch's traffic is that ratio times its algorithmic bytes
            roof["traffic"] = TRAFFIC_OVER_ALGORITHMIC_FP64 * bytes_pl
            roof["traffic_note"] = ("ncu dram__bytes_read.sum + dram__bytes_write.sum of the same kernel on the "
                                    "154k-node tube (181.0 MB per launch, 180.0 MB algorithmic), scaled to this "
                                    "launch by its algorithmic bytes")
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        try:
            dt, n_small = oracle_step_sample()
            cpu = {"value": 1.0 / (dt * s.n / n_small), "unit": UNIT, "cores": cpu_threads(), "kind": "oracle",
                   "sample": f"one oracle step (setup + SCR-FGMRES + mesh CG) on tube_small ({n_small} "
                             f"unknowns) in {dt:.2f} s, scaled x{n_small / s.n:.5f} to the {s.n}-unknown workload"}
        except Exception as e:  # pragma: no cover
            cpu = {"value": None, "unit": UNIT, "cores": 0, "kind": "oracle", "sample": f"failed: {e}"}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if prec == pkg.SCR_FP64 else "f64+f32",
        "data": "synthetic",
        "config": {"workload": f"{args.workload}: {describe_workload(args.workload)}, {s.n_v} nodes, {s.n} unknowns, "
                               f"{s.L.nb_rows} mesh nodes", "precision": args.precision,
                   "step": "scr_setup + scr_solve + mm_setup + mm_solve", "l2": "inputs > L2 (no flush)",
                   "parallelism": f"replicas x{world}",
                   "autotune": "decisions loaded from --tune-file" if tune_loaded else "timed at set-up"},
        "rel_res": rel_res, "outer_iters": st["outer_iters"], "inner_iters": st["a_iters"] + st["s_iters"] + st["i_iters"],
        "mesh_iters": st["mm_iters"], "setup_ms": st["setup_ms"], "solve_ms": st["solve_ms"],
        "dofs_iters_per_s": s.n * st["outer_iters"] * 1000.0 / st["solve_ms"],
        "mm_setup_ms": st["mm_setup_ms"], "mm_solve_ms": st["mm_solve_ms"],
        "gpu_launches": int(launches), "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "mixed": mixed,
        "batched": batched, "multi_rhs": multi, "assembly": assembly,
        "clocks": clocks, "inputs_build_s": t_in,
    }
    if args.tune_file and not tune_loaded and rank == 0:
        pkg.tune_save(args.tune_file)
    print(json.dumps(line))


if __name__ == "__main__":
    main()
