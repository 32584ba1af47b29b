"""Small, bounded cases for profiling single kernels of the path.

    python profcase.py --precision fp64 --n-ax 100 --reps 2

builds the 96 x (11 + 5) tube with `--n-ax` axial layers (100 layers:
154,337 nodes, A about 170 MB in FP64, larger than L2), sets up the solver
with the autotuner off (every product with the kernel `--group`, default
the scalar-row kernel with 2 lanes per row) and applies `--reps` V-cycles of
the A hierarchy; `--what solve` runs one full block solve instead, `--what
residual` evaluates the GPU residual assembly (element loop) `--reps` times,
`--what tangent` the GPU tangent assembly (element tangents, per-block sums
and the set-up of the solve on them) `--reps` times.  A
profiler capture of one kernel family (for example `k_spmv<3, 3, 1, 2,
double`) then sees only launches of that family on this moderate case.
"""
from __future__ import annotations

import argparse
import os
import sys

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--precision", choices=["fp64", "mixed"], default="fp64")
    ap.add_argument("--n-ax", type=int, default=100)
    ap.add_argument("--reps", type=int, default=2)
    ap.add_argument("--what", choices=["vcycle", "solve", "residual", "tangent"], default="vcycle")
    ap.add_argument("--group", type=int, default=102,
                    help="product kernel code for every matrix (102: scalar-row kernel, 2 lanes per row)")
    args = ap.parse_args()
    import torch

    import fsi_inputs as F
    import paper_2206_06996_gb300 as pkg

    if args.what == "tangent":
        s = F.tube_system("tube_large", n_ax=args.n_ax, keep_mesh=True)
        asm = F.Assembler(F.make_params(**{**F.PRESETS["tube_large"], "n_ax": args.n_ax}))
        v0, p0 = asm.initial_state()
        asm.close()
        with pkg.BlockSolver() as sol:
            sol.setup(s.A, s.B, s.C, s.D)
            sol.assembly_setup(s.mesh, s.params)
            v, p = torch.as_tensor(v0, device="cuda"), torch.as_tensor(p0, device="cuda")
            for _ in range(args.reps):
                sol.assemble_tangent(v, p)
            torch.cuda.synchronize()
        print("ok", s.mesh.n_elem)
        return
    if args.what == "residual":
        # the element loop on the same mesh: --reps residual evaluations
        s = F.tube_system("tube_large", n_ax=args.n_ax, keep_mesh=True)
        asm = F.Assembler(F.make_params(**{**F.PRESETS["tube_large"], "n_ax": args.n_ax}))
        v0, p0 = asm.initial_state()
        asm.close()
        with pkg.BlockSolver() as sol:
            sol.assembly_setup(s.mesh, s.params)
            v, p = torch.as_tensor(v0, device="cuda"), torch.as_tensor(p0, device="cuda")
            for _ in range(args.reps):
                R = sol.assemble_residual(v, p)
            torch.cuda.synchronize()
        print("ok", s.mesh.n_elem, float(R.norm()))
        return
    s = F.tube_system("tube_large", n_ax=args.n_ax)
    prec = pkg.SCR_MIXED if args.precision == "mixed" else pkg.SCR_FP64
    with pkg.BlockSolver(precision=prec, autotune=0, spmv_group=args.group) as sol:
        sol.setup(s.A, s.B, s.C, s.D)
        if args.what == "solve":
            x = sol.solve(torch.as_tensor(s.b, device="cuda"))
            out = float(x.norm())
        else:
            b = torch.as_tensor(s.b[: 3 * s.n_v], device="cuda").contiguous()
            for _ in range(args.reps):
                z = sol.amg_apply(pkg.SCR_HIER_A, b)
            out = float(z.norm())
        torch.cuda.synchronize()
    print("ok", s.n, out)


if __name__ == "__main__":
    main()
