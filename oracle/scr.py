"""SCR-preconditioned FGMRES and the mesh-motion AMG-CG (test
infrastructure only; the CPU reference of the whole solver path).

* Algorithm 1 (App. B): y = P_SCR^{-1} r
    1. solve A yhat_v = r_v  (GMRES + P_A, delta_A, n_A^max)
    2. r_p <- r_p - C yhat_v  (the garbled "C rhat_v" read as the solution
       of step 1, the only reading consistent with the LDU inverse)
    3. solve S y_p = r_p  (GMRES + P_S, delta_S, n_S^max), S applied by
       Algorithm 2
    4. r_v <- r_v - B y_p
    5. solve A y_v = r_v  (GMRES + P_A, delta_A, n_A^max)
* Algorithm 2 (App. B): S x_p = D x_p - C A^{-1} (B x_p) with A^{-1} an
  inner GMRES + P_I solve to delta_I.
* Outer level (Sec. 5.2.1): FGMRES on calA x = b preconditioned by P_SCR,
  tolerance delta, n^max.  P_A = P_I = AMG(A), P_S = AMG(Shat).
* SIMPLE (Sec. 5.2.1): P_SIMPLE = L diag(A, Shat) U_SIMPLE with
  L = [[I, 0], [C A^{-1}, I]] and U_SIMPLE = [[I, diag(A)^{-1} B], [0, I]];
  its inverse applies L^{-1} (one A solve), diag(A^{-1}, Shat^{-1}) (the
  same A solve and one GMRES + P_S solve with the explicit Shat, no inner
  level) and U_SIMPLE^{-1}:
      yhat_v = A^{-1} r_v, y_p = Shat^{-1} (r_p - C yhat_v),
      y_v = yhat_v - diag(A)^{-1} B y_p.
* SIMPLEC (Sec. 5.2.1): SIMPLE with diag(A) replaced, in Shat and in
  U_SIMPLE, by the diagonal lumped from the absolute values of A's entries,
  d_i = sum_j |a_ij|.
* Mesh motion (Sec. 5.2.2): CG + AMG(L) on the harmonic extension.
* Fixed-count A solves (options inner_vcycles, inter_vcycles): the paper's
  inner and intermediate solves are GMRES to a tolerance; with k > 0 they are
  k V-cycle-preconditioned Richardson steps instead, a fixed linear operator
  (valid under the flexible outer FGMRES; the reading is stated in DESIGN).
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import amg
from .krylov import fgmres, gmres, pcg, richardson
from .schur import schur_hat, simple_diagonal
from .sparse import BlockOperator, rel_residual, to_csr


@dataclasses.dataclass
class SolverOptions:
    """Solver settings of the paper's table of solver parameters with the
    outer tolerance tightened to 1e-8."""
    rtol: float = 1e-8
    max_it: int = 200
    restart: int = 30
    rtol_A: float = 1e-3
    rtol_S: float = 1e-3
    rtol_I: float = 1e-3
    max_A: int = 200
    max_S: int = 200
    max_I: int = 200
    restart_inner: int = 30
    amg_theta: float = 0.08
    amg_coarse: int = 64
    amg_max_levels: int = 10
    nu: int = 1
    amg_trunc: float = 0.3
    amg_pmax: int = 5
    smoother: str = "cheb"
    cheb_degree: int = 3
    precond: str = "scr"       # "scr" (Algorithm 1), "simple" or "simplec"
    inner_vcycles: int = 0     # Algorithm 2's A solve: 0 = GMRES to rtol_I, k = k Richardson steps
    inter_vcycles: int = 0     # Algorithm 1's A solves (steps 1, 5) and SIMPLE's: 0 = GMRES to rtol_A
    mm_rtol: float = 1e-8
    mm_max_it: int = 500


@dataclasses.dataclass
class Counters:
    outer: int = 0
    a_solves: int = 0
    a_iters: int = 0
    s_iters: int = 0
    i_iters: int = 0


class SCRSolver:
    def __init__(self, system, opts: SolverOptions | None = None):
        self.opts = opts or SolverOptions()
        self.op = BlockOperator.from_system(system)
        o = self.opts
        # SIMPLEC (Sec. 5.2.1): the lumped diagonal in Shat and in the update
        self.lumped = o.precond == "simplec"
        self.dsimple = simple_diagonal(self.op, self.lumped)
        self.Shat = schur_hat(self.op, self.lumped)
        self.amg_A = amg.setup(self.op.A, 3, o.amg_theta, o.amg_max_levels, o.amg_coarse, o.nu, o.nu,
                               o.amg_trunc, o.amg_pmax, o.smoother, o.cheb_degree)
        self.amg_S = amg.setup(self.Shat, 1, o.amg_theta, o.amg_max_levels, o.amg_coarse, o.nu, o.nu,
                               o.amg_trunc, o.amg_pmax, o.smoother, o.cheb_degree)
        self.cnt = Counters()

    # Algorithm 2 ------------------------------------------------------
    def apply_S(self, xp: np.ndarray) -> np.ndarray:
        o, op = self.opts, self.op
        xbar = op.B @ xp
        if o.inner_vcycles > 0:
            xt = richardson(lambda v: op.A @ v, xbar, lambda v: amg.vcycle(self.amg_A, v), o.inner_vcycles)
            self.cnt.i_iters += o.inner_vcycles
        else:
            xt, info = gmres(lambda v: op.A @ v, xbar, lambda v: amg.vcycle(self.amg_A, v),
                             tol=o.rtol_I, maxit=o.max_I, restart=o.restart_inner)
            self.cnt.i_iters += info.iters
        xbar = op.C @ xt
        xhat = op.D @ xp
        return xhat - xbar

    # Algorithm 1 ------------------------------------------------------
    def solve_A(self, rv: np.ndarray) -> np.ndarray:
        o, op = self.opts, self.op
        self.cnt.a_solves += 1
        if o.inter_vcycles > 0:
            self.cnt.a_iters += o.inter_vcycles
            return richardson(lambda v: op.A @ v, rv, lambda v: amg.vcycle(self.amg_A, v), o.inter_vcycles)
        y, info = gmres(lambda v: op.A @ v, rv, lambda v: amg.vcycle(self.amg_A, v),
                        tol=o.rtol_A, maxit=o.max_A, restart=o.restart_inner)
        self.cnt.a_iters += info.iters
        return y

    def apply_pc(self, r: np.ndarray) -> np.ndarray:
        o, op = self.opts, self.op
        rv, rp = op.split(np.asarray(r, dtype=np.float64))
        yv_hat = self.solve_A(rv)
        rp2 = rp - op.C @ yv_hat
        yp, info = gmres(self.apply_S, rp2, lambda v: amg.vcycle(self.amg_S, v),
                         tol=o.rtol_S, maxit=o.max_S, restart=o.restart_inner)
        self.cnt.s_iters += info.iters
        rv2 = rv - op.B @ yp
        yv = self.solve_A(rv2)
        return np.concatenate([yv, yp])

    # SIMPLE --------------------------------------------------------------
    def apply_simple(self, r: np.ndarray) -> np.ndarray:
        o, op = self.opts, self.op
        rv, rp = op.split(np.asarray(r, dtype=np.float64))
        yv_hat = self.solve_A(rv)
        rp2 = rp - op.C @ yv_hat
        yp, info = gmres(lambda v: self.Shat @ v, rp2, lambda v: amg.vcycle(self.amg_S, v),
                         tol=o.rtol_S, maxit=o.max_S, restart=o.restart_inner)
        self.cnt.s_iters += info.iters
        yv = yv_hat - (op.B @ yp) / self.dsimple
        return np.concatenate([yv, yp])

    # outer level --------------------------------------------------------
    def solve(self, b: np.ndarray, max_outer: int | None = None):
        o = self.opts
        pc = self.apply_simple if o.precond in ("simple", "simplec") else self.apply_pc
        x, info = fgmres(self.op.matvec, b, pc, tol=o.rtol,
                         maxit=o.max_it if max_outer is None else max_outer, restart=o.restart)
        self.cnt.outer += info.iters
        return x, info

    def rel_residual(self, x, b) -> float:
        return rel_residual(self.op, x, b)


class MeshSolver:
    """CG + AMG(L) on (L kron I3) U = g, vectors interleaved (n, 3)."""

    def __init__(self, system, opts: SolverOptions | None = None):
        self.opts = opts or SolverOptions()
        o = self.opts
        self.L = to_csr(system.L)
        self.H = amg.setup(self.L, 1, o.amg_theta, o.amg_max_levels, o.amg_coarse, o.nu, o.nu,
                           o.amg_trunc, o.amg_pmax, o.smoother, o.cheb_degree)

    def solve(self, g: np.ndarray, tol: float | None = None):
        o = self.opts
        n = self.L.shape[0]
        op = lambda v: (self.L @ v.reshape(n, 3)).reshape(-1)
        pc = lambda v: amg.vcycle(self.H, v.reshape(n, 3)).reshape(-1)
        return pcg(op, g, pc, tol=o.mm_rtol if tol is None else tol, maxit=o.mm_max_it)


def solve_system(system, opts: SolverOptions | None = None):
    """The whole CPU reference path: setup, SCR-FGMRES and the mesh CG."""
    s = SCRSolver(system, opts)
    x, info = s.solve(system.b)
    out = dict(x=x, info=info, counters=s.cnt)
    if system.L is not None:
        m = MeshSolver(system, opts)
        u, minfo = m.solve(system.mesh_b)
        out.update(u=u, mesh_info=minfo)
    return out
