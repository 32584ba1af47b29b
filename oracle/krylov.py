"""Krylov solvers (test infrastructure only).

FGMRES follows Saad (1993), the flexible variant the paper invokes for the
outer level because the SCR preconditioner varies between iterations
(Sec. 5.2.1): right preconditioning, the preconditioned vectors z_j are kept
and the update is x = x0 + Z y.  Orthogonalisation is classical
Gram-Schmidt applied twice; the Hessenberg least-squares problem is solved
with Givens rotations.  GMRES with a fixed preconditioner is the same
iteration (the stored z_j equal M^{-1} v_j).  Stopping rule: the residual
estimate |g_{j+1}| relative to ||b||, the unweighted l2 norm.
"""
from __future__ import annotations

import dataclasses
from typing import Callable

import numpy as np


@dataclasses.dataclass
class KrylovInfo:
    iters: int = 0
    rel_res: float = 0.0
    converged: bool = False
    restarts: int = 0


def fgmres(apply_op: Callable, b: np.ndarray, apply_pc: Callable | None = None,
           tol: float = 1e-8, maxit: int = 200, restart: int = 30,
           x0: np.ndarray | None = None, true_residual_check: bool = True):
    """Flexible GMRES(restart).  Returns (x, KrylovInfo)."""
    b = np.asarray(b, dtype=np.float64)
    n = b.shape[0]
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64)
    info = KrylovInfo()
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        info.converged = True
        return np.zeros(n), info
    pc = apply_pc if apply_pc is not None else (lambda v: v.copy())
    while True:
        r = b - apply_op(x) if np.any(x) else b.copy()
        beta = np.linalg.norm(r)
        info.rel_res = beta / bnorm
        if info.rel_res <= tol:
            info.converged = True
            return x, info
        if info.iters >= maxit:
            return x, info
        m = restart
        V = np.zeros((m + 1, n))
        Z = np.zeros((m, n))
        H = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        g = np.zeros(m + 1)
        V[0] = r / beta
        g[0] = beta
        k = 0
        for j in range(m):
            Z[j] = pc(V[j])
            w = apply_op(Z[j])
            # classical Gram-Schmidt, two passes
            h1 = V[: j + 1] @ w
            w = w - h1 @ V[: j + 1]
            h2 = V[: j + 1] @ w
            w = w - h2 @ V[: j + 1]
            H[: j + 1, j] = h1 + h2
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] > 0.0:
                V[j + 1] = w / H[j + 1, j]
            # apply the previous rotations to the new column
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            # new rotation annihilating H[j+1, j]
            a, c = H[j, j], H[j + 1, j]
            d = np.hypot(a, c)
            cs[j], sn[j] = (1.0, 0.0) if d == 0.0 else (a / d, c / d)
            H[j, j] = d
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            k = j + 1
            info.iters += 1
            info.rel_res = abs(g[j + 1]) / bnorm
            if info.rel_res <= tol or info.iters >= maxit or H[j, j] == 0.0:
                break
        # back substitution for y and update x = x0 + Z y
        y = np.zeros(k)
        for i in range(k - 1, -1, -1):
            y[i] = (g[i] - H[i, i + 1:k] @ y[i + 1:k]) / H[i, i] if H[i, i] != 0.0 else 0.0
        x = x + y @ Z[:k]
        info.restarts += 1
        if info.rel_res <= tol:
            if not true_residual_check:
                info.converged = True
                return x, info
            true = np.linalg.norm(b - apply_op(x)) / bnorm
            info.rel_res = true
            if true <= tol:
                info.converged = True
                return x, info
        if info.iters >= maxit:
            info.rel_res = np.linalg.norm(b - apply_op(x)) / bnorm
            info.converged = info.rel_res <= tol
            return x, info


def gmres(apply_op, b, apply_pc=None, tol=1e-3, maxit=200, restart=30):
    """Right-preconditioned GMRES(restart) with a fixed preconditioner;
    stops on the recurrence residual estimate (no extra true-residual
    product), as an inner solve does."""
    return fgmres(apply_op, b, apply_pc, tol=tol, maxit=maxit, restart=restart,
                  true_residual_check=False)


def pcg(apply_op, b, apply_pc=None, tol=1e-8, maxit=500):
    """Preconditioned conjugate gradients (Hestenes-Stiefel), x0 = 0,
    stopping on ||r_k|| / ||b||."""
    b = np.asarray(b, dtype=np.float64)
    info = KrylovInfo()
    x = np.zeros_like(b)
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        info.converged = True
        return x, info
    pc = apply_pc if apply_pc is not None else (lambda v: v.copy())
    r = b.copy()
    z = pc(r)
    p = z.copy()
    rz = r @ z
    while info.iters < maxit:
        q = apply_op(p)
        alpha = rz / (p @ q)
        x = x + alpha * p
        r = r - alpha * q
        info.iters += 1
        info.rel_res = np.linalg.norm(r) / bnorm
        if info.rel_res <= tol:
            info.converged = True
            break
        z = pc(r)
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, info


def richardson(apply_op, b, apply_pc, k: int):
    """k steps of Richardson's iteration preconditioned by M = apply_pc, from
    x = 0: x_1 = M b, x_{i+1} = x_i + M (b - A x_i).  With M linear the
    result is the fixed linear map sum_{i<k} (I - M A)^i M applied to b."""
    b = np.asarray(b, dtype=np.float64)
    x = apply_pc(b)
    for _ in range(k - 1):
        x = x + apply_pc(b - apply_op(x))
    return x

