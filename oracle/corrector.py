"""The segregated multi-corrector iteration of Sec. 3.5 with a fixed
tangent (test infrastructure only).

With the tangent K = alpha_m dR/dydot + alpha_f gamma dt dR/dy of the block
system (Dirichlet rows as identity rows) held fixed and the mesh fixed, each
iteration evaluates the residual R at the state (v, p at t_{n+alpha_f},
vdot at t_{n+alpha_m}, the solid displacement u), solves K x = -R (Dirichlet
velocity rows of the right-hand side zeroed) exactly, and moves the state by
the generalized-alpha weights of the rate increment (Sec. 3.4):
vdot += alpha_m x_v, v += alpha_f gamma dt x_v, p += alpha_f gamma dt x_p,
u += (alpha_f gamma dt)^2 / alpha_m x_v.  The residual is the generator's
element loop (the input module's assembly of the VMS formulation), plus the
traction m_k (a_k^T v) a_k of resistance outlets (Sec. 3.5: its derivative
is the rank-1 term c_k a_k a_k^T of the tangent, c_k = alpha_f gamma dt m_k).

``corrector_ale`` adds steps 3-4 of the multi-corrector stage (Sec. 3.5):
before each residual evaluation the mesh displacement at t_{n+1} is the
harmonic extension (Sec. 5.2.2: L uhat = 0 on the free fluid nodes) of the
solid displacement at t_{n+1} on the fluid-solid interface (zero on the other
Dirichlet mesh nodes), the mesh velocity at t_{n+1} follows from it, and the
residual sees the mesh velocity at t_{n+alpha_f} in its convective velocity.
The element geometry stays the reference configuration.

``tangent`` is the block Jacobian at an arbitrary state: the generator's
element loop with the consistent tangent (tau frozen at the state) and the
boundary conditions of the input convention (Dirichlet velocity nodes:
identity rows of A, their rows of B and their columns of A and C dropped).
With ``newton=True`` the loops re-assemble it at every iteration's state
before that iteration's solve (the paper's multi-corrector re-assembles the
left-hand side at each iteration), instead of holding the initial one.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spl

from .sparse import BlockOperator, to_csr


def genalpha_weights(rho_inf: float, dt: float):
    """alpha_m = (3 - rho_inf) / (2 (1 + rho_inf)), alpha_f = gamma =
    1 / (1 + rho_inf) (Sec. 3.4); returns (alpha_m, c_f, c_u)."""
    am = 0.5 * (3.0 - rho_inf) / (1.0 + rho_inf)
    af = ga = 1.0 / (1.0 + rho_inf)
    cf = af * ga * dt
    return am, cf, cf * cf / am


def mesh_displacement(L_raw, dir_m, g):
    """Harmonic extension of the Dirichlet data (Sec. 5.2.2): the rows of the
    free nodes solve (L_raw uhat)_i = 0, the Dirichlet nodes take g; each of
    the three components (g, uhat: n_fluid x 3 interleaved) separately."""
    L = L_raw.tocsr()
    dm = np.asarray(dir_m, dtype=bool)
    free = ~dm
    G = np.asarray(g, dtype=np.float64).reshape(-1, 3)
    U = G.copy()
    U[free] = 0.0
    if free.any():
        rhs = -(L[free][:, dm] @ G[dm])
        lu = spl.splu(L[free][:, free].tocsc())
        for c in range(3):
            U[free, c] = lu.solve(np.ascontiguousarray(rhs[:, c]))
    return U.ravel()


def mesh_velocity(uhat_n1, uhat_n, vhat_n, rho_inf: float, dt: float):
    """Step 4 of the multi-corrector stage (Sec. 3.5): vhat_{n+1} =
    (uhat_{n+1} - uhat_n) / (gamma dt) + (gamma - 1) / gamma vhat_n, then
    the value at the intermediate time, vhat_{n+alpha_f} = vhat_n +
    alpha_f (vhat_{n+1} - vhat_n); returns (vhat_{n+1}, vhat_{n+alpha_f})."""
    af = ga = 1.0 / (1.0 + rho_inf)
    v1 = (uhat_n1 - uhat_n) / (ga * dt) + (ga - 1.0) / ga * vhat_n
    return v1, vhat_n + af * (v1 - vhat_n)


def tangent(system, assembler, v, p, vdot=None, vhat=None):
    """(A, B, C, D) as scalar CSR matrices: the raw consistent tangent of the
    element loop at the state, K = alpha_m dR/dvdot + alpha_f gamma dt dR/dy
    (the solid displacement moving by (alpha_f gamma dt)^2 / alpha_m), with
    the Dirichlet velocity nodes' rows of A replaced by identity rows and
    their rows of B and columns of A and C removed."""
    am, cf, cu = genalpha_weights(system.params["rho_inf"], system.params["dt"])
    raw = assembler.evaluate(v, p, vd=vdot, vhat=vhat, cm=am, cf=cf, cu=cu, want_mat=True)
    dv = np.repeat(np.asarray(system.mesh.dir_v, dtype=bool), 3)
    keep = sp.diags((~dv).astype(np.float64))
    A = (keep @ to_csr(raw["A"]) @ keep + sp.diags(dv.astype(np.float64))).tocsr()
    B = (keep @ to_csr(raw["B"])).tocsr()
    C = (to_csr(raw["C"]) @ keep).tocsr()
    D = to_csr(raw["D"]).tocsr()
    return A, B, C, D


def corrector(system, assembler, v, p, vdot, u, n_iter: int, newton: bool = False):
    """n_iter corrector iterations; returns the final (v, p, vdot, u) and the
    right-hand-side norms before each solve and after the last update.  With
    newton=True the tangent is re-assembled at every iteration's state."""
    v, p, vdot, u, _, norms = _loop(system, assembler, v, p, vdot, u, n_iter, None, newton)
    return v, p, vdot, u, norms


def corrector_ale(system, assembler, v, p, vdot, u, n_iter: int, L_raw, fluid_id, dir_m, follow,
                  uhat_n, vhat_n, newton: bool = False):
    """As ``corrector`` with the mesh moving inside the loop.  The state
    enters at the same-Y predictor (Sec. 3.5), so u at entry is u_n; each
    iteration takes u_{n+1} = u_n + (u - u_n) / alpha_f, the Dirichlet data
    g_f = u_{n+1} at the fluid node f's node where follow[f] (zero at the
    other Dirichlet mesh nodes), uhat_{n+1} = mesh_displacement(g) and the
    mesh velocity of ``mesh_velocity``, scattered to the nodes of the fluid
    (zero elsewhere).  fluid_id maps a node to its fluid ordinal or -1.
    Returns (v, p, vdot, u, uhat_{n+1}, norms)."""
    mesh = dict(L=L_raw, fid=np.asarray(fluid_id), dir_m=np.asarray(dir_m, dtype=bool),
                follow=np.asarray(follow, dtype=bool), uhat_n=np.asarray(uhat_n, dtype=np.float64),
                vhat_n=np.asarray(vhat_n, dtype=np.float64))
    return _loop(system, assembler, v, p, vdot, u, n_iter, mesh, newton)


def _loop(system, assembler, v, p, vdot, u, n_iter, mesh, newton=False):
    op = BlockOperator.from_system(system)
    lu = None if newton else spl.splu(op.full().tocsc(), permc_spec="MMD_ATA")
    rho_inf, dt = system.params["rho_inf"], system.params["dt"]
    am, cf, cu = genalpha_weights(rho_inf, dt)
    af = 1.0 / (1.0 + rho_inf)
    v, p, vdot, u = (np.array(a, dtype=np.float64) for a in (v, p, vdot, u))
    dirichlet = np.repeat(np.asarray(system.mesh.dir_v, dtype=bool), 3)
    nv3 = v.size
    norms = []
    a_out = getattr(system, "a_out", None) or []
    c_out = getattr(system, "c_out", None) or []
    u_n = u.copy()
    uhat = None
    if mesh is not None:
        nodes = np.flatnonzero(mesh["fid"] >= 0)
        fl = mesh["fid"][nodes]
    for it in range(n_iter + 1):
        vhat = None
        if mesh is not None:
            # steps 3-4: mesh motion driven by the interface displacement
            u1 = (u_n + (u - u_n) / af).reshape(-1, 3)
            g = np.zeros((mesh["dir_m"].size, 3))
            g[fl] = u1[nodes]
            g[~mesh["follow"]] = 0.0
            uhat = mesh_displacement(mesh["L"], mesh["dir_m"], g.ravel())
            _, vh_f = mesh_velocity(uhat, mesh["uhat_n"], mesh["vhat_n"], rho_inf, dt)
            vhat = np.zeros((nv3 // 3, 3))
            vhat[nodes] = vh_f.reshape(-1, 3)[fl]
            vhat = vhat.ravel()
        R = assembler.evaluate(v, p, vd=vdot, u=u, vhat=vhat, want_mat=False)
        Rm = R["Rm"].copy()
        # resistance outlets: traction m_k (a_k^T v) a_k, m_k = c_k / c_f
        for a, c in zip(a_out, c_out):
            Rm += (c / cf) * float(a @ v) * a
        b = -np.concatenate([Rm, R["Rp"]])
        b[:nv3][dirichlet] = 0.0
        norms.append(float(np.linalg.norm(b)))
        if it == n_iter:
            break
        if newton:
            A, B, C, D = tangent(system, assembler, v, p, vdot, vhat)
            for a, c in zip(a_out, c_out):
                a = sp.csr_matrix(np.asarray(a, dtype=np.float64).reshape(-1, 1))
                A = (A + c * (a @ a.T)).tocsr()
            lu = spl.splu(sp.bmat([[A, B], [C, D]], format="csc"), permc_spec="MMD_ATA")
        x = lu.solve(b)
        vdot += am * x[:nv3]
        v += cf * x[:nv3]
        u += cu * x[:nv3]
        p += cf * x[nv3:]
    return v, p, vdot, u, uhat, norms
