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
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spl

from .sparse import BlockOperator


def genalpha_weights(rho_inf: float, dt: float):
    """alpha_m = (3 - rho_inf) / (2 (1 + rho_inf)), alpha_f = gamma =
    1 / (1 + rho_inf) (Sec. 3.4); returns (alpha_m, c_f, c_u)."""
    am = 0.5 * (3.0 - rho_inf) / (1.0 + rho_inf)
    af = ga = 1.0 / (1.0 + rho_inf)
    cf = af * ga * dt
    return am, cf, cf * cf / am


def corrector(system, assembler, v, p, vdot, u, n_iter: int):
    """n_iter corrector iterations; returns the final (v, p, vdot, u) and the
    right-hand-side norms before each solve and after the last update."""
    op = BlockOperator.from_system(system)
    lu = spl.splu(op.full().tocsc(), permc_spec="MMD_ATA")
    am, cf, cu = genalpha_weights(system.params["rho_inf"], system.params["dt"])
    v, p, vdot, u = (np.array(a, dtype=np.float64) for a in (v, p, vdot, u))
    dirichlet = np.repeat(np.asarray(system.mesh.dir_v, dtype=bool), 3)
    nv3 = v.size
    norms = []
    a_out = getattr(system, "a_out", None) or []
    c_out = getattr(system, "c_out", None) or []
    for it in range(n_iter + 1):
        R = assembler.evaluate(v, p, vd=vdot, u=u, want_mat=False)
        Rm = R["Rm"].copy()
        # resistance outlets: traction m_k (a_k^T v) a_k, m_k = c_k / c_f
        for a, c in zip(a_out, c_out):
            Rm += (c / cf) * float(a @ v) * a
        b = -np.concatenate([Rm, R["Rp"]])
        b[:nv3][dirichlet] = 0.0
        norms.append(float(np.linalg.norm(b)))
        if it == n_iter:
            break
        x = lu.solve(b)
        vdot += am * x[:nv3]
        v += cf * x[:nv3]
        u += cu * x[:nv3]
        p += cf * x[nv3:]
    return v, p, vdot, u, norms
