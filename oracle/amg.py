"""Smoothed-aggregation AMG (test infrastructure only).

The paper preconditions A, Shat and the mesh Laplacian with an AMG V-cycle
(Sec. 5.2, Table of BoomerAMG settings; P_A = P_I = AMG(A), P_S = AMG(Shat),
mesh CG + AMG in Sec. 5.2.2).  The solver here uses smoothed aggregation
instead of the paper's classical AMG; this module is the plain CPU
statement of that method (Vanek, Mandel, Brezina 1996):

1. strength graph: block i ~ j (i != j) is strong when
   ||A_ij|| >= theta * sqrt(||A_ii|| ||A_jj||), ||.|| the Frobenius norm of
   the block (the absolute value for scalar matrices);
2. aggregation: every node with a strong neighbour joins exactly one
   aggregate; nodes without one (for instance Dirichlet identity rows) are
   left out of the coarse space;
3. tentative prolongator: the near-nullspace of constants, one per
   component of a block, normalised on each aggregate:
   P_tent[i, a] = I_bs / sqrt(|a|) for node i in aggregate a;
4. smoothed prolongator P = (I - omega D^{-1} A) P_tent with D the scalar
   diagonal of A and omega = 4 / (3 lambda), lambda the Gershgorin bound
   max_i sum_j |a_ij| / |a_ii| of D^{-1} A;
5. Galerkin coarse operator A_c = P^T A P, restriction R = P^T;
6. V-cycle: l1-Jacobi smoothing x <- x + D_l1^{-1} (b - A x) with
   D_l1 = diag(sum_j |a_ij|), nu_pre sweeps from x = 0, residual,
   restriction, recursion, prolongation, nu_post sweeps; exact dense LU
   on the coarsest level.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp


@dataclasses.dataclass
class Level:
    A: sp.csr_matrix
    bs: int
    dl1: np.ndarray
    P: sp.csr_matrix | None = None
    R: sp.csr_matrix | None = None
    agg: np.ndarray | None = None
    omega: float = 0.0


@dataclasses.dataclass
class Hierarchy:
    levels: list
    coarse_lu: tuple
    nu_pre: int = 1
    nu_post: int = 1

    @property
    def n_levels(self) -> int:
        return len(self.levels)

    def operator_complexity(self) -> float:
        return sum(l.A.nnz for l in self.levels) / self.levels[0].A.nnz


def block_norms(A: sp.csr_matrix, bs: int):
    """(rows, cols, norms) of the bs x bs blocks of A."""
    if bs == 1:
        C = A.tocoo()
        return C.row, C.col, np.abs(C.data)
    B = sp.bsr_matrix(A, blocksize=(bs, bs))
    B.sort_indices()
    rows = np.repeat(np.arange(B.shape[0] // bs), np.diff(B.indptr))
    norms = np.sqrt((B.data ** 2).sum(axis=(1, 2)))
    return rows, B.indices.copy(), norms


def strength_graph(A: sp.csr_matrix, bs: int, theta: float) -> sp.csr_matrix:
    """Symmetric strong-connection graph over block rows (step 1)."""
    rows, cols, nrm = block_norms(A, bs)
    n = A.shape[0] // bs
    diag = np.zeros(n)
    on = rows == cols
    diag[rows[on]] = nrm[on]
    off = (rows != cols) & (nrm > 0)
    r, c, v = rows[off], cols[off], nrm[off]
    strong = v >= theta * np.sqrt(diag[r] * diag[c])
    S = sp.csr_matrix((v[strong], (r[strong], c[strong])), shape=(n, n))
    S = S.maximum(S.T).tocsr()     # symmetrise
    S.sort_indices()
    return S


def aggregate_greedy(S: sp.csr_matrix) -> np.ndarray:
    """Greedy aggregation (step 2): pass 1 makes an aggregate of every node
    whose strong neighbourhood is still free; pass 2 attaches each remaining
    node to the pass-1 aggregate of its strongest neighbour; pass 3 groups
    what is left with its free neighbours.  Returns agg[i] (-1: none)."""
    n = S.shape[0]
    ip, ix, dv = S.indptr, S.indices, S.data
    agg = -np.ones(n, dtype=np.int64)
    na = 0
    for i in range(n):
        nb = ix[ip[i]:ip[i + 1]]
        if nb.size == 0 or agg[i] >= 0:
            continue
        if np.all(agg[nb] < 0):
            agg[i] = na
            agg[nb] = na
            na += 1
    snap = agg.copy()
    for i in range(n):
        if agg[i] >= 0:
            continue
        nb = ix[ip[i]:ip[i + 1]]
        if nb.size == 0:
            continue
        w = dv[ip[i]:ip[i + 1]]
        cand = snap[nb] >= 0
        if np.any(cand):
            j = nb[cand][np.argmax(w[cand])]
            agg[i] = snap[j]
    for i in range(n):
        if agg[i] >= 0:
            continue
        nb = ix[ip[i]:ip[i + 1]]
        if nb.size == 0:
            continue
        agg[i] = na
        free = nb[agg[nb] < 0]
        agg[free] = na
        na += 1
    return agg


def tentative_prolongator(agg: np.ndarray, bs: int) -> sp.csr_matrix:
    """P_tent[i, a] = I_bs / sqrt(|a|) (step 3)."""
    n = agg.shape[0]
    na = int(agg.max()) + 1 if agg.size and agg.max() >= 0 else 0
    sizes = np.bincount(agg[agg >= 0], minlength=na).astype(np.float64)
    nodes = np.nonzero(agg >= 0)[0]
    rows = (nodes[:, None] * bs + np.arange(bs)[None, :]).ravel()
    cols = (agg[nodes][:, None] * bs + np.arange(bs)[None, :]).ravel()
    vals = np.repeat(1.0 / np.sqrt(sizes[agg[nodes]]), bs)
    return sp.csr_matrix((vals, (rows, cols)), shape=(n * bs, na * bs))


def gershgorin_dinv_a(A: sp.csr_matrix) -> float:
    """max_i sum_j |a_ij| / |a_ii| (an upper bound of rho(D^{-1} A))."""
    absrow = np.asarray(abs(A).sum(axis=1)).ravel()
    d = np.abs(A.diagonal())
    return float(np.max(absrow / d))


def smoothed_prolongator(A: sp.csr_matrix, Pt: sp.csr_matrix):
    """P = (I - omega D^{-1} A) P_tent, omega = 4/(3 lambda) (step 4)."""
    lam = gershgorin_dinv_a(A)
    omega = 4.0 / (3.0 * lam)
    Dinv = sp.diags(1.0 / A.diagonal())
    P = (Pt - omega * (Dinv @ (A @ Pt))).tocsr()
    P.sum_duplicates()
    P.sort_indices()
    return P, omega


def l1_diag(A: sp.csr_matrix) -> np.ndarray:
    return np.asarray(abs(A).sum(axis=1)).ravel()


def setup(A: sp.csr_matrix, bs: int, theta: float = 0.08, max_levels: int = 10,
          coarse_size: int = 64, nu_pre: int = 1, nu_post: int = 1) -> Hierarchy:
    """Build the hierarchy (steps 1-5); coarse_size counts block rows."""
    levels = []
    Al = A.tocsr()
    while True:
        lev = Level(A=Al, bs=bs, dl1=l1_diag(Al))
        levels.append(lev)
        nb = Al.shape[0] // bs
        if nb <= coarse_size or len(levels) >= max_levels:
            break
        S = strength_graph(Al, bs, theta)
        agg = aggregate_greedy(S)
        na = int(agg.max()) + 1 if agg.max() >= 0 else 0
        if na == 0 or na >= nb:
            break
        Pt = tentative_prolongator(agg, bs)
        P, omega = smoothed_prolongator(Al, Pt)
        R = P.T.tocsr()
        Ac = (R @ Al @ P).tocsr()
        Ac.sum_duplicates()
        Ac.sort_indices()
        lev.P, lev.R, lev.agg, lev.omega = P, R, agg, omega
        Al = Ac
    lu = sla.lu_factor(levels[-1].A.toarray())
    return Hierarchy(levels=levels, coarse_lu=lu, nu_pre=nu_pre, nu_post=nu_post)


def hierarchy_from_matrices(As, Ps, bs: int, nu_pre: int = 1, nu_post: int = 1) -> Hierarchy:
    """A hierarchy from given operators (A_0..A_L) and prolongators
    (P_0..P_{L-1}), e.g. ones exported from another implementation."""
    levels = []
    for l, A in enumerate(As):
        A = sp.csr_matrix(A)
        lev = Level(A=A, bs=bs, dl1=l1_diag(A))
        if l < len(Ps):
            lev.P = sp.csr_matrix(Ps[l])
            lev.R = lev.P.T.tocsr()
        levels.append(lev)
    lu = sla.lu_factor(levels[-1].A.toarray())
    return Hierarchy(levels=levels, coarse_lu=lu, nu_pre=nu_pre, nu_post=nu_post)


def vcycle(H: Hierarchy, b: np.ndarray, level: int = 0) -> np.ndarray:
    """One V-cycle from x = 0 (step 6); b may be (n,) or (n, k)."""
    lev = H.levels[level]
    b = np.asarray(b, dtype=np.float64)
    if level == H.n_levels - 1:
        return sla.lu_solve(H.coarse_lu, b)
    d = lev.dl1 if b.ndim == 1 else lev.dl1[:, None]
    x = np.zeros_like(b)
    for _ in range(H.nu_pre):
        x = x + (b - lev.A @ x) / d
    r = b - lev.A @ x
    ec = vcycle(H, lev.R @ r, level + 1)
    x = x + lev.P @ ec
    for _ in range(H.nu_post):
        x = x + (b - lev.A @ x) / d
    return x
