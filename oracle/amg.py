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
   max_i sum_j |a_ij| / |a_ii| of D^{-1} A, then truncated as the paper's
   AMG settings do for interpolation (truncation factor, at most P_max
   entries per row; table of AMG settings, Sec. 5.2): in each block row keep
   the blocks whose Frobenius norm is at least trunc times the row's largest
   and, among those, the P_max largest (ties: smaller column first); each
   scalar row is rescaled so that its sum is unchanged;
5. Galerkin coarse operator A_c = P^T A P, restriction R = P^T;
6. V-cycle: pre-smoothing from x = 0, residual, restriction, recursion,
   prolongation, post-smoothing; exact dense LU on the coarsest level.
   Smoothers: l1-Jacobi x <- x + D_l1^{-1} (b - A x), D_l1 = diag(sum_j
   |a_ij|) (nu sweeps), or Chebyshev of degree k on D^{-1} A over
   [lambda/30, lambda], lambda = 1.1 x the power-iteration estimate of the
   largest eigenvalue of D^{-1} A (20 iterations from a fixed start
   vector), written as the three-term recurrence of Chebyshev acceleration
   (Saad, Iterative Methods for Sparse Linear Systems, Alg. 12.1).
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
    dinv: np.ndarray | None = None   # 1 / diag(A)
    lam: float = 0.0                 # 1.1 x power-iteration estimate of rho(D^{-1} A)
    cheb: bool = True                # Chebyshev smoothing on this level (else l1-Jacobi)


@dataclasses.dataclass
class Hierarchy:
    levels: list
    coarse_lu: tuple
    nu_pre: int = 1
    nu_post: int = 1
    smoother: str = "l1"     # "l1" or "cheb"
    cheb_degree: int = 3

    @property
    def n_levels(self) -> int:
        return len(self.levels)


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


def truncate_to_pattern(P: sp.csr_matrix, bs: int, indptr: np.ndarray, indices: np.ndarray) -> sp.csr_matrix:
    """The truncation of step 4 with its kept block positions given (the
    block pattern indptr / indices, a subset of P's blocks in every row), as
    a numeric re-set-up keeps them: the kept blocks of each scalar row are
    rescaled by (sum of the row) / (sum of its kept entries)."""
    B = sp.bsr_matrix(P, blocksize=(bs, bs))
    B.sort_indices()
    nbr = B.shape[0] // bs
    rows = np.repeat(np.arange(nbr), np.diff(B.indptr))
    keep_set = set(zip(np.repeat(np.arange(nbr), np.diff(indptr)).tolist(), np.asarray(indices).tolist()))
    keep = np.array([(r, c) in keep_set for r, c in zip(rows.tolist(), B.indices.tolist())], dtype=bool)
    data = B.data.copy()
    s_all = np.zeros((nbr, bs))
    s_kept = np.zeros((nbr, bs))
    np.add.at(s_all, rows, data.sum(axis=2))
    np.add.at(s_kept, rows, (data * keep[:, None, None]).sum(axis=2))
    scale = np.where(s_kept != 0.0, s_all / np.where(s_kept != 0.0, s_kept, 1.0), 1.0)
    data = data * scale[rows][:, :, None]
    k = np.nonzero(keep)[0]
    ip = np.concatenate([[0], np.cumsum(np.bincount(rows[k], minlength=nbr))])
    out = sp.bsr_matrix((data[k], B.indices[k], ip), shape=P.shape).tocsr()
    out.sort_indices()
    return out


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


def truncate_prolongator(P: sp.csr_matrix, bs: int, trunc: float, pmax: int) -> sp.csr_matrix:
    """Interpolation truncation of step 4 (blocks of size bs)."""
    if trunc <= 0.0 and pmax <= 0:
        return P
    B = sp.bsr_matrix(P, blocksize=(bs, bs))
    B.sort_indices()
    nbr = B.shape[0] // bs
    rows = np.repeat(np.arange(nbr), np.diff(B.indptr))
    cols = B.indices
    norms = np.sqrt((B.data ** 2).sum(axis=(1, 2)))
    rowmax = np.zeros(nbr)
    np.maximum.at(rowmax, rows, norms)
    keep = (norms > 0) & (norms >= trunc * rowmax[rows])
    if pmax > 0:
        # rank within the row by (norm descending, column ascending)
        order = np.lexsort((cols, -norms, rows))
        rank = np.empty_like(order)
        start = B.indptr[rows[order]]
        rank[order] = np.arange(order.size) - start
        # ranks count every block; the candidate set is a prefix of that order
        cand_rank = np.zeros_like(rank)
        kept_sorted = keep[order]
        csum = np.cumsum(kept_sorted)
        row_first = B.indptr[:-1]
        before = np.zeros(nbr, dtype=np.int64)
        nz = np.diff(B.indptr) > 0
        before[nz] = (csum - kept_sorted)[row_first[nz] - 0]
        cand_rank[order] = csum - kept_sorted - before[rows[order]]
        keep &= cand_rank < pmax
    data = B.data.copy()
    # row sums per scalar row before and after
    s_all = np.zeros((nbr, bs))
    s_kept = np.zeros((nbr, bs))
    np.add.at(s_all, rows, data.sum(axis=2))
    np.add.at(s_kept, rows, (data * keep[:, None, None]).sum(axis=2))
    scale = np.where(s_kept != 0.0, s_all / np.where(s_kept != 0.0, s_kept, 1.0), 1.0)
    data = data * scale[rows][:, :, None]
    k = np.nonzero(keep)[0]
    indptr = np.concatenate([[0], np.cumsum(np.bincount(rows[k], minlength=nbr))])
    out = sp.bsr_matrix((data[k], cols[k], indptr), shape=P.shape).tocsr()
    out.sort_indices()
    return out


POWER_ITERS = 20


def power_start(n: int) -> np.ndarray:
    """Fixed start vector 1 + ((i * 2654435761) mod 2^32 mod 1000) / 1000."""
    i = np.arange(n, dtype=np.uint64)
    return 1.0 + (((i * np.uint64(2654435761)) % np.uint64(2 ** 32)) % np.uint64(1000)).astype(np.float64) / 1000.0


def power_lambda(A: sp.csr_matrix, dinv: np.ndarray, iters: int = POWER_ITERS) -> float:
    """Power iteration on D^{-1} A: v <- w / ||w||, w = D^{-1} A v, from the
    normalised fixed start vector; returns 1.1 ||w|| of the last step."""
    v = power_start(A.shape[0])
    v = v / np.linalg.norm(v)
    lam = 0.0
    for _ in range(iters):
        w = (A @ v) * dinv
        lam = np.linalg.norm(w)
        if lam == 0.0:
            break
        v = w / lam
    return 1.1 * lam


def cheb_coefficients(lam: float, degree: int):
    """theta and the (alpha_j, beta_j) of the Chebyshev recurrence on
    [lam/30, lam]."""
    lo, hi = lam / 30.0, lam
    theta, delta = (hi + lo) / 2.0, (hi - lo) / 2.0
    sigma = theta / delta
    rho = 1.0 / sigma
    steps = []
    for _ in range(degree - 1):
        rho_new = 1.0 / (2.0 * sigma - rho)
        steps.append((rho_new * rho, 2.0 * rho_new / delta))
        rho = rho_new
    return theta, steps


def cheb_smooth(A, dinv, lam, degree, x, b, from_zero: bool):
    """Degree-`degree` Chebyshev smoothing of A x = b (preconditioned by
    D^{-1}); x may be (n,) or (n, k)."""
    theta, steps = cheb_coefficients(lam, degree)
    dv = dinv if b.ndim == 1 else dinv[:, None]
    r = b * dv if from_zero else (b - A @ x) * dv
    d = r / theta
    x = d.copy() if from_zero else x + d
    for a, c in steps:
        r = r - (A @ d) * dv
        d = a * d + c * r
        x = x + d
    return x


def l1_diag(A: sp.csr_matrix) -> np.ndarray:
    return np.asarray(abs(A).sum(axis=1)).ravel()


# Chebyshev guard: the smoother's error propagation is run CHEB_GUARD_SWEEPS
# times on the homogeneous problem from the normalised power-iteration start
# vector; a level whose error grows beyond CHEB_GUARD_GROWTH uses l1-Jacobi
# instead (nonsymmetric coarse operators, e.g. Galerkin levels of Shat, can
# have eigenvalues of D^{-1} A off the interval [lam/30, lam], where the
# polynomial amplifies instead of damping).
CHEB_GUARD_SWEEPS = 5
CHEB_GUARD_GROWTH = 10.0


def cheb_guard_growth(A: sp.csr_matrix, dinv: np.ndarray, lam: float, degree: int) -> float:
    """||e_5|| for e_0 = the normalised start vector, e_{k+1} = the
    Chebyshev smoother applied to A e = 0 from e_k."""
    e = power_start(A.shape[0])
    e = e / np.linalg.norm(e)
    zero = np.zeros_like(e)
    for _ in range(CHEB_GUARD_SWEEPS):
        e = cheb_smooth(A, dinv, lam, degree, e, zero, False)
    return float(np.linalg.norm(e))


def _finish_levels(levels, smoother: str, cheb_degree: int = 3):
    for l, lev in enumerate(levels):
        lev.dinv = 1.0 / lev.A.diagonal()
        if smoother == "cheb":
            lev.lam = power_lambda(lev.A, lev.dinv)
            if l + 1 < len(levels):
                lev.cheb = cheb_guard_growth(lev.A, lev.dinv, lev.lam, cheb_degree) <= CHEB_GUARD_GROWTH


def setup(A: sp.csr_matrix, bs: int, theta: float = 0.08, max_levels: int = 10,
          coarse_size: int = 64, nu_pre: int = 1, nu_post: int = 1, trunc: float = 0.0,
          pmax: int = 0, smoother: str = "l1", cheb_degree: int = 3) -> Hierarchy:
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
        P = truncate_prolongator(P, bs, trunc, pmax)
        R = P.T.tocsr()
        Ac = (R @ Al @ P).tocsr()
        Ac.sum_duplicates()
        Ac.sort_indices()
        lev.P, lev.R, lev.agg, lev.omega = P, R, agg, omega
        Al = Ac
    lu = sla.lu_factor(levels[-1].A.toarray())
    _finish_levels(levels, smoother, cheb_degree)
    return Hierarchy(levels=levels, coarse_lu=lu, nu_pre=nu_pre, nu_post=nu_post, smoother=smoother,
                     cheb_degree=cheb_degree)


def hierarchy_from_matrices(As, Ps, bs: int, nu_pre: int = 1, nu_post: int = 1, smoother: str = "l1",
                            cheb_degree: int = 3) -> Hierarchy:
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
    _finish_levels(levels, smoother, cheb_degree)
    return Hierarchy(levels=levels, coarse_lu=lu, nu_pre=nu_pre, nu_post=nu_post, smoother=smoother,
                     cheb_degree=cheb_degree)


def vcycle(H: Hierarchy, b: np.ndarray, level: int = 0) -> np.ndarray:
    """One V-cycle from x = 0 (step 6); b may be (n,) or (n, k)."""
    lev = H.levels[level]
    b = np.asarray(b, dtype=np.float64)
    if level == H.n_levels - 1:
        return sla.lu_solve(H.coarse_lu, b)
    if H.smoother == "cheb" and lev.cheb:
        x = cheb_smooth(lev.A, lev.dinv, lev.lam, H.cheb_degree, None, b, True)
        r = b - lev.A @ x
        x = x + lev.P @ vcycle(H, lev.R @ r, level + 1)
        return cheb_smooth(lev.A, lev.dinv, lev.lam, H.cheb_degree, x, b, False)
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
