"""Schur complements and the block factorisation (test infrastructure only).

Sec. 5.2.1: calA = L D U with L = [[I, 0], [C A^{-1}, I]],
D = diag(A, S), U = [[I, A^{-1} B], [0, I]], S = D - C A^{-1} B, hence
calA^{-1} = [[I, -A^{-1}B], [0, I]] diag(A^{-1}, S^{-1}) [[I, 0], [-C A^{-1}, I]].
The sparse approximation used to build P_S is Shat = D - C diag(A)^{-1} B
with diag(A) the scalar diagonal of A; SIMPLEC replaces diag(A) by the
diagonal lumped from the absolute values of A's entries.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .sparse import BlockOperator


def simple_diagonal(op: BlockOperator, lumped: bool = False) -> np.ndarray:
    """The diagonal approximation of A used by Shat and P_SIMPLE: diag(A);
    lumped=True: the diagonal lumped from the absolute values of A's entries,
    d_i = sum_j |a_ij| (SIMPLEC, Sec. 5.2.1)."""
    if lumped:
        return np.asarray(abs(op.A).sum(axis=1)).ravel()
    return op.A.diagonal()


def schur_hat(op: BlockOperator, lumped: bool = False) -> sp.csr_matrix:
    """Shat = D - C diag(A)^{-1} B (Sec. 5.2.1); lumped=True takes the
    SIMPLEC diagonal instead of diag(A)."""
    dinv = sp.diags(1.0 / simple_diagonal(op, lumped))
    S = (op.D - op.C @ dinv @ op.B).tocsr()
    S.sum_duplicates()
    S.sort_indices()
    return S


def schur_exact_dense(op: BlockOperator) -> np.ndarray:
    """S = D - C A^{-1} B, dense (tiny systems only)."""
    A = op.A.toarray()
    return op.D.toarray() - op.C.toarray() @ np.linalg.solve(A, op.B.toarray())


def ldu_factors_dense(op: BlockOperator):
    """The three factors of the block LDU factorisation (Sec. 5.2.1)."""
    A, B, C = op.A.toarray(), op.B.toarray(), op.C.toarray()
    S = schur_exact_dense(op)
    nv, np_ = op.nv, op.np
    Ainv = np.linalg.inv(A)
    Lf = np.block([[np.eye(nv), np.zeros((nv, np_))], [C @ Ainv, np.eye(np_)]])
    Df = np.block([[A, np.zeros((nv, np_))], [np.zeros((np_, nv)), S]])
    Uf = np.block([[np.eye(nv), Ainv @ B], [np.zeros((np_, nv)), np.eye(np_)]])
    return Lf, Df, Uf


def scr_exact_apply(op: BlockOperator, r: np.ndarray) -> np.ndarray:
    """Algorithm 1 with every inner solve exact (dense): equals calA^{-1} r."""
    A = op.A.toarray()
    S = schur_exact_dense(op)
    rv, rp = op.split(np.asarray(r, dtype=np.float64))
    yv_hat = np.linalg.solve(A, rv)
    rp2 = rp - op.C @ yv_hat
    yp = np.linalg.solve(S, rp2)
    rv2 = rv - op.B @ yp
    yv = np.linalg.solve(A, rv2)
    return np.concatenate([yv, yp])


def simple_matrix_dense(op: BlockOperator, lumped: bool = False) -> np.ndarray:
    """P_SIMPLE = [[A, A diag(A)^{-1} B], [C, D]] (Sec. 5.2.1); lumped=True:
    P_SIMPLEC, the same with the lumped diagonal."""
    A, B, C, D = (M.toarray() for M in (op.A, op.B, op.C, op.D))
    dinv = np.diag(1.0 / simple_diagonal(op, lumped))
    return np.block([[A, A @ dinv @ B], [C, D]])


def simple_factored_dense(op: BlockOperator, lumped: bool = False) -> np.ndarray:
    """The factored form L diag(A, Shat) U_SIMPLE of P_SIMPLE (Sec. 5.2.1),
    U_SIMPLE = [[I, diag(A)^{-1} B], [0, I]] (lumped: the SIMPLEC diagonal in
    Shat and U)."""
    A, B, C = op.A.toarray(), op.B.toarray(), op.C.toarray()
    Sh = schur_hat(op, lumped).toarray()
    nv, np_ = op.nv, op.np
    Ainv = np.linalg.inv(A)
    dinv = np.diag(1.0 / simple_diagonal(op, lumped))
    Lf = np.block([[np.eye(nv), np.zeros((nv, np_))], [C @ Ainv, np.eye(np_)]])
    Df = np.block([[A, np.zeros((nv, np_))], [np.zeros((np_, nv)), Sh]])
    Uf = np.block([[np.eye(nv), dinv @ B], [np.zeros((np_, nv)), np.eye(np_)]])
    return Lf @ Df @ Uf


def simple_inverse_apply_dense(op: BlockOperator, r: np.ndarray, lumped: bool = False) -> np.ndarray:
    """P_SIMPLE^{-1} r with exact solves (dense): U_SIMPLE^{-1} diag(A, Shat)^{-1} L^{-1} r
    (lumped: P_SIMPLEC^{-1} r)."""
    A = op.A.toarray()
    Sh = schur_hat(op, lumped).toarray()
    rv, rp = op.split(np.asarray(r, dtype=np.float64))
    yv_hat = np.linalg.solve(A, rv)
    yp = np.linalg.solve(Sh, rp - op.C @ yv_hat)
    yv = yv_hat - (op.B @ yp) / simple_diagonal(op, lumped)
    return np.concatenate([yv, yp])
