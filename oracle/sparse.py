"""Block-sparse matrices for the oracle (test infrastructure only).

A block matrix arrives as (br, bc, row_ptr, col, val) with blocks stored
row-major one after another (the BSR container of ``fsi_inputs``).  The
oracle turns it into a scipy CSR matrix of scalars and uses scipy's
matrix-vector product as its library primitive.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def to_csr(M) -> sp.csr_matrix:
    """Scalar CSR of a block matrix (explicit zeros kept out)."""
    blocks = np.asarray(M.val, dtype=np.float64).reshape(-1, M.br, M.bc)
    out = sp.bsr_matrix((blocks, np.asarray(M.col), np.asarray(M.row_ptr)),
                        shape=(M.nb_rows * M.br, M.nb_cols * M.bc)).tocsr()
    out.sum_duplicates()
    return out


def bsr_matvec_by_definition(M, x: np.ndarray) -> np.ndarray:
    """y_I = sum_J M_IJ x_J over the stored blocks, written out block by
    block: the definition a block SpMV must reproduce."""
    x = np.asarray(x, dtype=np.float64)
    y = np.zeros(M.nb_rows * M.br)
    blocks = np.asarray(M.val).reshape(-1, M.br, M.bc)
    rows = np.repeat(np.arange(M.nb_rows), np.diff(M.row_ptr))
    xb = x.reshape(M.nb_cols, M.bc)[M.col]            # (nnzb, bc)
    contrib = np.einsum("nij,nj->ni", blocks, xb)      # (nnzb, br)
    yb = y.reshape(M.nb_rows, M.br)
    np.add.at(yb, rows, contrib)
    return y


class BlockOperator:
    """The 2x2 block matrix calA = [[A, B], [C, D]] of Sec. 5.2.1 with the
    vector split x = [x_v; x_p]."""

    def __init__(self, A, B, C, D, a_out=None, c_out=None):
        self.A_sparse = to_csr(A)
        self.A = self.A_sparse
        # resistance outlets (Sec. 3.5, outlet coupling matrix): the momentum
        # block is A + sum_k c_k a_k a_k^T, written out as explicit entries
        # on the outlet rows and columns
        if a_out is not None:
            for a, c in zip(a_out, c_out):
                a = sp.csr_matrix(np.asarray(a, dtype=np.float64).reshape(-1, 1))
                self.A = (self.A + c * (a @ a.T)).tocsr()
            self.A.sum_duplicates()
            self.A.sort_indices()
        self.B = to_csr(B)
        self.C = to_csr(C)
        self.D = to_csr(D)
        self.nv = self.A.shape[0]
        self.np = self.D.shape[0]
        self.n = self.nv + self.np

    @classmethod
    def from_system(cls, s) -> "BlockOperator":
        return cls(s.A, s.B, s.C, s.D, getattr(s, "a_out", None), getattr(s, "c_out", None))

    def split(self, x):
        return x[: self.nv], x[self.nv:]

    def matvec(self, x: np.ndarray) -> np.ndarray:
        xv, xp = self.split(x)
        return np.concatenate([self.A @ xv + self.B @ xp, self.C @ xv + self.D @ xp])

    def full(self) -> sp.csr_matrix:
        return sp.bmat([[self.A, self.B], [self.C, self.D]], format="csr")


def rel_residual(op: BlockOperator, x: np.ndarray, b: np.ndarray) -> float:
    """||b - calA x||_2 / ||b||_2 (unweighted l2 norm, as in the stopping
    criteria of the multi-corrector, Sec. 3.5)."""
    nb = np.linalg.norm(b)
    r = b - op.matvec(x)
    return float(np.linalg.norm(r) / nb) if nb > 0 else float(np.linalg.norm(r))
