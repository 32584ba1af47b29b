"""Exact solutions by sparse LU (test infrastructure only).

The SCR-FGMRES iteration of Sec. 5.2.1 approaches x* = calA^{-1} b; the
oracle's answer is that x* itself, obtained with SuperLU (a library sparse
LU with partial pivoting) on the assembled block matrix.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spl

from .sparse import BlockOperator, to_csr


def solve_block(s) -> np.ndarray:
    """x* with calA x* = b for a block system (Sec. 5.2.1)."""
    op = BlockOperator.from_system(s)
    K = op.full().tocsc()
    lu = spl.splu(K, permc_spec="MMD_ATA")
    return lu.solve(np.asarray(s.b, dtype=np.float64))


def solve_mesh(s) -> np.ndarray:
    """U with (L kron I3) U = g for the harmonic-extension system, each of
    the three displacement components solved with the same L (Sec. 2.2)."""
    L = to_csr(s.L).tocsc()
    lu = spl.splu(L, permc_spec="MMD_AT_PLUS_A")
    g = np.asarray(s.mesh_b, dtype=np.float64).reshape(-1, 3)
    return np.column_stack([lu.solve(g[:, c].copy()) for c in range(3)]).reshape(-1)


def solve_block_many(s, rhs) -> list[np.ndarray]:
    """x*_c with calA x*_c = b_c for several right-hand sides of one block
    system (one LU, one solve per column)."""
    op = BlockOperator.from_system(s)
    lu = spl.splu(op.full().tocsc(), permc_spec="MMD_ATA")
    return [lu.solve(np.asarray(b, dtype=np.float64)) for b in rhs]
