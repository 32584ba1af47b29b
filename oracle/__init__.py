"""CPU FP64 oracle for the SCR-FGMRES + AMG block solve and the mesh AMG-CG.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this
package: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may use it.  It shares no code with the CUDA library.

Contents (each function cites the passage of the paper it restates):

* ``sparse``  - block-sparse matrices as plain scipy operators, the block
                operator of Sec. 5.2.1 and its products by definition.
* ``direct``  - the exact solution x* = calA^{-1} b by a sparse LU
                (SuperLU), the definition of what the iterative path reaches.
* ``schur``   - the Schur complement S = D - C A^{-1} B and its sparse
                approximation Shat = D - C diag(A)^{-1} B (Sec. 5.2.1), the
                block LDU factorisation and its inverse, P_SIMPLE.
* ``krylov``  - FGMRES (Saad 1993) with classical Gram-Schmidt applied
                twice and Givens rotations, GMRES, preconditioned CG.
* ``amg``     - a plain smoothed-aggregation AMG (strength graph,
                greedy aggregation, tentative and smoothed prolongators,
                Galerkin products) and the V-cycle with l1-Jacobi smoothing.
* ``precision`` - the value an FP64 number takes when stored in binary32 or
                bfloat16 (the storage formats of the mixed-precision form).
* ``scr``     - Algorithm 1 (SCR preconditioner action) and Algorithm 2
                (matrix-free Schur complement action) of App. B, the outer
                FGMRES solve of Sec. 5.2.1 and the mesh-motion AMG-CG of
                Sec. 5.2.2.

Parity status: every function here is pinned by a ``-m "not gpu"`` test
(closed forms, brute force on tiny systems, invariants); see tests/.
"""
