"""GB300 (sm_103a) SCR-FGMRES + AMG solver for the vascular FSI block system.

Thin Python binding of the C ABI declared in ``include/scr_gb300.h``: it
marshals arguments (numpy arrays for host pointers, torch CUDA tensors for
device pointers) and calls the library; every arithmetic step of the solve
runs in the library's CUDA kernels.  There is no CPU fallback: importing a
solver without the built library raises.
"""
from .abi import (SCR_FP64, SCR_MIXED, SCR_PC_SCR, SCR_PC_SIMPLE, SCR_PC_SIMPLEC, SCR_HIER_A, SCR_HIER_SHAT, SCR_HIER_MESH,  # noqa: F401
                  SCR_EXPORT_OPERATOR, SCR_EXPORT_PROLONGATOR, SCR_EXPORT_AGGREGATES, SCR_EXPORT_ROOTS,
                  SCR_EXPORT_BLOCK_B, SCR_EXPORT_BLOCK_C, SCR_EXPORT_BLOCK_D,
                  ScrError, load_library, library_path)
from .solver import BlockSolver, DeviceBSR, bsr_spmv, bsr_spmv_noalloc, tune_load, tune_save  # noqa: F401

__all__ = ["BlockSolver", "DeviceBSR", "bsr_spmv", "ScrError", "load_library", "library_path",
           "SCR_FP64", "SCR_MIXED"]
