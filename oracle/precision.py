"""Storage formats of the mixed-precision form (test infrastructure only).

The paper computes in FP64 throughout; the mixed-precision form of this
library stores the preconditioner's matrices in narrower formats.  These
functions give the value a stored FP64 number takes in each format, by the
formats' definitions:

* binary32 (IEEE 754 single): round to nearest, ties to even;
* bfloat16: the upper 16 bits of a binary32 (sign, 8 exponent bits, 7
  stored mantissa bits), reached from the binary32 value by round to
  nearest, ties to even on the 16 discarded bits.

Values are returned as FP64 arrays holding the rounded numbers exactly.
"""
from __future__ import annotations

import numpy as np


def round_f32(a) -> np.ndarray:
    """FP64 -> binary32 -> FP64 (round to nearest even)."""
    return np.asarray(a, dtype=np.float64).astype(np.float32).astype(np.float64)


def round_bf16(a) -> np.ndarray:
    """FP64 -> binary32 -> bfloat16 -> FP64, each step round to nearest even.

    On the binary32 bit pattern u: add 0x7FFF plus the lowest kept bit
    (bit 16), then clear the 16 low bits; a carry out of the mantissa moves
    into the exponent, which is the correct rounding across a binade."""
    f = np.ascontiguousarray(np.asarray(a, dtype=np.float64).astype(np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)
