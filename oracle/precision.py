"""Rounding to bfloat16 (test infrastructure only).

The mixed-precision path stores the element moduli in bfloat16 (8 significant
bits, float32's exponent range) rounded to nearest, ties to even, directly
from the float64 value.  This module writes that rounding out from its
definition: scale the significand to [128, 256), round half to even, scale
back.  Results are returned as float64 values that bfloat16 represents exactly.
"""

import numpy as np


def round_to_bf16(x):
    """Round float64 values to the nearest bfloat16 (ties to even), as float64."""
    x = np.asarray(x, dtype=np.float64)
    m, e = np.frexp(x)  # x = m * 2**e with 0.5 <= |m| < 1
    return np.ldexp(np.rint(m * 256.0), e - 8)  # np.rint: half to even


def round_to_f32(x):
    """Round float64 values to the nearest float32, as float64."""
    return np.asarray(x, dtype=np.float64).astype(np.float32).astype(np.float64)
