"""Small numeric helpers shared by the GPU test modules."""
import numpy as np


def round_tf32(x):
    """FP32 values rounded to TF32 (10 mantissa bits), nearest with ties to even, on the
    bit pattern; infinities and NaNs unchanged."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    finite = (u & 0x7F800000) != 0x7F800000
    r = ((u + 0xFFF + ((u >> 13) & 1)) & 0xFFFFE000) & 0xFFFFFFFF
    return np.where(finite, r, u).astype(np.uint32).view(np.float32)
