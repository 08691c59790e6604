"""Element-wise error measure used beside the relative Frobenius norm in the
GPU parity tests: a Frobenius ratio of a large matrix can hide an error
confined to one block, the largest element error cannot."""

import numpy as np


def max_rel_err(got, ref):
    """max |got - ref| over every element (so over every block), divided by
    max |ref|."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    scale = np.max(np.abs(ref))
    return float(np.max(np.abs(got - ref)) / scale) if scale > 0 else float(np.max(np.abs(got)))
