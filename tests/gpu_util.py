"""Helpers for the GPU parity tests (test-only)."""
import numpy as np

import oracle


def to_dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda")


def classical_bound(A, B):
    """Elementwise bound 2 gamma_k |A||B| on the difference of two classical
    FP64 sums of the same products in different orders."""
    k = A.shape[1]
    return 2 * oracle.norms.gamma(k) * (np.abs(A) @ np.abs(B))
