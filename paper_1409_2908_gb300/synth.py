"""Seeded synthetic inputs (shared by tests, the smoke check and the
benchmark).  Holds no arithmetic of the method: only the value recipes.

  uniform     i.i.d. uniform[-1, 1] float64
  integer     round(4 u) with u uniform[-1, 1]: values in {-4..4}; every
              fast path is exact on these
  loguniform  sign * 10^U(-4, 4): magnitudes spread over eight decades

A and B come from separate streams of numpy's PCG64 generator, seeded from
(seed, stream), so both machines produce the same values.
"""
import numpy as np


def _rng(seed, stream):
    return np.random.Generator(np.random.PCG64([int(seed), int(stream)]))


def matrix(rows, cols, seed, stream=0, kind="uniform"):
    g = _rng(seed, stream)
    if kind == "uniform":
        return g.uniform(-1.0, 1.0, size=(rows, cols))
    if kind == "integer":
        return np.rint(4.0 * g.uniform(-1.0, 1.0, size=(rows, cols)))
    if kind == "loguniform":
        mag = 10.0 ** g.uniform(-4.0, 4.0, size=(rows, cols))
        sign = np.where(g.random(size=(rows, cols)) < 0.5, -1.0, 1.0)
        return sign * mag
    raise ValueError(f"unknown input kind {kind!r}")


def operands(m, k, n, seed, kind="uniform"):
    """(A, B): A is m x k from stream 0, B is k x n from stream 1."""
    return matrix(m, k, seed, 0, kind), matrix(k, n, seed, 1, kind)


def sample_indices(m, n, count, seed):
    """Row and column indices of `count` output entries to check."""
    g = _rng(seed, 7)
    return g.integers(0, m, size=count), g.integers(0, n, size=count)
