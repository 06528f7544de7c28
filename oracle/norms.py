"""Oracle: error norms (the paper measures no accuracy, Section 6; these
are the readings used throughout).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).
"""
import numpy as np


def rel_frobenius(C_hat, C):
    """e_F = ||C_hat - C||_F / ||C||_F."""
    d = np.linalg.norm(np.asarray(C_hat, np.float64) - np.asarray(C, np.float64))
    n = np.linalg.norm(np.asarray(C, np.float64))
    return float(d / n) if n else float(d)


def rel_max(C_hat, C, A, B):
    """e_max = max|C_hat - C| / (max|A| max|B| k), a normwise bound in the
    style used for Strassen-type error analyses."""
    k = A.shape[1]
    den = float(np.max(np.abs(A))) * float(np.max(np.abs(B))) * k
    return float(np.max(np.abs(np.asarray(C_hat) - np.asarray(C)))) / den if den else 0.0


def gamma(n, u=2.0 ** -53):
    """gamma_n = n u / (1 - n u), the classical dot-product error constant."""
    return n * u / (1 - n * u)
