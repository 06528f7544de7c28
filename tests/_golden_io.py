"""Readers for the text fixtures under tests/golden (test helpers only)."""
import os
import re
from fractions import Fraction

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _lines(name):
    with open(os.path.join(GOLDEN, name)) as fh:
        return [ln.split("#", 1)[0].strip() for ln in fh if ln.split("#", 1)[0].strip()]


def formulas_to_factors(name):
    """Turn written-out formulas (S_r = +-A.., T_r = +-B.., Cxy = +-M..) for a
    2x2 block algorithm into factor matrices (U, V, W) with rows in row-order
    vec: block 'Xab' (1-indexed) has row (a-1)*2 + (b-1)."""
    S, T, C = {}, {}, {}
    for ln in _lines(name):
        lhs, rhs = (p.strip() for p in ln.split("="))
        terms = re.findall(r"([+-]?)\s*([ABM])(\d+)", rhs)
        coeffs = {}
        for sign, sym, idx in terms:
            coeffs[(sym, idx)] = -1 if sign == "-" else 1
        if lhs.startswith("S"):
            S[int(lhs[1:])] = coeffs
        elif lhs.startswith("T"):
            T[int(lhs[1:])] = coeffs
        else:
            C[lhs[1:]] = coeffs
    R = len(S)

    def block_row(idx):
        a, b = int(idx[0]), int(idx[1])
        return (a - 1) * 2 + (b - 1)

    U = [[Fraction(0)] * R for _ in range(4)]
    V = [[Fraction(0)] * R for _ in range(4)]
    W = [[Fraction(0)] * R for _ in range(4)]
    for r in range(1, R + 1):
        for (sym, idx), c in S[r].items():
            U[block_row(idx)][r - 1] = Fraction(c)
        for (sym, idx), c in T[r].items():
            V[block_row(idx)][r - 1] = Fraction(c)
    for cidx, coeffs in C.items():
        for (sym, idx), c in coeffs.items():
            W[block_row(cidx)][int(idx) - 1] = Fraction(c)
    return U, V, W


def tensor_slices(name):
    """Frontal slices T_1..T_n as lists of integer rows."""
    out, cur = [], None
    for ln in _lines(name):
        if ln.startswith("T"):
            cur = []
            out.append(cur)
        else:
            cur.append([int(t) for t in ln.split()])
    return out


def table1(name="table1_algorithms.txt"):
    return [tuple(int(t) for t in ln.split()) for ln in _lines(name)]


def read_text(name):
    with open(os.path.join(GOLDEN, name)) as fh:
        return fh.read()
