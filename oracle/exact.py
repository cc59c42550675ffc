"""ORACLE — test infrastructure only.

Exact rational solution of X = P.X + B (Section 1) for tiny graphs: P has d/out_j at (i, j) for
each distinct link j -> i (Section 2.4 orientation; duplicates count once, a self-loop puts
d/out_j on the diagonal), and (I - P) X = B is solved by Gauss-Jordan elimination over
fractions.Fraction, so the result carries no rounding at all. Used only to write the golden
fixtures under tests/golden/.
"""
from __future__ import annotations

from fractions import Fraction


def exact_solve(n: int, edges, d: Fraction, B):
    links = sorted(set((int(s), int(t)) for s, t in edges))
    out = [0] * n
    for s, _ in links:
        out[s] += 1
    # A = I - P
    A = [[Fraction(int(i == j)) for j in range(n)] for i in range(n)]
    for s, t in links:
        A[t][s] -= d / out[s]
    rhs = [Fraction(b) for b in B]
    for col in range(n):
        piv = next(r for r in range(col, n) if A[r][col] != 0)
        if piv != col:
            A[col], A[piv] = A[piv], A[col]
            rhs[col], rhs[piv] = rhs[piv], rhs[col]
        inv = 1 / A[col][col]
        A[col] = [a * inv for a in A[col]]
        rhs[col] *= inv
        for r in range(n):
            if r != col and A[r][col] != 0:
                f = A[r][col]
                A[r] = [a - f * c for a, c in zip(A[r], A[col])]
                rhs[r] -= f * rhs[col]
    return rhs
