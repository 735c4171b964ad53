"""Independent numpy/fractions helpers used to pin the oracle.

Nothing here is shared with the oracle or the CUDA path: polynomials are handled in the
monomial basis with exact rational arithmetic where possible, and Gauss-Legendre rules
come from numpy.polynomial.legendre.leggauss.
"""
from fractions import Fraction

import numpy as np


def gl01(n):
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (x + 1.0), 0.5 * w


def mono_cell_average(coefs, a, b):
    """exact average over [a, b] of sum_k coefs[k] x^k (coefs may be Fractions)"""
    s = Fraction(0)
    for k, c in enumerate(coefs):
        s += Fraction(c) * (Fraction(b) ** (k + 1) - Fraction(a) ** (k + 1)) / (k + 1)
    return s / (Fraction(b) - Fraction(a))


def solve_exact(A, b):
    """Gaussian elimination over Fractions"""
    n = len(A)
    M = [list(map(Fraction, row)) + [Fraction(bv)] for row, bv in zip(A, b)]
    for c in range(n):
        p = next(i for i in range(c, n) if M[i][c] != 0)
        M[c], M[p] = M[p], M[c]
        for i in range(n):
            if i != c and M[i][c] != 0:
                f = M[i][c] / M[c][c]
                M[i] = [x - f * y for x, y in zip(M[i], M[c])]
    return [M[i][n] / M[i][i] for i in range(n)]


def poly_eval(coefs, x):
    return sum(float(c) * x ** k for k, c in enumerate(coefs))


def poly_deriv(coefs):
    return [k * c for k, c in enumerate(coefs)][1:]


def lagrange_values(nodes, x):
    """values of the Lagrange basis through `nodes` at points x: shape (len(x), len(nodes))"""
    x = np.atleast_1d(np.asarray(x, dtype=float))
    out = np.ones((len(x), len(nodes)))
    for l, xl in enumerate(nodes):
        for k, xk in enumerate(nodes):
            if k != l:
                out[:, l] *= (x - xk) / (xl - xk)
    return out


def lagrange_derivs(nodes, x):
    """first derivatives of the Lagrange basis at x (product rule)"""
    x = np.atleast_1d(np.asarray(x, dtype=float))
    n = len(nodes)
    out = np.zeros((len(x), n))
    for l in range(n):
        for m in range(n):
            if m == l:
                continue
            term = np.ones(len(x)) / (nodes[l] - nodes[m])
            for k in range(n):
                if k != l and k != m:
                    term *= (x - nodes[k]) / (nodes[l] - nodes[k])
            out[:, l] += term
    return out
