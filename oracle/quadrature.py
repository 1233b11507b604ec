"""Gauss-Legendre rule for the composite panel quadrature.

Sec. 5 (preamble) and Sec. 3.1: every boundary is discretised with 16-point
Gaussian panels.  The rule is taken from numpy's ``leggauss`` (a library
routine used as a step); the tests pin it by exact integration of
polynomials up to degree 31 and by the moments of [-1, 1].
"""
import numpy as np

NQ = 16  # points per panel (Sec. 5 preamble)


def gauss_legendre(n=NQ):
    """Return (nodes, weights) of the n-point Gauss-Legendre rule on [-1, 1],
    nodes ascending."""
    x, w = np.polynomial.legendre.leggauss(n)
    order = np.argsort(x)
    return x[order].astype(np.float64), w[order].astype(np.float64)
