"""Quadrature rules used by the oracle (the paper's Quadrature class, Sec. 4.2,
names numerical integration without fixing a rule).

* Segments: Gauss-Legendre on [0,1] (numpy's Legendre nodes, a library
  primitive), exact for polynomials of degree 2n-1.
* Triangles: collapsed (Duffy) Gauss rule on the reference triangle
  {xi, eta >= 0, xi + eta <= 1}: xi = a, eta = b (1 - a), weight
  w_a w_b (1 - a), with a, b n-point Gauss-Legendre on [0,1].  With n = 4 it
  integrates xi^p eta^q exactly for p + q <= 6; weights sum to 1/2.
"""
import numpy as np
from numpy.polynomial.legendre import leggauss


def gauss_legendre_01(n: int):
    x, w = leggauss(n)
    return 0.5 * (x + 1.0), 0.5 * w


def duffy_triangle(n: int = 4):
    """Points (nq, 2) as (xi, eta) and weights (nq,) on the reference triangle."""
    a, wa = gauss_legendre_01(n)
    b, wb = gauss_legendre_01(n)
    pts = np.empty((n * n, 2))
    wts = np.empty(n * n)
    k = 0
    for i in range(n):
        for j in range(n):
            pts[k] = (a[i], b[j] * (1.0 - a[i]))
            wts[k] = wa[i] * wb[j] * (1.0 - a[i])
            k += 1
    return pts, wts


def face_points(P: int, l: int) -> int:
    """Gauss points per face piece: ceil((P + l + 1) / 2) + 1, exact for the
    products psi * phi (degree l + P) with margin."""
    return (P + l + 2) // 2 + 1
