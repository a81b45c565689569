"""One-dimensional GLL / Gauss bases for the oracle (plain FP64 NumPy).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Sec. 3.3 of the paper discretises each hexahedral element with tensor-product
Lagrange polynomials on Gauss-Lobatto-Legendre (GLL) points, degree P for the
velocity and P-1 for the pressure; Sec. 2.4 places the SDC sub-nodes on GLL
points of the time step.  This module builds the 1D ingredients from their
textbook definitions:

* GLL points of degree P: the end points -1, 1 and the roots of L_P'(x)
  (L_P the Legendre polynomial), weights 2 / (P (P+1) L_P(x_i)^2);
* Gauss-Legendre points and weights (numpy's ``leggauss``), used for the
  over-integrated ("consistent integration") convection term of Sec. 3.3;
* Lagrange cardinal polynomials on arbitrary nodes, evaluated together with
  their first derivative by expanding the product definition
  l_j(x) = prod_{k != j} (x - x_k) / (x_j - x_k) with numpy polynomials.
"""
import numpy as np
from numpy.polynomial import legendre as npleg
from numpy.polynomial import polynomial as nppoly


def gll_nodes_weights(n):
    """n >= 2 GLL points on [-1, 1] (degree P = n-1) and their quadrature weights (the nodes of
    the basis of Sec. 3.3: degree P for the velocity, P-1 for the pressure; the
    collocation mass)."""
    if n < 2:
        raise ValueError("GLL rule needs at least two points")
    p = n - 1
    LP = npleg.Legendre.basis(p)
    interior = np.sort(np.real(LP.deriv().roots())) if p >= 2 else np.array([])
    x = np.concatenate([[-1.0], interior, [1.0]])
    w = 2.0 / (p * (p + 1) * LP(x) ** 2)
    return x, w


def gauss_nodes_weights(q):
    """q Gauss-Legendre points and weights on [-1, 1] (the consistent integration of the
    convective term, Sec. 3.3: ceil(3N/2) points per direction)."""
    x, w = npleg.leggauss(q)
    return x, w


def lagrange_polys(nodes):
    """Power-basis coefficients of the Lagrange cardinal polynomials on ``nodes`` (the nodal
    basis of Sec. 3.3)."""
    nodes = np.asarray(nodes, dtype=np.float64)
    polys = []
    for j, xj in enumerate(nodes):
        others = np.delete(nodes, j)
        num = nppoly.polyfromroots(others)
        den = np.prod(xj - others)
        polys.append(num / den)
    return polys


def lagrange_eval(nodes, pts, deriv=0):
    """Matrix E[i, j] = l_j^{(deriv)}(pts[i]) for the cardinal polynomials on ``nodes`` (Sec. 3.3:
    differentiation, interpolation between the P-1 and P bases and to the Gauss points)."""
    pts = np.asarray(pts, dtype=np.float64)
    polys = lagrange_polys(nodes)
    E = np.zeros((len(pts), len(polys)))
    for j, c in enumerate(polys):
        cc = c
        for _ in range(deriv):
            cc = nppoly.polyder(cc)
        E[:, j] = nppoly.polyval(pts, cc)
    return E


def lagrange_integrals(nodes, a, b):
    """int_a^b l_j(t) dt for every cardinal polynomial on ``nodes`` (exact polynomial integral;
    the SDC quadrature weights of Sec. 2.4 over each subinterval)."""
    out = []
    for c in lagrange_polys(nodes):
        ci = nppoly.polyint(c)
        out.append(nppoly.polyval(b, ci) - nppoly.polyval(a, ci))
    return np.array(out)


def over_integration_points(p):
    """Number of Gauss points per direction for the over-integrated convection term.

    Reading of "consistent integration" (Sec. 3.3): ceil(3 (P+1) / 2) Gauss points,
    the 3/2 rule on the P+1 nodes per direction.
    """
    return (3 * (p + 1) + 1) // 2
