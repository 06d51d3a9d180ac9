"""Reference element of the FR scheme on [0, 1] (test infrastructure only).

Sec. 2, Eqs. reference.element, ref.map, soln.points, soln.poly,
defn.lagrange, diff.matrix; App. B, Eq. correction.identities.

Everything is computed the plain way: nodes and weights come from numpy's
Gauss-Legendre routine (GL) or from the roots of P_N' (GLL), the Lagrange
polynomials from their product definition, D from the derivative of that
product, and the correction derivatives from the identity of App. B.
"""
import numpy as np
from numpy.polynomial import legendre as npleg


def gl_nodes_weights(N):
    """N+1 Gauss-Legendre nodes and weights mapped from [-1, 1] to [0, 1]
    (Eq. soln.points; exact for degree 2N+1)."""
    x, w = npleg.leggauss(N + 1)
    return (x + 1.0) / 2.0, w / 2.0


def gll_nodes_weights(N):
    """N+1 Gauss-Lobatto-Legendre nodes and weights on [0, 1] (N >= 1).

    Nodes: -1, +1 and the roots of P_N'; weights 2 / (N (N+1) P_N(x)^2) on
    [-1, 1]; exact for degree 2N-1 (Eq. soln.points)."""
    if N < 1:
        raise ValueError("GLL needs N >= 1")
    PN = npleg.Legendre.basis(N)
    interior = np.sort(np.real(PN.deriv().roots()))
    x = np.concatenate([[-1.0], interior, [1.0]])
    w = 2.0 / (N * (N + 1) * PN(x) ** 2)
    return (x + 1.0) / 2.0, w / 2.0


def lagrange(nodes, xi):
    """Values l_q(xi) of all Lagrange polynomials (Eq. defn.lagrange) at the
    points ``xi``; returns shape (len(xi), n)."""
    xi = np.atleast_1d(np.asarray(xi, dtype=float))
    n = len(nodes)
    out = np.ones((len(xi), n))
    for q in range(n):
        for p in range(n):
            if p != q:
                out[:, q] *= (xi - nodes[p]) / (nodes[q] - nodes[p])
    return out


def lagrange_deriv(nodes, xi):
    """Derivatives l_q'(xi): the product rule applied to Eq. defn.lagrange;
    returns shape (len(xi), n)."""
    xi = np.atleast_1d(np.asarray(xi, dtype=float))
    n = len(nodes)
    out = np.zeros((len(xi), n))
    for q in range(n):
        for m in range(n):
            if m == q:
                continue
            term = np.full(len(xi), 1.0 / (nodes[q] - nodes[m]))
            for p in range(n):
                if p != q and p != m:
                    term *= (xi - nodes[p]) / (nodes[q] - nodes[p])
            out[:, q] += term
    return out


class Basis:
    """Reference element tables for degree N and node family 'gl' or 'gll'.

    Attributes
    ----------
    xi, w  : nodes and quadrature weights on [0, 1]
    D      : D[i, j] = l_j'(xi_i)  (Eq. diff.matrix)
    l0, l1 : l_p(0), l_p(1)  (extrapolation to the element faces)
    gLp, gRp : g_L'(xi_p) = -l_p(0)/w_p, g_R'(xi_p) = l_p(1)/w_p
               (Eq. correction.identities; Radau for GL, g_2 for GLL)
    """

    def __init__(self, N, family="gl"):
        self.N = N
        self.n = N + 1
        self.family = family
        if family == "gl":
            self.xi, self.w = gl_nodes_weights(N)
        elif family == "gll":
            self.xi, self.w = gll_nodes_weights(N)
        else:
            raise ValueError(family)
        self.D = lagrange_deriv(self.xi, self.xi)
        self.l0 = lagrange(self.xi, [0.0])[0]
        self.l1 = lagrange(self.xi, [1.0])[0]
        self.gLp = -self.l0 / self.w
        self.gRp = self.l1 / self.w
