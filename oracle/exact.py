"""Exact solutions and error norms (test infrastructure only).

Variable-coefficient advection v_t + a(x) v_x = 0 (Sec. 5.1.3,
Eq. var.coeff.adv) is solved by characteristics: v(x, t) = v0(X) where the
foot X satisfies Phi(X) = Phi(x) - t with Phi(x) = int_0^x ds / a(s).

For the periodic coefficient a(x) = 1 + eps sin(k x), k = 2 pi / L, the
antiderivative is the classical closed form
  Phi(x) = 2 / (k s) * arctan((tan(k x / 2) + eps) / s),   s = sqrt(1 - eps^2),
continued across the poles of tan, and Phi(x + L) = Phi(x) + L / s.

The paper's own case a = x^-2 on [0.1, 1] has X = (x^3 - 3 t)^(1/3).
"""
import numpy as np

from .basis import gl_nodes_weights, lagrange


class SineCoefficient:
    """a(x) = 1 + eps sin(2 pi x / L)."""

    def __init__(self, eps=0.5, L=1.0):
        if not 0 <= eps < 1:
            raise ValueError("need 0 <= eps < 1 so that a > 0")
        self.eps, self.L = eps, L
        self.k = 2 * np.pi / L
        self.s = np.sqrt(1 - eps * eps)
        self.period = L / self.s

    def a(self, x):
        return 1.0 + self.eps * np.sin(self.k * x)

    def _psi(self, theta):
        """Continuous branch of arctan((tan(theta) + eps)/s) for theta in [0, pi]."""
        s, eps = self.s, self.eps
        th = np.asarray(theta, dtype=float)
        out = np.empty_like(th)
        mid = np.isclose(th, np.pi / 2, rtol=0, atol=1e-15)
        lo = (th < np.pi / 2) & ~mid
        hi = (th > np.pi / 2) & ~mid
        out[lo] = np.arctan((np.tan(th[lo]) + eps) / s)
        out[hi] = np.arctan((np.tan(th[hi]) + eps) / s) + np.pi
        out[mid] = np.pi / 2
        return out

    def phi(self, x):
        """Phi(x) = int_0^x ds / a(s), any real x."""
        x = np.asarray(x, dtype=float)
        m = np.floor(x / self.L)
        r = x - m * self.L
        theta = self.k * r / 2.0
        base = (2.0 / (self.k * self.s)) * (self._psi(theta) - self._psi(np.zeros(1))[0])
        return base + m * self.period

    def foot(self, x, t):
        """X with Phi(X) = Phi(x) - t (bisection; Phi is increasing)."""
        target = self.phi(x) - t
        lo = np.floor(target / self.period) * self.L - self.L
        hi = lo + 3 * self.L
        for _ in range(200):
            mid = 0.5 * (lo + hi)
            go = self.phi(mid) < target
            lo = np.where(go, mid, lo)
            hi = np.where(go, hi, mid)
        return 0.5 * (lo + hi)


def l2_error_1d(u_nodes, exact, xl, dx, nodes, nq=None):
    """L2 norm of (u_h - exact) over a 1D mesh: u_nodes (E, n) holds nodal
    values at ``nodes`` (reference [0, 1]); u_h is their Lagrange interpolant.
    Element integrals use an nq-point Gauss-Legendre rule (default n + 2)."""
    E, n = u_nodes.shape
    nq = nq or n + 2
    xq, wq = gl_nodes_weights(nq - 1)
    Lq = lagrange(nodes, xq)                       # (nq, n)
    uh = u_nodes @ Lq.T                            # (E, nq)
    x = xl + dx * (np.arange(E)[:, None] + xq[None, :])
    err = uh - exact(x)
    return np.sqrt(np.sum(dx * wq[None, :] * err * err))
