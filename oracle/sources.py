"""Source terms and the point-implicit solve of the IMEX inner stages
(test infrastructure only).

Sec. 2, Eq. con.law.source: u_t + f(u)_x = s(u).  With a double Butcher
tableau (Eq. imex.butcher) the inner stages of Eq. crkfr.inner treat the
source implicitly, one solution point at a time:

    u^(i) - dt a_ii s(u^(i)) = r^(i),
    r^(i) = u^n - dt sum_{j<i} a~_ij (local flux and non-conservative terms)_j
                + dt sum_{j<i} a_ij s(u^(j)),

and the final update adds dt S with the time-averaged source
S = sum_i b_i s(u^(i)) (Eqs. crkfr, avg.source).

Two sources, each with its analytic Jacobian:

  LinearDamping(K):  s = -K u on every evolved variable, the stiff model
      problem of App. A (Eq. advection.stiff.source) when the system is
      advection.
  ChezyFriction(C_f): s = (0, -C_f |v| v_1 [, -C_f |v| v_2]) with v the
      velocity (hu)/h, the friction term of the shallow-water model of
      Sec. 5.5; applied here to the shallow-water systems with bathymetry.

The stage equation is solved by Newton's method from the initial guess r,
iterated until the update stops shrinking (the plain definition of the
implicit stage; no closed form is used here).
"""
import numpy as np


class LinearDamping:
    name = "linear"

    def __init__(self, K):
        self.K = float(K)

    def source(self, u, c):
        return -self.K * u

    def jacobian(self, u, c):
        M = u.shape[0]
        J = np.zeros((M, M) + u.shape[1:])
        for k in range(M):
            J[k, k] = -self.K
        return J


class ChezyFriction:
    name = "chezy"

    def __init__(self, Cf):
        self.Cf = float(Cf)

    def source(self, u, c):
        h = u[0]
        vel = u[1:] / h
        speed = np.sqrt(np.sum(vel * vel, axis=0))
        return np.concatenate([np.zeros_like(h)[None], -self.Cf * speed * vel])

    def jacobian(self, u, c):
        """d s / d u for s_k = -C_f |m| m_k / h^2 (m the momentum vector)."""
        h, m = u[0], u[1:]
        M = u.shape[0]
        nm = np.sqrt(np.sum(m * m, axis=0))
        safe = np.where(nm > 0.0, nm, 1.0)
        J = np.zeros((M, M) + u.shape[1:])
        for k in range(1, M):
            J[k, 0] = 2.0 * self.Cf * nm * m[k - 1] / h ** 3
            for l in range(1, M):
                d = nm if k == l else 0.0
                J[k, l] = -self.Cf / h ** 2 * (d + np.where(nm > 0.0, m[k - 1] * m[l - 1] / safe,
                                                            0.0))
        return J


def point_implicit_solve(src, r, c, gamma, maxit=60):
    """u with u - gamma s(u) = r at every solution point (Newton, start r)."""
    u = np.array(r, dtype=np.result_type(r, float), copy=True)
    if gamma == 0.0:
        return u
    M = u.shape[0]
    last = np.inf
    for _ in range(maxit):
        G = u - gamma * src.source(u, c) - r
        J = -gamma * src.jacobian(u, c)
        for k in range(M):
            J[k, k] = J[k, k] + 1.0
        # batched M x M solve over the node axes
        Jm = np.moveaxis(J.reshape(M, M, -1), -1, 0)
        Gm = np.moveaxis(G.reshape(M, -1), -1, 0)[..., None]
        du = np.moveaxis(np.linalg.solve(Jm, Gm)[..., 0], 0, -1).reshape(u.shape)
        u = u - du
        size = np.max(np.abs(du) / (np.abs(u) + 1e-300)) if du.size else 0.0
        if size == 0.0 or size >= last:
            break
        last = size
    return u
