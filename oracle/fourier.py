"""Von Neumann analysis of cRK-FR for linear advection, giving CFL(N)
(test infrastructure only).

Sec. 5, remark under Eq. time.step.2d: CFL(N) is the optimal CFL number from
Fourier stability analysis; the paper takes it from the LWFR analysis because
cRK-FR is linearly equivalent to LWFR, but prints no values.  Reading used
here: for v_t + v_x = 0 written as the variable-coefficient system with a = 1
(Sec. 5.1.3), the amplification matrix G(kappa, nu) is obtained by applying
the oracle's own cRK-FR step, with dx = 1 and dt = nu, to the N+1 unit vectors
of one element of a Bloch wave with phase kappa per element.  CFL(N) is the
largest nu with spectral radius <= 1 + tau(N) over kappa_k = pi k / 256,
k = 0..256 (G(-kappa) is the complex conjugate of G(kappa)), found by 60
bisection halvings of [0, 2].  tau = 1e-12 for N <= 3.  For N = 4 the
scheme has a weak growth at mid wavenumbers (spectral radius - 1 below 1e-5
for nu up to the sharp high-wavenumber limit), so tau(4) = 1e-4 places the
limit at that sharp boundary.
"""
import numpy as np

from .crkfr import Scheme1D
from .systems import VarCoeffAdvection

KGRID = 256


def tolerance(N):
    return 1e-4 if N >= 4 else 1e-12


def amplification(N, nu, kappas, family="gl", tableau=None, source=None):
    """G(kappa, nu) for every kappa in ``kappas``; shape (K, N+1, N+1).
    ``tableau``/``source`` as for Scheme1D (a linear source keeps the step
    linear, so G is still its matrix)."""
    kappas = np.atleast_1d(np.asarray(kappas, dtype=float))
    sch = Scheme1D(VarCoeffAdvection(), N, 1.0, family=family, tableau=tableau, source=source)
    n, K = N + 1, len(kappas)
    # batch axis enumerates (kappa, column j); one element per Bloch period
    e = np.zeros((1, K, n, 1, n), dtype=complex)
    for j in range(n):
        e[0, :, j, 0, j] = 1.0
    e = e.reshape(1, K * n, 1, n)
    theta = np.repeat(kappas, n)
    c = np.ones((1, n))
    R = sch.residual(e, c, nu, bloch=theta)
    cols = (e - nu * R)[0, :, 0, :].reshape(K, n, n)   # [k, j, :] = G[k][:, j]
    return np.transpose(cols, (0, 2, 1))


def kappa_grid(kgrid=KGRID):
    return np.pi * np.arange(kgrid + 1) / kgrid


def spectral_radius(N, nu, family="gl", kgrid=KGRID, tableau=None, source=None):
    G = amplification(N, nu, kappa_grid(kgrid), family, tableau, source)
    return np.max(np.abs(np.linalg.eigvals(G)))


def stable(N, nu, family="gl", kgrid=KGRID, tol=None, tableau=None):
    tol = tolerance(N) if tol is None else tol
    return spectral_radius(N, nu, family, kgrid, tableau) <= 1.0 + tol


def cfl_number(N, family="gl", kgrid=KGRID, tol=None, halvings=60, tableau=None):
    """CFL(N) of the default tableau, or of an explicit tableau (A, b) given
    as ``tableau`` (for a source term: the explicit part of the IMEX
    tableau, the source being implicit)."""
    lo, hi = 0.0, 2.0
    for _ in range(halvings):
        mid = 0.5 * (lo + hi)
        if stable(N, mid, family, kgrid, tol, tableau):
            lo = mid
        else:
            hi = mid
    return lo
