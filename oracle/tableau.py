"""Explicit Butcher tableaux (A~, b~) used by the cRK-FR inner stages
(test infrastructure only).

Sec. 2, Eq. imex.butcher: A~ is strictly lower triangular; only the explicit
part is used because the hot path has no source term.  The paper prints the
explicit parts of HT(1,1,2) (App. C, Eq. ht112.butcher) and of
SSP3-IMEX(4,3,3) (App. C, Eq. ssp33.butcher) but does not say which explicit
method accompanies each degree in the non-stiff tests.  Reading used here:
order min(N+1, 4):

  N = 0   forward Euler (with N = 0 the local derivative vanishes, so any
          tableau gives the same scheme, the FV scheme of Eq. fr.fv)
  N = 1   explicit part of HT(1,1,2)
  N = 2   explicit part of SSP3-IMEX(4,3,3), kept with its printed null
          first stage
  N = 3   classical fourth-order Runge-Kutta
  N = 4   Butcher's six-stage fifth-order method

An order below N+1 is not an option: with RK4 at N = 4 the von Neumann
analysis of the oracle finds no usable CFL number (about 2e-4), because the
time-average polynomial sum_i b_i P_i(z) must match (e^z - 1)/z up to z^N
for the scheme to be linearly equivalent to LWFR (Sec. 5, under
Eq. time.step.2d).
"""
import numpy as np


def ht112_explicit():
    """App. C, Eq. ht112.butcher, explicit tableau."""
    A = np.array([[0.0, 0.0],
                  [1.0, 0.0]])
    b = np.array([0.5, 0.5])
    return A, b


def ssp3_imex433_explicit():
    """App. C, Eq. ssp33.butcher, explicit tableau (four stages, the first
    row and column are zero and b~_1 = 0)."""
    A = np.array([[0.0, 0.0, 0.0, 0.0],
                  [0.0, 0.0, 0.0, 0.0],
                  [0.0, 1.0, 0.0, 0.0],
                  [0.0, 0.25, 0.25, 0.0]])
    b = np.array([0.0, 1.0 / 6.0, 1.0 / 6.0, 2.0 / 3.0])
    return A, b


def rk4_classical():
    """The textbook fourth-order Runge-Kutta tableau."""
    A = np.array([[0.0, 0.0, 0.0, 0.0],
                  [0.5, 0.0, 0.0, 0.0],
                  [0.0, 0.5, 0.0, 0.0],
                  [0.0, 0.0, 1.0, 0.0]])
    b = np.array([1.0, 2.0, 2.0, 1.0]) / 6.0
    return A, b


def butcher_rk5():
    """Butcher's six-stage fifth-order explicit method."""
    A = np.zeros((6, 6))
    A[1, 0] = 1.0 / 4.0
    A[2, 0], A[2, 1] = 1.0 / 8.0, 1.0 / 8.0
    A[3, 1], A[3, 2] = -1.0 / 2.0, 1.0
    A[4, 0], A[4, 3] = 3.0 / 16.0, 9.0 / 16.0
    A[5, :5] = np.array([-3.0, 2.0, 12.0, -12.0, 8.0]) / 7.0
    b = np.array([7.0, 0.0, 32.0, 12.0, 32.0, 7.0]) / 90.0
    return A, b


def forward_euler():
    return np.array([[0.0]]), np.array([1.0])


def default_tableau(N):
    if N == 0:
        return forward_euler()
    if N == 1:
        return ht112_explicit()
    if N == 2:
        return ssp3_imex433_explicit()
    if N == 3:
        return rk4_classical()
    if N == 4:
        return butcher_rk5()
    raise ValueError("degree N must be 0..4")
