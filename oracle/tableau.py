"""Butcher tableaux of the cRK-FR inner stages (test infrastructure only).

Sec. 2, Eq. imex.butcher: A~ is strictly lower triangular (explicit part);
A is lower triangular (diagonally implicit part, used only for a source
term).  Without a source only the explicit part is used.  The paper prints the
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


class ImexTableau:
    """A double Butcher tableau (Sec. 2, Eq. imex.butcher): explicit (Ae, be)
    for the flux and non-conservative terms, diagonally implicit (Ai, bi)
    for the source."""

    def __init__(self, Ae, be, Ai, bi, name):
        self.Ae, self.be = np.asarray(Ae, float), np.asarray(be, float)
        self.Ai, self.bi = np.asarray(Ai, float), np.asarray(bi, float)
        self.name = name

    @property
    def stages(self):
        return len(self.be)


def ht112_imex():
    """App. C, Eq. ht112.butcher: explicit Heun, implicit part with a zero
    first row and the trapezoidal second row."""
    Ae, be = ht112_explicit()
    Ai = np.array([[0.0, 0.0],
                   [0.5, 0.5]])
    return ImexTableau(Ae, be, Ai, np.array([0.5, 0.5]), "HT(1,1,2)")


# App. C, Eq. ssp33.butcher: the three parameters of the implicit part, as
# printed (12 significant digits)
SSP3_ALPHA = 0.241694260788
SSP3_BETA = 0.0604235651970
SSP3_ETA = 0.12915286960590


def ssp3_imex433():
    """App. C, Eq. ssp33.butcher: both tableaux, four stages each.  Rows 2
    and 3 of the implicit part are the ones whose sums are the printed
    nodes c_2 = 0, c_3 = 1 (reading 7 of the package docstring: the printed
    rows contradict the printed nodes and the stated order and L-stability)."""
    Ae, be = ssp3_imex433_explicit()
    al, be_, et = SSP3_ALPHA, SSP3_BETA, SSP3_ETA
    Ai = np.array([[al, 0.0, 0.0, 0.0],
                   [-al, al, 0.0, 0.0],
                   [0.0, 1.0 - al, al, 0.0],
                   [be_, et, 0.5 - be_ - et - al, al]])
    return ImexTableau(Ae, be, Ai, be.copy(), "SSP3-IMEX(4,3,3)")


def imex_tableau(N):
    """Reading for a source term: SSP3-IMEX(4,3,3) at every degree, the
    scheme the paper uses for its stiff tests (Sec. 5.1, Sec. 5.2, at N = 3).
    Its explicit part has order 3, enough for N <= 2 and setting the time
    order for N >= 3.  HT(1,1,2) is not used by default: with a stiff
    source the cRK-FR step at N = 1 with HT(1,1,2) grows (spectral radius
    about 1.12 at K dt = 10 under the advective CFL number), in line with
    the paper's remark that HT(1,1,2) failed for very stiff relaxation
    (App. C)."""
    if 0 <= N <= 4:
        return ssp3_imex433()
    raise ValueError("degree N must be 0..4")


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
