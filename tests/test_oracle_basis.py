"""Pins of the oracle's reference element against closed forms and
textbook definitions (Sec. 2; App. B, Eq. correction.identities)."""
import numpy as np
import pytest
from numpy.polynomial import legendre as L

from oracle.basis import Basis, lagrange

DEGREES = [0, 1, 2, 3, 4]


def test_gl_n1_closed_form():
    bs = Basis(1, "gl")
    r = 1.0 / (2.0 * np.sqrt(3.0))
    assert np.allclose(bs.xi, [0.5 - r, 0.5 + r], atol=1e-15)
    assert np.allclose(bs.w, [0.5, 0.5], atol=1e-15)


def test_gll_n2_is_simpson():
    bs = Basis(2, "gll")
    assert np.allclose(bs.xi, [0.0, 0.5, 1.0], atol=1e-15)
    assert np.allclose(bs.w, [1 / 6, 2 / 3, 1 / 6], atol=1e-15)


@pytest.mark.parametrize("N", DEGREES)
@pytest.mark.parametrize("family", ["gl", "gll"])
def test_quadrature_exactness(N, family):
    """GL is exact to degree 2N+1 and GLL to 2N-1 (Eq. soln.points), and no
    further: the first failing degree identifies the family."""
    if family == "gll" and N == 0:
        pytest.skip("GLL needs N >= 1")
    bs = Basis(N, family)
    top = 2 * N + 1 if family == "gl" else 2 * N - 1
    for k in range(top + 1):
        assert abs(np.sum(bs.w * bs.xi ** k) - 1.0 / (k + 1)) < 1e-14
    k = top + 1
    assert abs(np.sum(bs.w * bs.xi ** k) - 1.0 / (k + 1)) > 1e-6


@pytest.mark.parametrize("N", DEGREES)
@pytest.mark.parametrize("family", ["gl", "gll"])
def test_diff_matrix_exact_on_polynomials(N, family):
    """D_ij = l_j'(xi_i) (Eq. diff.matrix) differentiates P_N exactly."""
    if family == "gll" and N == 0:
        pytest.skip("GLL needs N >= 1")
    bs = Basis(N, family)
    for k in range(N + 1):
        want = k * bs.xi ** (k - 1) if k > 0 else np.zeros_like(bs.xi)
        assert np.max(np.abs(bs.D @ bs.xi ** k - want)) < 1e-11
    assert np.max(np.abs(bs.D.sum(axis=1))) < 1e-11


@pytest.mark.parametrize("N", DEGREES)
def test_lagrange_cardinal_and_extrapolation(N):
    bs = Basis(N, "gl")
    assert np.allclose(lagrange(bs.xi, bs.xi), np.eye(N + 1), atol=1e-14)
    for k in range(N + 1):
        assert abs(bs.l1 @ bs.xi ** k - 1.0) < 1e-12
        assert abs(bs.l0 @ bs.xi ** k - (1.0 if k == 0 else 0.0)) < 1e-12


def _radau_left(k):
    """Huynh's right Radau polynomial R_{R,k} = (-1)^k/2 (P_k - P_{k-1}) on
    [-1, 1]; as g_L it is 1 at -1 and 0 at +1."""
    return ((-1) ** k / 2.0) * (L.Legendre.basis(k) - L.Legendre.basis(k - 1))


def _g2_left(k):
    """Huynh's g_2 = (k-1)/(2k-1) R_{R,k} + k/(2k-1) R_{R,k-1}."""
    return ((k - 1) / (2 * k - 1)) * _radau_left(k) + (k / (2 * k - 1)) * _radau_left(k - 1)


def _check_identity(bs, gL):
    """Compare g_L'(xi_p), g_R'(xi_p) on [0, 1] from the explicit polynomial
    (g_R(x) = g_L(-x); d/dxi = 2 d/dx) with Eq. correction.identities."""
    x = 2 * bs.xi - 1
    dgL = 2 * gL.deriv()(x)
    dgR = -2 * gL.deriv()(-x)
    assert gL(-1.0) == pytest.approx(1.0, abs=1e-14)
    assert gL(1.0) == pytest.approx(0.0, abs=1e-14)
    assert np.max(np.abs(dgL - bs.gLp)) < 1e-11 * max(1, np.max(np.abs(dgL)))
    assert np.max(np.abs(dgR - bs.gRp)) < 1e-11 * max(1, np.max(np.abs(dgR)))


@pytest.mark.parametrize("N", DEGREES)
def test_radau_identity_gl(N):
    _check_identity(Basis(N, "gl"), _radau_left(N + 1))


@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_g2_identity_gll(N):
    bs = Basis(N, "gll")
    _check_identity(bs, _g2_left(N + 1))
    # GLL + g_2 corrections only touch the end nodes (App. B, under Eq. fr.gll)
    assert np.allclose(bs.gRp[:-1], 0.0, atol=1e-12)
    assert np.allclose(bs.gLp[1:], 0.0, atol=1e-12)
