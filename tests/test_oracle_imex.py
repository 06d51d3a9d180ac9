"""Pins of the oracle's IMEX path (a source term treated implicitly in the
inner stages, Sec. 2 Eqs. crkfr.inner, crkfr, avg.source; App. A; App. C).

- the double tableaux against App. C as printed, with the reading of the
  SSP3-IMEX(4,3,3) implicit rows decided by the paper's own statements
  (third order, L-stable, the printed node column);
- App. A: with N = 0 and one-stage tableaux the scheme's amplification
  factors are the two printed closed forms (explicit and implicit source);
  with the real IMEX tableaux a stiff linear source decays under the
  advective CFL condition alone;
- closed-form solutions: linear damping of a uniform state (the stability
  function of the implicit tableau; the trapezoidal rule for HT(1,1,2)),
  Chezy friction of a uniform flow, m(t) = m0 / (1 + C_f |m0| t / h0^2),
  and damped advection u0(x - t) exp(-K t), each at the design order;
- a zero source gives the explicit scheme with the IMEX explicit part.
"""
import itertools
import json
import os

import numpy as np
import pytest

from oracle.basis import Basis
from oracle.crkfr import Scheme1D, Scheme2D
from oracle.fourier import amplification, kappa_grid
from oracle.sources import ChezyFriction, LinearDamping
from oracle.systems import ShallowWater1D, ShallowWater2D, VarCoeffAdvection
from oracle.tableau import (SSP3_ALPHA, SSP3_BETA, SSP3_ETA, ImexTableau, ht112_imex,
                            imex_tableau, ssp3_imex433)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "app_c_tableaux.json")


def _sym(x):
    env = {"alpha": SSP3_ALPHA, "beta": SSP3_BETA, "eta": SSP3_ETA}
    return float(eval(str(x), {"__builtins__": {}}, env))


def stability_function(A, b, z):
    """R(z) = 1 + z b^T (I - z A)^{-1} 1 (Dahlquist test problem)."""
    s = len(b)
    return 1.0 + z * b @ np.linalg.solve(np.eye(s) - z * A, np.ones(s))


def imex_order3_residuals(t):
    """Residuals of the IMEX order conditions through order 3: every
    combination of the two tableaux in b.1, b.c, b.(c c'), b.A c'."""
    Ae, be, Ai, bi = t.Ae, t.be, t.Ai, t.bi
    ce, ci = Ae.sum(1), Ai.sum(1)
    res = [be.sum() - 1, bi.sum() - 1]
    for b, c in itertools.product((be, bi), (ce, ci)):
        res.append(b @ c - 0.5)
    for b, c1, c2 in itertools.product((be, bi), (ce, ci), (ce, ci)):
        res.append(b @ (c1 * c2) - 1 / 3)
    for b, A, c in itertools.product((be, bi), (Ae, Ai), (ce, ci)):
        res.append(b @ A @ c - 1 / 6)
    return np.array(res)


# ---------------------------------------------------------------------------
# App. C tableaux
# ---------------------------------------------------------------------------
def test_ht112_implicit_as_printed():
    g = json.load(open(GOLDEN))["ht112"]
    t = ht112_imex()
    assert np.array_equal(t.Ai, np.array(g["A_implicit"], float))
    assert np.array_equal(t.bi, np.array(g["b_implicit"], float))
    assert np.array_equal(t.Ai.sum(1), np.array(g["c_implicit_printed"], float))


def test_ht112_stability_a_stable_not_l_stable():
    """App. C: the implicit part of HT(1,1,2) is A-stable but not L-stable.
    Its stability function is the trapezoidal rule's (1 + z/2) / (1 - z/2)."""
    t = ht112_imex()
    for z in (-0.3, -2.0, 1j, -5 + 3j):
        assert abs(stability_function(t.Ai, t.bi, z) - (1 + z / 2) / (1 - z / 2)) < 1e-15
    for y in np.linspace(-50, 50, 101):
        assert abs(stability_function(t.Ai, t.bi, 1j * y)) <= 1 + 1e-14
    assert abs(stability_function(t.Ai, t.bi, -1e6) + 1.0) < 1e-5


def test_ssp3_printed_rows_contradict_printed_nodes_and_claims():
    """The implicit rows 2 and 3 as printed do not sum to the printed nodes
    c_2 = 0, c_3 = 1, and the tableau so read is neither second order nor
    L-stable; App. C states third order and L-stability.  This is what
    decides the oracle's reading of those rows."""
    g = json.load(open(GOLDEN))["ssp3_imex433"]
    Ap = np.array([[_sym(x) for x in row] for row in g["A_implicit_printed"]])
    cp = np.array([_sym(x) for x in g["c_implicit_printed"]])
    b = np.array(g["b_implicit"], float)
    assert abs(Ap[1].sum() - cp[1]) > 0.2 and abs(Ap[2].sum() - cp[2]) > 0.05
    assert abs(b @ Ap.sum(1) - 0.5) > 0.02                       # not even order 2
    assert abs(stability_function(Ap, b, -1e10)) > 0.4            # not L-stable


def test_ssp3_reading_matches_printed_nodes_order3_l_stable():
    g = json.load(open(GOLDEN))["ssp3_imex433"]
    t = ssp3_imex433()
    # explicit part and weights as printed
    assert np.allclose(t.Ae, np.array(g["A_explicit"]), rtol=0, atol=1e-16)
    assert np.allclose(t.be, np.array(g["b_explicit"]), rtol=0, atol=1e-16)
    assert np.allclose(t.bi, np.array(g["b_implicit"]), rtol=0, atol=1e-16)
    assert np.allclose(t.Ae.sum(1), np.array(g["c_explicit_printed"]), rtol=0, atol=1e-16)
    # rows 1 and 4 as printed; row sums 1..3 equal the printed nodes
    Ap = np.array([[_sym(x) for x in row] for row in g["A_implicit_printed"]])
    assert np.array_equal(t.Ai[0], Ap[0]) and np.array_equal(t.Ai[3], Ap[3])
    cp = np.array([_sym(x) for x in g["c_implicit_printed"]])
    assert np.allclose(t.Ai.sum(1)[:3], cp[:3], rtol=0, atol=1e-16)
    # third order as a pair (with the 12-digit parameters)
    assert np.max(np.abs(imex_order3_residuals(t))) < 1e-11
    # L-stable: A-stable on the imaginary axis and R(-inf) = 0 to the
    # accuracy of the printed parameters
    for y in np.linspace(-100, 100, 201):
        assert abs(stability_function(t.Ai, t.bi, 1j * y)) <= 1 + 1e-12
    assert abs(stability_function(t.Ai, t.bi, -1e8)) < 1e-6
    assert abs(stability_function(t.Ai, t.bi, -1e12)) < 1e-9


def test_ht112_pair_order2():
    t = ht112_imex()
    r = imex_order3_residuals(t)
    assert np.max(np.abs(r[:6])) < 1e-15          # orders 1 and 2
    assert np.max(np.abs(r[6:])) > 1e-3           # not third order


# ---------------------------------------------------------------------------
# App. A: the model problem u_t + a u_x = -K u
# ---------------------------------------------------------------------------
def _one_stage(implicit):
    return ImexTableau([[0.0]], [1.0], [[1.0 if implicit else 0.0]], [1.0],
                       "backward" if implicit else "forward")


@pytest.mark.parametrize("implicit", [False, True])
def test_app_a_amplification_factors(implicit):
    """N = 0 (first-order upwind FV for a > 0, Sec. 3 under Eq. fr.fv) with
    the one-stage tableaux: the amplification factor is App. A's Eq.
    expl.evolution (source explicit) or Eq. implicit.evolution (source
    implicit) for every Fourier mode."""
    K, nu = 7.0, 0.6
    xi = np.linspace(-np.pi, np.pi, 33)
    G = amplification(0, nu, xi, tableau=_one_stage(implicit), source=LinearDamping(K))[:, 0, 0]
    adv = 1 - nu * (1 - np.exp(-1j * xi))
    expect = adv / (1 + K * nu) if implicit else adv - K * nu
    assert np.max(np.abs(G - expect)) < 1e-14


@pytest.mark.parametrize("N", [0, 1, 2, 3, 4])
def test_app_a_stiff_source_decays_under_advective_cfl(N):
    """App. A: with the source implicit, the model problem needs only the
    advective CFL condition.  With SSP3-IMEX(4,3,3) the cRK-FR amplification
    has spectral radius <= 1 for K dt from 0 to 1e8 at 0.9 CFL(N), and the
    L-stable implicit part damps the stiff limit."""
    import oracle.fourier as fr
    t = imex_tableau(N)
    nu = 0.9 * fr.cfl_number(N, tableau=(t.Ae, t.be), halvings=30)
    kap = kappa_grid(64)
    for Kdt in (0.0, 0.5, 4.0, 10.0, 1e3, 1e8):
        G = amplification(N, nu, kap, tableau=t, source=LinearDamping(Kdt / nu))
        rho = np.max(np.abs(np.linalg.eigvals(G)))
        assert rho <= 1 + 1e-12
        if Kdt == 1e8 and N >= 1:
            assert rho < 1e-3


def test_ht112_grows_under_stiff_source_at_n1():
    """App. C remarks that HT(1,1,2), A-stable but not L-stable, failed for
    very stiff relaxation.  The oracle's von Neumann analysis agrees: at
    N = 1 and 0.9 CFL(1) the step is stable for K dt <= 4 but grows for
    K dt = 10 and 100."""
    import oracle.fourier as fr
    t = ht112_imex()
    nu = 0.9 * fr.cfl_number(1, tableau=(t.Ae, t.be), halvings=30)
    rho = lambda Kdt: np.max(np.abs(np.linalg.eigvals(
        amplification(1, nu, kappa_grid(64), tableau=t, source=LinearDamping(Kdt / nu)))))
    assert rho(0.5) <= 1 + 1e-12 and rho(4.0) <= 1 + 1e-12
    assert rho(10.0) > 1.1 and rho(100.0) > 1.1


def test_app_a_explicit_source_needs_small_dt():
    """App. A: with the source explicit the step must also satisfy
    dt = O(1/K): K dt = 3 is unstable even for a tiny advective CFL."""
    G = amplification(0, 0.1, kappa_grid(32), tableau=_one_stage(False),
                      source=LinearDamping(30.0))
    assert np.max(np.abs(np.linalg.eigvals(G))) > 1.5


# ---------------------------------------------------------------------------
# closed forms
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("N", [1, 2, 3])
def test_uniform_linear_damping_is_the_stability_function(N):
    t = imex_tableau(N)
    E, n = 3, N + 1
    sch = Scheme1D(VarCoeffAdvection(), N, 1.0, source=LinearDamping(4.0))
    u = np.full((1, E, n), 1.7)
    c = np.ones((E, n))
    for dt in (0.01, 0.3, 50.0):
        out = sch.step(u, c, dt)
        R = stability_function(t.Ai, t.bi, -4.0 * dt)
        assert np.max(np.abs(out - 1.7 * R)) < 1e-13 * max(1.0, 4.0 * dt)
    # HT(1,1,2): the trapezoidal rule
    sch = Scheme1D(VarCoeffAdvection(), N, 1.0, tableau=ht112_imex(), source=LinearDamping(4.0))
    for dt in (0.01, 0.3, 50.0):
        z = -4.0 * dt
        assert np.max(np.abs(sch.step(u, c, dt) - 1.7 * (1 + z / 2) / (1 - z / 2))) < 1e-13 * max(1.0, -z)


def _chezy_errors(N, dim, Cf=0.05, h0=1.3, m0=(0.7, -0.4), T=20.0, steps=(20, 40, 80)):
    mm = np.array(m0[:dim])
    nm0 = np.sqrt(np.sum(mm * mm))
    errs = []
    for nst in steps:
        dt = T / nst
        n = N + 1
        if dim == 1:
            sch = Scheme1D(ShallowWater1D(9.81), N, 1e6, source=ChezyFriction(Cf))
            u = np.zeros((2, 3, n))
            c = np.zeros((3, n))
        else:
            sch = Scheme2D(ShallowWater2D(9.81), N, 1e6, 1e6, source=ChezyFriction(Cf))
            u = np.zeros((3, 2, 2, n, n))
            c = np.zeros((2, 2, n, n))
        u[0] = h0
        for k in range(dim):
            u[1 + k] = mm[k]
        for _ in range(nst):
            u = sch.step(u, c, dt)
        exact = mm / (1 + Cf * nm0 * T / h0 ** 2)
        got = np.array([u[1 + k].reshape(-1)[0] for k in range(dim)])
        errs.append(np.max(np.abs(got - exact)))
        assert np.max(np.abs(u[0] - h0)) < 1e-12
    return np.array(errs)


@pytest.mark.parametrize("N,order", [(1, 3), (2, 3), (3, 3)])
@pytest.mark.parametrize("dim", [1, 2])
def test_chezy_friction_uniform_flow_converges_to_closed_form(N, order, dim):
    """Uniform flow on a mesh so coarse that the flux terms vanish: the
    scheme is the IMEX tableau's implicit part applied to
    dm/dt = -C_f |m| m / h0^2, whose solution is m0 / (1 + C_f |m0| t / h0^2),
    direction preserved; the error falls at the tableau's order."""
    e = _chezy_errors(N, dim)
    rates = np.log2(e[:-1] / e[1:])
    assert abs(rates[-1] - order) < 0.1 and np.all(rates > order - 0.2), rates


@pytest.mark.parametrize("N,order", [(1, 2), (2, 3), (3, 3)])
def test_damped_advection_converges_to_exact(N, order):
    """App. A model problem with a = 1, K = 1: u = u0(x - t) exp(-t);
    L2 error at t = 0.5 falls at the scheme's order (N + 1 for N <= 2; the
    time order 3 of SSP3-IMEX(4,3,3) bounds N = 3 under a CFL time step)."""
    import oracle.fourier as fr
    t = imex_tableau(N)
    cfl = fr.cfl_number(N, tableau=(t.Ae, t.be), halvings=30)
    bs = Basis(N)
    errs = []
    for E in (8, 16, 32):
        dx = 1.0 / E
        x = (np.arange(E)[:, None] + bs.xi[None]) * dx
        u = np.sin(2 * np.pi * x)[None]
        c = np.ones_like(x)
        sch = Scheme1D(VarCoeffAdvection(), N, dx, source=LinearDamping(1.0))
        T = 0.5
        nst = int(np.ceil(T / (0.5 * cfl * dx)))
        dt = T / nst
        for _ in range(nst):
            u = sch.step(u, c, dt)
        ex = np.sin(2 * np.pi * (x - T)) * np.exp(-T)
        errs.append(np.sqrt(np.sum(bs.w * (u[0] - ex) ** 2) * dx))
    errs = np.array(errs)
    rates = np.log2(errs[:-1] / errs[1:])
    assert rates[-1] > order - 0.3, rates


def test_zero_source_is_the_explicit_scheme():
    for N in (1, 2, 3):
        E = 6
        dx = 1.0 / E
        bs = Basis(N)
        x = (np.arange(E)[:, None] + bs.xi[None]) * dx
        u = np.stack([1.0 + 0.1 * np.sin(2 * np.pi * x), 0.2 * np.cos(2 * np.pi * x)])
        c = 0.05 * np.sin(2 * np.pi * x)
        t = imex_tableau(N)
        a = Scheme1D(ShallowWater1D(9.81), N, dx, source=ChezyFriction(0.0)).step(u, c, 1e-3)
        b = Scheme1D(ShallowWater1D(9.81), N, dx, tableau=(t.Ae, t.be)).step(u, c, 1e-3)
        assert np.array_equal(a, b)


def test_source_needs_imex_tableau():
    with pytest.raises(ValueError):
        Scheme1D(VarCoeffAdvection(), 2, 0.1, tableau=(np.zeros((1, 1)), np.ones(1)),
                 source=LinearDamping(1.0))
