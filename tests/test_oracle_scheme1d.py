"""Pins of the oracle's 1D cRK-FR step against what the paper and the
mathematics fix: the N = 0 finite-volume reduction (App. B, Eq. fr.fv), the
semi-discrete FR scheme as dt -> 0 (Eq. general.non.conservative.fr.one), the
GLL/g_2 operator form (Eq. fr.non.cons.gll), the fully discrete HT(1,1,2)
scheme printed in App. C, conservation, constant states, the
characteristics solution and the design order (Sec. 5.1.3)."""
import numpy as np
import pytest
from scipy.integrate import quad

from oracle import fourier
from oracle.basis import Basis, lagrange
from oracle.crkfr import FROZEN, LITERAL, STAGEWISE, Scheme1D
from oracle.exact import SineCoefficient, l2_error_1d
from oracle.semidisc import rhs_1d
from oracle.systems import ShallowWater1D, VarCoeffAdvection

G = 9.81


def swe_data(E, N, seed=0, family="gl", L=10.0, amp_m=0.2):
    rng = np.random.default_rng(seed)
    bs = Basis(N, family)
    dx = L / E
    x = (np.arange(E)[:, None] + bs.xi[None, :]) * dx
    b = 0.3 * np.exp(-((x - 0.4 * L) ** 2) / 2.0) + 0.1 * np.sin(2 * np.pi * x / L)
    h = 1.0 + 0.1 * np.cos(2 * np.pi * x / L) - b + 0.01 * rng.standard_normal(x.shape)
    m = amp_m * np.sin(2 * np.pi * x / L) + 0.01 * rng.standard_normal(x.shape)
    return np.stack([h, m]), b, dx


def varadv_data(E, N, seed=0, family="gl"):
    rng = np.random.default_rng(seed)
    bs = Basis(N, family)
    dx = 1.0 / E
    x = (np.arange(E)[:, None] + bs.xi[None, :]) * dx
    a = 1.0 + 0.5 * np.sin(2 * np.pi * x)
    v = np.sin(2 * np.pi * x) + 0.05 * rng.standard_normal(x.shape)
    return v[None], a, dx


# ---------------------------------------------------------------------------
def fv_step(system, u, c, dt, dx):
    """First-order FV scheme of App. B, Eq. fr.fv, with the fluxes of
    Eqs. combined.num.flux and non.cons.num.flux.basic, forward Euler."""
    ue, ce = u[:, :, 0], c[:, 0]
    un, cn = np.roll(ue, -1, axis=-1), np.roll(ce, -1)     # right neighbour
    lam = np.maximum(system.speed(ue, ce), system.speed(un, cn))
    fnum = 0.5 * (system.flux(ue, ce) + system.flux(un, cn)) - 0.5 * lam * (un - ue)
    wnum_u, wnum_c = 0.5 * (ue + un), 0.5 * (ce + cn)
    right = fnum + system.ncprod(ue, ce, wnum_u, wnum_c)              # face e+1/2
    left = np.roll(fnum, 1, axis=-1) + system.ncprod(ue, ce, np.roll(wnum_u, 1, axis=-1),
                                                     np.roll(wnum_c, 1))  # face e-1/2
    return (ue - dt / dx * (right - left))[:, :, None]


@pytest.mark.parametrize("system,data", [(ShallowWater1D(G), swe_data),
                                         (VarCoeffAdvection(), varadv_data)])
def test_n0_reduces_to_finite_volume(system, data):
    u, c, dx = data(40, 0)
    sch = Scheme1D(system, 0, dx)
    dt = 0.3 * dx / np.max(system.speed(u[:, :, 0], c[:, 0]))
    got = sch.step(u, c, dt)
    want = fv_step(system, u, c, dt, dx)
    assert np.max(np.abs(got - want)) <= 1e-14 * np.max(np.abs(u))


@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_constant_state_is_preserved(N):
    E = 12
    u = np.stack([np.full((E, N + 1), 1.3), np.full((E, N + 1), 0.4)])
    b = np.full((E, N + 1), 0.2)
    sch = Scheme1D(ShallowWater1D(G), N, 0.1)
    out = sch.step(u, b, 0.01)
    # round-off of D applied to a constant: |D| eps |f| dt
    assert np.max(np.abs(out - u)) < 1e-13


@pytest.mark.parametrize("N", [1, 2, 3, 4])
@pytest.mark.parametrize("family", ["gl", "gll"])
def test_mass_conservation(N, family):
    """The h equation has no non-conservative term, so the discrete mass
    sum_e dx sum_p w_p h_ep is conserved; momentum too when b is constant."""
    u, b, dx = swe_data(30, N, family=family)
    sch = Scheme1D(ShallowWater1D(G), N, dx, family=family)
    w = sch.basis.w
    mass0 = np.sum(dx * w * u[0])
    dt = 0.3 * fourier.cfl_number(N, family) * dx / 4.0
    v = u
    for _ in range(10):
        v = sch.step(v, b, dt)
    assert abs(np.sum(dx * w * v[0]) - mass0) <= 1e-14 * abs(mass0)
    bflat = np.full_like(b, 0.25)
    mom0 = np.sum(dx * w * u[1])
    v = u
    for _ in range(10):
        v = sch.step(v, bflat, dt)
    assert abs(np.sum(dx * w * v[1]) - mom0) <= 1e-13 * np.max(np.abs(u[1])) * 10.0


@pytest.mark.parametrize("N", [1, 2, 3, 4])
@pytest.mark.parametrize("family", ["gl", "gll"])
def test_residual_tends_to_semidiscrete_rhs(N, family):
    """(u^{n+1} - u^n)/dt -> semi-discrete FR right-hand side with an O(dt)
    error (Eq. crkfr.non.cons.final vs Eq. general.non.conservative.fr.one)."""
    u, b, dx = swe_data(16, N, family=family)
    sys_ = ShallowWater1D(G)
    sch = Scheme1D(sys_, N, dx, family=family)
    rhs = rhs_1d(sys_, N, dx, u, b, family=family)
    errs = []
    for dt in (1e-4, 5e-5, 2.5e-5):
        errs.append(np.max(np.abs(-sch.residual(u, b, dt) - rhs)))
    assert errs[0] < 1e-2 * np.max(np.abs(rhs))
    assert 1.8 < errs[0] / errs[1] < 2.2 and 1.8 < errs[1] / errs[2] < 2.2


@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_gll_g2_operator_form(N):
    """With GLL nodes and g_2 the semi-discrete scheme equals
    du/dt + dFR f(u) + B(w) dFR w = 0 (App. B, Eq. fr.gll / Eq. fr.non.cons.gll)."""
    sys_ = ShallowWater1D(G)
    u, b, dx = swe_data(14, N, family="gll")
    bs = Basis(N, "gll")
    D = bs.D / dx
    f = sys_.flux(u, b)
    # end-node states: GLL nodes include both element ends
    um, up = np.roll(u[:, :, -1], 1, -1), u[:, :, 0]          # face e-1/2
    bm, bp = np.roll(b[:, -1], 1), b[:, 0]
    lam = np.maximum(sys_.speed(um, bm), sys_.speed(up, bp))
    fnum = 0.5 * (sys_.flux(um, bm) + sys_.flux(up, bp)) - 0.5 * lam * (up - um)
    unum, bnum = 0.5 * (um + up), 0.5 * (bm + bp)
    fnum_r, unum_r, bnum_r = (np.roll(x, -1, -1) for x in (fnum, unum, bnum))
    dfr_f = np.einsum("pj,...j->...p", D, f)
    dfr_f = dfr_f + ((fnum_r - f[:, :, -1])[..., None] * bs.gRp
                     + (fnum - f[:, :, 0])[..., None] * bs.gLp) / dx
    dfr_u = np.einsum("pj,...j->...p", D, u) + ((unum_r - u[:, :, -1])[..., None] * bs.gRp
                                                 + (unum - u[:, :, 0])[..., None] * bs.gLp) / dx
    dfr_b = np.einsum("pj,...j->...p", D, b) + ((bnum_r - b[:, -1])[..., None] * bs.gRp
                                                 + (bnum - b[:, 0])[..., None] * bs.gLp) / dx
    want = -(dfr_f + sys_.ncprod(u, b, dfr_u, dfr_b))
    got = rhs_1d(sys_, N, dx, u, b, family="gll")
    assert np.max(np.abs(got - want)) < 1e-12 * np.max(np.abs(want))


def test_ht112_printed_form_n1():
    """For N = 1 the scheme is the fully discrete HT(1,1,2) scheme printed in
    App. C (no source, flat bottom so B vanishes): u2 = u - dt dloc f(u),
    F = (f(u) + f(u2))/2, u^{n+1} = u - dt dFR F with the time-averaged
    Rusanov flux of Eq. numflux.cons."""
    sys_ = ShallowWater1D(G)
    u, _, dx = swe_data(20, 1)
    b = np.zeros_like(u[0])
    bs = Basis(1, "gl")
    D = bs.D / dx
    dt = 0.01
    dloc = lambda X: np.einsum("pj,...j->...p", D, X)
    u2 = u - dt * dloc(sys_.flux(u, b))
    F = 0.5 * (sys_.flux(u, b) + sys_.flux(u2, b))
    U = 0.5 * (u + u2)
    tr = lambda l, X: np.einsum("p,...p->...", l, X)
    Fm, Fp = np.roll(tr(bs.l1, F), 1, -1), tr(bs.l0, F)
    Um, Up = np.roll(tr(bs.l1, U), 1, -1), tr(bs.l0, U)
    zm, zp = np.roll(tr(bs.l1, u), 1, -1), tr(bs.l0, u)
    lam = np.maximum(sys_.speed(zm, 0 * zm[0]), sys_.speed(zp, 0 * zp[0]))
    Fnum = 0.5 * (Fm + Fp) - 0.5 * lam * (Up - Um)
    dfrF = dloc(F) + ((np.roll(Fnum, -1, -1) - tr(bs.l1, F))[..., None] * bs.gRp
                      + (Fnum - tr(bs.l0, F))[..., None] * bs.gLp) / dx
    want = u - dt * dfrF
    got = Scheme1D(sys_, 1, dx).step(u, b, dt)
    assert np.max(np.abs(got - want)) < 1e-14 * np.max(np.abs(u))


def test_face_readings_coincide_for_static_coefficient_b():
    """For v_t + a(x) v_x = 0, B depends only on the static a, so the frozen,
    literal and stagewise face terms are the same scheme (Sec. 3, around
    Eqs. bad.numflux.non.cons and good.numflux.non.cons)."""
    u, a, dx = varadv_data(20, 3)
    outs = [Scheme1D(VarCoeffAdvection(), 3, dx, nc_face=m).step(u, a, 0.002)
            for m in (FROZEN, LITERAL, STAGEWISE)]
    assert np.max(np.abs(outs[0] - outs[1])) < 1e-14
    assert np.max(np.abs(outs[0] - outs[2])) < 1e-14


def test_sampled_step_equals_full_step():
    u, b, dx = swe_data(25, 4)
    sch = Scheme1D(ShallowWater1D(G), 4, dx)
    full = sch.step(u, b, 0.003)
    elems = [0, 3, 11, 24]
    part = sch.step_elements(u, b, 0.003, elems)
    assert np.max(np.abs(part - full[:, elems])) < 1e-14


@pytest.mark.filterwarnings("ignore::scipy.integrate.IntegrationWarning")
def test_characteristic_map_closed_form():
    sc = SineCoefficient(0.5)
    for x in (0.0, 0.1, 0.37, 0.5, 0.73, 0.999, 1.3, -0.4, 2.25):
        q, _ = quad(lambda s: 1.0 / sc.a(s), 0.0, x, epsabs=1e-14, epsrel=1e-14, limit=200)
        assert sc.phi(np.array([x]))[0] == pytest.approx(q, abs=1e-12)
    X = sc.foot(np.array([0.3, 0.8]), 0.7)
    assert np.allclose(sc.phi(X), sc.phi(np.array([0.3, 0.8])) - 0.7, atol=1e-13)


def _varadv_error(N, E, T, cs=0.5):
    sc = SineCoefficient(0.5)
    bs = Basis(N, "gl")
    dx = 1.0 / E
    x = (np.arange(E)[:, None] + bs.xi[None, :]) * dx
    a, v = sc.a(x), np.sin(2 * np.pi * x)[None]
    sch = Scheme1D(VarCoeffAdvection(), N, dx)
    cfl = fourier.cfl_number(N)
    t = 0.0
    while t < T - 1e-14:
        dt = min(sch.compute_dt(v, a, cfl, cs), T - t)
        v = sch.step(v, a, dt)
        t += dt
    return l2_error_1d(v[0], lambda xx: np.sin(2 * np.pi * sc.foot(xx, T)), 0.0, dx, bs.xi)


@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_varadv_design_order(N):
    """Optimal order N+1 against the characteristics solution (Sec. 5.1.3)."""
    Es = [25, 50, 100] if N < 4 else [12, 24, 48]
    errs = np.array([_varadv_error(N, E, 0.5) for E in Es])
    rates = np.log2(errs[:-1] / errs[1:])
    assert rates[-1] > N + 1 - 0.3, (errs, rates)


def _swe_self_convergence(N, mode, Es, T=0.05):
    sys_ = ShallowWater1D(G)
    pts = np.linspace(0.013, 0.987, 37)
    vals = []
    for E in Es:
        dx = 1.0 / E
        sch = Scheme1D(sys_, N, dx, nc_face=mode)
        x = (np.arange(E)[:, None] + sch.basis.xi[None, :]) * dx
        b = 0.2 * np.exp(-((x - 0.5) ** 2) / (2 * 0.08 ** 2))
        u = np.stack([1.0 + 0.1 * np.sin(2 * np.pi * x) - b, 0.3 * np.cos(2 * np.pi * x)])
        dt0 = 0.5 * fourier.cfl_number(N) * dx / (0.5 + np.sqrt(G * 1.2))
        n = int(np.ceil(T / dt0))
        for _ in range(n):
            u = sch.step(u, b, T / n)
        e = np.floor(pts / dx).astype(int)
        Lm = lagrange(sch.basis.xi, pts / dx - e)
        vals.append(np.array([np.sum(u[:, e[i], :] * Lm[i], axis=-1) for i in range(len(pts))]))
    errs = np.array([np.max(np.abs(v - vals[-1])) for v in vals[:-1]])
    return np.log2(errs[:-1] / errs[1:])


@pytest.mark.slow
def test_swe_frozen_reading_keeps_order_literal_stalls():
    """Reading 1: with B depending on the evolving h, the literal extrapolation
    term is inconsistent (order about 1) while the frozen and stagewise
    readings give the design order N+1 on a smooth moving wave."""
    Es = [10, 20, 40, 80, 320]
    fr = _swe_self_convergence(3, FROZEN, Es)
    li = _swe_self_convergence(3, LITERAL, Es)
    st = _swe_self_convergence(3, STAGEWISE, Es)
    assert fr[-1] > 3.7 and st[-1] > 3.7
    assert li[-1] < 2.0
