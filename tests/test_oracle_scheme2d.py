"""Pins of the oracle's 2D (tensor-product) cRK-FR step: reduction to the 1D
scheme on y-invariant data, x/y symmetry, constant states, conservation,
sampled evaluation and the time step of Sec. 5, Eq. time.step.2d."""
import numpy as np
import pytest

from oracle.basis import Basis
from oracle.crkfr import Scheme1D, Scheme2D
from oracle.systems import ShallowWater1D, ShallowWater2D

G = 9.81


def swe2d_data(Ey, Ex, N, seed=0, L=8.0):
    rng = np.random.default_rng(seed)
    bs = Basis(N, "gl")
    dx, dy = L / Ex, L / Ey
    x = (np.arange(Ex)[None, :, None, None] + bs.xi[None, None, None, :]) * dx
    y = (np.arange(Ey)[:, None, None, None] + bs.xi[None, None, :, None]) * dy
    x, y = np.broadcast_arrays(x, y)
    b = 0.2 * np.exp(-((x - 3) ** 2 + (y - 5) ** 2) / 2.0) + 0.05 * np.sin(2 * np.pi * x / L)
    h = 1.0 + 0.05 * np.cos(2 * np.pi * (x + y) / L) - b + 0.01 * rng.standard_normal(x.shape)
    mx = 0.1 * np.sin(2 * np.pi * y / L) + 0.01 * rng.standard_normal(x.shape)
    my = 0.1 * np.cos(2 * np.pi * x / L) + 0.01 * rng.standard_normal(x.shape)
    return np.stack([h, mx, my]), b, dx, dy


@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_y_invariant_data_matches_1d(N):
    rng = np.random.default_rng(3)
    Ex, Ey, L = 10, 3, 5.0
    bs = Basis(N, "gl")
    dx = L / Ex
    x = (np.arange(Ex)[:, None] + bs.xi[None, :]) * dx
    b1 = 0.3 * np.exp(-((x - 2.0) ** 2))
    u1 = np.stack([1.0 - b1 + 0.02 * rng.standard_normal(x.shape),
                   0.2 * np.sin(2 * np.pi * x / L)])
    dt = 0.01
    want = Scheme1D(ShallowWater1D(G), N, dx).step(u1, b1, dt)
    n = N + 1
    tile = lambda a: np.broadcast_to(a[None, :, None, :], (Ey, Ex, n, n)).copy()
    u2 = np.stack([tile(u1[0]), tile(u1[1]), np.zeros((Ey, Ex, n, n))])
    got = Scheme2D(ShallowWater2D(G), N, dx, 0.7, family="gl").step(u2, tile(b1), dt)
    for v in range(2):
        assert np.max(np.abs(got[v] - want[v][None, :, None, :])) < 1e-13
    assert np.max(np.abs(got[2])) < 1e-13


@pytest.mark.parametrize("N", [2, 3])
def test_xy_transposition_symmetry(N):
    u, b, dx, dy = swe2d_data(5, 5, N)
    sch = Scheme2D(ShallowWater2D(G), N, dx, dy)
    out = sch.step(u, b, 0.005)
    T = lambda a: np.swapaxes(np.swapaxes(a, -4, -3), -2, -1)
    uT = np.stack([T(u[0]), T(u[2]), T(u[1])])
    outT = sch.step(uT, T(b), 0.005)
    want = np.stack([T(out[0]), T(out[2]), T(out[1])])
    assert np.max(np.abs(outT - want)) < 1e-14


@pytest.mark.parametrize("N", [1, 3, 4])
def test_constant_state_2d(N):
    n = N + 1
    u = np.stack([np.full((3, 4, n, n), 1.1), np.full((3, 4, n, n), 0.3),
                  np.full((3, 4, n, n), -0.2)])
    b = np.full((3, 4, n, n), 0.1)
    out = Scheme2D(ShallowWater2D(G), N, 0.5, 0.4).step(u, b, 0.005)
    assert np.max(np.abs(out - u)) < 1e-13


@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_mass_conservation_2d(N):
    u, b, dx, dy = swe2d_data(4, 6, N)
    sch = Scheme2D(ShallowWater2D(G), N, dx, dy)
    w = sch.basis.w
    mass = lambda v: np.sum(dx * dy * w[:, None] * w[None, :] * v[0])
    m0 = mass(u)
    v = u
    for _ in range(5):
        v = sch.step(v, b, 0.004)
    assert abs(mass(v) - m0) <= 1e-14 * abs(m0)


def test_sampled_step_equals_full_step_2d():
    u, b, dx, dy = swe2d_data(6, 5, 3)
    sch = Scheme2D(ShallowWater2D(G), 3, dx, dy)
    full = sch.step(u, b, 0.004)
    ey, ex = np.array([0, 2, 5, 5]), np.array([0, 4, 1, 4])
    part = sch.step_elements(u, b, 0.004, ey, ex)
    assert np.max(np.abs(part - full[:, ey, ex])) < 1e-14


def test_time_step_formula_2d():
    """Eq. time.step.2d: dt = Cs CFL / max_e(sigma_x(ubar)/dx + sigma_y(ubar)/dy)
    with the element means ubar = sum_pq w_p w_q u_pq."""
    u, b, dx, dy = swe2d_data(3, 4, 2)
    sch = Scheme2D(ShallowWater2D(G), 2, dx, dy)
    w = sch.basis.w
    best = 0.0
    for ey in range(3):
        for ex in range(4):
            h = np.sum(np.outer(w, w) * u[0, ey, ex])
            qx = np.sum(np.outer(w, w) * u[1, ey, ex])
            qy = np.sum(np.outer(w, w) * u[2, ey, ex])
            c = np.sqrt(G * h)
            best = max(best, (abs(qx / h) + c) / dx + (abs(qy / h) + c) / dy)
    assert sch.compute_dt(u, b, 0.17, 0.5) == pytest.approx(0.5 * 0.17 / best, rel=1e-14)


# ----------------------------------------------------------------------------
# Pins of the mixed-momentum flux components (hu)(hv)/h of flux_x and flux_y.
#
# On data that does not vary across one direction, with the tangential
# momentum a fixed multiple phi0 of the depth, every stage keeps that ratio:
# the tangential momentum's flux along the varying direction is phi0 times the
# normal momentum (the flux of h), its Rusanov term is phi0 times that of h
# (same speed, jump phi0 times h's), the non-conservative product has no row
# for it, and the invariant direction contributes only round-off.  So the step
# must return tangential momentum = phi0 * depth, while depth and normal
# momentum equal the 1D step.  A wrong factor, sign or denominator on the
# mixed term breaks the ratio.
# ----------------------------------------------------------------------------
PHI0 = 0.37


def _swe1d_line(N, Ex, L, seed):
    rng = np.random.default_rng(seed)
    bs = Basis(N, "gl")
    dx = L / Ex
    x = (np.arange(Ex)[:, None] + bs.xi[None, :]) * dx
    b1 = 0.3 * np.exp(-((x - 2.0) ** 2))
    h1 = 1.0 - b1 + 0.02 * rng.standard_normal(x.shape)
    m1 = 0.2 * np.sin(2 * np.pi * x / L) + 0.05 * rng.standard_normal(x.shape)
    return np.stack([h1, m1]), b1, dx


@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_mixed_momentum_flux_x_keeps_ratio(N):
    """y-invariant data with hv = phi0 h: flux_x[2] = (hu)(hv)/h = phi0 hu."""
    Ex, Ey, L, dt = 10, 3, 5.0, 0.01
    u1, b1, dx = _swe1d_line(N, Ex, L, 5)
    want = Scheme1D(ShallowWater1D(G), N, dx).step(u1, b1, dt)
    n = N + 1
    tile = lambda a: np.broadcast_to(a[None, :, None, :], (Ey, Ex, n, n)).copy()
    u2 = np.stack([tile(u1[0]), tile(u1[1]), PHI0 * tile(u1[0])])
    got = Scheme2D(ShallowWater2D(G), N, dx, 0.7, family="gl").step(u2, tile(b1), dt)
    for v in range(2):
        assert np.max(np.abs(got[v] - want[v][None, :, None, :])) < 1e-13
    assert np.max(np.abs(got[2] - PHI0 * got[0])) < 1e-13
    # the tangential momentum really moved (the pin is not vacuous)
    assert np.max(np.abs(got[2] - u2[2])) > 1e-4


@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_mixed_momentum_flux_y_keeps_ratio(N):
    """x-invariant data with hu = phi0 h: flux_y[1] = (hu)(hv)/h = phi0 hv."""
    Ex, Ey, L, dt = 3, 10, 5.0, 0.01
    u1, b1, dy = _swe1d_line(N, Ey, L, 6)
    want = Scheme1D(ShallowWater1D(G), N, dy).step(u1, b1, dt)
    n = N + 1
    # element (ey, ex), nodes (q, p): the 1D line runs along ey and q
    tile = lambda a: np.broadcast_to(a[:, None, :, None], (Ey, Ex, n, n)).copy()
    u2 = np.stack([tile(u1[0]), PHI0 * tile(u1[0]), tile(u1[1])])
    got = Scheme2D(ShallowWater2D(G), N, 0.9, dy, family="gl").step(u2, tile(b1), dt)
    assert np.max(np.abs(got[0] - want[0][:, None, :, None])) < 1e-13
    assert np.max(np.abs(got[2] - want[1][:, None, :, None])) < 1e-13
    assert np.max(np.abs(got[1] - PHI0 * got[0])) < 1e-13
    assert np.max(np.abs(got[1] - u2[1])) > 1e-4


@pytest.mark.parametrize("N", [2, 3])
def test_mixed_momentum_ratio_with_gll_nodes_and_source_free_wb_form(N):
    """The same ratio pin for GLL nodes and for the well-balanced form, whose
    fluxes carry the same mixed term."""
    from oracle.systems import ShallowWater2DWB
    Ex, Ey, L, dt = 8, 2, 5.0, 0.008
    rng = np.random.default_rng(11)
    bs = Basis(N, "gll")
    dx = L / Ex
    x = (np.arange(Ex)[:, None] + bs.xi[None, :]) * dx
    b1 = 0.25 * np.exp(-((x - 2.5) ** 2))
    h1 = 1.0 - b1 + 0.02 * rng.standard_normal(x.shape)
    m1 = 0.15 * np.cos(2 * np.pi * x / L)
    n = N + 1
    tile = lambda a: np.broadcast_to(a[None, :, None, :], (Ey, Ex, n, n)).copy()
    u2 = np.stack([tile(h1), tile(m1), PHI0 * tile(h1)])
    for system in (ShallowWater2D(G), ShallowWater2DWB(G)):
        got = Scheme2D(system, N, dx, 0.6, family="gll").step(u2, tile(b1), dt)
        assert np.max(np.abs(got[2] - PHI0 * got[0])) < 1e-13


# ----------------------------------------------------------------------------
# A genuinely 2D accuracy pin: a smooth wave along the diagonal.
#
# Data that depend on s = x + y only, with hu = hv = m(s), solve the 2D system
# exactly when (h, m) solve
#     h_t + 2 m_s = 0,   m_t + (2 m^2/h + g h^2/2)_s + g h b_s = 0,
# which is 1D shallow water in xi = s / sqrt(2) with normal momentum
# m_n = sqrt(2) m (d/dxi = sqrt(2) d/ds).  The periodic square [0, L]^2 is
# periodic in s with period L, i.e. in xi with period L / sqrt(2).  The 2D
# oracle on E x E quads must converge at order N + 1 to a fine 1D run in xi.
# ----------------------------------------------------------------------------
def _diag_fields(s, L):
    k = 2 * np.pi / L
    b = 0.1 * np.sin(k * s) + 0.05 * np.cos(2 * k * s)
    h = 1.0 + 0.08 * np.cos(k * s) - b
    m = 0.1 * np.sin(k * s + 0.3) * h
    return h, m, b


def _fine_1d_diag(L, T, N=4, E=160, cs=0.4):
    P = L / np.sqrt(2.0)
    bs = Basis(N, "gl")
    dxi = P / E
    xi = (np.arange(E)[:, None] + bs.xi[None, :]) * dxi
    h, m, b = _diag_fields(np.sqrt(2.0) * xi, L)
    u = np.stack([h, np.sqrt(2.0) * m])
    sch = Scheme1D(ShallowWater1D(G), N, dxi)
    from oracle.fourier import cfl_number
    dt0 = sch.compute_dt(u, b, cfl_number(N, "gl"), cs)
    nsteps = int(np.ceil(T / dt0))
    for _ in range(nsteps):
        u = sch.step(u, b, T / nsteps)
    return u, bs, dxi, E


def _eval_1d(u, bs, dxi, E, xi):
    """The fine solution's interpolating polynomial at the points ``xi``."""
    from oracle.basis import lagrange
    P = E * dxi
    xi = np.mod(xi, P)
    e = np.minimum((xi / dxi).astype(int), E - 1)
    r = xi / dxi - e
    lag = lagrange(bs.xi, r)                       # (S, n)
    return np.einsum("sn,vsn->vs", lag, u[:, e, :])


@pytest.mark.parametrize("N", [2, 3])
def test_diagonal_wave_converges_at_design_order(N):
    from oracle.fourier import cfl_number
    L, T, cs = 1.0, 0.06, 0.4
    fine = _fine_1d_diag(L, T)
    errs, sizes = [], [6, 12, 24]
    for E in sizes:
        bs = Basis(N, "gl")
        d = L / E
        x = (np.arange(E)[None, :, None, None] + bs.xi[None, None, None, :]) * d
        y = (np.arange(E)[:, None, None, None] + bs.xi[None, None, :, None]) * d
        x, y = np.broadcast_arrays(x, y)
        h, m, b = _diag_fields(x + y, L)
        u = np.stack([h, m, m])
        sch = Scheme2D(ShallowWater2D(G), N, d, d)
        dt0 = sch.compute_dt(u, b, cfl_number(N, "gl"), cs)
        nsteps = int(np.ceil(T / dt0))
        for _ in range(nsteps):
            u = sch.step(u, b, T / nsteps)
        ref = _eval_1d(*fine, ((x + y) / np.sqrt(2.0)).ravel())
        ref = np.stack([ref[0], ref[1] / np.sqrt(2.0), ref[1] / np.sqrt(2.0)]).reshape(u.shape)
        w2 = (bs.w[:, None] * bs.w[None, :]) * d * d
        errs.append(np.sqrt(np.sum(w2 * (u - ref) ** 2)))
    rates = [np.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    # measured: N = 2: 3.7e-3, 7.5e-4, 9.5e-5 (rates 2.3, 3.0);
    #           N = 3: 6.5e-4, 3.2e-5, 1.4e-6 (rates 4.4, 4.5)
    assert errs[-1] < {2: 2e-4, 3: 3e-6}[N], errs
    assert rates[-1] > N + 1 - 0.4, (errs, rates)


def test_mixed_momentum_pin_catches_a_planted_factor():
    """The ratio pin is not vacuous: an oracle whose mixed x-flux term carries a
    wrong factor (planted here, on the CPU) violates it."""
    class Wrong(ShallowWater2D):
        def flux_x(self, u, c):
            f = super().flux_x(u, c)
            f[2] = 1.1 * f[2]
            return f
    N, Ex, Ey, L, dt = 3, 10, 3, 5.0, 0.01
    u1, b1, dx = _swe1d_line(N, Ex, L, 5)
    n = N + 1
    tile = lambda a: np.broadcast_to(a[None, :, None, :], (Ey, Ex, n, n)).copy()
    u2 = np.stack([tile(u1[0]), tile(u1[1]), PHI0 * tile(u1[0])])
    got = Scheme2D(Wrong(G), N, dx, 0.7, family="gl").step(u2, tile(b1), dt)
    assert np.max(np.abs(got[2] - PHI0 * got[0])) > 1e-5
