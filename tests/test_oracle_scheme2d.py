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
