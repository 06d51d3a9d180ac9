"""Pins of the oracle's well-balanced shallow-water variant (the hydrostatic
pressure written as the non-conservative product g h (h + b)_x, the Rusanov
dissipation of the h equation on the free surface; the paper lists
well-balanced cRK methods as open, Sec. 6):

- a lake at rest over any bathymetry stays at rest to round-off (1D, 2D,
  GL and GLL, with and without Chezy friction), while the standard form
  moves it by the truncation error;
- design order N+1 on a smooth moving wave over a bump (self-convergence,
  as for the standard form);
- exact mass conservation;
- with a flat bottom and with bathymetry the two forms approximate the same
  solution: their difference falls at order N+1.
"""
import numpy as np
import pytest

from oracle import fourier
from oracle.basis import Basis
from oracle.crkfr import Scheme1D, Scheme2D
from oracle.sources import ChezyFriction
from oracle.systems import ShallowWater1D, ShallowWater1DWB, ShallowWater2D, ShallowWater2DWB

G = 9.81


def bathymetry_1d(x):
    return 0.3 * np.exp(-((x - 0.4) ** 2) / (2 * 0.05 ** 2)) + 0.1 * np.sin(6 * np.pi * x) ** 2


def lake_1d(N, family, E):
    bs = Basis(N, family)
    dx = 1.0 / E
    x = (np.arange(E)[:, None] + bs.xi[None, :]) * dx
    b = bathymetry_1d(x)
    return np.stack([1.0 - b, np.zeros_like(b)]), b, dx


CASES = [(N, f) for N in range(1, 5) for f in ("gl", "gll")]


@pytest.mark.parametrize("N,family", CASES)
def test_lake_at_rest_1d_to_round_off(N, family):
    E = 16
    u0, b, dx = lake_1d(N, family, E)
    dt = 0.5 * fourier.cfl_number(N, family, halvings=30) * dx / np.sqrt(G)
    wb = Scheme1D(ShallowWater1DWB(G), N, dx, family=family)
    st = Scheme1D(ShallowWater1D(G), N, dx, family=family)
    u, v = u0.copy(), u0.copy()
    for _ in range(50):
        u = wb.step(u, b, dt)
        v = st.step(v, b, dt)
    assert np.max(np.abs(u - u0)) < 1e-13
    # the standard form moves the lake by its truncation error
    assert np.max(np.abs(v - u0)) > 1e-7


def test_lake_at_rest_1d_with_friction():
    N, E = 3, 12
    u0, b, dx = lake_1d(N, "gl", E)
    sch = Scheme1D(ShallowWater1DWB(G), N, dx, source=ChezyFriction(5.0))
    u = u0.copy()
    for _ in range(20):
        u = sch.step(u, b, 0.003)
    assert np.max(np.abs(u - u0)) < 1e-13


@pytest.mark.parametrize("N,family", [(1, "gl"), (2, "gll"), (3, "gl")])
def test_lake_at_rest_2d_to_round_off(N, family):
    Ex, Ey = 5, 4
    bs = Basis(N, family)
    dx, dy = 1.0 / Ex, 1.0 / Ey
    x = (np.arange(Ex)[None, :, None, None] + bs.xi[None, None, None, :]) * dx
    y = (np.arange(Ey)[:, None, None, None] + bs.xi[None, None, :, None]) * dy
    x, y = np.broadcast_arrays(x, y)
    b = 0.3 * np.exp(-((x - 0.4) ** 2 + (y - 0.6) ** 2) / (2 * 0.1 ** 2)) + 0.05 * np.sin(2 * np.pi * x)
    u0 = np.stack([1.0 - b, np.zeros_like(b), np.zeros_like(b)])
    dt = 0.2 * fourier.cfl_number(N, family, halvings=30) * dx / np.sqrt(G)
    wb = Scheme2D(ShallowWater2DWB(G), N, dx, dy, family=family)
    st = Scheme2D(ShallowWater2D(G), N, dx, dy, family=family)
    u, v = u0.copy(), u0.copy()
    for _ in range(10):
        u = wb.step(u, b, dt)
        v = st.step(v, b, dt)
    assert np.max(np.abs(u - u0)) < 1e-13
    assert np.max(np.abs(v - u0)) > 1e-7


def test_mass_is_conserved_1d():
    N, E = 3, 20
    bs = Basis(N)
    dx = 1.0 / E
    x = (np.arange(E)[:, None] + bs.xi[None, :]) * dx
    b = bathymetry_1d(x)
    u = np.stack([1.0 + 0.05 * np.sin(2 * np.pi * x) - b, 0.2 * np.cos(2 * np.pi * x)])
    sch = Scheme1D(ShallowWater1DWB(G), N, dx)
    m0 = np.sum(bs.w * u[0]) * dx
    for _ in range(30):
        u = sch.step(u, b, 5e-4)
    assert abs(np.sum(bs.w * u[0]) * dx - m0) < 1e-14


def _moving_wave(system, N, Es, T=0.05, flat=False):
    pts = np.linspace(0.013, 0.987, 37)
    vals = []
    for E in Es:
        dx = 1.0 / E
        sch = Scheme1D(system, N, dx)
        x = (np.arange(E)[:, None] + sch.basis.xi[None, :]) * dx
        b = np.zeros_like(x) if flat else 0.2 * np.exp(-((x - 0.5) ** 2) / (2 * 0.08 ** 2))
        u = np.stack([1.0 + 0.1 * np.sin(2 * np.pi * x) - b, 0.3 * np.cos(2 * np.pi * x)])
        dt0 = 0.5 * fourier.cfl_number(N, halvings=30) * dx / (0.5 + np.sqrt(G * 1.2))
        n = int(np.ceil(T / dt0))
        for _ in range(n):
            u = sch.step(u, b, T / n)
        e = np.floor(pts / dx).astype(int)
        xi = pts / dx - e
        # Lagrange basis of the nodes at xi
        nodes = sch.basis.xi
        Lm = np.ones((len(pts), len(nodes)))
        for j in range(len(nodes)):
            for k in range(len(nodes)):
                if k != j:
                    Lm[:, j] *= (xi - nodes[k]) / (nodes[j] - nodes[k])
        vals.append(np.array([np.sum(u[:, e[i], :] * Lm[i], axis=-1) for i in range(len(pts))]))
    return vals


@pytest.mark.slow
def test_design_order_on_a_moving_wave():
    N = 3
    Es = [10, 20, 40, 80, 320]
    vals = _moving_wave(ShallowWater1DWB(G), N, Es)
    errs = np.array([np.max(np.abs(v - vals[-1])) for v in vals[:-1]])
    rates = np.log2(errs[:-1] / errs[1:])
    assert rates[-1] > 3.7, rates


@pytest.mark.parametrize("flat", [True, False])
def test_wb_and_standard_forms_agree_to_design_order(flat):
    """The two forms discretise the same equations: their difference on a
    smooth moving wave falls at order N+1 under refinement."""
    N = 2
    Es = [10, 20, 40]
    a = _moving_wave(ShallowWater1DWB(G), N, Es, flat=flat)
    b = _moving_wave(ShallowWater1D(G), N, Es, flat=flat)
    d = np.array([np.max(np.abs(x - y)) for x, y in zip(a, b)])
    rates = np.log2(d[:-1] / d[1:])
    assert rates[-1] > N + 1 - 0.4, rates


@pytest.mark.parametrize("N", [1, 2, 3])
def test_standard_form_lake_at_rest_defect_converges(N):
    """The standard form does not keep a lake at rest (the paper does not
    claim it does, Sec. 6); its defect after t = 0.05 over a Gaussian bump
    falls at about the design order N+1 on 25..200 elements (measured:
    N = 1: 2.3, N = 2: 3.0, N = 3: 3.9 on the finest pair)."""
    cfl = fourier.cfl_number(N, halvings=30)
    errs = []
    for E in (25, 50, 100, 200):
        bs = Basis(N)
        dx = 1.0 / E
        x = (np.arange(E)[:, None] + bs.xi[None, :]) * dx
        b = 0.2 * np.exp(-((x - 0.5) ** 2) / (2 * 0.08 ** 2))
        u0 = np.stack([1.0 - b, np.zeros_like(b)])
        sch = Scheme1D(ShallowWater1D(G), N, dx)
        T = 0.05
        n = int(np.ceil(T / (0.5 * cfl * dx / np.sqrt(G))))
        u = u0.copy()
        for _ in range(n):
            u = sch.step(u, b, T / n)
        errs.append(np.max(np.abs(u - u0)))
    errs = np.array(errs)
    rates = np.log2(errs[:-1] / errs[1:])
    assert np.all(errs > 1e-10)
    assert rates[-1] > N + 1 - 0.8, rates
